// Internal helpers shared by the libcfog translation units (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <cstdarg>
#include <cstdio>
#include <string>

#include "cfog.h"

namespace cfog {

// NVTX range over one C-ABI call (named after the call), visible in a
// profiler's timeline; without a tool attached it costs a pointer test.
struct TraceRange {
    explicit TraceRange(const char *name) { nvtxRangePushA(name); }
    ~TraceRange() { nvtxRangePop(); }
    TraceRange(const TraceRange &) = delete;
    TraceRange &operator=(const TraceRange &) = delete;
};
#define CFOG_TRACE(name) ::cfog::TraceRange cfog_trace_range_(name)

// Per-host-thread message behind cfog_last_error().
void set_error(const char *fmt, ...);
void clear_error();

inline cudaStream_t as_stream(void *s) { return reinterpret_cast<cudaStream_t>(s); }

// Check the launch that was just issued; map a failure to CFOG_E_CUDA.
inline cfog_status check_launch(const char *what) {
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        set_error("%s: %s", what, cudaGetErrorString(e));
        return CFOG_E_CUDA;
    }
    return CFOG_OK;
}

inline cfog_status check_cuda(cudaError_t e, const char *what) {
    if (e != cudaSuccess) {
        set_error("%s: %s", what, cudaGetErrorString(e));
        return CFOG_E_CUDA;
    }
    return CFOG_OK;
}

#define CFOG_REQUIRE(cond, ...)          \
    do {                                 \
        if (!(cond)) {                   \
            ::cfog::set_error(__VA_ARGS__); \
            return CFOG_E_INVAL;         \
        }                                \
    } while (0)

// Number of SMs of the current device (cached per device).
int sm_count();

// CTAs of `func` (threads per CTA, dynamic shared memory) that fit on one SM
// of the current device: the larger of the occupancy calculator's answer and
// an estimate from the kernel's registers and shared memory against the
// device's per-SM limits, at least 1.  Sizes persistent grids (a CTA that
// does not fit only starts later).
cfog_status persistent_ctas_per_sm(const void *func, int threads, int dyn_smem, int *out,
                                   const char *who);

// Raise a kernel's dynamic shared-memory limit to at least `bytes` on the
// current device.  The attribute call is made only when the limit grows, so
// steady-state launches (and stream captures after a first call) make none.
cfog_status ensure_dynamic_smem(const void *func, int bytes, const char *who);

}  // namespace cfog
