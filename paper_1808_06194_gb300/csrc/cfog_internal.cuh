// Internal helpers shared by the libcfog translation units (not part of the ABI).
#pragma once

#include <cuda_runtime.h>

#include <cstdarg>
#include <cstdio>
#include <string>

#include "cfog.h"

namespace cfog {

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

// Raise a kernel's dynamic shared-memory limit to at least `bytes` on the
// current device.  The attribute call is made only when the limit grows, so
// steady-state launches (and stream captures after a first call) make none.
cfog_status ensure_dynamic_smem(const void *func, int bytes, const char *who);

}  // namespace cfog
