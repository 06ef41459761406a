// Library-wide entry points: version, error string, defaults, feature layout.
#include "cfog_internal.cuh"

#include <algorithm>
#include <map>
#include <mutex>
#include <utility>

namespace cfog {

static thread_local std::string g_last_error;

void set_error(const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_last_error = buf;
}

void clear_error() { g_last_error.clear(); }

int sm_count() {
    static std::mutex mu;
    static int cached[64] = {0};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 148;
    std::lock_guard<std::mutex> lock(mu);
    if (cached[dev] == 0) {
        int n = 0;
        if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0)
            n = 148;
        cached[dev] = n;
    }
    return cached[dev];
}

cfog_status persistent_ctas_per_sm(const void *func, int threads, int dyn_smem, int *out,
                                   const char *who) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return check_cuda(e, who);
    int api = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&api, func, threads, dyn_smem);
    if (e != cudaSuccess) return check_cuda(e, who);
    cudaFuncAttributes fa;
    e = cudaFuncGetAttributes(&fa, func);
    if (e != cudaSuccess) return check_cuda(e, who);
    int smem_sm = 0, reserved = 0, regs_sm = 0, threads_sm = 0;
    cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
    cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev);
    cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, dev);
    cudaDeviceGetAttribute(&threads_sm, cudaDevAttrMaxThreadsPerMultiProcessor, dev);
    const long long smem_block = (long long)dyn_smem + (long long)fa.sharedSizeBytes + reserved;
    // registers are allocated per warp in units of 256 (8 per thread)
    const long long regs_block = (long long)((fa.numRegs + 7) / 8 * 8) * 32 * ((threads + 31) / 32);
    long long est = threads_sm / threads;
    if (smem_block > 0) est = std::min(est, (long long)smem_sm / smem_block);
    if (regs_block > 0) est = std::min(est, (long long)regs_sm / regs_block);
    *out = (int)std::max<long long>(1, std::max<long long>(api, est));
    return CFOG_OK;
}

cfog_status ensure_dynamic_smem(const void *func, int bytes, const char *who) {
    static std::mutex mu;
    static std::map<std::pair<const void *, int>, int> limits;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return check_cuda(e, who);
    std::lock_guard<std::mutex> lock(mu);
    int &cur = limits[std::make_pair(func, dev)];
    if (bytes <= cur) return CFOG_OK;
    e = cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e != cudaSuccess) {
        set_error("%s: cannot allow %d bytes of shared memory: %s", who, bytes,
                  cudaGetErrorString(e));
        return CFOG_E_CUDA;
    }
    // prefer the largest shared-memory carveout: the occupancy calculator
    // (which sizes the persistent grids) then counts every CTA that fits
    e = cudaFuncSetAttribute(func, cudaFuncAttributePreferredSharedMemoryCarveout,
                             cudaSharedmemCarveoutMaxShared);
    if (e != cudaSuccess) {
        set_error("%s: cannot set the shared-memory carveout: %s", who, cudaGetErrorString(e));
        return CFOG_E_CUDA;
    }
    cur = bytes;
    return CFOG_OK;
}

}  // namespace cfog

extern "C" {

int32_t cfog_version(void) { return CFOG_API_VERSION; }

const char *cfog_last_error(void) { return cfog::g_last_error.c_str(); }

cfog_status cfog_default_params(cfog_params *p) {
    if (!p) {
        cfog::set_error("cfog_default_params: p is NULL");
        return CFOG_E_INVAL;
    }
    p->m = 9;             // Sec. V-C
    p->sigma = 0.8f;      // Sec. V-C
    p->eps = 1e-6f;       // reading: absolute guard of the L2 normalisation
    p->gauss_radius = 3;  // reading: ceil(3 sigma)
    p->orientation = CFOG_ORIENT_EQ2;   // Eq. 2, the scheme the paper's method uses
    return CFOG_OK;
}

size_t cfog_feature_layout(int32_t h, int32_t w, int32_t m, int64_t *row_pitch,
                           int64_t *plane_pitch) {
    if (h <= 0 || w <= 0 || m <= 0 || m > 64) return 0;
    // rows padded to 32 floats (128 B) so every row starts on a 128 B boundary
    int64_t rp = ((int64_t)w + 31) / 32 * 32;
    int64_t pp = rp * (int64_t)h;
    if (row_pitch) *row_pitch = rp;
    if (plane_pitch) *plane_pitch = pp;
    return (size_t)(pp * m) * sizeof(float);
}

}  // extern "C"
