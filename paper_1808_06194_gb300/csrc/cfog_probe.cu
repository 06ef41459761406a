// Measurement helper, not part of the method: an FP32 fused multiply-add
// throughput probe.  It gives the measured denominator of the FP32-ALU
// roofline fraction the benchmark reports for the FFT matcher.
//
// Every thread runs eight independent FMA chains (scalar fmaf, or four packed
// f32x2 chains) for `iters` iterations of 16 unrolled steps, so issue, not
// latency, bounds the loop.  The result is written only when it is exactly
// zero, which the compiler cannot rule out, so no chain is removed and almost
// nothing is stored.
#include "cfog_internal.cuh"

#include <cstdint>

namespace cfog {
namespace {

constexpr int kProbeThreads = 256;
constexpr int kProbeUnroll = 16;

template <bool PACKED>
__global__ void __launch_bounds__(kProbeThreads) fma_probe_kernel(int iters, float *out) {
    const float seed = 1.0f + 1e-6f * (float)threadIdx.x;
    float s = 0.f;
    if constexpr (PACKED) {
        float2 a[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) a[k] = make_float2(seed + k, seed - k);
        const float2 b = make_float2(0.9999999f, 0.9999998f), c = make_float2(1e-7f, 2e-7f);
        for (int i = 0; i < iters; ++i) {
#pragma unroll
            for (int u = 0; u < kProbeUnroll; ++u)
#pragma unroll
                for (int k = 0; k < 4; ++k) a[k] = __ffma2_rn(a[k], b, c);
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) s += a[k].x + a[k].y;
    } else {
        float a[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) a[k] = seed + k;
        const float b = 0.9999999f, c = 1e-7f;
        for (int i = 0; i < iters; ++i) {
#pragma unroll
            for (int u = 0; u < kProbeUnroll; ++u)
#pragma unroll
                for (int k = 0; k < 8; ++k) a[k] = fmaf(a[k], b, c);
        }
#pragma unroll
        for (int k = 0; k < 8; ++k) s += a[k];
    }
    if (s == 0.f) out[0] = s;
}

}  // namespace
}  // namespace cfog

extern "C" cfog_status cfog_probe_fp32_fma(int32_t blocks, int32_t iters, int32_t packed,
                                           float *out_dev, double *flops, void *stream) {
    CFOG_TRACE("cfog_probe_fp32_fma");
    CFOG_REQUIRE(blocks >= 1 && blocks <= (1 << 20), "cfog_probe_fp32_fma: blocks = %d", blocks);
    CFOG_REQUIRE(iters >= 1 && iters <= (1 << 24), "cfog_probe_fp32_fma: iters = %d", iters);
    CFOG_REQUIRE(out_dev, "cfog_probe_fp32_fma: out_dev is NULL");
    cudaStream_t s = cfog::as_stream(stream);
    if (packed)
        cfog::fma_probe_kernel<true><<<blocks, cfog::kProbeThreads, 0, s>>>(iters, out_dev);
    else
        cfog::fma_probe_kernel<false><<<blocks, cfog::kProbeThreads, 0, s>>>(iters, out_dev);
    // 8 FMAs (2 flops each) per unrolled step and thread, in either form
    if (flops)
        *flops = (double)blocks * cfog::kProbeThreads * (double)iters * cfog::kProbeUnroll * 8.0 * 2.0;
    return cfog::check_launch("cfog_probe_fp32_fma: launch");
}
