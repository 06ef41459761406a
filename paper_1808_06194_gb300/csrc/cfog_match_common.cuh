// Device code shared by the FFT matcher (cfog_match.cu) and the BF16
// tensor-core matcher (cfog_bf16.cu): launch arguments, job views, block
// reductions, the sub-pixel fit.  Internal to libcfog.
#pragma once

#include <cuda_runtime.h>

#include <cfloat>
#include <climits>
#include <cmath>
#include <cstdint>

#include "cfog.h"
#include "cfog_internal.cuh"

namespace cfog {

constexpr float kRescoreRel = 2e-5f; // FFT nomination band, relative to sum T^2 + N^2
constexpr int kMaxCand = 8;
constexpr int kCandBuf = 64;

struct MatchArgs {
    // single feature pair (cfog_match) ...
    const float *ref;
    const float *ref_sq;
    int ref_h, ref_w;
    int64_t ref_rp, ref_pp;
    const float *sen;
    const float *sen_sq;
    int sen_h, sen_w;
    int64_t sen_rp, sen_pp;
    // ... or a device table of jobs (cfog_match_batched)
    const cfog_job *jobs;
    const int *job_of_cp;
    int n_jobs;
    int m;
    const cfog_point *cps;
    const int *tmpl;
    const int *radius;
    const cfog_point *prior;
    int n;
    cfog_match_result *out;
    float *surface;
    int surf_side;   // 2 * radius_max + 1
    int tmpl_max, radius_max;  // launch bounds the shared memory was sized for
    int smem_bytes;  // dynamic shared memory of the launch
    int plan_table;  // tuned-plan table the FFT kernel consults (-1: none)
    long long wait_limit;  // cycle limit of each bounded device-side wait
    int stall_cp;    // failure-detection test: this CP waits on a barrier nothing
                     // arrives at, until wait_limit (-1: none)
};

// Failure-detection test hook of the tensor-core path (host state, read at
// launch): the CP to stall and the wait limit in cycles.
void bf16_test_hook(int *stall_cp, long long *wait_limit);


// n / d for 0 <= n < 2^16, 1 <= d < 2^16: one multiply-high with
// ceil(2^32 / d), exact because n * d < 2^32.
struct FastDiv {
    unsigned mul;
    int d;
    __device__ explicit FastDiv(int dd) : d(dd) {
        mul = dd > 1 ? (unsigned)((0x100000000ull + (unsigned)dd - 1) / (unsigned)dd) : 0u;
    }
    __device__ __forceinline__ int div(int n) const { return d > 1 ? (int)__umulhi((unsigned)n, mul) : n; }
};

struct JobView {
    const float *ref, *ref_sq, *sen, *sen_sq;
    int ref_h, ref_w, sen_h, sen_w;
    int64_t ref_rp, ref_pp, sen_rp, sen_pp;
    bool ok;
};

__device__ __forceinline__ JobView job_view(const MatchArgs &A, int cp) {
    JobView v;
    if (!A.jobs) {
        v.ref = A.ref; v.ref_sq = A.ref_sq; v.ref_h = A.ref_h; v.ref_w = A.ref_w;
        v.ref_rp = A.ref_rp; v.ref_pp = A.ref_pp;
        v.sen = A.sen; v.sen_sq = A.sen_sq; v.sen_h = A.sen_h; v.sen_w = A.sen_w;
        v.sen_rp = A.sen_rp; v.sen_pp = A.sen_pp;
        v.ok = true;
        return v;
    }
    const int j = A.job_of_cp ? A.job_of_cp[cp] : 0;
    v.ok = j >= 0 && j < A.n_jobs;
    const cfog_job &J = A.jobs[v.ok ? j : 0];
    v.ref = J.ref.data; v.ref_sq = J.ref.sqnorm; v.ref_h = J.ref.h; v.ref_w = J.ref.w;
    v.ref_rp = J.ref.row_pitch; v.ref_pp = J.ref.plane_pitch;
    v.sen = J.sen.data; v.sen_sq = J.sen.sqnorm; v.sen_h = J.sen.h; v.sen_w = J.sen.w;
    v.sen_rp = J.sen.row_pitch; v.sen_pp = J.sen.plane_pitch;
    v.ok = v.ok && J.ref.m == A.m && J.sen.m == A.m && v.ref && v.sen && v.sen_sq;
    return v;
}

// ------------------------------------------------------------ reductions --
template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Block-wide sum (fixed tree: deterministic).  `red` holds NT/32 values.
template <int NT, typename T>
__device__ __forceinline__ T block_sum(T v, T *red) {
    v = warp_sum(v);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) red[warp] = v;
    __syncthreads();
    T t = (threadIdx.x < NT / 32) ? red[threadIdx.x] : T(0);
    if (warp == 0) t = warp_sum(t);
    if (threadIdx.x == 0) red[0] = t;
    __syncthreads();
    const T r = red[0];
    __syncthreads();
    return r;
}

// Block-wide argmin over (value, index): smaller value, then smaller index.
template <int NT>
__device__ __forceinline__ void block_argmin(float v, int idx, float *redv, int *redi, float &bv, int &bi) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float ov = __shfl_xor_sync(0xffffffffu, v, o);
        const int oi = __shfl_xor_sync(0xffffffffu, idx, o);
        if (ov < v || (ov == v && oi < idx)) {
            v = ov;
            idx = oi;
        }
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) {
        redv[warp] = v;
        redi[warp] = idx;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        float b = redv[0];
        int bix = redi[0];
        for (int w = 1; w < NT / 32; ++w)
            if (redv[w] < b || (redv[w] == b && redi[w] < bix)) {
                b = redv[w];
                bix = redi[w];
            }
        redv[0] = b;
        redi[0] = bix;
    }
    __syncthreads();
    bv = redv[0];
    bi = redi[0];
    __syncthreads();
}

// ------------------------------------------------------------- sub-pixel --
// Least-squares quadratic a + b x + c y + d x^2 + e xy + g y^2 on the 3 x 3
// grid {-1,0,1}^2 (Sec. V-B), in closed form: b = sum x f / 6,
// c = sum y f / 6, e = sum xy f / 4, d = sum x^2 f / 2 - sum f / 3,
// g = sum y^2 f / 2 - sum f / 3.  Stationary point if the Hessian is positive
// definite and the point stays in [-1, 1]^2; otherwise 1-D parabolas clamped
// to [-0.5, 0.5].
__device__ __forceinline__ void subpixel_fit(const double *f, double &ox, double &oy) {
    double s0 = 0, sxf = 0, syf = 0, sxyf = 0, sxxf = 0, syyf = 0;
    for (int j = 0; j < 3; ++j)
        for (int i = 0; i < 3; ++i) {
            const double x = i - 1, y = j - 1, v = f[j * 3 + i];
            s0 += v;
            sxf += x * v;
            syf += y * v;
            sxyf += x * y * v;
            sxxf += x * x * v;
            syyf += y * y * v;
        }
    const double b = sxf / 6.0, c = syf / 6.0, e = sxyf / 4.0;
    const double d = sxxf / 2.0 - s0 / 3.0, g = syyf / 2.0 - s0 / 3.0;
    const double h11 = 2.0 * d, h22 = 2.0 * g, h12 = e;
    const double det = h11 * h22 - h12 * h12;
    if (h11 > 0.0 && det > 0.0) {
        const double px = -(h22 * b - h12 * c) / det;
        const double py = -(h11 * c - h12 * b) / det;
        if (fabs(px) <= 1.0 && fabs(py) <= 1.0) {
            ox = px;
            oy = py;
            return;
        }
    }
    const double denx = f[3] - 2.0 * f[4] + f[5], deny = f[1] - 2.0 * f[4] + f[7];
    double qx = denx > 0.0 ? (f[3] - f[5]) / (2.0 * denx) : 0.0;
    double qy = deny > 0.0 ? (f[1] - f[7]) / (2.0 * deny) : 0.0;
    ox = fmin(0.5, fmax(-0.5, qx));
    oy = fmin(0.5, fmax(-0.5, qy));
}


// Error-free transformation (TwoSum): s + e equals a + b exactly.
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
    s = a + b;
    const float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}

// Block-wide sum of per-thread FP32 partial sums carried as (hi, lo) pairs
// through a fixed tree of TwoSum steps (deterministic, close to exactly
// rounded without FP64).  `red` holds NT/32 float2.
template <int NT>
__device__ __forceinline__ float block_sum_comp(float v, float2 *red) {
    float hi = v, lo = 0.f;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float oh = __shfl_xor_sync(0xffffffffu, hi, o);
        const float ol = __shfl_xor_sync(0xffffffffu, lo, o);
        float sum, err;
        two_sum(hi, oh, sum, err);
        hi = sum;
        lo = (lo + ol) + err;
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) red[warp] = make_float2(hi, lo);
    __syncthreads();
    if (threadIdx.x == 0) {
        float h = red[0].x, l = red[0].y;
        for (int w = 1; w < NT / 32; ++w) {
            float sum, err;
            two_sum(h, red[w].x, sum, err);
            h = sum;
            l = (l + red[w].y) + err;
        }
        red[0] = make_float2(h + l, 0.f);
    }
    __syncthreads();
    const float r = red[0].x;
    __syncthreads();
    return r;
}

// Block-wide compensated sums of K per-thread values at once (the first n are
// used): the same fixed TwoSum tree as block_sum_comp for each value, with one
// exchange through shared memory.  out[c] (shared) receives sum c.
template <int NT, int K>
__device__ __forceinline__ void block_sum_comp_n(const float *v, int n, float2 (*red)[NT / 32],
                                                 float *out) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int c = 0; c < K; ++c) {
        if (c >= n) break;
        float hi = v[c], lo = 0.f;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const float oh = __shfl_xor_sync(0xffffffffu, hi, o);
            const float ol = __shfl_xor_sync(0xffffffffu, lo, o);
            float sum, err;
            two_sum(hi, oh, sum, err);
            hi = sum;
            lo = (lo + ol) + err;
        }
        if (lane == 0) red[c][warp] = make_float2(hi, lo);
    }
    __syncthreads();
    if (threadIdx.x < n) {
        const int c = threadIdx.x;
        float h = red[c][0].x, l = red[c][0].y;
        for (int w = 1; w < NT / 32; ++w) {
            float sum, err;
            two_sum(h, red[c][w].x, sum, err);
            h = sum;
            l = (l + red[c][w].y) + err;
        }
        out[c] = h + l;
    }
}

// Launch the BF16 direct-correlation matcher (cfog_bf16.cu): one CTA per CP
// when `order` is null, otherwise persistent CTAs draining the queue.
cfog_status launch_bf16_direct(const MatchArgs &a, int *counter, const int *order, cudaStream_t s);

}  // namespace cfog
