// K9: iterative outlier rejection with a polynomial mapping model (Sec. IV,
// outlier rejection): fit the model to the kept CPs by least squares, compute
// the residuals and the RMSE, drop the CP with the largest residual, repeat
// until the RMSE is below the threshold.
//
// One CTA of 256 threads per job.  The FP64 normal equations are reduced once
// (warp-cooperative: each lane owns up to three of the 75 sums, the CPs'
// monomial vectors are staged per warp in shared memory); after that a removal
// subtracts the dropped CP's terms.  Warp 0 solves by Cholesky in FP64.  The
// residuals of the first fit are evaluated once in FP64 and stored as FP32,
// with the CP's FP32 (u, v), in shared memory when the largest job fits
// (11520 CPs), else in the workspace;
// each later round evaluates only the change of the model, sum_t (c_t - c0_t)
// phi_t, in FP32, whose magnitude is that of the outliers' pull, so the
// residuals keep an absolute error of order 1e-5 px.  Reductions use a fixed
// per-thread assignment and a fixed tree, so results are deterministic.
#include "cfog_internal.cuh"

#include <algorithm>
#include <climits>
#include <cmath>
#include <cstdint>

namespace cfog {
namespace {

constexpr int RT = 256;
constexpr int RW = RT / 32;
constexpr int kMaxT = 10;                                    // cubic: 10 monomials
constexpr int kMaxS = kMaxT * (kMaxT + 1) / 2 + 2 * kMaxT;   // 55 + 20 sums
constexpr int kPsi = kMaxT + 2;                              // phi_0..phi_{T-1}, x', y'
constexpr size_t kCacheMax = 180 * 1024;   // per-CP state in shared memory up to 11520 CPs per job

template <int DEG>
struct PolyDim {
    static constexpr int T = (DEG + 1) * (DEG + 2) / 2;
    static constexpr int TM = T * (T + 1) / 2;   // upper triangle of the normal matrix
    static constexpr int S = TM + 2 * T;         // + the two right-hand sides
};

// Monomials of total degree <= DEG in the order 1, u, v, u^2, uv, v^2, u^3,
// u^2 v, u v^2, v^3; each product is formed left to right (u^2 v = (u u) v,
// u v^2 = (u v) v).
template <int DEG, typename F>
__device__ __forceinline__ void basis(F u, F v, F *phi) {
    phi[0] = F(1);
    if constexpr (DEG >= 1) {
        phi[1] = u;
        phi[2] = v;
    }
    if constexpr (DEG >= 2) {
        phi[3] = u * u;
        phi[4] = u * v;
        phi[5] = v * v;
    }
    if constexpr (DEG >= 3) {
        phi[6] = phi[3] * u;
        phi[7] = phi[3] * v;
        phi[8] = phi[4] * v;
        phi[9] = phi[5] * v;
    }
}

// Sum s of the normal equations is sum_i psi_a psi_b over the kept CPs, with
// psi = (phi_0..phi_{T-1}, x', y').
__device__ __forceinline__ void sum_pair(int s, int T, int &a, int &b) {
    const int TM = T * (T + 1) / 2;
    if (s < TM) {
        int idx = s;
        a = 0;
        while (idx >= T - a) {
            idx -= T - a;
            ++a;
        }
        b = a + idx;
    } else if (s < TM + T) {
        a = s - TM;
        b = T;
    } else {
        a = s - TM - T;
        b = T + 1;
    }
}

struct RejectShared {
    double psi[RW][32][kPsi + 1];   // staged monomial vectors, one row per lane
    double part[RW][kMaxS];         // per-warp partial sums
    double S[kMaxS];                // normal equations (packed) and right-hand sides
    double A[kMaxT][kMaxT + 1];     // Cholesky factor (lower triangle)
    double dinv[kMaxT];             // 1 / L_kk
    double coef[2 * kMaxT];         // current model
    double c0[2 * kMaxT];           // first fit
    double cnew[2 * kMaxT];         // candidate after a removal
    double psi_rm[kPsi];            // monomial vector of the CP being dropped
    double red_d[RW];
    float dcf[2 * kMaxT];           // coef - c0 in FP32
    float red_e[RW];
    int red_i[RW];
    unsigned char pa[kMaxS], pb[kMaxS];
    int xmin, xmax, ymin, ymax, n_valid;
    int kept, n_removed, n_fits, status, done, solve_ok, worst;
    double rmse;
};

// Psi vector of CP i in FP64 (the CP must be valid).
template <int DEG>
__device__ __forceinline__ void cp_psi(const cfog_point *cps, const cfog_match_result *res, int i,
                                       double cx, double cy, double sc, double *ps) {
    constexpr int T = PolyDim<DEG>::T;
    const double x = (double)cps[i].x, y = (double)cps[i].y;
    const double u = (x - cx) / sc, v = (y - cy) / sc;
    basis<DEG>(u, v, ps);
    ps[T] = x + (double)res[i].sub_dx;
    ps[T + 1] = y + (double)res[i].sub_dy;
}

// Warp 0: Cholesky of the T x T normal matrix held packed in sh.S, then the
// two triangular solves into out[0..T) (x') and out[kMaxT..kMaxT+T) (y').
// Sets sh.solve_ok.  Singular when a pivot is not above 1e-12 of the largest
// diagonal entry.  Each pivot costs one reciprocal square root; the solves
// multiply by the stored reciprocals.
template <int T>
__device__ void solve_warp(RejectShared &sh, double *out) {
    const int lane = threadIdx.x & 31;
    for (int e = lane; e < T * T; e += 32) {
        const int i = e / T, j = e - (e / T) * T;
        const int a = i < j ? i : j, b = i < j ? j : i;
        sh.A[i][j] = sh.S[a * T - a * (a - 1) / 2 + (b - a)];
    }
    __syncwarp();
    double dmax = 0.0;
    for (int i = 0; i < T; ++i) dmax = fmax(dmax, sh.A[i][i]);
    const double tol = 1e-12 * dmax;
    bool ok = dmax > 0.0;
    for (int k = 0; k < T && ok; ++k) {
        const double d = sh.A[k][k];
        ok = d > tol && isfinite(d);
        if (!ok) break;
        const double inv = rsqrt(d);   // 1 / L_kk
        __syncwarp();
        if (lane > k && lane < T) sh.A[lane][k] *= inv;
        if (lane == 0) {
            sh.A[k][k] = d * inv;
            sh.dinv[k] = inv;
        }
        __syncwarp();
        const int rem = T - k - 1;
        for (int e = lane; e < rem * rem; e += 32) {
            const int i = k + 1 + e / rem, j = k + 1 + (e - (e / rem) * rem);
            if (j <= i) sh.A[i][j] -= sh.A[i][k] * sh.A[j][k];
        }
        __syncwarp();
    }
    if (ok && lane < 2) {
        const int base = T * (T + 1) / 2 + lane * T;
        double z[T];
#pragma unroll
        for (int i = 0; i < T; ++i) {
            double acc = sh.S[base + i];
#pragma unroll
            for (int k = 0; k < i; ++k) acc -= sh.A[i][k] * z[k];
            z[i] = acc * sh.dinv[i];
        }
#pragma unroll
        for (int i = T - 1; i >= 0; --i) {
            double acc = z[i];
#pragma unroll
            for (int k = i + 1; k < T; ++k) acc -= sh.A[k][i] * z[k];
            z[i] = acc * sh.dinv[i];
        }
#pragma unroll
        for (int i = 0; i < T; ++i) out[lane * kMaxT + i] = z[i];
    }
    if (lane == 0) sh.solve_ok = ok ? 1 : 0;
    __syncwarp();
}

template <int DEG>
__global__ void __launch_bounds__(RT) reject_kernel(const cfog_point *__restrict__ cps,
                                                    const cfog_match_result *__restrict__ res,
                                                    const int32_t *__restrict__ job_start, double thr,
                                                    int min_keep, uint8_t *keep,
                                                    int32_t *__restrict__ order,
                                                    cfog_poly_model *__restrict__ models,
                                                    float4 *__restrict__ work, int cached) {
    constexpr int T = PolyDim<DEG>::T;
    constexpr int S = PolyDim<DEG>::S;
    __shared__ RejectShared sh;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int b0 = job_start[blockIdx.x], e0 = job_start[blockIdx.x + 1];
    const int nj = e0 - b0;
    // per-CP state (u, v, first-fit residual), x = NaN for a CP not kept: in
    // shared memory when the launch reserved room for the largest job
    extern __shared__ float4 wcache[];
    float4 *wb = cached ? wcache : work + b0;

    if (tid == 0) {
        sh.xmin = sh.ymin = INT_MAX;
        sh.xmax = sh.ymax = INT_MIN;
        sh.n_valid = 0;
    }
    if (tid < S) {
        int a, b;
        sum_pair(tid, T, a, b);
        sh.pa[tid] = (unsigned char)a;
        sh.pb[tid] = (unsigned char)b;
    }
    __syncthreads();

    // bounding box of the valid CPs; keep = valid
    {
        int xmn = INT_MAX, xmx = INT_MIN, ymn = INT_MAX, ymx = INT_MIN, cnt = 0;
        for (int i = b0 + tid; i < e0; i += RT) {
            const bool ok = res[i].status == CFOG_CP_OK;
            keep[i] = ok ? 1 : 0;
            if (!ok) continue;
            const cfog_point p = cps[i];
            xmn = min(xmn, p.x);
            xmx = max(xmx, p.x);
            ymn = min(ymn, p.y);
            ymx = max(ymx, p.y);
            ++cnt;
        }
        atomicMin(&sh.xmin, xmn);
        atomicMax(&sh.xmax, xmx);
        atomicMin(&sh.ymin, ymn);
        atomicMax(&sh.ymax, ymx);
        atomicAdd(&sh.n_valid, cnt);
    }
    __syncthreads();
    const int n_valid = sh.n_valid;
    double cx = 0.0, cy = 0.0, sc = 1.0;
    if (n_valid > 0) {
        cx = 0.5 * ((double)sh.xmin + (double)sh.xmax);
        cy = 0.5 * ((double)sh.ymin + (double)sh.ymax);
        sc = fmax(0.5 * ((double)sh.xmax - (double)sh.xmin), 0.5 * ((double)sh.ymax - (double)sh.ymin));
        if (!(sc > 0.0)) sc = 1.0;
    }

    // normal equations over the valid CPs, warp-cooperative
    {
        double acc[3] = {0.0, 0.0, 0.0};
        for (int base = b0 + warp * 32; base < e0; base += RT) {
            const int i = base + lane;
            double ps[kPsi];
#pragma unroll
            for (int q = 0; q < kPsi; ++q) ps[q] = 0.0;
            if (i < e0 && res[i].status == CFOG_CP_OK) cp_psi<DEG>(cps, res, i, cx, cy, sc, ps);
#pragma unroll
            for (int q = 0; q < T + 2; ++q) sh.psi[warp][lane][q] = ps[q];
            __syncwarp();
            for (int c = 0; c < 32; ++c) {
#pragma unroll
                for (int q = 0; q < 3; ++q) {
                    const int s = lane + 32 * q;
                    if (s < S) acc[q] = fma(sh.psi[warp][c][sh.pa[s]], sh.psi[warp][c][sh.pb[s]], acc[q]);
                }
            }
            __syncwarp();
        }
#pragma unroll
        for (int q = 0; q < 3; ++q)
            if (lane + 32 * q < S) sh.part[warp][lane + 32 * q] = acc[q];
    }
    __syncthreads();
    if (tid < S) {
        double v = 0.0;
        for (int w = 0; w < RW; ++w) v += sh.part[w][tid];
        sh.S[tid] = v;
    }
    if (tid < 2 * kMaxT) sh.coef[tid] = 0.0;
    if (tid == 0) {
        sh.kept = n_valid;
        sh.n_removed = 0;
        sh.n_fits = 1;
        sh.status = CFOG_REJECT_SINGULAR;
        sh.rmse = -1.0;
        sh.done = 0;
        sh.solve_ok = 0;
    }
    __syncthreads();
    if (n_valid > 0 && warp == 0) solve_warp<T>(sh, sh.c0);
    __syncthreads();
    const bool first_ok = n_valid > 0 && sh.solve_ok;
    if (first_ok) {
        if (tid < 2 * kMaxT) sh.coef[tid] = sh.c0[tid];
        // first-fit residuals in FP64, stored as FP32 with the FP32 (u, v)
        for (int i = b0 + tid; i < e0; i += RT) {
            if (res[i].status != CFOG_CP_OK) {
                wb[i - b0] = make_float4(__int_as_float(0x7fc00000), 0.f, 0.f, 0.f);
                continue;
            }
            double ps[kPsi];
            cp_psi<DEG>(cps, res, i, cx, cy, sc, ps);
            double px = 0.0, py = 0.0;
#pragma unroll
            for (int t = 0; t < T; ++t) {
                px = fma(sh.c0[t], ps[t], px);
                py = fma(sh.c0[kMaxT + t], ps[t], py);
            }
            wb[i - b0] = make_float4((float)ps[1], (float)ps[2],
                                     (float)(ps[T] - px), (float)(ps[T + 1] - py));
        }
    }
    __syncthreads();

    const int floor_n = max(min_keep, T);
    while (first_ok) {
        if (tid < 2 * kMaxT) sh.dcf[tid] = (float)(sh.coef[tid] - sh.c0[tid]);
        __syncthreads();
        // residual round: compensated FP32 sum of e^2, largest e^2 (lowest index on ties)
        float s_hi = 0.f, s_lo = 0.f, best = -1.f;
        int bi = INT_MAX;
#pragma unroll 4
        for (int k = tid; k < nj; k += RT) {
            const float4 w = wb[k];
            if (isnan(w.x)) continue;
            const int i = b0 + k;
            float ph[kMaxT];
            basis<DEG>(w.x, w.y, ph);
            float dx = 0.f, dy = 0.f;
#pragma unroll
            for (int t = 0; t < T; ++t) {
                dx = fmaf(sh.dcf[t], ph[t], dx);
                dy = fmaf(sh.dcf[kMaxT + t], ph[t], dy);
            }
            const float ex = w.z - dx, ey = w.w - dy;
            const float e2 = fmaf(ex, ex, ey * ey);
            const float t = s_hi + e2;
            const float bp = t - s_hi;
            s_lo += (s_hi - (t - bp)) + (e2 - bp);
            s_hi = t;
            if (e2 > best) {
                best = e2;
                bi = i;
            }
        }
        double ssum = (double)s_hi + (double)s_lo;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            ssum += __shfl_xor_sync(0xffffffffu, ssum, o);
            const float ob = __shfl_xor_sync(0xffffffffu, best, o);
            const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
            if (ob > best || (ob == best && oi < bi)) {
                best = ob;
                bi = oi;
            }
        }
        if (lane == 0) {
            sh.red_d[warp] = ssum;
            sh.red_e[warp] = best;
            sh.red_i[warp] = bi;
        }
        __syncthreads();
        if (tid == 0) {
            double tot = 0.0;
            float bb = -1.f;
            int ii = INT_MAX;
            for (int w = 0; w < RW; ++w) {
                tot += sh.red_d[w];
                if (sh.red_e[w] > bb || (sh.red_e[w] == bb && sh.red_i[w] < ii)) {
                    bb = sh.red_e[w];
                    ii = sh.red_i[w];
                }
            }
            sh.rmse = sqrt(tot / (double)sh.kept);
            if (ii == INT_MAX || !isfinite(sh.rmse)) {
                sh.status = CFOG_REJECT_SINGULAR;   // non-finite residuals: no ranking
                sh.done = 1;
            } else if (sh.rmse < thr) {
                sh.status = CFOG_REJECT_OK;
                sh.done = 1;
            } else if (sh.kept - 1 < floor_n) {
                sh.status = CFOG_REJECT_MIN_KEEP;
                sh.done = 1;
            } else {
                sh.worst = ii;
                cp_psi<DEG>(cps, res, ii, cx, cy, sc, sh.psi_rm);
            }
        }
        __syncthreads();
        if (sh.done) break;
        if (tid < S) sh.S[tid] -= sh.psi_rm[sh.pa[tid]] * sh.psi_rm[sh.pb[tid]];
        __syncthreads();
        if (warp == 0) solve_warp<T>(sh, sh.cnew);
        __syncthreads();
        const bool ok = sh.solve_ok;
        if (ok && tid < 2 * kMaxT) sh.coef[tid] = sh.cnew[tid];
        if (tid == 0) {
            ++sh.n_fits;
            if (ok) {
                keep[sh.worst] = 0;
                wb[sh.worst - b0].x = __int_as_float(0x7fc00000);
                if (order) order[b0 + sh.n_removed] = sh.worst;
                ++sh.n_removed;
                --sh.kept;
            } else {
                sh.status = CFOG_REJECT_SINGULAR;   // the removal is not made
                sh.done = 1;
            }
        }
        __syncthreads();
        if (sh.done) break;
    }
    __syncthreads();

    if (tid == 0) {
        cfog_poly_model md;
        md.status = sh.status;
        md.terms = T;
        md.n_valid = n_valid;
        md.n_kept = first_ok ? sh.kept : n_valid;
        md.n_removed = sh.n_removed;
        md.n_fits = sh.n_fits;
        md.rmse = first_ok ? sh.rmse : -1.0;
        md.cx = cx;
        md.cy = cy;
        md.scale = sc;
        for (int t = 0; t < kMaxT; ++t) {
            md.coef_x[t] = first_ok && t < T ? sh.coef[t] : 0.0;
            md.coef_y[t] = first_ok && t < T ? sh.coef[kMaxT + t] : 0.0;
        }
        models[blockIdx.x] = md;
    }
}

size_t offsets_bytes(int32_t n_jobs) { return ((size_t)(n_jobs + 1) * sizeof(int32_t) + 255) / 256 * 256; }

}  // namespace
}  // namespace cfog

extern "C" size_t cfog_reject_workspace_bytes(int32_t n_cps, int32_t n_jobs) {
    if (n_cps < 0 || n_jobs < 0) return 0;
    return cfog::offsets_bytes(n_jobs) + (size_t)n_cps * sizeof(float4);
}

extern "C" cfog_status cfog_reject_outliers(const cfog_point *cps_dev, const cfog_match_result *res_dev,
                                            const int32_t *job_start, int32_t n_jobs, int32_t degree,
                                            double rmse_threshold, int32_t min_keep, uint8_t *keep_dev,
                                            int32_t *order_dev, cfog_poly_model *models_dev,
                                            void *work_dev, size_t work_bytes, void *stream) {
    CFOG_TRACE("cfog_reject_outliers");
    using namespace cfog;
    CFOG_REQUIRE(n_jobs >= 0, "cfog_reject_outliers: n_jobs = %d < 0", n_jobs);
    if (n_jobs == 0) return CFOG_OK;
    CFOG_REQUIRE(job_start, "cfog_reject_outliers: job_start is null");
    CFOG_REQUIRE(degree >= 1 && degree <= 3, "cfog_reject_outliers: degree %d not in 1..3", degree);
    CFOG_REQUIRE(rmse_threshold >= 0.0, "cfog_reject_outliers: rmse_threshold must be >= 0");
    CFOG_REQUIRE(min_keep >= 0, "cfog_reject_outliers: min_keep = %d < 0", min_keep);
    CFOG_REQUIRE(job_start[0] >= 0, "cfog_reject_outliers: job_start[0] = %d < 0", job_start[0]);
    for (int32_t j = 0; j < n_jobs; ++j)
        CFOG_REQUIRE(job_start[j + 1] >= job_start[j],
                     "cfog_reject_outliers: job_start decreases at job %d", j);
    const int32_t n_cps = job_start[n_jobs];
    if (n_cps > 0) CFOG_REQUIRE(cps_dev && res_dev && keep_dev, "cfog_reject_outliers: null CP array");
    CFOG_REQUIRE(models_dev && work_dev, "cfog_reject_outliers: null models or workspace");
    const size_t need = cfog_reject_workspace_bytes(n_cps, n_jobs);
    if (work_bytes < need) {
        set_error("cfog_reject_outliers: workspace of %zu bytes, %zu needed", work_bytes, need);
        return CFOG_E_NOMEM;
    }
    CFOG_REQUIRE(reinterpret_cast<uintptr_t>(work_dev) % 256 == 0,
                 "cfog_reject_outliers: workspace not 256-byte aligned");
    cudaStream_t st = as_stream(stream);
    int32_t *off_dev = static_cast<int32_t *>(work_dev);
    float4 *w4 = reinterpret_cast<float4 *>(static_cast<unsigned char *>(work_dev) + offsets_bytes(n_jobs));
    int32_t max_job = 0;
    for (int32_t j = 0; j < n_jobs; ++j) max_job = std::max(max_job, job_start[j + 1] - job_start[j]);
    const size_t cache = (size_t)max_job * sizeof(float4);
    const int cached = cache <= kCacheMax ? 1 : 0;
    const int dyn = cached ? (int)cache : 0;
    const void *fn = degree == 1 ? (const void *)reject_kernel<1>
                   : degree == 2 ? (const void *)reject_kernel<2> : (const void *)reject_kernel<3>;
    cfog_status s = ensure_dynamic_smem(fn, dyn, "cfog_reject_outliers");
    if (s != CFOG_OK) return s;
    s = check_cuda(cudaMemcpyAsync(off_dev, job_start, (size_t)(n_jobs + 1) * sizeof(int32_t),
                                               cudaMemcpyHostToDevice, st),
                               "cfog_reject_outliers: copy of job_start");
    if (s != CFOG_OK) return s;
    switch (degree) {
        case 1:
            reject_kernel<1><<<n_jobs, RT, dyn, st>>>(cps_dev, res_dev, off_dev, rmse_threshold, min_keep,
                                                      keep_dev, order_dev, models_dev, w4, cached);
            break;
        case 2:
            reject_kernel<2><<<n_jobs, RT, dyn, st>>>(cps_dev, res_dev, off_dev, rmse_threshold, min_keep,
                                                      keep_dev, order_dev, models_dev, w4, cached);
            break;
        default:
            reject_kernel<3><<<n_jobs, RT, dyn, st>>>(cps_dev, res_dev, off_dev, rmse_threshold, min_keep,
                                                      keep_dev, order_dev, models_dev, w4, cached);
            break;
    }
    return check_launch("cfog_reject_outliers: launch");
}
