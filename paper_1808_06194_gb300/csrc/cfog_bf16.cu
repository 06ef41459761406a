// K5: BF16 direct correlation on the tcgen05 tensor cores (Eq. 3 in its
// direct form), FP32 accumulation in tensor memory, then FP32 re-scoring.
//
// For one CP with template T (N x N x m) and window S ((N+2r)^2 x m, origin
// at shift -r) the correlation C(dx, dy) = sum_{y,k,x'} T_k(y,x') S_k(y+dy, x'+dx)
// is one GEMM  D[dx][dy] = sum_K A[dx][K] B[K][dy]  with K = (k, y'', x'):
//   A[dx][(k,y'',x')] = S_k(y'', x' + dx)           (im2col of window row y'')
//   B[(k,y'',x')][dy] = T_k(y'' - dy, x')           (Toeplitz: zero outside 0..N-1)
// M = 128 rows (dx; 2r+1 used), N_g = 2r+1 rounded up to 16 columns (dy),
// K = m * (N+2r) * N_x (N_x = N rounded up to 16).  Both operands are K-major,
// no swizzle, and neither is materialised as a matrix:
//   * A: each window row is stored as 8 shifted copies, chunk (c, b) = the 8
//     values at columns 8c + b .. 8c + b + 7, at byte (c*8 + b)*16.  The 8 rows
//     dx = 8a..8a+7 of K-chunk c' are then chunks (b, c'+a), b = 0..7: one
//     contiguous 128-byte core matrix, so both descriptor strides are 128 B.
//   * B: the template of channel k is stored flipped, row j holding template
//     row W-1-j (zero outside the template), chunk-major: K-chunk c' of row j
//     at byte (c' * JB + j) * 16.  The B tile of window row y'' starts at row
//     j = W-1-y'': consecutive dy are consecutive rows, 16 B apart.
// One thread issues the MMAs of a staged group of window rows and commits them
// to an mbarrier; every wait is bounded.  The epilogue reads D from tensor
// memory, forms S(v) = sum T^2 + box(||D_sen||^2) - 2 C(v) in FP32, takes the
// 8 smallest, re-scores them and the 3 x 3 neighbourhood of the winner by
// direct FP32 SSD (compensated reduction), and fits the sub-pixel offset.
#include "cfog_match_common.cuh"
#include "cfog_tc.cuh"

#include <cuda_bf16.h>

#include <cstdint>

namespace cfog {
namespace {

constexpr int BT = 128;        // threads per CTA (4 warps, one per TMEM lane quadrant)
constexpr int BG = 8;          // window rows staged per MMA group
constexpr int BM = 128;        // MMA M
constexpr int kTmemCols = 128; // >= N_g for r <= 32
constexpr int kTop = 8;
constexpr long long kWaitCycles = 2000000000ll;   // ~1 s at 2 GHz

struct Geom {
    int N, r, L, W, Nx, Ng, CA, JB;
    int a_bytes, b_bytes;
};

__host__ __device__ inline Geom make_geom(int N, int r) {
    Geom g;
    g.N = N;
    g.r = r;
    g.L = 2 * r + 1;
    g.W = N + 2 * r;
    g.Nx = (N + 15) / 16 * 16;
    g.Ng = (g.L + 15) / 16 * 16;
    g.CA = (g.Nx + BM) / 8;
    g.JB = g.W + g.Ng - 1;
    g.a_bytes = BG * g.CA * 128;
    g.b_bytes = (g.Nx / 8) * g.JB * 16;
    return g;
}

// dynamic shared memory: [B operand][A operand] reused as box-sum rows,
// then the L x L surface
__host__ __device__ inline int geom_smem(const Geom &g) {
    int ops = g.b_bytes + g.a_bytes;
    const int rows = g.W * g.L * 4;
    if (rows > ops) ops = rows;
    ops = (ops + 127) / 128 * 128;
    return ops + g.L * g.L * 4;
}

// Wait for the mbarrier phase with a cycle limit; false if it ran out.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *mbar, uint32_t parity) {
    const long long t0 = clock64();
    while (!mbar_try_wait(mbar, parity)) {
        if (clock64() - t0 > kWaitCycles) return false;
    }
    return true;
}

__device__ __forceinline__ uint32_t pack_bf16x2(float lo, float hi) {
    const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<const uint32_t *>(&v);
}

struct Bf16Shared {
    uint64_t mbar;
    uint32_t tmem;
    int error;
    uint32_t phase;
    int next;
    float red_f[BT / 32];
    int red_i[BT / 32];
    float2 red_c[BT / 32];
    int ncand;
    int cand_idx[kTop + 9];
    float cand_ssd[kTop + 9];
};

// Direct FP32 SSD of lag index li (compensated block reduction).
__device__ float direct_ssd(const JobView &J, int m, int N, int r, int ry0, int rx0, int sy0,
                            int sx0, int li, Bf16Shared &sh) {
    const int Lside = 2 * r + 1;
    const int vy = li / Lside - r, vx = li % Lside - r;
    const int NN = N * N;
    float acc = 0.f;
    for (int e = threadIdx.x; e < m * NN; e += BT) {
        const int k = e / NN, rem = e - k * NN;
        const int y = rem / N, x = rem - y * N;
        const float a = __ldg(J.ref + (int64_t)k * J.ref_pp + (int64_t)(ry0 + y) * J.ref_rp + (rx0 + x));
        const float b = __ldg(J.sen + (int64_t)k * J.sen_pp + (int64_t)(sy0 + r + vy + y) * J.sen_rp +
                              (sx0 + r + vx + x));
        const float d = a - b;
        acc = fmaf(d, d, acc);
    }
    return block_sum_comp<BT>(acc, sh.red_c);
}

// Match one CP with the whole CTA (tensor memory already allocated).
__device__ void match_one_bf16(const MatchArgs &A, const int cp, Bf16Shared &sh,
                               unsigned char *smem) {
    const int tid = threadIdx.x;
    const JobView J = job_view(A, cp);
    const int N = A.tmpl[cp], r = A.radius[cp];
    const int px = A.cps[cp].x, py = A.cps[cp].y;
    const int qx = A.prior ? A.prior[cp].x : 0, qy = A.prior ? A.prior[cp].y : 0;
    const int m = A.m;

    cfog_match_result res;
    res.dx = qx;
    res.dy = qy;
    res.sub_dx = (float)qx;
    res.sub_dy = (float)qy;
    res.ssd = INFINITY;
    res.status = CFOG_CP_OOB;
    const int t0 = N / 2;
    const int ry0 = py - t0, rx0 = px - t0;
    const int sy0 = py + qy - t0 - r, sx0 = px + qx - t0 - r;
    const bool inside = J.ok && N >= 1 && r >= 0 && N <= A.tmpl_max && r <= A.radius_max &&
                        ry0 >= 0 && rx0 >= 0 && ry0 + N <= J.ref_h && rx0 + N <= J.ref_w &&
                        sy0 >= 0 && sx0 >= 0 && sy0 + N + 2 * r <= J.sen_h &&
                        sx0 + N + 2 * r <= J.sen_w;
    if (!inside || sh.error) {
        if (sh.error) res.status = CFOG_CP_TIMEOUT;
        if (tid == 0) A.out[cp] = res;
        return;
    }
    const Geom g = make_geom(N, r);
    unsigned char *bbuf = smem;
    unsigned char *abuf = smem + g.b_bytes;
    const int ops = (max(g.b_bytes + g.a_bytes, g.W * g.L * 4) + 127) / 128 * 128;
    float *surf = reinterpret_cast<float *>(smem + ops);
    float *rows = reinterpret_cast<float *>(smem);   // box-sum rows, after the MMAs
    const uint32_t bbase = smem_u32(bbuf), abase = smem_u32(abuf);
    const uint32_t idesc = mma_idesc(BM, g.Ng);
    const int kchunks = g.Nx / 8;

    bool first = true;
    for (int k = 0; k < m && !sh.error; ++k) {
        const float *tk = J.ref + (int64_t)k * J.ref_pp;
        const float *sk = J.sen + (int64_t)k * J.sen_pp;
        // B: flipped, zero-padded template of channel k
        for (int e = tid; e < kchunks * g.JB; e += BT) {
            const int c = e / g.JB, j = e - c * g.JB;
            const int y = g.W - 1 - j;
            float v[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int x = 8 * c + u;
                v[u] = (y >= 0 && y < N && x < N) ? __ldg(tk + (int64_t)(ry0 + y) * J.ref_rp + (rx0 + x)) : 0.f;
            }
            uint4 w;
            w.x = pack_bf16x2(v[0], v[1]);
            w.y = pack_bf16x2(v[2], v[3]);
            w.z = pack_bf16x2(v[4], v[5]);
            w.w = pack_bf16x2(v[6], v[7]);
            *reinterpret_cast<uint4 *>(bbuf + (size_t)(c * g.JB + j) * 16) = w;
        }
        for (int g0 = 0; g0 < g.W && !sh.error; g0 += BG) {
            const int G = min(BG, g.W - g0);
            // A: 8 shifted copies of each window row of the group
            for (int e = tid; e < G * g.CA * 8; e += BT) {
                const int row = e / (g.CA * 8), rem = e - row * (g.CA * 8);
                const int c = rem >> 3, b = rem & 7;
                const float *srow = sk + (int64_t)(sy0 + g0 + row) * J.sen_rp + sx0;
                float v[8];
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    const int x = 8 * c + b + u;
                    v[u] = x < g.W ? __ldg(srow + x) : 0.f;
                }
                uint4 w;
                w.x = pack_bf16x2(v[0], v[1]);
                w.y = pack_bf16x2(v[2], v[3]);
                w.z = pack_bf16x2(v[4], v[5]);
                w.w = pack_bf16x2(v[6], v[7]);
                *reinterpret_cast<uint4 *>(abuf + (size_t)(row * g.CA + c) * 128 + b * 16) = w;
            }
            fence_proxy_async();
            __syncthreads();
            if (tid == 0) {
                tc_fence_after();
                for (int row = 0; row < G; ++row) {
                    const int yy = g0 + row;
                    for (int i = 0; i < g.Nx / 16; ++i) {
                        const uint64_t ad = smem_desc(abase + (uint32_t)((row * g.CA + 2 * i) * 128), 128, 128);
                        const uint64_t bd = smem_desc(bbase + (uint32_t)((2 * i * g.JB + (g.W - 1 - yy)) * 16),
                                                      (uint32_t)(g.JB * 16), 128);
                        mma_bf16(sh.tmem, ad, bd, idesc, first ? 0u : 1u);
                        first = false;
                    }
                }
                mma_commit(&sh.mbar);
            }
            // every thread waits for the group's MMAs before the buffers are reused;
            // after a time-out, one more bounded wait lets MMAs still in flight end
            bool ok = mbar_wait_bounded(&sh.mbar, sh.phase);
            if (!ok) {
                mbar_wait_bounded(&sh.mbar, sh.phase);
                sh.error = 1;
            }
            tc_fence_after();
            __syncthreads();
            if (tid == 0) sh.phase ^= 1u;
            __syncthreads();
        }
    }
    if (sh.error) {
        if (tid == 0) {
            res.status = CFOG_CP_TIMEOUT;
            A.out[cp] = res;
        }
        return;
    }
    // epilogue: C(dx, dy) = D[dx][dy] from tensor memory into the surface buffer
    const int L = g.L;
    {
        const int warp = tid >> 5, lane = tid & 31;
        const int dx = warp * 32 + lane;
        for (int c0 = 0; c0 < g.Ng; c0 += 16) {
            float v[16];
            tmem_ld16(sh.tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
            if (dx < L) {
#pragma unroll
                for (int u = 0; u < 16; ++u)
                    if (c0 + u < L) surf[(c0 + u) * L + dx] = v[u];   // [dy][dx]
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    // sum T^2 and the box sums B(v) of ||D_sen||^2, FP32
    float tt_part = 0.f;
    for (int e = tid; e < m * N * N; e += BT) {
        const int k = e / (N * N), rem = e - k * N * N;
        const int y = rem / N, x = rem - y * N;
        const float a = __ldg(J.ref + (int64_t)k * J.ref_pp + (int64_t)(ry0 + y) * J.ref_rp + (rx0 + x));
        tt_part = fmaf(a, a, tt_part);
    }
    const float tt = block_sum_comp<BT>(tt_part, sh.red_c);
    for (int e = tid; e < g.W * L; e += BT) {
        const int yy = e / L, vx = e - yy * L;
        const float *q = J.sen_sq + (int64_t)(sy0 + yy) * J.sen_rp + sx0 + vx;
        float acc = 0.f;
        for (int x = 0; x < N; ++x) acc += __ldg(q + x);
        rows[e] = acc;
    }
    __syncthreads();
    for (int e = tid; e < L * L; e += BT) {
        const int vy = e / L, vx = e - vy * L;
        float box = 0.f;
        for (int y = 0; y < N; ++y) box += rows[(vy + y) * L + vx];
        surf[e] = tt + box - 2.0f * surf[e];   // surf[e] held C at [dy = vy][dx = vx]
    }
    __syncthreads();
    if (A.surface) {
        const int Lmax = A.surf_side;
        float *dst = A.surface + (int64_t)cp * Lmax * Lmax;
        const int off = (Lmax - L) / 2;
        for (int e = tid; e < L * L; e += BT) {
            const int vy = e / L, vx = e - vy * L;
            dst[(vy + off) * Lmax + (vx + off)] = surf[e];
        }
    }
    // the kTop smallest BF16 scores, re-scored directly in FP32
    if (tid == 0) sh.ncand = 0;
    for (int t = 0; t < kTop && t < L * L; ++t) {
        float bv = INFINITY;
        int bi = INT_MAX;
        for (int e = tid; e < L * L; e += BT) {
            bool taken = false;
            for (int c = 0; c < t; ++c) taken |= sh.cand_idx[c] == e;
            const float v = surf[e];
            if (!taken && (v < bv || (v == bv && e < bi))) {
                bv = v;
                bi = e;
            }
        }
        float smin;
        int imin;
        block_argmin<BT>(bv, bi, sh.red_f, sh.red_i, smin, imin);
        if (tid == 0) {
            sh.cand_idx[t] = imin;
            sh.ncand = t + 1;
        }
        __syncthreads();
    }
    const int ncand = sh.ncand;
    for (int c = 0; c < ncand; ++c) {
        const float s = direct_ssd(J, m, N, r, ry0, rx0, sy0, sx0, sh.cand_idx[c], sh);
        if (tid == 0) sh.cand_ssd[c] = s;
    }
    __syncthreads();
    int win = sh.cand_idx[0];
    float win_ssd = sh.cand_ssd[0];
    for (int c = 1; c < ncand; ++c)
        if (sh.cand_ssd[c] < win_ssd || (sh.cand_ssd[c] == win_ssd && sh.cand_idx[c] < win)) {
            win = sh.cand_idx[c];
            win_ssd = sh.cand_ssd[c];
        }
    const int vy = win / L - r, vx = win % L - r;
    const bool edge = vx == -r || vx == r || vy == -r || vy == r;
    float nb[9];
    if (!edge) {
        for (int j = -1; j <= 1; ++j)
            for (int i = -1; i <= 1; ++i) {
                const int li = (vy + r + j) * L + (vx + r + i);
                float s = INFINITY;
                for (int c = 0; c < ncand; ++c)
                    if (sh.cand_idx[c] == li) s = sh.cand_ssd[c];
                if (s == INFINITY) s = direct_ssd(J, m, N, r, ry0, rx0, sy0, sx0, li, sh);
                nb[(j + 1) * 3 + (i + 1)] = s;
            }
    }
    if (tid == 0) {
        res.dx = qx + vx;
        res.dy = qy + vy;
        res.ssd = win_ssd;
        double ox = 0.0, oy = 0.0;
        if (edge) {
            res.status = CFOG_CP_EDGE_PEAK;
        } else {
            double f[9];
            for (int i = 0; i < 9; ++i) f[i] = (double)nb[i];
            subpixel_fit(f, ox, oy);
            res.status = CFOG_CP_OK;
        }
        res.sub_dx = (float)((double)res.dx + ox);
        res.sub_dy = (float)((double)res.dy + oy);
        A.out[cp] = res;
    }
    __syncthreads();
}

// One CTA per CP (order == nullptr) or persistent CTAs over a queue.
__global__ void __launch_bounds__(BT) match_bf16_kernel(const MatchArgs A, int *counter,
                                                         const int *order) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ Bf16Shared sh;
    const int tid = threadIdx.x;
    if (tid < 32) {
        tmem_alloc(&sh.tmem, kTmemCols);
        tmem_relinquish();
    }
    if (tid == 0) {
        mbar_init(&sh.mbar, 1);
        fence_mbar_init();
        sh.error = 0;
        sh.phase = 0;
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (!order) {
        if (blockIdx.x < A.n) match_one_bf16(A, blockIdx.x, sh, smem_raw);
    } else {
        for (;;) {
            if (tid == 0) sh.next = atomicAdd(counter, 1);
            __syncthreads();
            const int i = sh.next;
            __syncthreads();
            if (i >= A.n) break;
            match_one_bf16(A, order[i], sh, smem_raw);
            __syncthreads();
        }
    }
    tc_fence_before();
    __syncthreads();
    if (tid < 32) tmem_dealloc(sh.tmem, kTmemCols);
}

}  // namespace

cfog_status launch_bf16_direct(const MatchArgs &a, int *counter, const int *order, cudaStream_t s) {
    if (a.tmpl_max > 128) {
        set_error("cfog_match: BF16 direct precision supports templates up to 128 (tmpl_max %d)",
                  a.tmpl_max);
        return CFOG_E_UNSUPPORTED;
    }
    // shared memory for the largest (N, r) the launch allows
    int smem = 0;
    for (int N = 1; N <= a.tmpl_max; ++N) {
        const Geom g = make_geom(N, a.radius_max);
        const int b = geom_smem(g);
        smem = b > smem ? b : smem;
    }
    // at least 60 KB per CTA keeps at most 3 CTAs (3 x 128 TMEM columns) on an SM
    smem = smem < 60 * 1024 ? 60 * 1024 : smem;
    if (smem > 200 * 1024) {
        set_error("cfog_match: BF16 direct plan needs %d bytes of shared memory", smem);
        return CFOG_E_UNSUPPORTED;
    }
    cfog_status st = ensure_dynamic_smem(reinterpret_cast<const void *>(match_bf16_kernel), smem,
                                         "cfog_match (bf16)");
    if (st != CFOG_OK) return st;
    int grid = a.n;
    if (order) {
        int per_sm = 0;
        st = check_cuda(cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                            &per_sm, reinterpret_cast<const void *>(match_bf16_kernel), BT, smem),
                        "cfog_match (bf16): occupancy");
        if (st != CFOG_OK) return st;
        per_sm = per_sm < 1 ? 1 : (per_sm > 512 / kTmemCols ? 512 / kTmemCols : per_sm);
        const long long cap = (long long)sm_count() * per_sm;
        grid = (int)(a.n < cap ? a.n : cap);
    }
    match_bf16_kernel<<<grid, BT, smem, s>>>(a, counter, order);
    return check_launch("cfog_match (bf16): launch");
}

}  // namespace cfog
