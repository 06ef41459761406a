// K5: BF16 direct correlation on the tcgen05 tensor cores (Eq. 3 in its
// direct form), FP32 accumulation in tensor memory, then FP32 re-scoring.
//
// For one CP with template T (N x N x m) and window S ((N+2r)^2 x m, origin
// at shift -r) the correlation C(dx, dy) = sum_{y,k,x'} T_k(y,x') S_k(y+dy, x'+dx)
// is a sum of GEMMs over the window rows.  Each MMA step takes J window rows
// y0 .. y0+J-1 (J = 2 when 2r+1 <= 64, else 1) stacked along M:
//   D[(dx, j)][c] += sum_{k, x'} A[(dx, j)][(k, x')] B[(k, x')][c]
//   A[(dx, j)][(k, x')] = S_k(y0 + j, x' + dx)      (im2col of window row y0+j)
//   B[(k, x')][c]       = T_k(y0 + J-1 - c, x')     (Toeplitz: zero outside 0..N-1)
// Row (dx, j) and column c pair window row y0+j with template row
// y0+J-1-c, i.e. the lag dy = c + j - (J-1), the same for every step, so
//   C(dx, dy) = sum_j D[(dx, j)][dy + J-1 - j].
// M = 128 rows: 64 dx for each of two window rows (J = 2), or 128 dx (J = 1);
// N_g = 2r+J rounded up to 16 columns; K = m * N_x per step (N_x = N rounded
// up to 16), and ceil((N+2r)/J) steps per channel.  Stacking two window rows
// halves the MMAs per CP at the same cost per instruction (a tcgen05.mma of
// up to 96 columns takes the same time at M = 64 and at M = 128).  Both
// operands are K-major, no swizzle, and neither is materialised as a matrix:
//   * A: each window row is stored as 8 shifted copies, chunk (c, b) = the 8
//     values at columns 8c + b .. 8c + b + 7.  The J rows of a step are
//     interleaved chunk by chunk: chunk (j, c, b) at byte ((c*J + j)*8 + b)*16.
//     The 8 rows dx = 8a..8a+7 of window row j and K-chunk c' are then chunks
//     (j, c'+a, b), b = 0..7: one contiguous 128-byte core matrix at
//     (c'+a)*J*128 + j*128, so with the rows of D ordered (a, j, b) the core
//     matrices along M are 128 B apart and those along K J*128 B apart.
//   * B: the template of channel k is stored flipped, row i holding template
//     row W+J-2-i (zero outside the template), chunk-major: K-chunk c' of row
//     i at byte (c' * JB + i) * 16.  The B tile of the step at window row y0
//     starts at row i = W-1-y0: consecutive columns are consecutive rows.
// Row (dx, j) of D sits in tensor-memory lane 8 (J (dx / 8) + j) + dx % 8.
// Each channel's template and window are read as coalesced 8-value chunks
// and converted to BF16 in registers; the rows of B outside the template are
// cleared once per CP.
// The CTA is warp-specialised: four builder warps stage each channel and
// build groups of window rows into a ring of three A slots (one full/empty
// mbarrier pair per slot), and a fifth warp issues each full slot's MMAs
// (descriptors advanced by integer adds, one elected lane) and commits them
// to the slot's empty barrier, so the next groups are built while the tensor
// core runs; every wait is bounded.  The epilogue reads D from tensor
// memory, forms S(v) = sum T^2 + box(||D_sen||^2) - 2 C(v) in FP32, takes the
// 8 smallest, re-scores them and the 3 x 3 neighbourhood of the smallest by
// direct FP32 SSD in one pass over the channels (the lags' window region and
// the template staged in shared memory by cp.async, compensated reductions),
// and fits the sub-pixel offset.
#include "cfog_match_common.cuh"
#include "cfog_tc.cuh"

#include <cuda_bf16.h>

#include <atomic>
#include <cstdint>

namespace cfog {
namespace {

constexpr int kBuilderWarps = 4;   // warps 0-3: staging, A build, epilogue (one per TMEM lane quadrant)
constexpr int kBuilders = 32 * kBuilderWarps;
constexpr int BT = kBuilders + 32; // threads per CTA: the builders and the MMA-issuing warp
constexpr int BG = 4;          // window rows per MMA group
constexpr int NBUF = 3;        // A slots in the ring
constexpr int kTmemCols = 256; // the accumulators: up to 4 x N_g columns
constexpr int kMaxAcc = 4;     // independent accumulators the MMA steps rotate over
constexpr int kTop = 8;
constexpr int kMaxSet = kTop + 9;   // top-8 plus the 3 x 3 neighbourhood of the BF16 minimum
// Bound of the BF16 surface error, relative to sum T^2 + N^2 >= E(v): rounding
// both operands to BF16 (unit roundoff 2^-9) moves each product by at most
// about 2^-8 of |T W|, and sum |T W| <= E(v) / 2, so |dS(v)| <= 2^-8 E(v); two
// lags differ by at most twice that, and a factor 2 more covers the FP32
// accumulation.  Lags whose BF16 score is farther than this above the minimum
// cannot be the FP32 minimum and are not re-scored.
constexpr float kBf16Band = 1.0f / 64.0f;
constexpr long long kWaitCycles = 2000000000ll;   // ~1 s at 2 GHz

struct Geom {
    int N, r, L, W, Nx, Ng, MM, J, DXR, CA, JB, Wp;
    int nacc;   // accumulators the MMA steps rotate over (columns nacc * Ng <= kTmemCols)
    int a_bytes, b_bytes, w_bytes;
};

__host__ __device__ inline Geom make_geom(int N, int r) {
    Geom g;
    g.N = N;
    g.r = r;
    g.L = 2 * r + 1;
    g.W = N + 2 * r;
    g.Nx = (N + 15) / 16 * 16;
    g.J = g.L <= 64 ? 2 : 1;                 // window rows stacked along M
    g.MM = 128;                              // MMA M: rows (dx, j) of the accumulator
    g.DXR = g.MM / g.J;                      // dx rows per window row
    g.Ng = (g.L + g.J - 1 + 15) / 16 * 16;
    g.nacc = kTmemCols / g.Ng < kMaxAcc ? kTmemCols / g.Ng : kMaxAcc;
    g.CA = (g.Nx + g.DXR) / 8;
    g.JB = g.W + g.Ng - 1;
    g.Wp = (g.W + 7) / 8 * 8;
    g.a_bytes = BG * g.CA * 128;             // one A buffer (BG window rows, BG % J == 0)
    g.b_bytes = (g.Nx / 8) * g.JB * 16;
    // the window channel in BF16, then a zero row (the second row of a step
    // past the window when W is odd) and a zero tail: the A build reads up to
    // 4 CA + 4 words from a row start without bounds tests
    g.w_bytes = ((g.W + 1) * g.Wp * 2 + (4 * g.CA + 4) * 4 + 15) / 16 * 16;
    return g;
}

// dynamic shared memory: [B operand][window][A slots 0..NBUF-1], the
// front reused after the MMAs for the ||D_sen||^2 window and its box-sum rows
// (and the FP32 window while re-scoring), then the L x L surface
__host__ __device__ inline int geom_ops(const Geom &g) {
    int ops = g.b_bytes + g.w_bytes + NBUF * g.a_bytes;
    const int box = (g.W * g.W + g.W * g.L) * 4;
    if (box > ops) ops = box;
    return (ops + 127) / 128 * 128;
}
__host__ __device__ inline int geom_smem(const Geom &g) { return geom_ops(g) + g.L * g.L * 4; }

// Stage the rows [0, rows) x [0, cols) of a row-major FP32 image block into
// shared memory (row pitch cols); the caller synchronises afterwards.
__device__ __forceinline__ void stage_block(float *dst, const float *src, int64_t rp, int rows, int cols) {
    for (int e = threadIdx.x; e < rows * cols; e += BT) {
        const int y = e / cols, x = e - y * cols;
        cp_async4(dst + e, src + (int64_t)y * rp + x);
    }
    cp_async_wait_all();
}

// Wait for the mbarrier phase with a cycle limit; false if it ran out.  Each
// probe may suspend the thread for up to 2 us (it resumes when the phase
// completes), so waiting threads leave the issue slots to the working warps.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *mbar, uint32_t parity, long long limit) {
    const long long t0 = clock64();
    while (!mbar_try_wait_sleep(mbar, parity, 2000u)) {
        if (clock64() - t0 > limit) return false;
    }
    return true;
}

// The nk MMAs of one step (K steps of 16 along the template row); the first
// one overwrites the accumulator unless acc0.
template <int NK>
__device__ __forceinline__ void issue_step(uint32_t dcol, uint64_t ar, uint64_t br, uint32_t da,
                                           uint32_t db, uint32_t idesc, uint32_t acc0) {
#pragma unroll
    for (int i = 0; i < NK; ++i)
        mma_bf16(dcol, ar + (uint64_t)(i * da), br + (uint64_t)(i * db), idesc, i == 0 ? acc0 : 1u);
}

// Named barrier 1 over the builder warps (the MMA-issuing warp does not take
// part); the _or form returns whether any builder thread passed true.
__device__ __forceinline__ void builders_sync() {
    asm volatile("bar.sync 1, %0;" ::"n"(kBuilders) : "memory");
}
__device__ __forceinline__ bool builders_sync_or(bool v) {
    int r;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\t"
        "setp.ne.b32 p, %1, 0;\n\t"
        "bar.red.or.pred q, 1, %2, p;\n\t"
        "selp.b32 %0, 1, 0, q;\n\t}\n"
        : "=r"(r) : "r"((int)v), "n"(kBuilders) : "memory");
    return r != 0;
}

__device__ __forceinline__ uint32_t pack_bf16x2(float lo, float hi) {
    const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<const uint32_t *>(&v);
}

struct Bf16Shared {
    uint64_t mbar_full[NBUF];    // slot b built: one arrival per builder warp
    uint64_t mbar_empty[NBUF];   // slot b's MMAs complete: the issuer's commit
    uint64_t mbar_idle;   // never arrived at: the failure-detection test waits on it
    uint32_t tmem;
    int error;            // a wait gave up: no more MMAs in this CTA
    int ierr;             // the issuer's wait for a full slot gave up
    uint32_t phase[NBUF];    // parity of the next empty[b] phase (builders)
    uint32_t fphase[NBUF];   // parity of the next full[b] phase (issuer)
    int pending[NBUF];    // slot b has a commit not yet seen complete
    int next;
    float red_f[BT / 32];
    int red_i[BT / 32];
    float2 red_c[BT / 32];
    int ncand;
    int cand_idx[kMaxSet];
    float cand_ssd[kMaxSet];
    int miss_idx[9];
    float miss_ssd[9];
};

// 16-byte asynchronous global -> shared copy (both addresses 16-byte aligned)
__device__ __forceinline__ void cp_async16(void *dst_smem, const float *src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(dst_smem)), "l"(src)
                 : "memory");
}

// Stage rows [0, rows) x columns [0, cols) of an image block whose first
// column is `col0` of rows `src` (row pitch rp) into shared memory: with
// `vec`, from column col0 & ~3 in 16-byte copies to a row pitch rounded up
// to 4 floats (the caller indexes from col0 & 3); otherwise 4-byte copies at
// pitch cols.  The caller waits and synchronises.
__device__ __forceinline__ void stage_rows(float *dst, const float *src, int64_t rp, int col0,
                                           int rows, int cols, bool vec) {
    if (vec) {
        const int a0 = col0 & ~3;
        const int pw = ((col0 - a0) + cols + 3) & ~3;
        const int q = pw / 4;
        for (int e = threadIdx.x; e < rows * q; e += BT) {
            const int y = e / q, x4 = e - y * q;
            cp_async16(dst + y * pw + 4 * x4, src + (int64_t)y * rp + a0 + 4 * x4);
        }
    } else {
        for (int e = threadIdx.x; e < rows * cols; e += BT) {
            const int y = e / cols, x = e - y * cols;
            cp_async4(dst + e, src + (int64_t)y * rp + col0 + x);
        }
    }
}

// Direct FP32 SSD (Eq. 3) of up to kMaxSet lags at once, channel by channel.
// When the template and the bounding box of the lags' windows fit in the
// `cap` bytes at wsm, both are staged in shared memory by asynchronous copies
// (16-byte copies from 16-byte aligned column starts when the volumes'
// pitches allow) and every template value is compared with each lag's window
// value there, warps over template rows and lanes over columns; otherwise the
// whole search window is staged and the template read from global memory.
// The element order of each thread is fixed by (N, r) and the path, so the
// result does not depend on the batch; the per-lag sums end in compensated
// block reductions.
template <int KS>
__device__ void rescore_set_k(const JobView &J, int m, int N, int r, int ry0, int rx0, int sy0,
                              int sx0, const int *idx, int n, float *out, float *wsm, int cap,
                              Bf16Shared &sh) {
    const int Lside = 2 * r + 1, W = N + 2 * r;
    // slots n .. KS-1 repeat lag 0: computed, never reported, so the inner
    // loops carry no per-slot test.  Lags 2h and 2h+1 share one packed
    // (f32x2) subtraction and fused multiply-add: t + (-w) and each lane's
    // FMA round exactly as the scalar t - w and fmaf.
    constexpr int KP = (KS + 1) / 2;
    int oy[KS], ox[KS];
    float2 acc2[KP];
    int y_lo = Lside, y_hi = 0, x_lo = Lside, x_hi = 0;
#pragma unroll
    for (int c = 0; c < KS; ++c) {
        const int li = c < n ? idx[c] : idx[0];
        oy[c] = li / Lside;   // r + vy
        ox[c] = li % Lside;   // r + vx
        if (c < n) {
            y_lo = min(y_lo, oy[c]);
            y_hi = max(y_hi, oy[c]);
            x_lo = min(x_lo, ox[c]);
            x_hi = max(x_hi, ox[c]);
        }
    }
    // window rows/columns the lags touch: [y_lo, y_hi + N) x [x_lo, x_hi + N)
    const int UH = N + y_hi - y_lo, UW = N + x_hi - x_lo;
    const int wc0 = sx0 + x_lo;        // first staged window column (image)
    // 16-byte copies need 16-byte aligned rows and must stay inside the row pitch
    const bool vec = ((J.sen_rp | J.sen_pp | J.ref_rp | J.ref_pp) & 3) == 0 &&
                     ((reinterpret_cast<uintptr_t>(J.sen) | reinterpret_cast<uintptr_t>(J.ref)) & 15) == 0 &&
                     (wc0 & ~3) + ((((wc0 & 3) + UW + 3) & ~3)) <= J.sen_rp &&
                     (rx0 & ~3) + ((((rx0 & 3) + N + 3) & ~3)) <= J.ref_rp;
#pragma unroll
    for (int h = 0; h < KP; ++h) acc2[h] = make_float2(0.f, 0.f);
    const int wsh = vec ? (wc0 & 3) : 0, tsh = vec ? (rx0 & 3) : 0;   // column shifts
    const int wpw = vec ? ((wsh + UW + 3) & ~3) : UW;                 // staged pitches
    const int tpw = vec ? ((tsh + N + 3) & ~3) : N;
    const bool packed = n > 0 && ((long long)UH * wpw + (long long)N * tpw) * 4 <= cap;
    if (packed) {
#pragma unroll
        for (int c = 0; c < KS; ++c) {
            oy[c] -= y_lo;
            ox[c] += wsh - x_lo;
        }
    }
    const int ww = packed ? wpw : W;  // row pitch of the staged window
    float *tsm = wsm + UH * wpw;      // staged template (packed path)
    int off[KS];                      // window offset of each lag in the staged window
#pragma unroll
    for (int c = 0; c < KS; ++c) off[c] = oy[c] * ww + ox[c];
    constexpr int U = 4;              // template loads in flight per thread (global path)
    const FastDiv divN(N);
    for (int k = 0; k < m; ++k) {
        const float *sk = J.sen + (int64_t)k * J.sen_pp;
        const float *tk = J.ref + (int64_t)k * J.ref_pp;
        __syncthreads();
        if (packed) {
            stage_rows(wsm, sk + (int64_t)(sy0 + y_lo) * J.sen_rp, J.sen_rp, wc0, UH, UW, vec);
            stage_rows(tsm, tk + (int64_t)ry0 * J.ref_rp, J.ref_rp, rx0, N, N, vec);
            cp_async_wait_all();
        } else {
            stage_block(wsm, sk + (int64_t)sy0 * J.sen_rp + sx0, J.sen_rp, W, W);
        }
        __syncthreads();
        if (packed) {
            // both operands in shared memory: warps take template rows, lanes
            // take columns; every lag's window value is at a fixed offset
            const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
            for (int y = warp; y < N; y += BT / 32) {
                const float *trow = tsm + y * tpw + tsh;
                const float *wrow = wsm + y * ww;
                for (int x = lane; x < N; x += 32) {
                    const float t = trow[x];
                    const float *wr = wrow + x;
#pragma unroll
                    for (int h = 0; h < KP; ++h) {
                        const float w0 = wr[off[2 * h]];
                        const float w1 = 2 * h + 1 < KS ? wr[off[2 * h + 1]] : w0;
                        const float2 d = __fadd2_rn(make_float2(t, t), make_float2(-w0, -w1));
                        acc2[h] = __ffma2_rn(d, d, acc2[h]);
                    }
                }
            }
            continue;
        }
        for (int e0 = threadIdx.x; e0 < N * N; e0 += U * BT) {
            float t[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int e = e0 + u * BT;
                const int y = divN.div(e), x = e - y * N;
                t[u] = e >= N * N ? 0.f : __ldg(tk + (int64_t)(ry0 + y) * J.ref_rp + (rx0 + x));
            }
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int e = e0 + u * BT;
                if (e >= N * N) break;
                const int y = divN.div(e), x = e - y * N;
                const float *wr = wsm + y * ww + x;
#pragma unroll
                for (int h = 0; h < KP; ++h) {
                    const float w0 = wr[off[2 * h]];
                    const float w1 = 2 * h + 1 < KS ? wr[off[2 * h + 1]] : w0;
                    const float2 d = __fadd2_rn(make_float2(t[u], t[u]), make_float2(-w0, -w1));
                    acc2[h] = __ffma2_rn(d, d, acc2[h]);
                }
            }
        }
    }
#pragma unroll
    for (int c = 0; c < KS; ++c) {
        if (c < n) {   // n is uniform across the CTA
            const float v = block_sum_comp<BT>((c & 1) ? acc2[c >> 1].y : acc2[c >> 1].x, sh.red_c);
            if (threadIdx.x == 0) out[c] = v;
        }
    }
    __syncthreads();
}

__device__ void rescore_set(const JobView &J, int m, int N, int r, int ry0, int rx0, int sy0,
                            int sx0, const int *idx, int n, float *out, float *wsm, int cap,
                            Bf16Shared &sh) {
    // the usual set is the 3 x 3 neighbourhood of the BF16 minimum
    if (n <= 9)
        rescore_set_k<9>(J, m, N, r, ry0, rx0, sy0, sx0, idx, n, out, wsm, cap, sh);
    else
        rescore_set_k<kMaxSet>(J, m, N, r, ry0, rx0, sy0, sx0, idx, n, out, wsm, cap, sh);
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
    if (cp == A.stall_cp) {
        // failure-detection test: a bounded wait that cannot succeed (no MMA
        // is outstanding, so the CTA may go on with its next CP)
        if (!mbar_wait_bounded(&sh.mbar_idle, 0u, A.wait_limit)) res.status = CFOG_CP_TIMEOUT;
        __syncthreads();
        if (tid == 0) A.out[cp] = res;
        return;
    }
    const Geom g = make_geom(N, r);
    unsigned char *bbuf = smem;
    __nv_bfloat16 *wbuf = reinterpret_cast<__nv_bfloat16 *>(smem + g.b_bytes);
    unsigned char *abuf0 = smem + g.b_bytes + g.w_bytes;
    float *surf = reinterpret_cast<float *>(smem + geom_ops(g));
    float *sqw = reinterpret_cast<float *>(smem);   // ||D_sen||^2 window, after the MMAs
    float *rows = sqw + g.W * g.W;                  // its box-sum rows
    const uint32_t bbase = smem_u32(bbuf), abase0 = smem_u32(abuf0);
    const int kchunks = g.Nx / 8;

    // The channel loop runs as two roles joined by a pair of mbarriers per A
    // slot: the builder warps 0-3 stage each channel and build the slots
    // (full[b]: one arrival per builder warp), and lane 0 of warp 4 issues a
    // slot's MMAs once it is full and commits them to empty[b].  Neither role
    // waits for the other at a CTA barrier, so the next slots are built while
    // the tensor core works through the earlier ones.  Every wait is bounded;
    // a wait that gives up ends its role's work for the CP, and the CTA then
    // reports TIMEOUT for this CP and every later one without further MMAs.
    float tt_part = 0.f;   // sum T^2, accumulated while the template is staged
    // The rows of B outside the template are zero for every channel: cleared
    // once per CP by the builders (every MMA of the previous CP has
    // completed; their proxy fences before each full arrival cover these
    // writes too), then each channel writes the N template rows only.
    const int warp = tid >> 5, lane = tid & 31;
    if (warp < kBuilderWarps) {
        for (int e = tid; e < g.b_bytes / 16; e += kBuilders)
            reinterpret_cast<uint4 *>(bbuf)[e] = make_uint4(0u, 0u, 0u, 0u);
        // the staged window's zero row and tail (never written by staging)
        const int w0 = g.W * g.Wp * 2 / 16;   // W * Wp * 2 is a multiple of 16
        for (int e = w0 + tid; e < g.w_bytes / 16; e += kBuilders)
            reinterpret_cast<uint4 *>(wbuf)[e] = make_uint4(0u, 0u, 0u, 0u);
    }
    const int ngrp = (g.W + BG - 1) / BG;   // A groups per channel
    if (warp < kBuilderWarps) {
        // empty[b] parities and commits not yet seen complete, tracked by
        // every builder warp (lane 0 waits, the warp shares the outcome)
        uint32_t ph[NBUF];
        bool pending[NBUF];
#pragma unroll
        for (int b = 0; b < NBUF; ++b) {
            ph[b] = sh.phase[b];
            pending[b] = false;
        }
        bool failed = false;
        auto wait_empty = [&](int b) {
            if (!pending[b] || failed) return;
            int ok = 1;
            if (lane == 0) ok = mbar_wait_bounded(&sh.mbar_empty[b], ph[b], A.wait_limit) ? 1 : 0;
            ok = __shfl_sync(0xffffffffu, ok, 0);
            if (ok) {
                ph[b] ^= 1u;
                pending[b] = false;
            } else {
                failed = true;
            }
        };
        constexpr int U = 4;   // 8-value chunks loaded per thread before converting
        // A build: lane b of each group of 8 lanes (an octet) writes copy b
        const int oct = tid >> 3, b = tid & 7;
        const int q_off = b >> 1;
        const uint32_t sel = (b & 1) ? 0x5432u : 0x3210u;
        const int wq = g.Wp / 2;          // 32-bit words per staged window row
        const int cstride = g.J * 128;    // bytes between the chunks of one row
        const FastDiv divCA(g.CA);
        // the window of channel k in BF16, zero in the pad columns [W, Wp)
        auto stage_window = [&](int k) {
            const float *sk = J.sen + (int64_t)k * J.sen_pp;
            const int wch = g.Wp / 8;
            const int nwt = g.W * wch;
            const FastDiv divW(wch);
            for (int e0 = tid; e0 < nwt; e0 += U * kBuilders) {
                float v[U][8];
#pragma unroll
                for (int h = 0; h < U; ++h) {
                    const int e = e0 + h * kBuilders;
                    const int y = divW.div(e), c = e - y * wch;
                    const float *src = sk + (int64_t)(sy0 + y) * J.sen_rp + (sx0 + 8 * c);
#pragma unroll
                    for (int u = 0; u < 8; ++u) v[h][u] = (e < nwt && 8 * c + u < g.W) ? __ldg(src + u) : 0.f;
                }
#pragma unroll
                for (int h = 0; h < U; ++h) {
                    const int e = e0 + h * kBuilders;
                    if (e >= nwt) break;
                    const int y = divW.div(e), c = e - y * wch;
                    uint4 w;
                    w.x = pack_bf16x2(v[h][0], v[h][1]);
                    w.y = pack_bf16x2(v[h][2], v[h][3]);
                    w.z = pack_bf16x2(v[h][4], v[h][5]);
                    w.w = pack_bf16x2(v[h][6], v[h][7]);
                    *reinterpret_cast<uint4 *>(wbuf + y * g.Wp + 8 * c) = w;
                }
            }
        };
        // The window is read by the builders only, so channel k+1's window
        // is staged as soon as every builder has built channel k's last
        // group, while that channel's last MMAs still run; B is read by the
        // MMAs and is rewritten only after they have completed.
        stage_window(0);
        for (int k = 0; k < m; ++k) {
            const float *tk = J.ref + (int64_t)k * J.ref_pp;
            // B is rewritten: every MMA of the previous channel must have
            // completed
#pragma unroll
            for (int bb = 0; bb < NBUF; ++bb) wait_empty(bb);
            failed = builders_sync_or(failed);   // one decision for the builders
            if (failed) break;
            // B: flipped template of channel k, template row y at row W+J-2-y;
            // consecutive threads read consecutive 8-value chunks of one row
            const int nbt = N * kchunks;
            const FastDiv divK(kchunks);
            for (int e0 = tid; e0 < nbt; e0 += U * kBuilders) {
                float v[U][8];
#pragma unroll
                for (int h = 0; h < U; ++h) {
                    const int e = e0 + h * kBuilders;
                    const int y = divK.div(e), c = e - y * kchunks;
                    const float *src = tk + (int64_t)(ry0 + y) * J.ref_rp + (rx0 + 8 * c);
#pragma unroll
                    for (int u = 0; u < 8; ++u) v[h][u] = (e < nbt && 8 * c + u < N) ? __ldg(src + u) : 0.f;
                }
#pragma unroll
                for (int h = 0; h < U; ++h) {
                    const int e = e0 + h * kBuilders;
                    if (e >= nbt) break;
                    const int y = divK.div(e), c = e - y * kchunks;
#pragma unroll
                    for (int u = 0; u < 8; ++u) tt_part = fmaf(v[h][u], v[h][u], tt_part);
                    uint4 w;
                    w.x = pack_bf16x2(v[h][0], v[h][1]);
                    w.y = pack_bf16x2(v[h][2], v[h][3]);
                    w.z = pack_bf16x2(v[h][4], v[h][5]);
                    w.w = pack_bf16x2(v[h][6], v[h][7]);
                    *reinterpret_cast<uint4 *>(bbuf + (size_t)(c * g.JB + (g.W + g.J - 2 - y)) * 16) = w;
                }
            }
            builders_sync();
            for (int gi = 0; gi < ngrp; ++gi) {
                const int bsel = gi % NBUF;
                const int g0 = gi * BG;
                const int G = min(BG, g.W - g0);
                wait_empty(bsel);
                if (failed) continue;   // idle to the end of the channel
                // A: 8 shifted copies of each window row of the group, the J
                // rows of a step interleaved chunk by chunk.  Copy b of chunk
                // c holds columns 8c+b .. 8c+b+7 (zero past Wp); the 8 lanes
                // of an octet fill one 128-byte core matrix without bank
                // conflicts: lane b reads the five 32-bit words (BF16 pairs)
                // from column 8c + 2(b/2) and, for odd b, shifts the pairs by
                // one value with a byte permute.  Columns past Wp come from
                // the next staged row (or the zero row and tail): finite
                // values that only reach rows dx >= 2r+1, which are never
                // read, or meet the zero columns N .. N_x-1 of B.  A step's
                // row past the window (odd W) is the zero row.  Items (row,
                // chunk) run over the octets; each octet loads four items
                // before storing.
                const int GR = (G + g.J - 1) / g.J * g.J;
                const int nit = GR * g.CA;
                unsigned char *abuf = abuf0 + bsel * g.a_bytes;
                constexpr int UB = 4;
                for (int it0 = oct; it0 < nit; it0 += (kBuilders / 8) * UB) {
                    uint32_t x[UB][5];
                    int off[UB];
#pragma unroll
                    for (int u = 0; u < UB; ++u) {
                        const int it = it0 + (kBuilders / 8) * u;
                        const int row = it < nit ? divCA.div(it) : 0;   // past nit: loaded, not stored
                        const int c = it < nit ? it - row * g.CA : 0;
                        const int pj = g.J == 2 ? (row & 1) : 0;
                        const uint32_t *wr = reinterpret_cast<const uint32_t *>(wbuf) +
                                             (size_t)(g0 + row) * wq;
                        const int q0 = 4 * c + q_off;
#pragma unroll
                        for (int j = 0; j < 5; ++j) x[u][j] = wr[q0 + j];
                        off[u] = ((row - pj) * g.CA + pj) * 128 + c * cstride + b * 16;
                    }
#pragma unroll
                    for (int u = 0; u < UB; ++u) {
                        if (it0 + (kBuilders / 8) * u < nit)
                            *reinterpret_cast<uint4 *>(abuf + off[u]) =
                                make_uint4(__byte_perm(x[u][0], x[u][1], sel), __byte_perm(x[u][1], x[u][2], sel),
                                           __byte_perm(x[u][2], x[u][3], sel), __byte_perm(x[u][3], x[u][4], sel));
                    }
                }
                // each lane's writes become visible to the tensor core's
                // (async-proxy) reads, then one arrival for the warp
                fence_proxy_async();
                __syncwarp();
                if (lane == 0) mbar_arrive(&sh.mbar_full[bsel]);
                pending[bsel] = true;
            }
            if (k + 1 < m) {
                builders_sync();   // every builder is done with channel k's window
                stage_window(k + 1);
            }
        }
        bool any_pending = false;
#pragma unroll
        for (int bb = 0; bb < NBUF; ++bb) {
            wait_empty(bb);
            any_pending = any_pending || pending[bb];
        }
        // one decision for the builders; a commit still outstanding makes the
        // error sticky (every later CP of this CTA reports TIMEOUT without MMAs)
        failed = builders_sync_or(failed || any_pending);
        if (tid == 0) {
#pragma unroll
            for (int bb = 0; bb < NBUF; ++bb) {
                sh.phase[bb] = ph[bb];
                sh.pending[bb] = pending[bb];
            }
            if (failed) sh.error = 1;
        }
    } else if (lane == 0) {
        // lane 0 of warp 4, the MMA issuer: per full slot, the group's MMAs,
        // then one commit to the slot's empty barrier (operands computed once
        // per step, the K steps unrolled).  Step s (J window rows) accumulates into
        // accumulator s % nacc (columns (s % nacc) * Ng), so consecutive steps
        // do not wait for one another's accumulation; the first MMA of each
        // accumulator overwrites it.
        uint32_t fph[NBUF];
#pragma unroll
        for (int b = 0; b < NBUF; ++b) fph[b] = sh.fphase[b];
        const uint32_t tmem0 = sh.tmem;
        const uint32_t idesc = mma_idesc(g.MM, g.Ng);
        const int nk = g.Nx / 16;
        const uint32_t da = (uint32_t)(16 * g.J), db = (uint32_t)(2 * g.JB);   // per K step
        int step = 0, acc = 0;
        bool ifail = false;
        for (int k = 0; k < m && !ifail; ++k) {
            for (int gi = 0; gi < ngrp; ++gi) {
                const int bsel = gi % NBUF;
                const int g0 = gi * BG;
                const int G = min(BG, g.W - g0);
                const int GR = (G + g.J - 1) / g.J * g.J;
                if (!mbar_wait_bounded(&sh.mbar_full[bsel], fph[bsel], A.wait_limit)) {
                    ifail = true;
                    break;
                }
                fph[bsel] ^= 1u;
                tc_fence_after();
                // descriptors of the group's first operands; the start address
                // field (16-byte units, low 14 bits) then advances by adds:
                // one step's A is J rows of CA chunks of 128 B, one K step two
                // chunks of each row; B moves one 16-byte row per window row
                // and 2 JB rows per K step
                const uint64_t a0 = smem_desc(abase0 + (uint32_t)(bsel * g.a_bytes),
                                              (uint32_t)(g.J * 128), 128);
                const uint64_t b0 = smem_desc(bbase + (uint32_t)((g.W - 1 - g0) * 16),
                                              (uint32_t)(g.JB * 16), 128);
                for (int row = 0; row < GR; row += g.J, ++step) {
                    const uint32_t dcol = tmem0 + (uint32_t)(acc * g.Ng);
                    const uint32_t acc0 = step < g.nacc ? 0u : 1u;
                    const uint64_t ar = a0 + (uint64_t)(row * g.CA * 8);
                    const uint64_t br = b0 - (uint64_t)row;
                    switch (nk) {
                        case 1: issue_step<1>(dcol, ar, br, da, db, idesc, acc0); break;
                        case 2: issue_step<2>(dcol, ar, br, da, db, idesc, acc0); break;
                        case 3: issue_step<3>(dcol, ar, br, da, db, idesc, acc0); break;
                        case 4: issue_step<4>(dcol, ar, br, da, db, idesc, acc0); break;
                        case 5: issue_step<5>(dcol, ar, br, da, db, idesc, acc0); break;
                        case 6: issue_step<6>(dcol, ar, br, da, db, idesc, acc0); break;
                        case 7: issue_step<7>(dcol, ar, br, da, db, idesc, acc0); break;
                        default: issue_step<8>(dcol, ar, br, da, db, idesc, acc0); break;
                    }
                    if (++acc == g.nacc) acc = 0;
                }
                mma_commit(&sh.mbar_empty[bsel]);
            }
        }
#pragma unroll
        for (int b = 0; b < NBUF; ++b) sh.fphase[b] = fph[b];
        if (ifail) sh.ierr = 1;
    }
    __syncthreads();
    if (tid == 0 && sh.ierr) sh.error = 1;
    __syncthreads();
    tc_fence_after();
    if (sh.error) {
        if (tid == 0) {
            res.status = CFOG_CP_TIMEOUT;
            A.out[cp] = res;
        }
        return;
    }
    // epilogue: C(dx, dy) = sum_j D[(dx, j)][dy + J-1 - j] from tensor memory
    // into the surface buffer
    const int L = g.L;
    {
        // lane 32 w + l holds row (dx, j): for J = 1 dx = 32 w + l; for J = 2
        // dx = 16 w + 8 (l / 16) + l % 8 and j = (l / 8) % 2, so the two rows
        // of one dx sit in lanes l and l ^ 8 of the same warp
        const int dx = g.J == 1 ? warp * 32 + lane : warp * 16 + 8 * (lane >> 4) + (lane & 7);
        const bool j0 = g.J == 1 || (lane & 8) == 0;
        // accumulators written by at least one step (all of them unless the
        // CP has fewer steps than accumulators)
        const long long n_step = (long long)m * ((g.W + g.J - 1) / g.J);
        const int nused = n_step < g.nacc ? (int)n_step : g.nacc;
        float carry = 0.f;   // J = 2: the partner row's value at the previous column
        for (int c0 = 0; c0 < g.Ng && warp < kBuilderWarps; c0 += 16) {
            float v[16];
            tmem_ld16(sh.tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
            for (int a = 1; a < nused; ++a) {
                float w[16];
                tmem_ld16(sh.tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(a * g.Ng + c0), w);
#pragma unroll
                for (int u = 0; u < 16; ++u) v[u] += w[u];
            }
            if (g.J == 1) {
                if (dx < L) {
#pragma unroll
                    for (int u = 0; u < 16; ++u)
                        if (c0 + u < L) surf[(c0 + u) * L + dx] = v[u];   // [dy][dx]
                }
            } else {
                // column c holds dy = c - 1 for j = 0 and dy = c for j = 1
#pragma unroll
                for (int u = 0; u < 16; ++u) {
                    const float pv = __shfl_xor_sync(0xffffffffu, v[u], 8);
                    const int dy = c0 + u - 1;
                    if (j0 && dx < L && dy >= 0 && dy < L) surf[dy * L + dx] = v[u] + carry;
                    carry = pv;
                }
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    // sum T^2 and the box sums B(v) of ||D_sen||^2 (separable sliding sums), FP32
    const float tt = block_sum_comp<BT>(tt_part, sh.red_c);
    stage_block(sqw, J.sen_sq + (int64_t)sy0 * J.sen_rp + sx0, J.sen_rp, g.W, g.W);
    __syncthreads();
    for (int yy = tid; yy < g.W; yy += BT) {
        const float *q = sqw + yy * g.W;
        float acc = 0.f;
        for (int x = 0; x < N; ++x) acc += q[x];
        rows[yy * L] = acc;
        for (int vx = 1; vx < L; ++vx) {
            acc += q[vx + N - 1] - q[vx - 1];
            rows[yy * L + vx] = acc;
        }
    }
    __syncthreads();
    for (int vx = tid; vx < L; vx += BT) {
        float acc = 0.f;
        for (int y = 0; y < N; ++y) acc += rows[y * L + vx];
        surf[vx] = tt + acc - 2.0f * surf[vx];   // surf held C at [dy][dx]
        for (int vy = 1; vy < L; ++vy) {
            acc += rows[(vy + N - 1) * L + vx] - rows[(vy - 1) * L + vx];
            surf[vy * L + vx] = tt + acc - 2.0f * surf[vy * L + vx];
        }
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
    // the smallest BF16 scores (at most kTop, and only those within the BF16
    // error band of the minimum) and the 3 x 3 neighbourhood of the smallest,
    // re-scored directly in FP32 in one pass
    const float band = kBf16Band * (tt + (float)N * (float)N);
    float s0 = 0.f;
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
        if (t == 0) s0 = smin;
        if (t > 0 && !(smin <= s0 + band)) break;   // uniform: every thread has smin
        if (tid == 0) {
            sh.cand_idx[t] = imin;
            sh.ncand = t + 1;
        }
        __syncthreads();
    }
    if (tid == 0) {
        const int b0 = sh.cand_idx[0];
        const int by = b0 / L, bx = b0 % L;
        int n = sh.ncand;
        for (int j = -1; j <= 1; ++j)
            for (int i = -1; i <= 1; ++i) {
                const int yy = by + j, xx = bx + i;
                if (yy < 0 || yy >= L || xx < 0 || xx >= L) continue;
                const int li = yy * L + xx;
                bool have = false;
                for (int c = 0; c < n; ++c) have |= sh.cand_idx[c] == li;
                if (!have) sh.cand_idx[n++] = li;
            }
        sh.ncand = n;
    }
    __syncthreads();
    const int ncand = sh.ncand;
    float *wsm = reinterpret_cast<float *>(smem);   // operand region is free now
    rescore_set(J, m, N, r, ry0, rx0, sy0, sx0, sh.cand_idx, ncand, sh.cand_ssd, wsm, geom_ops(g), sh);
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
        // neighbours of the winner not re-scored yet (only when the FP32
        // winner differs from the BF16 minimum)
        if (tid == 0) {
            int nm = 0;
            for (int j = -1; j <= 1; ++j)
                for (int i = -1; i <= 1; ++i) {
                    const int li = (vy + r + j) * L + (vx + r + i);
                    bool have = false;
                    for (int c = 0; c < ncand; ++c) have |= sh.cand_idx[c] == li;
                    if (!have) sh.miss_idx[nm++] = li;
                }
            sh.ncand = nm;   // reused as the count of missing lags
        }
        __syncthreads();
        const int nmiss = sh.ncand;
        if (nmiss > 0)
            rescore_set(J, m, N, r, ry0, rx0, sy0, sx0, sh.miss_idx, nmiss, sh.miss_ssd, wsm, geom_ops(g), sh);
        for (int j = -1; j <= 1; ++j)
            for (int i = -1; i <= 1; ++i) {
                const int li = (vy + r + j) * L + (vx + r + i);
                float sv = INFINITY;
                for (int c = 0; c < ncand; ++c)
                    if (sh.cand_idx[c] == li) sv = sh.cand_ssd[c];
                for (int c = 0; c < nmiss; ++c)
                    if (sh.miss_idx[c] == li) sv = sh.miss_ssd[c];
                nb[(j + 1) * 3 + (i + 1)] = sv;
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
__global__ void __launch_bounds__(BT, 2) match_bf16_kernel(const MatchArgs A, int *counter,
                                                         const int *order) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ Bf16Shared sh;
    const int tid = threadIdx.x;
    if (tid < 32) {
        tmem_alloc(&sh.tmem, kTmemCols);
        tmem_relinquish();
    }
    if (tid == 0) {
        for (int b = 0; b < NBUF; ++b) {
            mbar_init(&sh.mbar_full[b], kBuilderWarps);
            mbar_init(&sh.mbar_empty[b], 1);
            sh.phase[b] = 0;
            sh.fphase[b] = 0;
            sh.pending[b] = 0;
        }
        mbar_init(&sh.mbar_idle, 1);
        fence_mbar_init();
        sh.error = 0;
        sh.ierr = 0;
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
    // before the tensor memory is released, every commit must have completed:
    // a CTA whose wait gave up waits once more (bounded) for what is left
    if (sh.error) {
        for (int b = 0; b < NBUF; ++b)
            if (sh.pending[b]) mbar_wait_bounded(&sh.mbar_empty[b], sh.phase[b], A.wait_limit);
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
    for (int N = 1; N <= a.tmpl_max; ++N)
        for (int r = 0; r <= a.radius_max; ++r) {
            const int b = geom_smem(make_geom(N, r));
            smem = b > smem ? b : smem;
        }
    // at least 60 KB per CTA keeps at most 3 CTAs (3 x 128 TMEM columns) on an SM
    smem = smem < 60 * 1024 ? 60 * 1024 : smem;
    // 226 KB leaves the static shared memory within the 227 KB a CTA may use
    if (smem > 226 * 1024) {
        set_error("cfog_match: BF16 direct plan needs %d bytes of shared memory", smem);
        return CFOG_E_UNSUPPORTED;
    }
    cfog_status st = ensure_dynamic_smem(reinterpret_cast<const void *>(match_bf16_kernel), smem,
                                         "cfog_match (bf16)");
    if (st != CFOG_OK) return st;
    int grid = a.n;
    if (order) {
        int per_sm = 0;
        st = persistent_ctas_per_sm(reinterpret_cast<const void *>(match_bf16_kernel), BT, smem,
                                    &per_sm, "cfog_match (bf16): occupancy");
        if (st != CFOG_OK) return st;
        per_sm = per_sm < 1 ? 1 : (per_sm > 512 / kTmemCols ? 512 / kTmemCols : per_sm);
        const long long cap = (long long)sm_count() * per_sm;
        grid = (int)(a.n < cap ? a.n : cap);
    }
    MatchArgs b = a;
    bf16_test_hook(&b.stall_cp, &b.wait_limit);
    match_bf16_kernel<<<grid, BT, smem, s>>>(b, counter, order);
    return check_launch("cfog_match (bf16): launch");
}

namespace {
std::atomic<int> g_stall_cp{-1};
std::atomic<long long> g_wait_limit{kWaitCycles};
}  // namespace

void bf16_test_hook(int *stall_cp, long long *wait_limit) {
    *stall_cp = g_stall_cp.load();
    *wait_limit = g_wait_limit.load();
}

}  // namespace cfog

extern "C" cfog_status cfog_test_inject_wait_timeout(int32_t cp, int64_t wait_cycles) {
    CFOG_REQUIRE(cp >= -1, "cfog_test_inject_wait_timeout: cp = %d", cp);
    CFOG_REQUIRE(wait_cycles >= 1000 && wait_cycles <= (int64_t)cfog::kWaitCycles,
                 "cfog_test_inject_wait_timeout: wait_cycles %lld outside [1000, %lld]",
                 (long long)wait_cycles, (long long)cfog::kWaitCycles);
    cfog::g_stall_cp.store(cp);
    cfog::g_wait_limit.store(cp < 0 ? cfog::kWaitCycles : (long long)wait_cycles);
    return CFOG_OK;
}

namespace cfog {

}  // namespace cfog
