// K3 + K4 + K6: SSD template matching of control points by FP32 FFT
// correlation (Sec. III-G, Eq. 3-9) with argmin and sub-pixel fit (Sec. V-B).
//
// One CTA matches one CP.  For the template T (N x N x m, reference CFOG) and
// the search window S ((N+2r) x (N+2r) x m, sensed CFOG) Eq. 5 gives
//     S(v) = sum T^2 + sum_window ||D_sen||^2 - 2 sum_x T(x) S(x + v).
// Eq. 9 evaluates the correlation with a 3-D FFT over (x, y, channel); only
// channel lag 0 is a match, and the 3-D correlation at channel lag 0 equals
// the sum over channels of the 2-D correlations, so the channel FFT is not
// needed.  Per channel k the template block (real part) and its window
// (imaginary part) share one complex 2-D FFT; the two spectra are separated
// by Hermitian symmetry and conj(T_k) S_k is accumulated with weight -2; one
// inverse 2-D FFT then yields -2 C(v) at every lag.  The box sums of
// ||D_sen||^2 (the middle term of Eq. 5) come from two separable sliding-sum
// passes before the FFTs, and S(v) = sum T^2 + B(v) - 2 C(v).
// The FFT surface nominates the minimum; lags within a relative 2e-5 of it
// are re-scored directly (FP32 differences and sums, compensated block
// reduction), so the argmin is decided at the precision of the features.  The quadratic sub-pixel fit runs
// in FP64 on the 3 x 3 neighbourhood.
//
// Each FFT length is P = A * B: a decimation-in-frequency pass of radix A at
// stride B (then twiddles) and a pass of radix B on contiguous runs, each a
// register DFT (cfog_fft.cuh) with one shared-memory read and write per
// element.  The gather of the template and window is fused into the first row
// pass.  The spectrum stays in the two-digit reversed order (position
// a*B + b holds frequency a + A*b); the inverse runs the passes backwards, so
// no reordering pass exists.  The plane's row pitch is odd and every pass maps
// consecutive threads to consecutive columns or rows so that shared-memory
// accesses are free of bank conflicts.  Each thread keeps its share of the
// half-spectrum accumulator in registers across all channels and blocks.
#include "cfog_internal.cuh"
#include "cfog_fft.cuh"
#include "cfog_match_common.cuh"
#include "cfog_tc.cuh"
#include "cfog_plan.cuh"

#include <cuda.h>

#include <cfloat>
#include <climits>
#include <cmath>
#include <cstdint>
#include <algorithm>
#include <array>
#include <cstring>
#include <map>
#include <mutex>
#include <vector>

namespace cfog {
namespace {

// Kernel variants: threads per CTA, CTAs per SM, and the bound on the FFT
// plane P_y * P_x (which bounds shared memory and the accumulator items each
// thread holds in registers).
template <int ID_, int NT_, int MINB_, int MAXE_, bool TM_ = false>
struct Variant {
    static constexpr int ID = ID_;    // CFOG_MATCH_VARIANT_* value
    static constexpr int NT = NT_;
    static constexpr int MINB = MINB_;
    static constexpr int MAXE = MAXE_;
    static constexpr int XI = (MAXE_ / 2 + kMaxFft + NT_ - 1) / NT_;
    static constexpr bool TM = TM_;   // accumulator in tensor memory instead of registers
};
using VarWide = Variant<CFOG_MATCH_VARIANT_WIDE, 512, 1, 16384>;         // one CP per SM, large planes
using VarPair = Variant<CFOG_MATCH_VARIANT_PAIR, 256, 2, 9216>;          // two CPs per SM, planes up to 96 x 96
using VarTrio = Variant<CFOG_MATCH_VARIANT_TRIO, 256, 3, 7680, true>;    // three CPs per SM, accumulator in TMEM
using VarPairT = Variant<CFOG_MATCH_VARIANT_PAIRT, 256, 2, 9216, true>;  // pair geometry, accumulator in TMEM
constexpr int kNumVariants = 4;

__host__ __device__ inline int variant_maxe(int v) {
    return v == CFOG_MATCH_VARIANT_PAIR || v == CFOG_MATCH_VARIANT_PAIRT ? 9216
           : v == CFOG_MATCH_VARIANT_TRIO                             ? 7680
                                                                      : 16384;
}

// Dynamic shared memory one CP of plan p needs in variant V: the TMEM
// variants keep the accumulator positions in tensor memory, not in a table.
template <class V>
__host__ __device__ inline int variant_smem_bytes(const MatchPlan &p, int r) {
    return V::TM ? p.y.P * plane_ld(p) * 8 + (p.y.P + p.x.P) * 8 + (2 * r + 1) * (2 * r + 1) * 4
                 : plan_smem_bytes(p, r);
}

// Tuned plans (the autotuner's choices), one table per variant: entry
// [N][r] = (m << 16) | (plan code + 1), 0 = none (the cost model decides).
__device__ int32_t g_plan_override[kNumVariants][kMaxFft + 1][33];

// Tensor-memory layout of a TM variant: each warp group (warps w and w+4 share
// a 32-lane quadrant) owns a column window; X (2 floats per item) then the
// packed positions (1 per item), each rounded up to 16 columns.
template <class V>
struct TmemLayout {
    static constexpr int NX16 = (2 * V::XI + 15) / 16;
    static constexpr int NP16 = (V::XI + 15) / 16;
    static constexpr int GROUP = (NX16 + NP16) * 16 <= 64 ? 64 : 128;
    static constexpr int COLS = GROUP * (V::NT / 128);   // power of two for NT = 256
    static_assert((NX16 + NP16) * 16 <= GROUP, "TMEM window too small");
};
constexpr int kTrioTmemCols = TmemLayout<VarTrio>::COLS;
// ------------------------------------------------------------ FFT passes --
// Everything one fused gather + first row pass needs about the block.
struct GatherSrc {
    const float *t;   // template channel plane (reference)
    int64_t t_rp;
    int ty0, tx0;     // template block origin in the reference image
    int bh, bw;       // template block extent
    const float *w;   // window plane (sensed channel or ||D||^2)
    int64_t w_rp;
    int wy0, wx0;     // window origin in the sensed image
    int wh, ww;       // window extent
};

// Row pass 1 (radix A at stride B) fused with the gather.  Butterfly (row, j),
// j fastest: global reads are row segments, shared accesses are contiguous.
template <int NT, int A>
__device__ __forceinline__ void row_fwd_s1(float2 *plane, int ld, const float2 *tw, int B, int Py,
                                           const GatherSrc &g, float &tt) {
    const FastDiv divB(B);
    const int total = Py * B;
    for (int b = threadIdx.x; b < total; b += NT) {
        const int row = divB.div(b), j = b - row * B;
        float2 *p = plane + row * ld + j;
        if (row >= g.wh) {
#pragma unroll
            for (int a = 0; a < A; ++a) p[a * B] = make_float2(0.f, 0.f);
            continue;
        }
        float2 x[A];
        const float *trow = g.t + (int64_t)(g.ty0 + row) * g.t_rp + g.tx0;
        const float *wrow = g.w + (int64_t)(g.wy0 + row) * g.w_rp + g.wx0;
        const bool trow_ok = row < g.bh;
#pragma unroll
        for (int a = 0; a < A; ++a) {
            const int col = j + a * B;
            float re = 0.f, im = 0.f;
            if (trow_ok && col < g.bw) re = __ldg(trow + col);
            if (col < g.ww) im = __ldg(wrow + col);
            x[a] = make_float2(re, im);
        }
#pragma unroll
        for (int a = 0; a < A; ++a) tt = fmaf(x[a].x, x[a].x, tt);
        rdft<A, false>(x);
#pragma unroll
        for (int a = 1; a < A; ++a) x[a] = c_mul(x[a], tw[a * j]);
#pragma unroll
        for (int a = 0; a < A; ++a) p[a * B] = x[a];
    }
}

// Row pass 2 (radix B, contiguous runs) over rows [0, nrows), rows fastest.
template <int NT, int Bv, bool INV>
__device__ __forceinline__ void row_s2(float2 *plane, int ld, int A, int nrows) {
    const FastDiv divR(nrows);
    const int total = nrows * A;
    for (int b = threadIdx.x; b < total; b += NT) {
        const int a = divR.div(b), row = b - a * nrows;
        float2 *p = plane + row * ld + a * Bv;
        float2 x[Bv];
#pragma unroll
        for (int u = 0; u < Bv; ++u) x[u] = p[u];
        rdft<Bv, INV>(x);
#pragma unroll
        for (int u = 0; u < Bv; ++u) p[u] = x[u];
    }
}

// Inverse row pass 1 (conjugate twiddles, then inverse radix A at stride B)
// over rows [0, nrows), j fastest.
template <int NT, int A>
__device__ __forceinline__ void row_inv_s1(float2 *plane, int ld, const float2 *tw, int B, int nrows) {
    const FastDiv divB(B);
    const int total = nrows * B;
    for (int b = threadIdx.x; b < total; b += NT) {
        const int row = divB.div(b), j = b - row * B;
        float2 *p = plane + row * ld + j;
        float2 x[A];
#pragma unroll
        for (int a = 0; a < A; ++a) x[a] = p[a * B];
#pragma unroll
        for (int a = 1; a < A; ++a) x[a] = c_mul_conj(x[a], tw[a * j]);
        rdft<A, true>(x);
#pragma unroll
        for (int a = 0; a < A; ++a) p[a * B] = x[a];
    }
}

// Column pass 1 (radix A at stride B rows), columns fastest.  Forward: DFT
// then twiddles; inverse: conjugate twiddles then inverse DFT.
template <int NT, int A, bool INV>
__device__ __forceinline__ void col_s1(float2 *plane, int ld, const float2 *tw, int B, int Px) {
    const FastDiv divP(Px);
    const int total = Px * B;
    for (int b = threadIdx.x; b < total; b += NT) {
        const int j = divP.div(b), c = b - j * Px;
        float2 *p = plane + j * ld + c;
        const int step = B * ld;
        float2 x[A];
#pragma unroll
        for (int a = 0; a < A; ++a) x[a] = p[a * step];
        if (INV) {
#pragma unroll
            for (int a = 1; a < A; ++a) x[a] = c_mul_conj(x[a], tw[a * j]);
            rdft<A, true>(x);
        } else {
            rdft<A, false>(x);
#pragma unroll
            for (int a = 1; a < A; ++a) x[a] = c_mul(x[a], tw[a * j]);
        }
#pragma unroll
        for (int a = 0; a < A; ++a) p[a * step] = x[a];
    }
}

// Column pass 2 (radix B on contiguous rows), columns fastest.
template <int NT, int Bv, bool INV>
__device__ __forceinline__ void col_s2(float2 *plane, int ld, int A, int Px) {
    const FastDiv divP(Px);
    const int total = Px * A;
    for (int b = threadIdx.x; b < total; b += NT) {
        const int a = divP.div(b), c = b - a * Px;
        float2 *p = plane + a * Bv * ld + c;
        float2 x[Bv];
#pragma unroll
        for (int u = 0; u < Bv; ++u) x[u] = p[u * ld];
        rdft<Bv, INV>(x);
#pragma unroll
        for (int u = 0; u < Bv; ++u) p[u * ld] = x[u];
    }
}

#define CFOG_RADIX_SWITCH(R, CALL)                    \
    switch (R) {                                      \
        case 2: { constexpr int RR = 2; CALL; } break;  \
        case 3: { constexpr int RR = 3; CALL; } break;  \
        case 4: { constexpr int RR = 4; CALL; } break;  \
        case 5: { constexpr int RR = 5; CALL; } break;  \
        case 6: { constexpr int RR = 6; CALL; } break;  \
        case 8: { constexpr int RR = 8; CALL; } break;  \
        case 9: { constexpr int RR = 9; CALL; } break;  \
        case 10: { constexpr int RR = 10; CALL; } break; \
        case 12: { constexpr int RR = 12; CALL; } break; \
        case 15: { constexpr int RR = 15; CALL; } break; \
        default: { constexpr int RR = 16; CALL; } break; \
    }

// exp(-2 pi i k / P) with the argument reduced to one quadrant, so that
// sincospif sees an exactly scaled value in [0, 1/4)
__device__ __forceinline__ float2 twiddle(int k, int P) {
    const int q = (4 * k) / P;
    const int rem = 4 * k - q * P;
    float s, c;
    sincospif(0.5f * ((float)rem / (float)P), &s, &c);
    float cs, sn;
    switch (q & 3) {
        case 0: cs = c; sn = s; break;
        case 1: cs = -s; sn = c; break;
        case 2: cs = -c; sn = -s; break;
        default: cs = s; sn = -c; break;
    }
    return make_float2(cs, -sn);
}

// Sliding sums of one row segment: out[lx] = sum of q[lx .. lx+N-1] for lx in
// [l0, l1), from global (GLOBAL) or shared memory.  The first window sum runs
// in four interleaved partial sums (a shorter dependent chain); the rest
// slide by one value in and one out.
template <bool GLOBAL>
__device__ __forceinline__ void row_sliding_sum(const float *q, int N, int l0, int l1, float *out) {
    auto at = [&](int i) { return GLOBAL ? __ldg(q + i) : q[i]; };
    float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f;
    int x = 0;
    for (; x + 3 < N; x += 4) {
        a0 += at(l0 + x);
        a1 += at(l0 + x + 1);
        a2 += at(l0 + x + 2);
        a3 += at(l0 + x + 3);
    }
    for (; x < N; ++x) a0 += at(l0 + x);
    float acc = (a0 + a1) + (a2 + a3);
    out[l0] = acc;
    for (int lx = l0 + 1; lx < l1; ++lx) {
        acc += at(lx + N - 1) - at(lx - 1);
        out[lx] = acc;
    }
}

// position of frequency f after the forward passes of one axis
__device__ __forceinline__ int freq_pos(int f, const FftDim &d) { return (f % d.A) * d.B + f / d.A; }

// ------------------------------------------------------------------ kernel --
template <int NT>
struct CoreShared {
    float red_f[NT / 32];
    int red_i[NT / 32];
    float2 red_c[NT / 32];
    float2 red_cn[kMaxCand][NT / 32];
    int cand_n;
    int cand_idx[kCandBuf];
    float cand_val[kCandBuf];
    float cand_ssd[kMaxCand];
    int64_t cand_off[kMaxCand];
    MatchPlan plan;
    int ok;
    int next;
    uint32_t tmem;
};

// Match control point `cp` with the whole CTA.  Every branch that returns
// early is uniform across the CTA.
template <class V>
__device__ __forceinline__ void match_one(const MatchArgs &A, const int cp, CoreShared<V::NT> &sh,
                          unsigned char *smem_raw) {
    constexpr int NT = V::NT;
    constexpr int XI = V::XI;
    const int tid = threadIdx.x;
    const JobView J = job_view(A, cp);
    const int N = A.tmpl[cp], r = A.radius[cp];
    const int px = A.cps[cp].x, py = A.cps[cp].y;
    const int qx = A.prior ? A.prior[cp].x : 0, qy = A.prior ? A.prior[cp].y : 0;
    const int m = A.m;
    const int Lside = 2 * r + 1;

    cfog_match_result res;
    res.dx = qx;
    res.dy = qy;
    res.sub_dx = (float)qx;
    res.sub_dy = (float)qy;
    res.ssd = INFINITY;
    res.status = CFOG_CP_OOB;

    const int t0 = N / 2;
    const int ry0 = py - t0, rx0 = px - t0;                 // template origin in ref
    const int sy0 = py + qy - t0 - r, sx0 = px + qx - t0 - r; // window origin in sen
    // a CP outside the launch bounds would need more shared memory than the
    // launch has: it is reported out of bounds and never touches the buffers
    const bool inside = J.ok && N >= 1 && r >= 0 && N <= A.tmpl_max && r <= A.radius_max &&
                        ry0 >= 0 && rx0 >= 0 && ry0 + N <= J.ref_h && rx0 + N <= J.ref_w &&
                        sy0 >= 0 && sx0 >= 0 && sy0 + N + 2 * r <= J.sen_h &&
                        sx0 + N + 2 * r <= J.sen_w;
    if (!inside) {
        if (tid == 0) A.out[cp] = res;
        return;
    }
    // The plan of this class: the tuned plan when the table holds one for m
    // and it fits the launch's shared memory; otherwise the cost model's
    // search, lanes 0..15 of warp 0 each costing one block split.  Every
    // input is uniform over the warp, so the branch is too.
    if (tid < 32) {
        MatchPlan p;
        long long c = -1;
        bool tuned = false;
        if (A.plan_table >= 0) {
            const int e = g_plan_override[A.plan_table][N][r];
            if (e != 0 && (e >> 16) == m) {
                c = plan_for_code(N, r, m, (e & 0xffff) - 1, V::MAXE, &p);
                tuned = c >= 0 && variant_smem_bytes<V>(p, r) <= A.smem_bytes;
            }
        }
        if (tuned) {
            if (tid == 0) {
                sh.plan = p;
                sh.ok = 1;
            }
        } else {
            c = -1;
            if (tid < kNbMax * kNbMax)
                c = plan_for_split(N, r, m, tid / kNbMax + 1, tid % kNbMax + 1, V::MAXE, &p);
            long long bc = c < 0 ? LLONG_MAX : c;
            int bl = tid;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const long long oc = __shfl_xor_sync(0xffffffffu, bc, o);
                const int ol = __shfl_xor_sync(0xffffffffu, bl, o);
                if (oc < bc || (oc == bc && ol < bl)) {
                    bc = oc;
                    bl = ol;
                }
            }
            if (tid == bl && c >= 0) sh.plan = p;
            if (tid == 0) sh.ok = bc != LLONG_MAX;
        }
    }
    __syncthreads();
    if (!sh.ok) {
        if (tid == 0) A.out[cp] = res;
        return;
    }
    const MatchPlan plan = sh.plan;
    const FftDim &DY = plan.y;
    const FftDim &DX = plan.x;
    const int Py = DY.P, Px = DX.P;
    const int ld = Px + 1;
    const int Hx = Px / 2 + 1;
    const int nitems = Py * Hx;

    float2 *plane = reinterpret_cast<float2 *>(smem_raw);
    float2 *twx = plane + Py * ld;
    float2 *twy = twx + Px;
    unsigned *postab = reinterpret_cast<unsigned *>(twy + Py);   // [nitems] (register variants)
    float *bbox = V::TM ? reinterpret_cast<float *>(twy + Py)
                        : reinterpret_cast<float *>(postab + nitems);   // [Lside^2]

    for (int i = tid; i < Px; i += NT) twx[i] = twiddle(i, Px);
    for (int i = tid; i < Py; i += NT) twy[i] = twiddle(i, Py);

    // Box sums B(v) of ||D_sen||^2 over the template window at every lag
    // (the second term of Eq. 5), by separable sliding sums in FP32: row sums
    // R[y][lx] in the plane (free until the first FFT), then column sums.
    // When it fits beside R, the ||D_sen||^2 window is first staged in the
    // plane by cp.async (odd row pitch: one row per thread, no bank
    // conflicts); the sums take the same values in the same order either way.
    {
        float *rsum = reinterpret_cast<float *>(plane);   // [W][Lside]
        const int Wn = N + 2 * r;
        const int sp = Wn | 1;
        float *sqw = rsum + Wn * Lside;                    // [W][sp]
        const bool staged = (long long)Wn * (sp + Lside) <= 2LL * Py * ld;
        if (staged) {
            for (int e = tid; e < Wn * Wn; e += NT) {
                const int y = e / Wn, x = e - y * Wn;
                cp_async4(sqw + y * sp + x, J.sen_sq + (int64_t)(sy0 + y) * J.sen_rp + (sx0 + x));
            }
            cp_async_wait_all();
            __syncthreads();
        }
        // rows: two threads per window row, each sliding over half the lags
        const int lh = (Lside + 1) / 2;
        for (int it = tid; it < 2 * Wn; it += NT) {
            const int y = it >> 1, l0 = (it & 1) * lh, l1 = min(Lside, l0 + lh);
            if (l0 >= l1) continue;
            if (staged)
                row_sliding_sum<false>(sqw + y * sp, N, l0, l1, rsum + y * Lside);
            else
                row_sliding_sum<true>(J.sen_sq + (int64_t)(sy0 + y) * J.sen_rp + sx0, N, l0, l1,
                                      rsum + y * Lside);
        }
        __syncthreads();
        // columns: up to eight threads per lag column, each sliding over a
        // segment of the row lags
        const int nseg = max(1, min(8, NT / Lside));
        const int ls = (Lside + nseg - 1) / nseg;
        for (int it = tid; it < Lside * nseg; it += NT) {
            const int lx = it % Lside, l0 = (it / Lside) * ls, l1 = min(Lside, l0 + ls);
            if (l0 >= l1) continue;
            float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f;
            int y = 0;
            for (; y + 3 < N; y += 4) {
                a0 += rsum[(l0 + y) * Lside + lx];
                a1 += rsum[(l0 + y + 1) * Lside + lx];
                a2 += rsum[(l0 + y + 2) * Lside + lx];
                a3 += rsum[(l0 + y + 3) * Lside + lx];
            }
            for (; y < N; ++y) a0 += rsum[(l0 + y) * Lside + lx];
            float acc = (a0 + a1) + (a2 + a3);
            bbox[l0 * Lside + lx] = acc;
            for (int ly = l0 + 1; ly < l1; ++ly) {
                acc += rsum[(ly + N - 1) * Lside + lx] - rsum[(ly - 1) * Lside + lx];
                bbox[ly * Lside + lx] = acc;
            }
        }
        __syncthreads();
    }

    // accumulator items: frequencies (fy, fx) with fx <= Px/2; item `it` is
    // owned by thread it % NT.  postab[it] packs the plane positions of f and
    // -f as two 16-bit fields.  The items live in registers, or (TM variants)
    // in this warp's tensor-memory columns: X at [0, 32), positions at [32, 48)
    // of the warp group's 64 columns, one lane per thread.
    float2 X[V::TM ? 1 : XI];
    uint32_t tx = 0;
    if constexpr (V::TM) {
        using TL = TmemLayout<V>;
        tx = sh.tmem + ((uint32_t)((tid >> 5) & 3) * 32u << 16) + (uint32_t)(tid >> 7) * TL::GROUP;
        float z[16];
#pragma unroll
        for (int k = 0; k < 16; ++k) z[k] = 0.f;
#pragma unroll
        for (int c = 0; c < TL::NX16; ++c) tmem_st16(tx + 16 * c, z);
        const FastDiv divH(Hx);
#pragma unroll
        for (int c = 0; c < TL::NP16; ++c) {
            float pf[16];
#pragma unroll
            for (int u = 0; u < 16; ++u) {
                const int k = 16 * c + u;
                const int it = tid + k * NT;
                unsigned pk = 0u;
                if (k < XI && it < nitems) {
                    const int fy = divH.div(it), fx = it - fy * Hx;
                    const int gy = fy ? Py - fy : 0, gx = fx ? Px - fx : 0;
                    pk = (unsigned)(freq_pos(fy, DY) * ld + freq_pos(fx, DX)) |
                         ((unsigned)(freq_pos(gy, DY) * ld + freq_pos(gx, DX)) << 16);
                }
                pf[u] = __uint_as_float(pk);
            }
            tmem_st16(tx + 16 * (TL::NX16 + c), pf);
        }
        tmem_wait_st();
    } else {
#pragma unroll
        for (int k = 0; k < XI; ++k) X[k] = make_float2(0.f, 0.f);
        const FastDiv divH(Hx);
        for (int it = tid; it < nitems; it += NT) {
            const int fy = divH.div(it), fx = it - fy * Hx;
            const int gy = fy ? Py - fy : 0, gx = fx ? Px - fx : 0;
            const unsigned p1 = (unsigned)(freq_pos(fy, DY) * ld + freq_pos(fx, DX));
            const unsigned p2 = (unsigned)(freq_pos(gy, DY) * ld + freq_pos(gx, DX));
            postab[it] = p1 | (p2 << 16);
        }
    }
    __syncthreads();

    float tt_part = 0.f;   // sum T^2, per thread
    for (int iby = 0; iby < DY.nb; ++iby) {
        const int by0 = iby * DY.bs;
        const int bh = min(DY.bs, N - by0);
        for (int ibx = 0; ibx < DX.nb; ++ibx) {
            const int bx0 = ibx * DX.bs;
            const int bw = min(DX.bs, N - bx0);
            GatherSrc g;
            g.t_rp = J.ref_rp;
            g.ty0 = ry0 + by0;
            g.tx0 = rx0 + bx0;
            g.bh = bh;
            g.bw = bw;
            g.w_rp = J.sen_rp;
            g.wy0 = sy0 + by0;
            g.wx0 = sx0 + bx0;
            g.wh = bh + 2 * r;
            g.ww = bw + 2 * r;
            const int nrows = min(Py, g.wh);
            for (int k = 0; k < m; ++k) {
                g.t = J.ref + (int64_t)k * J.ref_pp;
                g.w = J.sen + (int64_t)k * J.sen_pp;
                // forward 2-D FFT of (template + i window)
                CFOG_RADIX_SWITCH(DX.A, (row_fwd_s1<NT, RR>(plane, ld, twx, DX.B, Py, g, tt_part)));
                __syncthreads();
                if (DX.B > 1) {
                    CFOG_RADIX_SWITCH(DX.B, (row_s2<NT, RR, false>(plane, ld, DX.A, nrows)));
                    __syncthreads();
                }
                CFOG_RADIX_SWITCH(DY.A, (col_s1<NT, RR, false>(plane, ld, twy, DY.B, Px)));
                __syncthreads();
                if (DY.B > 1) {
                    CFOG_RADIX_SWITCH(DY.B, (col_s2<NT, RR, false>(plane, ld, DY.A, Px)));
                    __syncthreads();
                }
                // separate the spectra of T and S and accumulate w * conj(T) S
                const float wgt = -0.5f;   // -2 / 4
                if constexpr (V::TM) {
                    using TL = TmemLayout<V>;
                    float xa[16 * TL::NX16], pf[16 * TL::NP16];
#pragma unroll
                    for (int c = 0; c < TL::NX16; ++c) tmem_ld16_nowait(tx + 16 * c, xa + 16 * c);
#pragma unroll
                    for (int c = 0; c < TL::NP16; ++c) tmem_ld16_nowait(tx + 16 * (TL::NX16 + c), pf + 16 * c);
                    tmem_wait_ld();
#pragma unroll
                    for (int q = 0; q < XI; ++q) {
                        if (tid + q * NT < nitems) {
                            const unsigned pk = __float_as_uint(pf[q]);
                            const float2 z1 = plane[pk & 0xffffu];
                            const float2 z2 = plane[pk >> 16];
                            const float2 t2 = make_float2(z1.x + z2.x, z1.y - z2.y);
                            const float2 s2 = make_float2(z1.y + z2.y, z2.x - z1.x);
                            xa[2 * q] = fmaf(wgt, fmaf(t2.x, s2.x, t2.y * s2.y), xa[2 * q]);
                            xa[2 * q + 1] = fmaf(wgt, fmaf(t2.x, s2.y, -t2.y * s2.x), xa[2 * q + 1]);
                        }
                    }
#pragma unroll
                    for (int c = 0; c < TL::NX16; ++c) tmem_st16(tx + 16 * c, xa + 16 * c);
                    tmem_wait_st();
                } else {
#pragma unroll
                    for (int q = 0; q < XI; ++q) {
                        if (tid + q * NT < nitems) {
                            const unsigned pk = postab[tid + q * NT];
                            const float2 z1 = plane[pk & 0xffffu];
                            const float2 z2 = plane[pk >> 16];
                            const float2 t2 = make_float2(z1.x + z2.x, z1.y - z2.y);     // 2 T
                            const float2 s2 = make_float2(z1.y + z2.y, z2.x - z1.x);     // 2 S
                            X[q].x = fmaf(wgt, fmaf(t2.x, s2.x, t2.y * s2.y), X[q].x);
                            X[q].y = fmaf(wgt, fmaf(t2.x, s2.y, -t2.y * s2.x), X[q].y);
                        }
                    }
                }
                __syncthreads();
            }
        }
    }

    // Hermitian completion into the plane, then the inverse passes backwards
    {
        const FastDiv divH(Hx);
        if constexpr (V::TM) {
            using TL = TmemLayout<V>;
            float xa[16 * TL::NX16], pf[16 * TL::NP16];
#pragma unroll
            for (int c = 0; c < TL::NX16; ++c) tmem_ld16_nowait(tx + 16 * c, xa + 16 * c);
#pragma unroll
            for (int c = 0; c < TL::NP16; ++c) tmem_ld16_nowait(tx + 16 * (TL::NX16 + c), pf + 16 * c);
            tmem_wait_ld();
#pragma unroll
            for (int q = 0; q < XI; ++q) {
                const int it = tid + q * NT;
                if (it < nitems) {
                    const int fy = divH.div(it), fx = it - fy * Hx;
                    const unsigned pk = __float_as_uint(pf[q]);
                    plane[pk & 0xffffu] = make_float2(xa[2 * q], xa[2 * q + 1]);
                    if (fx != 0 && 2 * fx != Px) plane[pk >> 16] = make_float2(xa[2 * q], -xa[2 * q + 1]);
                }
            }
        } else {
#pragma unroll
            for (int q = 0; q < XI; ++q) {
                const int it = tid + q * NT;
                if (it < nitems) {
                    const int fy = divH.div(it), fx = it - fy * Hx;
                    const unsigned pk = postab[it];
                    plane[pk & 0xffffu] = X[q];
                    if (fx != 0 && 2 * fx != Px) plane[pk >> 16] = make_float2(X[q].x, -X[q].y);
                }
            }
        }
    }
    __syncthreads();
    if (DY.B > 1) {
        CFOG_RADIX_SWITCH(DY.B, (col_s2<NT, RR, true>(plane, ld, DY.A, Px)));
        __syncthreads();
    }
    CFOG_RADIX_SWITCH(DY.A, (col_s1<NT, RR, true>(plane, ld, twy, DY.B, Px)));
    __syncthreads();
    if (DX.B > 1) {
        CFOG_RADIX_SWITCH(DX.B, (row_s2<NT, RR, true>(plane, ld, DX.A, Lside)));
        __syncthreads();
    }
    CFOG_RADIX_SWITCH(DX.A, (row_inv_s1<NT, RR>(plane, ld, twx, DX.B, Lside)));
    __syncthreads();

    const float tt = block_sum<NT>(tt_part, sh.red_f);
    const float inv_area = 1.0f / ((float)Py * (float)Px);
    const int L2 = Lside * Lside;
    const FastDiv divL(Lside);
    auto surf_at = [&](int i) {
        const int ly = divL.div(i), lx = i - ly * Lside;
        return tt + bbox[i] + plane[ly * ld + lx].x * inv_area;
    };
    float bv = INFINITY;
    int bi = INT_MAX;
    for (int i = tid; i < L2; i += NT) {
        const float sv = surf_at(i);
        if (sv < bv || (sv == bv && i < bi)) {
            bv = sv;
            bi = i;
        }
    }
    if (tid == 0) sh.cand_n = 0;
    float smin;
    int imin;
    block_argmin<NT>(bv, bi, sh.red_f, sh.red_i, smin, imin);

    // lags inside the nomination band are re-scored directly
    const float band = kRescoreRel * (tt + (float)N * (float)N);
    for (int i = tid; i < L2; i += NT) {
        const float sv = surf_at(i);
        if (sv <= smin + band) {
            const int slot = atomicAdd(&sh.cand_n, 1);
            if (slot < kCandBuf) {
                sh.cand_idx[slot] = i;
                sh.cand_val[slot] = sv;
            }
        }
    }
    __syncthreads();
    int ncand = min(sh.cand_n, kCandBuf);
    if (tid == 0) {
        // order by (FFT value, index) and keep the best kMaxCand
        for (int a = 1; a < ncand; ++a) {
            const int ii = sh.cand_idx[a];
            const float vv = sh.cand_val[a];
            int b = a - 1;
            while (b >= 0 && (sh.cand_val[b] > vv || (sh.cand_val[b] == vv && sh.cand_idx[b] > ii))) {
                sh.cand_idx[b + 1] = sh.cand_idx[b];
                sh.cand_val[b + 1] = sh.cand_val[b];
                --b;
            }
            sh.cand_idx[b + 1] = ii;
            sh.cand_val[b + 1] = vv;
        }
    }
    __syncthreads();
    ncand = min(ncand, kMaxCand);
    int win = imin;
    float win_ssd = smin;
    if (ncand > 1) {
        // one pass over the template per group of up to four candidates: each
        // template value is read once per group and compared with the window
        // value at every candidate lag of the group.  Eight elements per thread
        // are loaded before any is used, so the loads overlap; each thread
        // still visits its elements in the order e = tid, tid + NT, ...
        const int NN = N * N;
        if (tid < ncand) {
            const int li = sh.cand_idx[tid];
            const int vy = li / Lside - r, vx = li - (li / Lside) * Lside - r;
            sh.cand_off[tid] = (int64_t)vy * J.sen_rp + vx;
        }
        __syncthreads();
        float acc[kMaxCand];
#pragma unroll
        for (int c = 0; c < kMaxCand; ++c) acc[c] = 0.f;
        const FastDiv divN(N);
        constexpr int U = 8;
        if (ncand == 2) {
            // the usual near tie, two lags: sixteen elements per thread in
            // flight per round (the features were read long ago and mostly
            // come from DRAM), same element order, so the same sums
            constexpr int U2 = 16;
            const int64_t o0 = sh.cand_off[0], o1 = sh.cand_off[1];
            float a0 = 0.f, a1 = 0.f;
            for (int k = 0; k < m; ++k) {
                const float *tp = J.ref + (int64_t)k * J.ref_pp + (int64_t)ry0 * J.ref_rp + rx0;
                const float *wp = J.sen + (int64_t)k * J.sen_pp + (int64_t)(sy0 + r) * J.sen_rp + (sx0 + r);
                for (int e0 = tid; e0 < NN; e0 += U2 * NT) {
                    float ta[U2], w0[U2], w1[U2];
#pragma unroll
                    for (int u = 0; u < U2; ++u) {
                        const int e = e0 + u * NT;
                        const bool ok = e < NN;
                        const int y = divN.div(e), x = e - y * N;
                        const float *wq = wp + (int64_t)y * J.sen_rp + x;
                        ta[u] = ok ? __ldg(tp + (int64_t)y * J.ref_rp + x) : 0.f;
                        w0[u] = ok ? __ldg(wq + o0) : 0.f;
                        w1[u] = ok ? __ldg(wq + o1) : 0.f;
                    }
#pragma unroll
                    for (int u = 0; u < U2; ++u) {
                        const float d0 = ta[u] - w0[u], d1 = ta[u] - w1[u];
                        a0 = fmaf(d0, d0, a0);
                        a1 = fmaf(d1, d1, a1);
                    }
                }
            }
            acc[0] = a0;
            acc[1] = a1;
        }
#pragma unroll
        for (int cg = 0; cg < kMaxCand; cg += 4) {
            if (cg >= ncand || ncand == 2) break;
            const int nc = min(4, ncand - cg);
            int64_t off4[4];
#pragma unroll
            for (int c = 0; c < 4; ++c) off4[c] = sh.cand_off[cg + (c < nc ? c : 0)];
            float a4[4] = {0.f, 0.f, 0.f, 0.f};
            for (int k = 0; k < m; ++k) {
                const float *tp = J.ref + (int64_t)k * J.ref_pp + (int64_t)ry0 * J.ref_rp + rx0;
                const float *wp = J.sen + (int64_t)k * J.sen_pp + (int64_t)(sy0 + r) * J.sen_rp + (sx0 + r);
                for (int e0 = tid; e0 < NN; e0 += U * NT) {
                    float ta[U], wb[U][4];
#pragma unroll
                    for (int u = 0; u < U; ++u) {
                        const int e = e0 + u * NT;
                        const bool ok = e < NN;
                        const int y = divN.div(e), x = e - y * N;
                        ta[u] = ok ? __ldg(tp + (int64_t)y * J.ref_rp + x) : 0.f;
                        const float *wq = wp + (int64_t)y * J.sen_rp + x;
#pragma unroll
                        for (int c = 0; c < 4; ++c) wb[u][c] = ok && c < nc ? __ldg(wq + off4[c]) : 0.f;
                    }
#pragma unroll
                    for (int u = 0; u < U; ++u) {
#pragma unroll
                        for (int c = 0; c < 4; ++c) {
                            const float d = ta[u] - wb[u][c];
                            a4[c] = fmaf(d, d, a4[c]);
                        }
                    }
                }
            }
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                if (cg == 0) acc[c] = a4[c];
                else if (c + 4 < kMaxCand) acc[c + 4] = a4[c];
            }
        }
        block_sum_comp_n<NT, kMaxCand>(acc, ncand, sh.red_cn, sh.cand_ssd);
        __syncthreads();
        if (tid == 0) {
            int bc = 0;
            for (int c = 1; c < ncand; ++c)
                if (sh.cand_ssd[c] < sh.cand_ssd[bc] ||
                    (sh.cand_ssd[c] == sh.cand_ssd[bc] && sh.cand_idx[c] < sh.cand_idx[bc]))
                    bc = c;
            sh.red_i[0] = sh.cand_idx[bc];
            sh.red_f[0] = sh.cand_ssd[bc];
        }
        __syncthreads();
        win = sh.red_i[0];
        win_ssd = sh.red_f[0];
        __syncthreads();
    }

    if (A.surface) {
        const int Lmax = A.surf_side;
        float *dst = A.surface + (int64_t)cp * Lmax * Lmax;
        const int off = (Lmax - Lside) / 2;
        for (int i = tid; i < L2; i += NT) {
            const int ly = divL.div(i), lx = i - ly * Lside;
            dst[(ly + off) * Lmax + (lx + off)] = surf_at(i);
        }
    }

    if (tid == 0) {
        const int vy = win / Lside - r, vx = win - (win / Lside) * Lside - r;
        res.dx = qx + vx;
        res.dy = qy + vy;
        res.ssd = win_ssd;
        double ox = 0.0, oy = 0.0;
        if (vx == -r || vx == r || vy == -r || vy == r) {
            res.status = CFOG_CP_EDGE_PEAK;
        } else {
            double f[9];
            for (int j = -1; j <= 1; ++j)
                for (int i = -1; i <= 1; ++i)
                    f[(j + 1) * 3 + (i + 1)] = (double)surf_at((vy + r + j) * Lside + (vx + r + i));
            subpixel_fit(f, ox, oy);
            res.status = CFOG_CP_OK;
        }
        res.sub_dx = (float)((double)res.dx + ox);
        res.sub_dy = (float)((double)res.dy + oy);
        A.out[cp] = res;
    }
}

// One CTA per CP, in CP order.
template <class V>
__global__ void __launch_bounds__(V::NT, V::MINB) match_fft_kernel(const MatchArgs A) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ CoreShared<V::NT> sh;
    if (blockIdx.x < A.n) match_one<V>(A, blockIdx.x, sh, smem_raw);
}

// Persistent CTAs draining a queue of CPs: slot i of the queue is CP order[i];
// the next slot is taken with one atomic on `counter` (no waiting).
template <class V>
__global__ void __launch_bounds__(V::NT, V::MINB)
match_persistent_kernel(const MatchArgs A, int *__restrict__ counter, const int *__restrict__ order) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ CoreShared<V::NT> sh;
    if constexpr (V::TM) {
        if (threadIdx.x < 32) {
            tmem_alloc(&sh.tmem, TmemLayout<V>::COLS);
            tmem_relinquish();
        }
        tc_fence_before();
        __syncthreads();
        tc_fence_after();
    }
    for (;;) {
        if (threadIdx.x == 0) sh.next = atomicAdd(counter, 1);
        __syncthreads();
        const int i = sh.next;
        __syncthreads();
        if (i >= A.n) break;
        match_one<V>(A, order[i], sh, smem_raw);
        __syncthreads();
    }
    if constexpr (V::TM) {
        tc_fence_before();
        __syncthreads();
        if (threadIdx.x < 32) tmem_dealloc(sh.tmem, TmemLayout<V>::COLS);
    }
}

// Queue order for the persistent kernel: CPs sorted by search-window side
// N + 2r, largest first (a proxy of their FFT cost), so that the expensive CPs
// start early and the cheap ones fill the tail.  One CTA: histogram over the
// window side, exclusive scan, scatter.  Also resets the queue counter.
constexpr int kOrderThreads = 1024;
constexpr int kSideMax = kMaxFft + 64;

__global__ void __launch_bounds__(kOrderThreads)
order_queue_kernel(const int *__restrict__ tmpl, const int *__restrict__ radius, int n,
                   int *__restrict__ counter, int *__restrict__ order) {
    __shared__ int hist[kSideMax + 2];
    for (int i = threadIdx.x; i < kSideMax + 2; i += kOrderThreads) hist[i] = 0;
    if (threadIdx.x == 0) *counter = 0;
    __syncthreads();
    auto key = [&](int i) {
        const int side = tmpl[i] + 2 * radius[i];
        const int s = side < 0 ? 0 : (side > kSideMax ? kSideMax : side);
        return kSideMax - s;   // descending side
    };
    for (int i = threadIdx.x; i < n; i += kOrderThreads) atomicAdd(&hist[key(i)], 1);
    __syncthreads();
    if (threadIdx.x == 0) {
        int acc = 0;
        for (int b = 0; b <= kSideMax; ++b) {
            const int c = hist[b];
            hist[b] = acc;
            acc += c;
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += kOrderThreads) order[atomicAdd(&hist[key(i)], 1)] = i;
}

// ------------------------------------------------------------------- host --
// Host mirror of the tuned-plan tables and the AUTO variant choices.
struct Tuning {
    std::mutex mu;
    int32_t plan[kNumVariants][kMaxFft + 1][33] = {};
    int count[kNumVariants] = {};
    unsigned gen = 1;   // bumped by every change of the plan tables
    std::map<std::array<int, 4>, int> auto_variant;   // (m, tmpl_max, radius_max, precision)
};
Tuning &tuning() {
    static Tuning t;
    return t;
}

// Tuned plan code of (variant, N, r) for m, or -1.
int tuned_code(int v, int N, int r, int m) {
    const int e = tuning().plan[v - 1][N][r];
    return (e != 0 && (e >> 16) == m) ? (e & 0xffff) - 1 : -1;
}

// Largest dynamic shared memory over every class (N <= tmpl_max, r <=
// radius_max) of a launch, for the cost-model plan and any tuned plan alike
// (a device whose table was not written uses the cost model).
template <class V>
int max_plan_smem(int tmpl_max, int radius_max, int m) {
    static std::mutex mu;
    static std::map<std::array<unsigned, 4>, int> cache;
    Tuning &T = tuning();
    std::lock_guard<std::mutex> tl(T.mu);
    std::lock_guard<std::mutex> lock(mu);
    const std::array<unsigned, 4> key{(unsigned)tmpl_max, (unsigned)radius_max, (unsigned)m, T.gen};
    auto it = cache.find(key);
    if (it != cache.end()) return it->second;
    int best = 0;
    for (int N = 1; N <= tmpl_max; ++N)
        for (int r = 0; r <= radius_max; ++r) {
            MatchPlan p;
            if (!make_plan_host(N, r, m, V::MAXE, &p)) return -1;
            int b = variant_smem_bytes<V>(p, r);
            const int e = T.plan[V::ID - 1][N][r];
            if (e != 0 && (e >> 16) == m && plan_for_code(N, r, m, (e & 0xffff) - 1, V::MAXE, &p) >= 0)
                b = std::max(b, variant_smem_bytes<V>(p, r));
            best = b > best ? b : best;
        }
    cache[key] = best;
    return best;
}

// Whether the kernel should consult variant V's tuned-plan table.
template <class V>
int plan_table_of() {
    Tuning &T = tuning();
    std::lock_guard<std::mutex> lock(T.mu);
    return T.count[V::ID - 1] > 0 ? V::ID - 1 : -1;
}

struct Launch {
    const void *kernel;
    int threads;
    int smem;
    int plan_table;
};

template <class V>
cfog_status prepare(bool persistent, int tmpl_max, int radius_max, int m, Launch *L) {
    const int smem = max_plan_smem<V>(tmpl_max, radius_max, m);
    if (smem <= 0) {
        set_error("cfog_match: no FFT plan for tmpl_max %d radius_max %d", tmpl_max, radius_max);
        return CFOG_E_INVAL;
    }
    L->kernel = persistent ? reinterpret_cast<const void *>(match_persistent_kernel<V>)
                           : reinterpret_cast<const void *>(match_fft_kernel<V>);
    L->threads = V::NT;
    L->smem = smem;
    L->plan_table = plan_table_of<V>();
    return ensure_dynamic_smem(L->kernel, smem, "cfog_match");
}

// The variant AUTO runs for a launch class: the autotuner's choice if one is
// recorded, else WIDE (it plans every class with the fewest template blocks).
int auto_variant(int m, int tmpl_max, int radius_max, int precision) {
    Tuning &T = tuning();
    std::lock_guard<std::mutex> lock(T.mu);
    auto it = T.auto_variant.find({m, tmpl_max, radius_max, precision});
    return it != T.auto_variant.end() ? it->second : CFOG_MATCH_VARIANT_WIDE;
}

cfog_status check_common(int32_t n, const void *cps, const void *tmpl, const void *radius,
                         const void *out, int32_t tmpl_max, int32_t radius_max, int32_t m,
                         int32_t precision, int32_t variant) {
    CFOG_REQUIRE(n >= 0, "cfog_match: n = %d < 0", n);
    CFOG_REQUIRE(n == 0 || (cps && tmpl && radius && out), "cfog_match: null CP array");
    CFOG_REQUIRE(m >= 1 && m <= 64, "cfog_match: m = %d outside [1, 64]", m);
    CFOG_REQUIRE(tmpl_max >= 1 && tmpl_max <= kMaxFft, "cfog_match: tmpl_max %d outside [1, %d]",
                 tmpl_max, kMaxFft);
    CFOG_REQUIRE(radius_max >= 0 && radius_max <= 32, "cfog_match: radius_max %d outside [0, 32]",
                 radius_max);
    CFOG_REQUIRE(n <= (1 << 30), "cfog_match: n too large");
    CFOG_REQUIRE(variant >= 0 && variant <= 4, "cfog_match: unknown variant %d", variant);
    CFOG_REQUIRE(precision == CFOG_PREC_FP32_FFT || precision == CFOG_PREC_BF16_DIRECT,
                 "cfog_match: unknown precision %d", precision);
    if (precision == CFOG_PREC_BF16_DIRECT && tmpl_max > 128) {
        set_error("cfog_match: BF16 direct precision supports templates up to 128 (tmpl_max %d)",
                  tmpl_max);
        return CFOG_E_UNSUPPORTED;
    }
    return CFOG_OK;
}

}  // namespace
}  // namespace cfog

using namespace cfog;

extern "C" cfog_status cfog_match(const cfog_features *ref, const cfog_features *sen,
                                  const cfog_point *cps_dev, int32_t n, const int32_t *tmpl_dev,
                                  const int32_t *radius_dev, int32_t tmpl_max, int32_t radius_max,
                                  const cfog_point *prior_dev, int32_t precision,
                                  cfog_match_result *out_dev, float *surface_dev, void *stream) {
    CFOG_TRACE("cfog_match");
    CFOG_REQUIRE(ref && sen, "cfog_match: ref and sen must be non-NULL");
    CFOG_REQUIRE(ref->m == sen->m, "cfog_match: channel counts %d/%d", ref->m, sen->m);
    cfog_status st = check_common(n, cps_dev, tmpl_dev, radius_dev, out_dev, tmpl_max, radius_max,
                                  ref->m, precision, 0);
    if (st != CFOG_OK || n == 0) return st;
    CFOG_REQUIRE(ref->data && sen->data && sen->sqnorm, "cfog_match: null feature pointer");

    MatchArgs a{};
    a.ref = ref->data;
    a.ref_sq = ref->sqnorm;
    a.ref_h = ref->h;
    a.ref_w = ref->w;
    a.ref_rp = ref->row_pitch;
    a.ref_pp = ref->plane_pitch;
    a.sen = sen->data;
    a.sen_sq = sen->sqnorm;
    a.sen_h = sen->h;
    a.sen_w = sen->w;
    a.sen_rp = sen->row_pitch;
    a.sen_pp = sen->plane_pitch;
    a.jobs = nullptr;
    a.job_of_cp = nullptr;
    a.n_jobs = 0;
    a.m = ref->m;
    a.cps = cps_dev;
    a.tmpl = tmpl_dev;
    a.radius = radius_dev;
    a.prior = prior_dev;
    a.n = n;
    a.out = out_dev;
    a.surface = surface_dev;
    a.surf_side = 2 * radius_max + 1;
    a.tmpl_max = tmpl_max;
    a.radius_max = radius_max;
    a.plan_table = -1;
    if (precision == CFOG_PREC_BF16_DIRECT) return launch_bf16_direct(a, nullptr, nullptr, as_stream(stream));
    Launch L;
    st = prepare<VarWide>(false, tmpl_max, radius_max, a.m, &L);
    if (st != CFOG_OK) return st;
    a.smem_bytes = L.smem;
    a.plan_table = L.plan_table;
    match_fft_kernel<VarWide><<<n, L.threads, L.smem, as_stream(stream)>>>(a);
    return check_launch("cfog_match: launch");
}

extern "C" size_t cfog_match_workspace_bytes(int32_t n) {
    if (n < 0) return 0;
    return 256 + (size_t)n * sizeof(int32_t);
}

extern "C" cfog_status cfog_match_batched(const cfog_job *jobs_dev, int32_t n_jobs,
                                          const int32_t *job_of_cp_dev, const cfog_point *cps_dev,
                                          int32_t n, const int32_t *tmpl_dev,
                                          const int32_t *radius_dev, int32_t tmpl_max,
                                          int32_t radius_max, int32_t m,
                                          const cfog_point *prior_dev, int32_t precision,
                                          int32_t variant, cfog_match_result *out_dev,
                                          void *workspace_dev, size_t workspace_bytes,
                                          void *stream) {
    CFOG_TRACE("cfog_match_batched");
    cfog_status st = check_common(n, cps_dev, tmpl_dev, radius_dev, out_dev, tmpl_max, radius_max,
                                  m, precision, variant);
    if (st != CFOG_OK || n == 0) return st;
    CFOG_REQUIRE(jobs_dev && n_jobs >= 1, "cfog_match_batched: empty job table");
    CFOG_REQUIRE(workspace_dev, "cfog_match_batched: workspace is NULL");
    if (workspace_bytes < cfog_match_workspace_bytes(n)) {
        set_error("cfog_match_batched: workspace %zu bytes < %zu needed", workspace_bytes,
                  cfog_match_workspace_bytes(n));
        return CFOG_E_NOMEM;
    }
    CFOG_REQUIRE(((uintptr_t)workspace_dev & 255) == 0,
                 "cfog_match_batched: workspace must be 256-byte aligned");
    MatchArgs a{};
    a.jobs = jobs_dev;
    a.job_of_cp = job_of_cp_dev;
    a.n_jobs = n_jobs;
    a.m = m;
    a.cps = cps_dev;
    a.tmpl = tmpl_dev;
    a.radius = radius_dev;
    a.prior = prior_dev;
    a.n = n;
    a.out = out_dev;
    a.surface = nullptr;
    a.surf_side = 2 * radius_max + 1;
    a.tmpl_max = tmpl_max;
    a.radius_max = radius_max;
    a.plan_table = -1;
    const int v = variant == 0 ? auto_variant(m, tmpl_max, radius_max, precision) : variant;
    int *counter = static_cast<int *>(workspace_dev);
    int *order = reinterpret_cast<int *>(static_cast<char *>(workspace_dev) + 256);
    cudaStream_t s = as_stream(stream);
    if (precision == CFOG_PREC_BF16_DIRECT) {
        order_queue_kernel<<<1, kOrderThreads, 0, s>>>(tmpl_dev, radius_dev, n, counter, order);
        st = check_launch("cfog_match_batched: order launch");
        if (st != CFOG_OK) return st;
        return launch_bf16_direct(a, counter, order, s);
    }
    Launch L;
    st = v == CFOG_MATCH_VARIANT_PAIR    ? prepare<VarPair>(true, tmpl_max, radius_max, m, &L)
         : v == CFOG_MATCH_VARIANT_TRIO  ? prepare<VarTrio>(true, tmpl_max, radius_max, m, &L)
         : v == CFOG_MATCH_VARIANT_PAIRT ? prepare<VarPairT>(true, tmpl_max, radius_max, m, &L)
                                         : prepare<VarWide>(true, tmpl_max, radius_max, m, &L);
    if (st != CFOG_OK) return st;
    a.smem_bytes = L.smem;
    a.plan_table = L.plan_table;
    int per_sm = 0;
    st = persistent_ctas_per_sm(L.kernel, L.threads, L.smem, &per_sm,
                                "cfog_match_batched: occupancy");
    if (st != CFOG_OK) return st;
    // persistent TMEM variants hold their columns for life: at most 512 / 128 per SM
    if (v == CFOG_MATCH_VARIANT_TRIO && per_sm > 512 / kTrioTmemCols) per_sm = 512 / kTrioTmemCols;
    if (v == CFOG_MATCH_VARIANT_PAIRT && per_sm > 512 / TmemLayout<VarPairT>::COLS)
        per_sm = 512 / TmemLayout<VarPairT>::COLS;
    const int grid = (int)std::min<long long>((long long)n, (long long)sm_count() * per_sm);
    order_queue_kernel<<<1, kOrderThreads, 0, s>>>(tmpl_dev, radius_dev, n, counter, order);
    st = check_launch("cfog_match_batched: order launch");
    if (st != CFOG_OK) return st;
    if (v == CFOG_MATCH_VARIANT_PAIR)
        match_persistent_kernel<VarPair><<<grid, L.threads, L.smem, s>>>(a, counter, order);
    else if (v == CFOG_MATCH_VARIANT_TRIO)
        match_persistent_kernel<VarTrio><<<grid, L.threads, L.smem, s>>>(a, counter, order);
    else if (v == CFOG_MATCH_VARIANT_PAIRT)
        match_persistent_kernel<VarPairT><<<grid, L.threads, L.smem, s>>>(a, counter, order);
    else
        match_persistent_kernel<VarWide><<<grid, L.threads, L.smem, s>>>(a, counter, order);
    return check_launch("cfog_match_batched: launch");
}

// Plan of (N, r, m) in variant v: the tuned plan if one is recorded (host
// mirror), else the cost model's.
static bool plan_in_use(int tmpl, int radius, int m, int v, MatchPlan *p) {
    const int maxe = variant_maxe(v);
    int code;
    {
        Tuning &T = tuning();
        std::lock_guard<std::mutex> lock(T.mu);
        code = tuned_code(v, tmpl, radius, m);
    }
    if (code >= 0 && plan_for_code(tmpl, radius, m, code, maxe, p) >= 0) return true;
    return make_plan_host(tmpl, radius, m, maxe, p);
}

static int plan_smem_of(int v, const MatchPlan &p, int r) {
    return v == CFOG_MATCH_VARIANT_TRIO || v == CFOG_MATCH_VARIANT_PAIRT
               ? variant_smem_bytes<VarTrio>(p, r)
               : plan_smem_bytes(p, r);
}

static void plan_row(const MatchPlan &p, int v, int r, int32_t *out8) {
    out8[0] = p.y.nb;
    out8[1] = p.x.nb;
    out8[2] = p.y.P;
    out8[3] = p.x.P;
    out8[4] = p.y.bs;
    out8[5] = p.x.bs;
    out8[6] = (p.y.B > 1 ? 2 : 1) + (p.x.B > 1 ? 2 : 1);
    out8[7] = plan_smem_of(v, p, r);
}

#define CFOG_CHECK_CLASS(who, tmpl, radius, m)                                                \
    CFOG_REQUIRE(tmpl >= 1 && tmpl <= kMaxFft && radius >= 0 && radius <= 32 && m >= 1 && m <= 64, \
                 who ": (N=%d, r=%d, m=%d) outside the supported range", tmpl, radius, m)

extern "C" cfog_status cfog_plan_info(int32_t tmpl, int32_t radius, int32_t m, int32_t variant,
                                      int32_t *out8) {
    CFOG_REQUIRE(out8, "cfog_plan_info: out8 is NULL");
    CFOG_CHECK_CLASS("cfog_plan_info", tmpl, radius, m);
    CFOG_REQUIRE(variant >= 0 && variant <= 4, "cfog_plan_info: unknown variant %d", variant);
    const int v = variant == 0 ? CFOG_MATCH_VARIANT_WIDE : variant;
    MatchPlan p;
    CFOG_REQUIRE(plan_in_use(tmpl, radius, m, v, &p), "cfog_plan_info: no plan");
    plan_row(p, v, radius, out8);
    return CFOG_OK;
}

extern "C" cfog_status cfog_plan_candidates(int32_t tmpl, int32_t radius, int32_t m,
                                            int32_t variant, int32_t max_out, int32_t *out9,
                                            int32_t *n_out) {
    CFOG_REQUIRE(out9 && n_out, "cfog_plan_candidates: null output");
    CFOG_CHECK_CLASS("cfog_plan_candidates", tmpl, radius, m);
    CFOG_REQUIRE(variant >= 1 && variant <= 4, "cfog_plan_candidates: variant %d not in 1..4",
                 variant);
    CFOG_REQUIRE(max_out >= 0, "cfog_plan_candidates: max_out = %d", max_out);
    std::vector<std::pair<long long, int>> c;
    for (int code = 0; code < kPlanCodes; ++code) {
        MatchPlan p;
        const long long cost = plan_for_code(tmpl, radius, m, code, variant_maxe(variant), &p);
        if (cost >= 0) c.emplace_back(cost, code);
    }
    std::sort(c.begin(), c.end());
    // distinct plans only (two codes can name the same plan when a block
    // split degenerates), in order of the model's cost
    int n = 0;
    std::vector<MatchPlan> seen;
    for (const auto &e : c) {
        if (n >= max_out) break;
        MatchPlan p;
        plan_for_code(tmpl, radius, m, e.second, variant_maxe(variant), &p);
        bool dup = false;
        for (const MatchPlan &q : seen)
            dup = dup || (q.y.nb == p.y.nb && q.x.nb == p.x.nb && q.y.P == p.y.P && q.x.P == p.x.P);
        if (dup) continue;
        seen.push_back(p);
        out9[9 * n] = e.second;
        plan_row(p, variant, radius, out9 + 9 * n + 1);
        ++n;
    }
    *n_out = n;
    return CFOG_OK;
}

extern "C" cfog_status cfog_match_set_plan(int32_t variant, int32_t m, int32_t tmpl,
                                           int32_t radius, int32_t code) {
    CFOG_TRACE("cfog_match_set_plan");
    CFOG_CHECK_CLASS("cfog_match_set_plan", tmpl, radius, m);
    CFOG_REQUIRE(variant >= 1 && variant <= 4, "cfog_match_set_plan: variant %d not in 1..4",
                 variant);
    MatchPlan p;
    CFOG_REQUIRE(code == -1 || plan_for_code(tmpl, radius, m, code, variant_maxe(variant), &p) >= 0,
                 "cfog_match_set_plan: code %d names no feasible plan for (N=%d, r=%d, m=%d)", code,
                 tmpl, radius, m);
    const int32_t e = code < 0 ? 0 : (int32_t)((m << 16) | (code + 1));
    Tuning &T = tuning();
    std::lock_guard<std::mutex> lock(T.mu);
    const size_t off = (((size_t)(variant - 1) * (kMaxFft + 1) + tmpl) * 33 + radius) * sizeof(int32_t);
    cfog_status st = check_cuda(cudaMemcpyToSymbol(g_plan_override, &e, sizeof(e), off),
                                "cfog_match_set_plan: table write");
    if (st != CFOG_OK) return st;
    int32_t &h = T.plan[variant - 1][tmpl][radius];
    T.count[variant - 1] += (e != 0) - (h != 0);
    h = e;
    ++T.gen;
    return CFOG_OK;
}

extern "C" cfog_status cfog_match_set_auto_variant(int32_t m, int32_t tmpl_max,
                                                   int32_t radius_max, int32_t precision,
                                                   int32_t variant) {
    CFOG_CHECK_CLASS("cfog_match_set_auto_variant", tmpl_max, radius_max, m);
    CFOG_REQUIRE(variant >= 0 && variant <= 4, "cfog_match_set_auto_variant: variant %d", variant);
    CFOG_REQUIRE(precision == CFOG_PREC_FP32_FFT || precision == CFOG_PREC_BF16_DIRECT,
                 "cfog_match_set_auto_variant: unknown precision %d", precision);
    Tuning &T = tuning();
    std::lock_guard<std::mutex> lock(T.mu);
    const std::array<int, 4> key{m, tmpl_max, radius_max, precision};
    if (variant == 0)
        T.auto_variant.erase(key);
    else
        T.auto_variant[key] = variant;
    return CFOG_OK;
}

extern "C" int32_t cfog_match_auto_variant(int32_t m, int32_t tmpl_max, int32_t radius_max,
                                           int32_t precision) {
    return auto_variant(m, tmpl_max, radius_max, precision);
}

extern "C" cfog_status cfog_match_clear_tuning(void) {
    CFOG_TRACE("cfog_match_clear_tuning");
    Tuning &T = tuning();
    std::lock_guard<std::mutex> lock(T.mu);
    static int32_t zeros[kNumVariants][kMaxFft + 1][33];
    cfog_status st = check_cuda(cudaMemcpyToSymbol(g_plan_override, zeros, sizeof(zeros)),
                                "cfog_match_clear_tuning: table write");
    if (st != CFOG_OK) return st;
    std::memset(T.plan, 0, sizeof(T.plan));
    for (int &c : T.count) c = 0;
    T.auto_variant.clear();
    ++T.gen;
    return CFOG_OK;
}

// ------------------------------------------------ allocation-free variant --
// Batched matching for callers that cannot allocate device memory.  The
// queue scratch of cfog_match_batched (a counter and the order of up to
// kNoAllocMaxCps CPs) lives in this file-scope array instead of a caller
// workspace.  Every GPU that loads the library holds it until the process
// exits.  In host code the symbol is only a host-side stand-in: the device
// address comes from cudaGetSymbolAddress, looked up with the device current.
// The address belongs to one CUDA context (a device reset, or a second
// context on the same device, loads the module again elsewhere), so the
// cached address is keyed by the driver's context ID, which is never reused
// within a process; a call from another context looks the address up again.
namespace cfog {
namespace {
constexpr int kNoAllocMaxCps = 65536;
constexpr size_t kNoAllocBytes = 256 + (size_t)kNoAllocMaxCps * sizeof(int32_t);
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

struct NoAllocSlot {
    void *ptr;
    unsigned long long ctx_id;   // 0: unknown, never matches
};
std::mutex g_noalloc_mu;
NoAllocSlot g_noalloc[64] = {};

// ID of the current CUDA context (0 if there is none or the driver calls are
// unavailable).  The two driver functions are resolved through the runtime,
// so the library does not link libcuda itself.
unsigned long long current_ctx_id() {
    using GetCurrentFn = CUresult (*)(CUcontext *);
    using GetIdFn = CUresult (*)(CUcontext, unsigned long long *);
    static GetCurrentFn get_current = [] {
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) !=
                cudaSuccess || q != cudaDriverEntryPointSuccess)
            f = nullptr;
        return reinterpret_cast<GetCurrentFn>(f);
    }();
    static GetIdFn get_id = [] {
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) !=
                cudaSuccess || q != cudaDriverEntryPointSuccess)
            f = nullptr;
        return reinterpret_cast<GetIdFn>(f);
    }();
    CUcontext ctx = nullptr;
    unsigned long long id = 0;
    if (!get_current || !get_id || get_current(&ctx) != CUDA_SUCCESS || !ctx) return 0;
    if (get_id(ctx, &id) != CUDA_SUCCESS) return 0;
    return id;
}

// Device address of g_noalloc_scratch in the current context (looked up on
// the first call made in that context).
cfog_status noalloc_scratch(void **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return check_cuda(e, "cfog_match_batched_noalloc: cudaGetDevice");
    if (dev < 0 || dev >= 64) {
        set_error("cfog_match_batched_noalloc: device %d outside the supported range [0, 64)", dev);
        return CFOG_E_UNSUPPORTED;
    }
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    const unsigned long long id = current_ctx_id();
    if (g_noalloc[dev].ptr && id != 0 && g_noalloc[dev].ctx_id == id) {
        *out = g_noalloc[dev].ptr;
        return CFOG_OK;
    }
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p)
        return check_cuda(e != cudaSuccess ? e : cudaErrorInvalidSymbol,
                          "cfog_match_batched_noalloc: cudaGetSymbolAddress");
    // the lookup makes the device's primary context current if none was
    g_noalloc[dev].ptr = p;
    g_noalloc[dev].ctx_id = id != 0 ? id : current_ctx_id();
    *out = p;
    return CFOG_OK;
}
}  // namespace
}  // namespace cfog

extern "C" int32_t cfog_match_batched_noalloc_max_cps(void) { return kNoAllocMaxCps; }

extern "C" cfog_status cfog_match_batched_noalloc(const cfog_job *jobs_dev, int32_t n_jobs,
                                                  const int32_t *job_of_cp_dev,
                                                  const cfog_point *cps_dev, int32_t n,
                                                  const int32_t *tmpl_dev,
                                                  const int32_t *radius_dev, int32_t tmpl_max,
                                                  int32_t radius_max, int32_t m,
                                                  const cfog_point *prior_dev, int32_t precision,
                                                  int32_t variant, cfog_match_result *out_dev,
                                                  void *stream) {
    CFOG_TRACE("cfog_match_batched_noalloc");
    if (n > kNoAllocMaxCps) {
        set_error("cfog_match_batched_noalloc: n = %d CPs exceeds the built-in scratch for %d CPs;"
                  " split the batch or use cfog_match_batched with a workspace",
                  n, kNoAllocMaxCps);
        return CFOG_E_INVAL;
    }
    void *scratch = nullptr;
    if (n > 0) {
        cfog_status st = noalloc_scratch(&scratch);
        if (st != CFOG_OK) return st;
    }
    return cfog_match_batched(jobs_dev, n_jobs, job_of_cp_dev, cps_dev, n, tmpl_dev, radius_dev,
                              tmpl_max, radius_max, m, prior_dev, precision, variant, out_dev,
                              scratch, kNoAllocBytes, stream);
}
