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
// by Hermitian symmetry and conj(T_k) S_k is accumulated with weight -2.  The
// box sum of ||D_sen||^2 is one more such channel (an all-ones template,
// weight +1).  One inverse 2-D FFT then yields S(v) - sum T^2 at every lag.
// The FFT surface nominates the minimum; lags within a relative 2e-5 of it
// are re-scored by direct FP32 differences summed in FP64, so the argmin is
// decided at the precision of the features.  The quadratic sub-pixel fit runs
// in FP64 on the 3 x 3 neighbourhood.
//
// FFTs are in-place mixed-radix (2, 3, 4, 5) decimation-in-frequency passes in
// shared memory; the spectrum stays in digit-reversed order and the inverse
// runs the decimation-in-time passes in reverse, so no reordering pass exists.
#include "cfog_internal.cuh"
#include "cfog_plan.cuh"

#include <cfloat>
#include <climits>
#include <cmath>
#include <cstdint>
#include <mutex>

namespace cfog {
namespace {

constexpr int MT = 512;              // threads per CTA
constexpr float kRescoreRel = 2e-5f; // FFT nomination band, relative to sum T^2 + N^2
constexpr int kMaxCand = 8;
constexpr int kCandBuf = 64;

struct MatchArgs {
    const float *ref;
    const float *ref_sq;
    int ref_h, ref_w;
    int64_t ref_rp, ref_pp;
    const float *sen;
    const float *sen_sq;
    int sen_h, sen_w;
    int64_t sen_rp, sen_pp;
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
};

// ---------------------------------------------------------------- complex --
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ float2 cmulconj(float2 a, float2 b) {  // a * conj(b)
    return make_float2(fmaf(a.x, b.x, a.y * b.y), fmaf(a.y, b.x, -a.x * b.y));
}
// multiply by -i (forward) or +i (inverse)
template <bool INV>
__device__ __forceinline__ float2 rot90(float2 a) {
    return INV ? make_float2(-a.y, a.x) : make_float2(a.y, -a.x);
}

// exp(-2 pi i k / P), argument reduced to a quadrant so sincospif sees [0, 1/4)
__device__ float2 twiddle(int k, int P) {
    k %= P;
    const int q = (4 * k) / P;
    const int rem = 4 * k - q * P;
    float s, c;
    sincospif(0.5f * ((float)rem / (float)P), &s, &c);
    float cs, sn;  // cos, sin of 2 pi k / P
    switch (q) {
        case 0: cs = c; sn = s; break;
        case 1: cs = -s; sn = c; break;
        case 2: cs = -c; sn = -s; break;
        default: cs = s; sn = -c; break;
    }
    return make_float2(cs, -sn);
}

// ------------------------------------------------------------ butterflies --
template <bool INV>
__device__ __forceinline__ void dft2(float2 *x) {
    const float2 a = x[0], b = x[1];
    x[0] = cadd(a, b);
    x[1] = csub(a, b);
}

template <bool INV>
__device__ __forceinline__ void dft4(float2 *x) {
    const float2 s02 = cadd(x[0], x[2]), d02 = csub(x[0], x[2]);
    const float2 s13 = cadd(x[1], x[3]), d13 = rot90<INV>(csub(x[1], x[3]));
    x[0] = cadd(s02, s13);
    x[2] = csub(s02, s13);
    x[1] = cadd(d02, d13);
    x[3] = csub(d02, d13);
}

template <bool INV>
__device__ __forceinline__ void dft3(float2 *x) {
    const float s3 = 0.86602540378443864676f;
    const float2 t1 = cadd(x[1], x[2]);
    const float2 t2 = csub(x[1], x[2]);
    const float2 y0 = cadd(x[0], t1);
    const float2 mm = make_float2(fmaf(-0.5f, t1.x, x[0].x), fmaf(-0.5f, t1.y, x[0].y));
    const float2 b = rot90<INV>(make_float2(s3 * t2.x, s3 * t2.y));
    x[0] = y0;
    x[1] = cadd(mm, b);
    x[2] = csub(mm, b);
}

template <bool INV>
__device__ __forceinline__ void dft5(float2 *x) {
    const float c1 = 0.30901699437494742410f, c2 = -0.80901699437494742410f;
    const float s1 = 0.95105651629515357212f, s2 = 0.58778525229247312917f;
    const float2 t1 = cadd(x[1], x[4]), t2 = cadd(x[2], x[3]);
    const float2 t3 = csub(x[1], x[4]), t4 = csub(x[2], x[3]);
    const float2 y0 = cadd(x[0], cadd(t1, t2));
    const float2 a1 = make_float2(fmaf(c2, t2.x, fmaf(c1, t1.x, x[0].x)), fmaf(c2, t2.y, fmaf(c1, t1.y, x[0].y)));
    const float2 a2 = make_float2(fmaf(c1, t2.x, fmaf(c2, t1.x, x[0].x)), fmaf(c1, t2.y, fmaf(c2, t1.y, x[0].y)));
    const float2 b1 = rot90<INV>(make_float2(fmaf(s1, t3.x, s2 * t4.x), fmaf(s1, t3.y, s2 * t4.y)));
    const float2 b2 = rot90<INV>(make_float2(fmaf(s2, t3.x, -s1 * t4.x), fmaf(s2, t3.y, -s1 * t4.y)));
    x[0] = y0;
    x[1] = cadd(a1, b1);
    x[4] = csub(a1, b1);
    x[2] = cadd(a2, b2);
    x[3] = csub(a2, b2);
}

template <int R, bool INV>
__device__ __forceinline__ void dft(float2 *x) {
    if (R == 2) dft2<INV>(x);
    else if (R == 3) dft3<INV>(x);
    else if (R == 4) dft4<INV>(x);
    else dft5<INV>(x);
}

// One radix-R stage over `nlines` independent lines of length P.
// DIF (forward): butterfly then twiddle.  DIT (inverse): conj twiddle then
// butterfly.  ROWMAP: consecutive threads walk along a line (contiguous rows);
// otherwise consecutive threads take consecutive lines (columns).
template <int R, bool INV, bool ROWMAP>
__device__ __forceinline__ void fft_stage(float2 *buf, int P, int L, int n_s, const float2 *tw,
                                          int nlines, int line_stride, int elem_stride) {
    const int per_line = P / R;
    const int total = nlines * per_line;
    const int tstep = P / n_s;
    for (int b = threadIdx.x; b < total; b += MT) {
        int line, q;
        if (ROWMAP) {
            line = b / per_line;
            q = b - line * per_line;
        } else {
            q = b / nlines;
            line = b - q * nlines;
        }
        const int seg = q / L, j = q - seg * L;
        float2 *p = buf + line * line_stride + (seg * n_s + j) * elem_stride;
        const int es = L * elem_stride;
        float2 x[R];
#pragma unroll
        for (int a = 0; a < R; ++a) x[a] = p[a * es];
        if (INV) {
#pragma unroll
            for (int a = 1; a < R; ++a) {
                const float2 t = tw[a * j * tstep];   // a*j < n_s, so the index is < P
                x[a] = cmul(x[a], make_float2(t.x, -t.y));
            }
            dft<R, INV>(x);
        } else {
            dft<R, INV>(x);
#pragma unroll
            for (int a = 1; a < R; ++a) x[a] = cmul(x[a], tw[a * j * tstep]);
        }
#pragma unroll
        for (int a = 0; a < R; ++a) p[a * es] = x[a];
    }
}

template <bool INV, bool ROWMAP>
__device__ void fft_lines(float2 *buf, const FftDim &d, const float2 *tw, int nlines, int line_stride,
                          int elem_stride) {
    if (!INV) {
        int n_s = d.P;
        for (int s = 0; s < d.ns; ++s) {
            const int R = d.rad[s], L = n_s / R;
            switch (R) {
                case 2: fft_stage<2, INV, ROWMAP>(buf, d.P, L, n_s, tw, nlines, line_stride, elem_stride); break;
                case 3: fft_stage<3, INV, ROWMAP>(buf, d.P, L, n_s, tw, nlines, line_stride, elem_stride); break;
                case 4: fft_stage<4, INV, ROWMAP>(buf, d.P, L, n_s, tw, nlines, line_stride, elem_stride); break;
                default: fft_stage<5, INV, ROWMAP>(buf, d.P, L, n_s, tw, nlines, line_stride, elem_stride); break;
            }
            n_s = L;
            __syncthreads();
        }
    } else {
        int nss[kMaxStages];
        int n_s = d.P;
        for (int s = 0; s < d.ns; ++s) {
            nss[s] = n_s;
            n_s /= d.rad[s];
        }
        for (int s = d.ns - 1; s >= 0; --s) {
            const int R = d.rad[s], L = nss[s] / R;
            switch (R) {
                case 2: fft_stage<2, INV, ROWMAP>(buf, d.P, L, nss[s], tw, nlines, line_stride, elem_stride); break;
                case 3: fft_stage<3, INV, ROWMAP>(buf, d.P, L, nss[s], tw, nlines, line_stride, elem_stride); break;
                case 4: fft_stage<4, INV, ROWMAP>(buf, d.P, L, nss[s], tw, nlines, line_stride, elem_stride); break;
                default: fft_stage<5, INV, ROWMAP>(buf, d.P, L, nss[s], tw, nlines, line_stride, elem_stride); break;
            }
            __syncthreads();
        }
    }
}

// digit-reversed position of frequency f after the DIF passes
__device__ __forceinline__ int dif_position(int f, const FftDim &d) {
    int p = 0, n = d.P;
    for (int s = 0; s < d.ns; ++s) {
        const int R = d.rad[s];
        const int a = f % R;
        f /= R;
        n /= R;
        p += a * n;
    }
    return p;
}

// ------------------------------------------------------------ reductions --
template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Block-wide sum (fixed tree: deterministic).  `red` holds MT/32 values.
template <typename T>
__device__ T block_sum(T v, T *red) {
    v = warp_sum(v);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) red[warp] = v;
    __syncthreads();
    T t = (threadIdx.x < MT / 32) ? red[threadIdx.x] : T(0);
    if (warp == 0) t = warp_sum(t);
    if (threadIdx.x == 0) red[0] = t;
    __syncthreads();
    const T r = red[0];
    __syncthreads();
    return r;
}

// Block-wide argmin over (value, index): smaller value, then smaller index.
__device__ void block_argmin(float v, int idx, float *redv, int *redi, float &bv, int &bi) {
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
        for (int w = 1; w < MT / 32; ++w)
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
__device__ void subpixel_fit(const double *f, double &ox, double &oy) {
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

// ------------------------------------------------------------------ kernel --
__global__ void __launch_bounds__(MT, 1) match_fft_kernel(const MatchArgs A) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ float red_f[MT / 32];
    __shared__ int red_i[MT / 32];
    __shared__ double red_d[MT / 32];
    __shared__ int cand_n;
    __shared__ int cand_idx[kCandBuf];
    __shared__ float cand_val[kCandBuf];
    __shared__ double cand_ssd[kMaxCand];
    __shared__ MatchPlan s_plan;
    __shared__ int s_ok;

    const int cp = blockIdx.x;
    if (cp >= A.n) return;
    const int tid = threadIdx.x;
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
    const bool inside = N >= 1 && r >= 0 && N <= A.tmpl_max && r <= A.radius_max && ry0 >= 0 && rx0 >= 0 && ry0 + N <= A.ref_h &&
                        rx0 + N <= A.ref_w && sy0 >= 0 && sx0 >= 0 &&
                        sy0 + N + 2 * r <= A.sen_h && sx0 + N + 2 * r <= A.sen_w;
    if (!inside) {
        if (tid == 0) A.out[cp] = res;
        return;
    }
    // plan search: lanes 0..15 of warp 0 each cost one block split
    if (tid < 32) {
        MatchPlan p;
        long long c = -1;
        if (tid < kNbMax * kNbMax) c = plan_for_split(N, r, m, tid / kNbMax + 1, tid % kNbMax + 1, &p);
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
        if (tid == bl && c >= 0) s_plan = p;
        if (tid == 0) s_ok = bc != LLONG_MAX;
    }
    __syncthreads();
    if (!s_ok) {
        if (tid == 0) A.out[cp] = res;
        return;
    }
    const MatchPlan plan = s_plan;
    const FftDim &dy_ = plan.y;
    const FftDim &dx_ = plan.x;
    const int Py = dy_.P, Px = dx_.P, ld = Px;
    const int Hx = Px / 2 + 1;

    float2 *plane = reinterpret_cast<float2 *>(smem_raw);
    float2 *X = plane + Py * Px;
    float2 *twx = X + Py * Hx;
    float2 *twy = twx + kMaxFft;
    int *posx = reinterpret_cast<int *>(twy + kMaxFft);
    int *posy = posx + kMaxFft;
    float *surf = reinterpret_cast<float *>(X);   // reused after the inverse FFT

    for (int i = tid; i < Px; i += MT) {
        twx[i] = twiddle(i, Px);
        posx[i] = dif_position(i, dx_);
    }
    for (int i = tid; i < Py; i += MT) {
        twy[i] = twiddle(i, Py);
        posy[i] = dif_position(i, dy_);
    }
    for (int i = tid; i < Py * Hx; i += MT) X[i] = make_float2(0.f, 0.f);
    __syncthreads();

    float tt_part = 0.f;   // sum T^2, per thread
    for (int iby = 0; iby < dy_.nb; ++iby) {
        const int by0 = iby * dy_.bs;
        const int bh = min(dy_.bs, N - by0);
        for (int ibx = 0; ibx < dx_.nb; ++ibx) {
            const int bx0 = ibx * dx_.bs;
            const int bw = min(dx_.bs, N - bx0);
            const int wh = bh + 2 * r, ww = bw + 2 * r;
            for (int k = 0; k <= m; ++k) {
                const bool feat = k < m;
                const float *tsrc = A.ref + (int64_t)k * A.ref_pp;
                const float *wsrc = feat ? A.sen + (int64_t)k * A.sen_pp : A.sen_sq;
                for (int e = tid; e < Py * Px; e += MT) {
                    const int y = e / Px, x = e - y * Px;
                    float re = 0.f, im = 0.f;
                    if (y < bh && x < bw) {
                        if (feat) {
                            re = __ldg(tsrc + (int64_t)(ry0 + by0 + y) * A.ref_rp + (rx0 + bx0 + x));
                            tt_part = fmaf(re, re, tt_part);
                        } else {
                            re = 1.f;
                        }
                    }
                    if (y < wh && x < ww)
                        im = __ldg(wsrc + (int64_t)(sy0 + by0 + y) * A.sen_rp + (sx0 + bx0 + x));
                    plane[e] = make_float2(re, im);
                }
                __syncthreads();
                // forward 2-D FFT: rows that hold data, then all columns
                fft_lines<false, true>(plane, dx_, twx, min(Py, wh), ld, 1);
                fft_lines<false, false>(plane, dy_, twy, Px, 1, ld);
                // separate the spectra of T and S and accumulate w * conj(T) S
                const float wgt = feat ? -0.5f : 0.25f;   // (-2 or +1) / 4
                for (int it = tid; it < Py * Hx; it += MT) {
                    const int fy = it / Hx, fx = it - fy * Hx;
                    const float2 z1 = plane[posy[fy] * ld + posx[fx]];
                    const int gy = fy ? Py - fy : 0, gx = fx ? Px - fx : 0;
                    const float2 z2 = plane[posy[gy] * ld + posx[gx]];
                    const float2 t2 = make_float2(z1.x + z2.x, z1.y - z2.y);     // 2 T
                    const float2 s2 = make_float2(z1.y + z2.y, z2.x - z1.x);     // 2 S
                    const float2 c = make_float2(fmaf(t2.x, s2.x, t2.y * s2.y),
                                                 fmaf(t2.x, s2.y, -t2.y * s2.x));  // conj(2T) 2S
                    float2 acc = X[it];
                    acc.x = fmaf(wgt, c.x, acc.x);
                    acc.y = fmaf(wgt, c.y, acc.y);
                    X[it] = acc;
                }
                __syncthreads();
            }
        }
    }

    // Hermitian completion into the plane (digit-reversed order), inverse FFT
    for (int it = tid; it < Py * Hx; it += MT) {
        const int fy = it / Hx, fx = it - fy * Hx;
        const float2 v = X[it];
        plane[posy[fy] * ld + posx[fx]] = v;
        if (fx != 0 && 2 * fx != Px) {
            const int gy = fy ? Py - fy : 0;
            plane[posy[gy] * ld + posx[Px - fx]] = make_float2(v.x, -v.y);
        }
    }
    __syncthreads();
    fft_lines<true, false>(plane, dy_, twy, Px, 1, ld);
    fft_lines<true, true>(plane, dx_, twx, Lside, ld, 1);

    const float tt = block_sum(tt_part, red_f);
    const float inv_area = 1.0f / ((float)Py * (float)Px);
    const int L2 = Lside * Lside;
    float bv = INFINITY;
    int bi = INT_MAX;
    for (int i = tid; i < L2; i += MT) {
        const int ly = i / Lside, lx = i - ly * Lside;
        const float s = tt + plane[ly * ld + lx].x * inv_area;
        surf[i] = s;
        if (s < bv || (s == bv && i < bi)) {
            bv = s;
            bi = i;
        }
    }
    if (tid == 0) cand_n = 0;
    float smin;
    int imin;
    block_argmin(bv, bi, red_f, red_i, smin, imin);

    // lags inside the nomination band are re-scored directly
    const float band = kRescoreRel * (tt + (float)N * (float)N);
    for (int i = tid; i < L2; i += MT) {
        if (surf[i] <= smin + band) {
            const int slot = atomicAdd(&cand_n, 1);
            if (slot < kCandBuf) {
                cand_idx[slot] = i;
                cand_val[slot] = surf[i];
            }
        }
    }
    __syncthreads();
    int ncand = min(cand_n, kCandBuf);
    if (tid == 0) {
        // order by (FFT value, index) and keep the best kMaxCand
        for (int a = 1; a < ncand; ++a) {
            const int ii = cand_idx[a];
            const float vv = cand_val[a];
            int b = a - 1;
            while (b >= 0 && (cand_val[b] > vv || (cand_val[b] == vv && cand_idx[b] > ii))) {
                cand_idx[b + 1] = cand_idx[b];
                cand_val[b + 1] = cand_val[b];
                --b;
            }
            cand_idx[b + 1] = ii;
            cand_val[b + 1] = vv;
        }
    }
    __syncthreads();
    ncand = min(ncand, kMaxCand);
    int win = imin;
    double win_ssd = (double)smin;
    if (ncand > 1) {
        const int NN = N * N;
        for (int c = 0; c < ncand; ++c) {
            const int li = cand_idx[c];
            const int vy = li / Lside - r, vx = li - (li / Lside) * Lside - r;
            double acc = 0.0;
            for (int e = tid; e < m * NN; e += MT) {
                const int k = e / NN, rem = e - k * NN;
                const int y = rem / N, x = rem - y * N;
                const float a = __ldg(A.ref + (int64_t)k * A.ref_pp + (int64_t)(ry0 + y) * A.ref_rp + (rx0 + x));
                const float b = __ldg(A.sen + (int64_t)k * A.sen_pp +
                                      (int64_t)(sy0 + r + vy + y) * A.sen_rp + (sx0 + r + vx + x));
                const float d = a - b;
                acc += (double)(d * d);
            }
            const double s = block_sum(acc, red_d);
            if (tid == 0) cand_ssd[c] = s;
        }
        __syncthreads();
        if (tid == 0) {
            int bc = 0;
            for (int c = 1; c < ncand; ++c)
                if (cand_ssd[c] < cand_ssd[bc] || (cand_ssd[c] == cand_ssd[bc] && cand_idx[c] < cand_idx[bc]))
                    bc = c;
            red_i[0] = cand_idx[bc];
            red_d[0] = cand_ssd[bc];
        }
        __syncthreads();
        win = red_i[0];
        win_ssd = red_d[0];
    }

    if (A.surface) {
        const int Lmax = A.surf_side;
        float *dst = A.surface + (int64_t)cp * Lmax * Lmax;
        const int off = (Lmax - Lside) / 2;
        for (int i = tid; i < L2; i += MT) {
            const int ly = i / Lside, lx = i - ly * Lside;
            dst[(ly + off) * Lmax + (lx + off)] = surf[i];
        }
    }

    if (tid == 0) {
        const int vy = win / Lside - r, vx = win - (win / Lside) * Lside - r;
        res.dx = qx + vx;
        res.dy = qy + vy;
        res.ssd = (float)win_ssd;
        double ox = 0.0, oy = 0.0;
        if (vx == -r || vx == r || vy == -r || vy == r) {
            res.status = CFOG_CP_EDGE_PEAK;
        } else {
            double f[9];
            for (int j = -1; j <= 1; ++j)
                for (int i = -1; i <= 1; ++i) f[(j + 1) * 3 + (i + 1)] = (double)surf[(vy + r + j) * Lside + (vx + r + i)];
            subpixel_fit(f, ox, oy);
            res.status = CFOG_CP_OK;
        }
        res.sub_dx = (float)((double)res.dx + ox);
        res.sub_dy = (float)((double)res.dy + oy);
        A.out[cp] = res;
    }
}

// Host-side plan cache: the largest shared-memory need over all (N, r) up to
// the launch bounds, memoised per (tmpl_max, radius_max, m).
int max_plan_smem(int tmpl_max, int radius_max, int m) {
    static std::mutex mu;
    static int cache[kMaxFft + 1][33];
    static int cache_m[kMaxFft + 1][33];
    std::lock_guard<std::mutex> lock(mu);
    if (cache_m[tmpl_max][radius_max] == m && cache[tmpl_max][radius_max] > 0)
        return cache[tmpl_max][radius_max];
    int best = 0;
    for (int N = 1; N <= tmpl_max; ++N)
        for (int r = 0; r <= radius_max; ++r) {
            MatchPlan p;
            if (!make_plan_host(N, r, m, &p)) return -1;
            const int b = plan_smem_bytes(p);
            best = b > best ? b : best;
        }
    cache[tmpl_max][radius_max] = best;
    cache_m[tmpl_max][radius_max] = m;
    return best;
}

}  // namespace
}  // namespace cfog

extern "C" cfog_status cfog_match(const cfog_features *ref, const cfog_features *sen,
                                  const cfog_point *cps_dev, int32_t n, const int32_t *tmpl_dev,
                                  const int32_t *radius_dev, int32_t tmpl_max, int32_t radius_max,
                                  const cfog_point *prior_dev, int32_t precision,
                                  cfog_match_result *out_dev, float *surface_dev, void *stream) {
    using namespace cfog;
    CFOG_REQUIRE(ref && sen, "cfog_match: ref and sen must be non-NULL");
    CFOG_REQUIRE(n >= 0, "cfog_match: n = %d < 0", n);
    if (n == 0) return CFOG_OK;
    CFOG_REQUIRE(ref->data && sen->data && sen->sqnorm, "cfog_match: null feature pointer");
    CFOG_REQUIRE(cps_dev && tmpl_dev && radius_dev && out_dev, "cfog_match: null CP array");
    CFOG_REQUIRE(ref->m == sen->m && ref->m >= 1 && ref->m <= 64, "cfog_match: channel counts %d/%d",
                 ref->m, sen->m);
    CFOG_REQUIRE(tmpl_max >= 1 && tmpl_max <= kMaxFft, "cfog_match: tmpl_max %d outside [1, %d]",
                 tmpl_max, kMaxFft);
    CFOG_REQUIRE(radius_max >= 0 && radius_max <= 32, "cfog_match: radius_max %d outside [0, 32]",
                 radius_max);
    CFOG_REQUIRE(n <= (1 << 30), "cfog_match: n too large");
    if (precision == CFOG_PREC_BF16_DIRECT) {
        set_error("cfog_match: BF16 direct precision is not available in this build");
        return CFOG_E_UNSUPPORTED;
    }
    CFOG_REQUIRE(precision == CFOG_PREC_FP32_FFT, "cfog_match: unknown precision %d", precision);

    const int smem = max_plan_smem(tmpl_max, radius_max, ref->m);
    CFOG_REQUIRE(smem > 0, "cfog_match: no FFT plan for tmpl_max %d radius_max %d", tmpl_max,
                 radius_max);
    cfog_status fs = ensure_dynamic_smem(reinterpret_cast<const void *>(match_fft_kernel), smem,
                                         "cfog_match");
    if (fs != CFOG_OK) return fs;

    MatchArgs a;
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
    match_fft_kernel<<<n, MT, smem, as_stream(stream)>>>(a);
    return check_launch("cfog_match: launch");
}

extern "C" cfog_status cfog_plan_info(int32_t tmpl, int32_t radius, int32_t m, int32_t *out8) {
    using namespace cfog;
    CFOG_REQUIRE(out8, "cfog_plan_info: out8 is NULL");
    CFOG_REQUIRE(tmpl >= 1 && tmpl <= kMaxFft && radius >= 0 && radius <= 32 && m >= 1 && m <= 64,
                 "cfog_plan_info: (N=%d, r=%d, m=%d) outside the supported range", tmpl, radius, m);
    MatchPlan p;
    CFOG_REQUIRE(make_plan_host(tmpl, radius, m, &p), "cfog_plan_info: no plan");
    out8[0] = p.y.nb;
    out8[1] = p.x.nb;
    out8[2] = p.y.P;
    out8[3] = p.x.P;
    out8[4] = p.y.bs;
    out8[5] = p.x.bs;
    out8[6] = p.y.ns + p.x.ns;
    out8[7] = plan_smem_bytes(p);
    return CFOG_OK;
}
