// Register-resident DFTs of small composite sizes for the shared-memory FFTs
// of the matcher.  rdft<R, INV>(x) transforms R complex values held in
// registers and leaves the result in natural order:
//     forward  y_f = sum_a x_a exp(-2 pi i a f / R)
//     inverse  y_f = sum_a x_a exp(+2 pi i a f / R)   (unnormalised)
// Prime sizes 2, 3, 5 and size 4 are written out; a composite R = R1 * R2 is
// one decimation-in-frequency step (R1-point DFTs at stride R2, twiddles,
// R2-point DFTs) followed by a compile-time reordering.  All indices are
// compile-time constants after unrolling, so x stays in registers.
#pragma once

#include <cuda_runtime.h>

namespace cfog {

// ------------------------------------------------- compile-time sin / cos --
// Taylor series on [-pi, pi]; 30 terms are far below double rounding there.
constexpr double kPiD = 3.14159265358979323846264338327950288;

constexpr double cx_sin(double x) {
    double term = x, sum = x;
    for (int n = 1; n < 30; ++n) {
        term *= -x * x / ((2.0 * n) * (2.0 * n + 1.0));
        sum += term;
    }
    return sum;
}

constexpr double cx_cos(double x) {
    double term = 1.0, sum = 1.0;
    for (int n = 1; n < 30; ++n) {
        term *= -x * x / ((2.0 * n - 1.0) * (2.0 * n));
        sum += term;
    }
    return sum;
}

// exp(-2 pi i k / R) for k in [0, R): real and imaginary parts
constexpr double tw_angle(int k, int R) {
    double a = 2.0 * kPiD * (double)(k % R) / (double)R;
    return a > kPiD ? a - 2.0 * kPiD : a;
}
constexpr float tw_re(int k, int R) { return (float)cx_cos(tw_angle(k, R)); }
constexpr float tw_im(int k, int R) { return (float)(-cx_sin(tw_angle(k, R))); }

template <int R>
struct TwTable {
    float re[R > 0 ? R : 1];
    float im[R > 0 ? R : 1];
    constexpr TwTable() : re(), im() {
        for (int k = 0; k < R; ++k) {
            re[k] = tw_re(k, R);
            im[k] = tw_im(k, R);
        }
    }
};

// ------------------------------------------------------------- complex ops --
// Complex add and subtract as packed FP32x2 operations (one instruction for
// both parts, same rounding as two scalar operations; a - b is b * -1 + a with
// an exact product).
__device__ __forceinline__ float2 c_add(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 c_sub(float2 a, float2 b) {
    return __ffma2_rn(b, make_float2(-1.f, -1.f), a);
}
__device__ __forceinline__ float2 c_mul(float2 a, float2 b) {
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ float2 c_mul_conj(float2 a, float2 b) {  // a * conj(b)
    return make_float2(fmaf(a.x, b.x, a.y * b.y), fmaf(a.y, b.x, -a.x * b.y));
}
// multiply by -i (forward) or +i (inverse)
template <bool INV>
__device__ __forceinline__ float2 c_rot(float2 a) {
    return INV ? make_float2(-a.y, a.x) : make_float2(a.y, -a.x);
}

// ------------------------------------------------------------ base kernels --
template <bool INV>
__device__ __forceinline__ void base2(float2 *x) {
    const float2 a = x[0], b = x[1];
    x[0] = c_add(a, b);
    x[1] = c_sub(a, b);
}

template <bool INV>
__device__ __forceinline__ void base3(float2 *x) {
    const float s3 = 0.86602540378443864676f;
    const float2 t1 = c_add(x[1], x[2]);
    const float2 t2 = c_sub(x[1], x[2]);
    const float2 y0 = c_add(x[0], t1);
    const float2 mm = make_float2(fmaf(-0.5f, t1.x, x[0].x), fmaf(-0.5f, t1.y, x[0].y));
    const float2 b = c_rot<INV>(make_float2(s3 * t2.x, s3 * t2.y));
    x[0] = y0;
    x[1] = c_add(mm, b);
    x[2] = c_sub(mm, b);
}

template <bool INV>
__device__ __forceinline__ void base4(float2 *x) {
    const float2 s02 = c_add(x[0], x[2]), d02 = c_sub(x[0], x[2]);
    const float2 s13 = c_add(x[1], x[3]), d13 = c_rot<INV>(c_sub(x[1], x[3]));
    x[0] = c_add(s02, s13);
    x[2] = c_sub(s02, s13);
    x[1] = c_add(d02, d13);
    x[3] = c_sub(d02, d13);
}

template <bool INV>
__device__ __forceinline__ void base5(float2 *x) {
    const float c1 = 0.30901699437494742410f, c2 = -0.80901699437494742410f;
    const float s1 = 0.95105651629515357212f, s2 = 0.58778525229247312917f;
    const float2 t1 = c_add(x[1], x[4]), t2 = c_add(x[2], x[3]);
    const float2 t3 = c_sub(x[1], x[4]), t4 = c_sub(x[2], x[3]);
    const float2 y0 = c_add(x[0], c_add(t1, t2));
    const float2 a1 = make_float2(fmaf(c2, t2.x, fmaf(c1, t1.x, x[0].x)), fmaf(c2, t2.y, fmaf(c1, t1.y, x[0].y)));
    const float2 a2 = make_float2(fmaf(c1, t2.x, fmaf(c2, t1.x, x[0].x)), fmaf(c1, t2.y, fmaf(c2, t1.y, x[0].y)));
    const float2 b1 = c_rot<INV>(make_float2(fmaf(s1, t3.x, s2 * t4.x), fmaf(s1, t3.y, s2 * t4.y)));
    const float2 b2 = c_rot<INV>(make_float2(fmaf(s2, t3.x, -s1 * t4.x), fmaf(s2, t3.y, -s1 * t4.y)));
    x[0] = y0;
    x[1] = c_add(a1, b1);
    x[4] = c_sub(a1, b1);
    x[2] = c_add(a2, b2);
    x[3] = c_sub(a2, b2);
}

// first factor of a composite size (the stride radix of its DIF step)
template <int R> struct Split { static constexpr int R1 = 1; };
template <> struct Split<6> { static constexpr int R1 = 2; };
template <> struct Split<8> { static constexpr int R1 = 2; };
template <> struct Split<9> { static constexpr int R1 = 3; };
template <> struct Split<10> { static constexpr int R1 = 2; };
template <> struct Split<12> { static constexpr int R1 = 4; };
template <> struct Split<15> { static constexpr int R1 = 3; };
template <> struct Split<16> { static constexpr int R1 = 4; };

template <int R, bool INV>
__device__ __forceinline__ void rdft(float2 *x);

template <int R, bool INV>
__device__ __forceinline__ void rdft_composite(float2 *x) {
    constexpr int R1 = Split<R>::R1;
    constexpr int R2 = R / R1;
    constexpr TwTable<R> tw{};
    float2 u[R];
#pragma unroll
    for (int j = 0; j < R2; ++j) {
        float2 col[R1];
#pragma unroll
        for (int a = 0; a < R1; ++a) col[a] = x[j + a * R2];
        rdft<R1, INV>(col);
#pragma unroll
        for (int a = 0; a < R1; ++a) {
            const int k = (a * j) % R;
            float2 w = make_float2(tw.re[k], INV ? -tw.im[k] : tw.im[k]);
            u[a * R2 + j] = (k == 0) ? col[a] : c_mul(col[a], w);
        }
    }
#pragma unroll
    for (int a = 0; a < R1; ++a) {
        float2 row[R2];
#pragma unroll
        for (int b = 0; b < R2; ++b) row[b] = u[a * R2 + b];
        rdft<R2, INV>(row);
#pragma unroll
        for (int b = 0; b < R2; ++b) x[a + R1 * b] = row[b];
    }
}

template <int R, bool INV>
__device__ __forceinline__ void rdft(float2 *x) {
    if constexpr (R == 1) {
    } else if constexpr (R == 2) {
        base2<INV>(x);
    } else if constexpr (R == 3) {
        base3<INV>(x);
    } else if constexpr (R == 4) {
        base4<INV>(x);
    } else if constexpr (R == 5) {
        base5<INV>(x);
    } else {
        rdft_composite<R, INV>(x);
    }
}

}  // namespace cfog
