// Per-pixel orientation binning shared by the CFOG kernel (first scheme of
// Sec. III-F, Fig. 7) and the pixel-wise HOG kernel (Sec. III-C): the
// gradient magnitude is shared between the two orientation bins next to the
// gradient's orientation, bins centred on k*pi/M and wrapping at pi.
#pragma once

#include <cuda_runtime.h>

#include "cfog.h"

namespace cfog {

constexpr float kPiF = 3.14159265358979f;

// What phase 1 keeps per gradient cell: (gx, gy) for Eq. 2; for the binned
// scheme the magnitude and the orientation folded into [0, pi) in bin widths,
// t in [0, M).
template <int ORI, int M>
__device__ __forceinline__ float2 grad_cell(float gx, float gy) {
    if constexpr (ORI == CFOG_ORIENT_BINS) {
        const float mag = sqrtf(fmaf(gx, gx, gy * gy));
        float phi = atan2f(gy, gx);
        if (phi < 0.f) phi += kPiF;
        float t = phi * ((float)M / kPiF);
        if (t >= (float)M) t -= (float)M;
        return make_float2(mag, t);
    } else {
        return make_float2(gx, gy);
    }
}

// Weight of bin k for orientation t (bin widths): 1 - circular distance,
// clamped at 0, so only the two bins next to t receive the magnitude.
template <int M>
__device__ __forceinline__ float bin_w(float t, int k) {
    float d = fabsf(t - (float)k);
    d = fminf(d, (float)M - d);
    return fmaxf(0.f, 1.f - d);
}

}  // namespace cfog
