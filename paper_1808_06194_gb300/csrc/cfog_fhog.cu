// K10: pixel-wise HOG (Sec. III-C), the FHOG descriptor of the framework.
//
// At every pixel, a block centred on it of 2 x 2 cells of C x C pixels; the
// gradient orientation in [0, 180) degrees is quantised into 9 bins; each
// block pixel adds its gradient magnitude to the bins next to its position and
// orientation by trilinear interpolation, and the 36 bins are L2-normalised.
// The spatial part of the interpolation is a bilinear weight between the two
// cell centres of an axis, at -C/2 and +C/2 from the pixel, over block offsets
// -C..C; the orientation part is the two-bin split of the first orientation
// scheme of Sec. III-F (bins centred on k*pi/9).  Both are separable, so the
// block histogram of every pixel is a correlation of the 9 binned channels
// with one 1-D cell kernel per axis, computed once per tile:
//   phase 0  input tile + halo of C+1 pixels in shared memory,
//   phase 1  (magnitude, orientation in bin widths) on the (TH+2C) x (TW+2C)
//            gradient region,
//   phase 2  binned channels formed in registers, correlated along x with the
//            two cell kernels -> 18 planes (bin, cell column) in shared memory,
//   phase 3  correlation along y with the two cell kernels -> 36 values per
//            pixel in registers, L2 normalisation, stores of the 36 planes and
//            the ||D||^2 plane.
// Replicate borders: every gradient-region cell stands for the clamped image
// pixel, so block pixels outside the image repeat the edge pixel.
#include "cfog_internal.cuh"
#include "cfog_orient.cuh"

#include <cmath>
#include <cstdint>

namespace cfog {
namespace {

constexpr int FW = 32;      // output tile width
constexpr int FH = 16;      // output tile height
constexpr int FNT = 256;    // threads per CTA
constexpr int FRUN = 4;     // outputs per phase-2 work item
constexpr int FM = 9;       // orientation bins
constexpr int FD = 36;      // 2 x 2 cells x 9 bins
constexpr int FSTRIP = 2;   // rows per phase-3 work item

template <int C>
struct FSmem {
    static constexpr int GH = FH + 2 * C;        // gradient / x-pass rows
    static constexpr int GW = FW + 2 * C;        // gradient columns
    static constexpr int IH = GH + 2;            // input tile rows
    static constexpr int IW = GW + 2;            // input tile columns
    static constexpr int GXY_BYTES = GH * GW * 8;
    static constexpr int HX_FLOATS = 2 * FM * GH * FW;   // [bin][cell column][GH][FW]
    static constexpr int BYTES = GXY_BYTES + HX_FLOATS * 4;
    static_assert(IH * IW <= HX_FLOATS, "input tile aliases the x-pass buffer");
};

// Weight of block offset d in [-C, C] for the cell centred at -C/2 (cell 0)
// or +C/2 (cell 1): 1 - |d - centre| / C, zero when negative.  Exact in FP32
// for C = 4 and 8.
template <int C>
__device__ __forceinline__ constexpr float cell_w(int cell, int d) {
    const float c = cell ? 0.5f * (float)C : -0.5f * (float)C;
    const float v = 1.f - ((float)d - c < 0.f ? c - (float)d : (float)d - c) / (float)C;
    return v > 0.f ? v : 0.f;
}

__device__ __forceinline__ int clampi_f(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

template <typename T>
__device__ __forceinline__ float load_px_f(const T *p) { return static_cast<float>(__ldg(p)); }

template <int C, typename TIn>
// 32 x 16 tiles: ~86 KB of shared memory and at most 128 registers, so two
// CTAs share an SM
__global__ void __launch_bounds__(FNT, 2)
fhog_kernel(const TIn *__restrict__ img, int h, int w, int64_t pitch, float *__restrict__ out,
            float *__restrict__ sqn, int64_t row_pitch, int64_t plane_pitch, float eps) {
    using S = FSmem<C>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float2 *gmt = reinterpret_cast<float2 *>(smem_raw);                       // [GH][GW]
    float *hx = reinterpret_cast<float *>(smem_raw + S::GXY_BYTES);           // [FM][2][GH][FW]
    float *tile = hx;                                                         // [IH][IW], phases 0-1

    const int tid = threadIdx.x;
    const int x0 = blockIdx.x * FW, y0 = blockIdx.y * FH;
    const int oy = y0 - (C + 1), ox = x0 - (C + 1);

    // phase 0: input tile at clamped coordinates
    for (int i = tid; i < S::IH * S::IW; i += FNT) {
        const int ty = i / S::IW, tx = i - ty * S::IW;
        const int gy = clampi_f(oy + ty, 0, h - 1), gx = clampi_f(ox + tx, 0, w - 1);
        tile[i] = load_px_f(img + (int64_t)gy * pitch + gx);
    }
    __syncthreads();

    // phase 1: gradients of the clamped image pixel of each gradient cell,
    // kept as (magnitude, orientation in bin widths)
    for (int i = tid; i < S::GH * S::GW; i += FNT) {
        const int j = i / S::GW, c = i - j * S::GW;
        const int cy = clampi_f(y0 - C + j, 0, h - 1), cx = clampi_f(x0 - C + c, 0, w - 1);
        const int yu = clampi_f(cy - 1, 0, h - 1) - oy, yd = clampi_f(cy + 1, 0, h - 1) - oy;
        const int xl = clampi_f(cx - 1, 0, w - 1) - ox, xr = clampi_f(cx + 1, 0, w - 1) - ox;
        const int ty = cy - oy, tx = cx - ox;
        const float gxv = tile[ty * S::IW + xr] - tile[ty * S::IW + xl];
        const float gyv = tile[yd * S::IW + tx] - tile[yu * S::IW + tx];
        gmt[i] = grad_cell<CFOG_ORIENT_BINS, FM>(gxv, gyv);
    }
    __syncthreads();

    // phase 2: binned channels in registers, correlated along x with the two
    // cell kernels
    constexpr int NRUN = FW / FRUN;
    constexpr int SPAN = FRUN + 2 * C;
    for (int it = tid; it < S::GH * NRUN; it += FNT) {
        const int j = it / NRUN, q = it - j * NRUN;
        const float2 *src = gmt + j * S::GW + q * FRUN;
        float mg[SPAN], tt[SPAN];
#pragma unroll
        for (int u = 0; u < SPAN; ++u) {
            const float2 v = src[u];
            mg[u] = v.x;
            tt[u] = v.y;
        }
#pragma unroll
        for (int k = 0; k < FM; ++k) {
            float g[SPAN];
#pragma unroll
            for (int u = 0; u < SPAN; ++u) g[u] = bin_w<FM>(tt[u], k) * mg[u];
#pragma unroll
            for (int cell = 0; cell < 2; ++cell) {
                float o[FRUN];
#pragma unroll
                for (int cc = 0; cc < FRUN; ++cc) {
                    float acc = 0.f;
#pragma unroll
                    for (int d = -C; d <= C; ++d) {
                        const float wv = cell_w<C>(cell, d);
                        if (wv != 0.f) acc = fmaf(wv, g[cc + C + d], acc);
                    }
                    o[cc] = acc;
                }
                *reinterpret_cast<float4 *>(hx + ((k * 2 + cell) * S::GH + j) * FW + q * FRUN) =
                    make_float4(o[0], o[1], o[2], o[3]);
            }
        }
    }
    __syncthreads();

    // phase 3: correlation along y, L2 normalisation, stores
    const int c = tid % FW;
    const int x = x0 + c;
    for (int s0 = tid / FW; s0 * FSTRIP < FH; s0 += FNT / FW) {
        const int r0 = s0 * FSTRIP;
        float v[FD][FSTRIP];
#pragma unroll
        for (int k = 0; k < FM; ++k) {
#pragma unroll
            for (int cx = 0; cx < 2; ++cx) {
                float col[FSTRIP + 2 * C];
#pragma unroll
                for (int u = 0; u < FSTRIP + 2 * C; ++u) col[u] = hx[((k * 2 + cx) * S::GH + r0 + u) * FW + c];
#pragma unroll
                for (int cy = 0; cy < 2; ++cy) {
#pragma unroll
                    for (int i = 0; i < FSTRIP; ++i) {
                        float acc = 0.f;
#pragma unroll
                        for (int d = -C; d <= C; ++d) {
                            const float wv = cell_w<C>(cy, d);
                            if (wv != 0.f) acc = fmaf(wv, col[i + C + d], acc);
                        }
                        v[(cy * 2 + cx) * FM + k][i] = acc;
                    }
                }
            }
        }
        if (x >= w) continue;
#pragma unroll
        for (int i = 0; i < FSTRIP; ++i) {
            const int y = y0 + r0 + i;
            if (y >= h) break;
            float ss = 0.f;
#pragma unroll
            for (int e = 0; e < FD; ++e) ss = fmaf(v[e][i], v[e][i], ss);
            const float inv = 1.0f / (sqrtf(ss) + eps);
            float dd = 0.f;
            float *o = out + (int64_t)y * row_pitch + x;
#pragma unroll
            for (int e = 0; e < FD; ++e) {
                const float dv = v[e][i] * inv;
                dd = fmaf(dv, dv, dd);
                __stcs(o + e * plane_pitch, dv);
            }
            __stcs(sqn + (int64_t)y * row_pitch + x, dd);
        }
    }
}

template <int C, typename TIn>
cfog_status launch_fhog(const cfog_image *img, const cfog_features *out, float eps, cudaStream_t st) {
    auto kern = fhog_kernel<C, TIn>;
    constexpr int bytes = FSmem<C>::BYTES;
    cfog_status fs = ensure_dynamic_smem(reinterpret_cast<const void *>(kern), bytes, "cfog_extract_fhog");
    if (fs != CFOG_OK) return fs;
    dim3 grid((img->w + FW - 1) / FW, (img->h + FH - 1) / FH);
    kern<<<grid, FNT, bytes, st>>>(static_cast<const TIn *>(img->data), img->h, img->w, img->pitch,
                                   out->data, out->sqnorm, out->row_pitch, out->plane_pitch, eps);
    return check_launch("cfog_extract_fhog: launch");
}

template <int C>
cfog_status fhog_dtype(const cfog_image *img, const cfog_features *out, float eps, cudaStream_t st) {
    if (img->dtype == CFOG_DTYPE_F32) return launch_fhog<C, float>(img, out, eps, st);
    return launch_fhog<C, uint16_t>(img, out, eps, st);
}

}  // namespace
}  // namespace cfog

extern "C" cfog_status cfog_extract_fhog(const cfog_image *img, int32_t cell, float eps,
                                         const cfog_features *out, void *stream) {
    CFOG_TRACE("cfog_extract_fhog");
    using namespace cfog;
    const char *who = "cfog_extract_fhog";
    CFOG_REQUIRE(img && out, "%s: img and out must be non-NULL", who);
    CFOG_REQUIRE(img->data && out->data && out->sqnorm, "%s: null data pointer", who);
    CFOG_REQUIRE(img->h > 0 && img->w > 0, "%s: empty image %dx%d", who, img->h, img->w);
    CFOG_REQUIRE(img->pitch >= img->w, "%s: pitch %lld < width %d", who, (long long)img->pitch, img->w);
    CFOG_REQUIRE(img->dtype == CFOG_DTYPE_F32 || img->dtype == CFOG_DTYPE_U16, "%s: unknown dtype %d",
                 who, img->dtype);
    CFOG_REQUIRE(out->m == 36 && out->h == img->h && out->w == img->w,
                 "%s: output %dx%dx%d, need 36 x %d x %d", who, out->m, out->h, out->w, img->h, img->w);
    CFOG_REQUIRE(out->row_pitch >= out->w && out->plane_pitch >= out->row_pitch * out->h,
                 "%s: bad output pitches", who);
    CFOG_REQUIRE(eps >= 0.f, "%s: eps must be >= 0", who);
    CFOG_REQUIRE(img->h <= (1 << 24) && img->w <= (1 << 24), "%s: image too large", who);
    cudaStream_t st = as_stream(stream);
    if (cell == 8) return fhog_dtype<8>(img, out, eps, st);
    if (cell == 4) return fhog_dtype<4>(img, out, eps, st);
    set_error("%s: cell %d not compiled (4, 8)", who, cell);
    return CFOG_E_UNSUPPORTED;
}
