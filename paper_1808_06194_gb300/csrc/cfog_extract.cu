// K1: fused CFOG extraction (Sec. III-F, Eq. 2, Fig. 9).
//
// One CTA produces a TH x TW tile of the CFOG volume.  The input tile plus a
// halo of R+1 pixels is staged in shared memory; then, without leaving the SM:
//   phase 1  gx, gy by [-1,0,1] on the (TH+2R) x (TW+2R) gradient region,
//   phase 2  one work item per (gradient row, channel pair): the two oriented
//            channels |cos t_k gx + sin t_k gy| (Eq. 2), or the binned
//            channels of the first scheme (Fig. 7), are formed once per
//            pixel of the row and filtered horizontally by the Gaussian in a
//            sliding register window,
//   phase 3  vertical Gaussian, circular [1,2,1] across k, L2 normalisation
//            and coalesced stores of the m planes and the ||D||^2 plane.
// Replicate borders: every gradient-region pixel stands for the clamped image
// pixel, so out-of-image taps repeat the edge value of the channel image,
// exactly as a separable filter with clamp-to-edge indexing does.
// The Z kernel is applied as [1,2,1] with the guard 4 eps in the norm: the
// same D as [1,2,1]/4 with eps, since scaling by 4 is exact in FP32.  The
// norm uses the approximate square-root and reciprocal units (a few ulp).
#include "cfog_internal.cuh"
#include "cfog_orient.cuh"

#include <cmath>
#include <cstdint>

namespace cfog {
namespace {

constexpr int TW = 32;       // output tile width (columns)
constexpr int TH = 32;       // output tile height (rows)
constexpr int NT = 256;      // threads per CTA
constexpr int STRIP = TH / (NT / TW);  // rows per thread in phase 3 (4)

struct ExtractArgs {
    float taps[9];   // normalised Gaussian taps, t = -R..R
    float cs[16];    // cos(k pi / m)
    float sn[16];    // sin(k pi / m)
    float eps;
};

__device__ __forceinline__ int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

template <typename T>
__device__ __forceinline__ float load_px(const T *p) { return static_cast<float>(__ldg(p)); }

// Four consecutive pixels from a 4-element-aligned address.
__device__ __forceinline__ float4 load4(const float *p) { return __ldg(reinterpret_cast<const float4 *>(p)); }
__device__ __forceinline__ float4 load4(const uint16_t *p) {
    const uint2 v = __ldg(reinterpret_cast<const uint2 *>(p));
    return make_float4((float)(v.x & 0xffffu), (float)(v.x >> 16), (float)(v.y & 0xffffu),
                       (float)(v.y >> 16));
}

// Shared-memory layout.  Row pitches are odd (in 8-byte units for the
// gradient plane and the channel-pair planes, in 4-byte units for the single
// channel of odd m), so that a warp walking down rows (phase 2) or across
// columns (phase 3) touches distinct banks.
template <int M, int R>
struct Smem {
    static constexpr int GH = TH + 2 * R;          // gradient / h-pass rows
    static constexpr int GW = TW + 2 * R;          // gradient columns
    static constexpr int GWP = GW | 1;             // gradient-plane row pitch (float2)
    static constexpr int HP = TW + 1;              // h-pass row pitch
    static constexpr int NPAIR = M / 2;            // channel pairs (2p, 2p+1)
    static constexpr int IH = TH + 2 * (R + 1);    // input tile rows
    static constexpr int IW = TW + 2 * (R + 1);    // input tile columns
    static constexpr int GXY_BYTES = GH * GWP * 8;
    static constexpr int PAIR_FLOATS = GH * HP * 2;   // one channel-pair plane
    static constexpr int HX_FLOATS = NPAIR * PAIR_FLOATS + (M & 1) * GH * HP;
    static constexpr int BYTES = GXY_BYTES + HX_FLOATS * 4;
    static_assert(IH * IW <= HX_FLOATS, "input tile aliases the h-pass buffer");
};

template <int M, int R, typename TIn, int ORI>
// 32 x 32 tiles: ~56 KB of shared memory and at most 64 registers, so four
// CTAs (32 warps) share an SM and hide each other's input-tile loads
__global__ void __launch_bounds__(NT, 4)
cfog_fused_kernel(const TIn *__restrict__ img, int h, int w, int64_t pitch,
                  float *__restrict__ out, float *__restrict__ sqn, int64_t row_pitch,
                  int64_t plane_pitch, int row0, int row1, const ExtractArgs args) {
    using S = Smem<M, R>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float2 *gxy = reinterpret_cast<float2 *>(smem_raw);                       // [GH][GWP]
    float *hx = reinterpret_cast<float *>(smem_raw + S::GXY_BYTES);           // pair planes, single plane
    float2 *hx2 = reinterpret_cast<float2 *>(hx);                             // [NPAIR][GH][HP]
    float *hx1 = hx + S::NPAIR * S::PAIR_FLOATS;                              // [GH][HP] (odd m)
    float *tile = hx;                                                         // [IH][IW], phase 0-1

    const int tid = threadIdx.x;
    const int x0 = blockIdx.x * TW;
    const int y0 = row0 + blockIdx.y * TH;
    const int oy = y0 - (R + 1);   // image row of tile row 0
    const int ox = x0 - (R + 1);

    // interior tiles need no border clamping
    const bool interior = ox >= 0 && oy >= 0 && ox + S::IW <= w && oy + S::IH <= h;

    // phase 0: stage the input tile (clamped coordinates); four pixels per
    // load where the rows allow aligned vector loads
    const bool vec = interior && (S::IW % 4) == 0 && (ox & 3) == 0 && (pitch & 3) == 0 &&
                     ((reinterpret_cast<uintptr_t>(img) & (4 * sizeof(TIn) - 1)) == 0);
    if (vec) {
        constexpr int QW = S::IW / 4;
        for (int i = tid; i < S::IH * QW; i += NT) {
            const int ty = i / QW, tq = i - ty * QW;
            reinterpret_cast<float4 *>(tile)[i] = load4(img + (int64_t)(oy + ty) * pitch + (ox + 4 * tq));
        }
    } else if (interior) {
        for (int i = tid; i < S::IH * S::IW; i += NT) {
            const int ty = i / S::IW, tx = i - ty * S::IW;
            tile[i] = load_px(img + (int64_t)(oy + ty) * pitch + (ox + tx));
        }
    } else {
        for (int i = tid; i < S::IH * S::IW; i += NT) {
            const int ty = i / S::IW, tx = i - ty * S::IW;
            const int gy = clampi(oy + ty, 0, h - 1), gx = clampi(ox + tx, 0, w - 1);
            tile[i] = load_px(img + (int64_t)gy * pitch + gx);
        }
    }
    __syncthreads();

    // phase 1: gradients at the clamped image pixel of each gradient-region cell
    if (interior) {
        for (int i = tid; i < S::GH * S::GW; i += NT) {
            const int j = i / S::GW, c = i - j * S::GW;
            const float *t = tile + (j + 1) * S::IW + (c + 1);
            gxy[j * S::GWP + c] = grad_cell<ORI, M>(t[1] - t[-1], t[S::IW] - t[-S::IW]);
        }
    } else {
        for (int i = tid; i < S::GH * S::GW; i += NT) {
            const int j = i / S::GW, c = i - j * S::GW;
            const int cy = clampi(y0 - R + j, 0, h - 1), cx = clampi(x0 - R + c, 0, w - 1);
            const int yu = clampi(cy - 1, 0, h - 1) - oy, yd = clampi(cy + 1, 0, h - 1) - oy;
            const int xl = clampi(cx - 1, 0, w - 1) - ox, xr = clampi(cx + 1, 0, w - 1) - ox;
            const int ty = cy - oy, tx = cx - ox;
            const float gxv = tile[ty * S::IW + xr] - tile[ty * S::IW + xl];
            const float gyv = tile[yd * S::IW + tx] - tile[yu * S::IW + tx];
            gxy[j * S::GWP + c] = grad_cell<ORI, M>(gxv, gyv);
        }
    }
    __syncthreads();

    // phase 2: per (gradient row j, channel pair p) the channels of the row's
    // GW pixels, each formed once, and the horizontal Gaussian of its TW
    // outputs from a sliding window of 2R+1 values.  Work items run j fastest
    // so that a warp shares p.  Odd m: the last item kind is the single
    // channel m-1.
    constexpr int KW = 2 * R + 1;
    constexpr int NKIND = (M + 1) / 2;
    for (int it = tid; it < S::GH * NKIND; it += NT) {
        const int p = it / S::GH, j = it - p * S::GH;
        const float2 *src = gxy + j * S::GWP;
        if (p < S::NPAIR) {
            const int k = 2 * p;
            const float2 c2 = make_float2(args.cs[k], args.cs[k + 1]);
            const float2 s2 = make_float2(args.sn[k], args.sn[k + 1]);
            auto chan = [&](int u) {
                const float2 v = src[u];
                if constexpr (ORI == CFOG_ORIENT_BINS) {
                    return make_float2(bin_w<M>(v.y, k) * v.x, bin_w<M>(v.y, k + 1) * v.x);
                } else {
                    float2 pr = __fmul2_rn(make_float2(v.x, v.x), c2);
                    pr = __ffma2_rn(make_float2(v.y, v.y), s2, pr);
                    return make_float2(fabsf(pr.x), fabsf(pr.y));
                }
            };
            float2 win[KW];
#pragma unroll
            for (int u = 0; u < KW - 1; ++u) win[u] = chan(u);
            float2 *dst = hx2 + (p * S::GH + j) * S::HP;
#pragma unroll
            for (int cc = 0; cc < TW; ++cc) {
                win[(cc + KW - 1) % KW] = chan(cc + KW - 1);
                float2 acc = make_float2(0.f, 0.f);
#pragma unroll
                for (int t = 0; t < KW; ++t)
                    acc = __ffma2_rn(make_float2(args.taps[t], args.taps[t]), win[(cc + t) % KW], acc);
                dst[cc] = acc;
            }
        } else {
            constexpr int k = M - 1;
            const float ck = args.cs[k], sk = args.sn[k];
            auto chan = [&](int u) {
                const float2 v = src[u];
                return ORI == CFOG_ORIENT_BINS ? bin_w<M>(v.y, k) * v.x : fabsf(fmaf(sk, v.y, ck * v.x));
            };
            float win[KW];
#pragma unroll
            for (int u = 0; u < KW - 1; ++u) win[u] = chan(u);
            float *dst = hx1 + j * S::HP;
#pragma unroll
            for (int cc = 0; cc < TW; ++cc) {
                win[(cc + KW - 1) % KW] = chan(cc + KW - 1);
                float acc = 0.f;
#pragma unroll
                for (int t = 0; t < KW; ++t) acc = fmaf(args.taps[t], win[(cc + t) % KW], acc);
                dst[cc] = acc;
            }
        }
    }
    __syncthreads();

    // phase 3: vertical Gaussian, Z kernel, L2 norm, stores
    const int c = tid % TW;
    const int r0 = (tid / TW) * STRIP;
    float v[M][STRIP];
#pragma unroll
    for (int p = 0; p < S::NPAIR; ++p) {
        float2 col[STRIP + 2 * R];
#pragma unroll
        for (int u = 0; u < STRIP + 2 * R; ++u) col[u] = hx2[(p * S::GH + r0 + u) * S::HP + c];
#pragma unroll
        for (int i = 0; i < STRIP; ++i) {
            float2 acc = make_float2(0.f, 0.f);
#pragma unroll
            for (int t = 0; t <= 2 * R; ++t)
                acc = __ffma2_rn(make_float2(args.taps[t], args.taps[t]), col[i + t], acc);
            v[2 * p][i] = acc.x;
            v[2 * p + 1][i] = acc.y;
        }
    }
    if (M & 1) {
        constexpr int k = M - 1;
        float col[STRIP + 2 * R];
#pragma unroll
        for (int u = 0; u < STRIP + 2 * R; ++u) col[u] = hx1[(r0 + u) * S::HP + c];
#pragma unroll
        for (int i = 0; i < STRIP; ++i) {
            float acc = 0.f;
#pragma unroll
            for (int t = 0; t <= 2 * R; ++t) acc = fmaf(args.taps[t], col[i + t], acc);
            v[k][i] = acc;
        }
    }
    const int x = x0 + c;
    if (x >= w) return;
    const float eps4 = 4.0f * args.eps;
#pragma unroll
    for (int i = 0; i < STRIP; ++i) {
        const int y = y0 + r0 + i;
        if (y >= row1) break;
        float hz[M];
        float ss = 0.f;
#pragma unroll
        for (int k = 0; k < M; ++k) {
            const int km = (k + M - 1) % M, kp = (k + 1) % M;
            hz[k] = v[km][i] + 2.0f * v[k][i] + v[kp][i];
            ss = fmaf(hz[k], hz[k], ss);
        }
        // 1 / (||h|| + 4 eps) from the approximate square root and reciprocal
        // units (a few ulp; the norm of a unit vector needs no more)
        const float nrm = ss > 0.f ? ss * rsqrtf(ss) : 0.f;
        const float inv = __fdividef(1.0f, nrm + eps4);
        float dd = 0.f;
        float *o = out + (int64_t)y * row_pitch + x;
#pragma unroll
        for (int k = 0; k < M; ++k) {
            const float d = hz[k] * inv;
            dd = fmaf(d, d, dd);
            __stcs(o + k * plane_pitch, d);
        }
        __stcs(sqn + (int64_t)y * row_pitch + x, dd);
    }
}

template <int M, int R, typename TIn, int ORI>
cfog_status launch_extract(const cfog_image *img, const cfog_features *out, const ExtractArgs &a,
                           int row0, int row1, cudaStream_t st) {
    auto kern = cfog_fused_kernel<M, R, TIn, ORI>;
    constexpr int bytes = Smem<M, R>::BYTES;
    cfog_status fs = ensure_dynamic_smem(reinterpret_cast<const void *>(kern), bytes, "cfog_extract");
    if (fs != CFOG_OK) return fs;
    dim3 grid((img->w + TW - 1) / TW, (row1 - row0 + TH - 1) / TH);
    kern<<<grid, NT, bytes, st>>>(static_cast<const TIn *>(img->data), img->h, img->w, img->pitch,
                                   out->data, out->sqnorm, out->row_pitch, out->plane_pitch, row0,
                                   row1, a);
    return check_launch("cfog_extract: launch");
}

template <int M, int R, int ORI>
cfog_status dispatch_dtype(const cfog_image *img, const cfog_features *out, const ExtractArgs &a,
                           int row0, int row1, cudaStream_t st) {
    if (img->dtype == CFOG_DTYPE_F32) return launch_extract<M, R, float, ORI>(img, out, a, row0, row1, st);
    return launch_extract<M, R, uint16_t, ORI>(img, out, a, row0, row1, st);
}

template <int M, int R>
cfog_status dispatch_dtype(int ori, const cfog_image *img, const cfog_features *out,
                           const ExtractArgs &a, int row0, int row1, cudaStream_t st) {
    if constexpr (R == 3) {
        if (ori == CFOG_ORIENT_BINS)
            return dispatch_dtype<M, R, CFOG_ORIENT_BINS>(img, out, a, row0, row1, st);
    } else if (ori == CFOG_ORIENT_BINS) {
        set_error("cfog_extract: the binned orientation scheme is compiled for gauss_radius 3 only");
        return CFOG_E_UNSUPPORTED;
    }
    return dispatch_dtype<M, R, CFOG_ORIENT_EQ2>(img, out, a, row0, row1, st);
}

template <int M>
cfog_status dispatch_radius(int R, int ori, const cfog_image *img, const cfog_features *out,
                            const ExtractArgs &a, int row0, int row1, cudaStream_t st) {
    switch (R) {
        case 2: return dispatch_dtype<M, 2>(ori, img, out, a, row0, row1, st);
        case 3: return dispatch_dtype<M, 3>(ori, img, out, a, row0, row1, st);
        case 4: return dispatch_dtype<M, 4>(ori, img, out, a, row0, row1, st);
    }
    set_error("cfog_extract: gauss_radius %d not compiled (2, 3, 4)", R);
    return CFOG_E_UNSUPPORTED;
}

}  // namespace
}  // namespace cfog

namespace cfog {
namespace {

cfog_status extract_impl(const cfog_image *img, const cfog_params *p, const cfog_features *out,
                         int row0, int row1, void *stream, const char *who) {
    cfog_params def;
    cfog_default_params(&def);
    if (!p) p = &def;
    CFOG_REQUIRE(img && out, "%s: img and out must be non-NULL", who);
    CFOG_REQUIRE(img->data && out->data && out->sqnorm, "%s: null data pointer", who);
    CFOG_REQUIRE(img->h > 0 && img->w > 0, "%s: empty image %dx%d", who, img->h, img->w);
    CFOG_REQUIRE(img->pitch >= img->w, "%s: pitch %lld < width %d", who, (long long)img->pitch,
                 img->w);
    CFOG_REQUIRE(img->dtype == CFOG_DTYPE_F32 || img->dtype == CFOG_DTYPE_U16,
                 "%s: unknown dtype %d", who, img->dtype);
    CFOG_REQUIRE(out->h == img->h && out->w == img->w && out->m == p->m,
                 "%s: output %dx%dx%d does not match image %dx%d, m=%d", who, out->m, out->h,
                 out->w, img->h, img->w, p->m);
    CFOG_REQUIRE(out->row_pitch >= out->w && out->plane_pitch >= out->row_pitch * out->h,
                 "%s: bad output pitches", who);
    CFOG_REQUIRE(p->sigma > 0.f && p->eps >= 0.f, "%s: sigma must be > 0, eps >= 0", who);
    CFOG_REQUIRE(p->orientation == CFOG_ORIENT_EQ2 || p->orientation == CFOG_ORIENT_BINS,
                 "%s: unknown orientation scheme %d", who, p->orientation);
    CFOG_REQUIRE(img->h <= (1 << 24) && img->w <= (1 << 24), "%s: image too large", who);
    CFOG_REQUIRE(row0 >= 0 && row0 <= row1 && row1 <= img->h, "%s: rows [%d, %d) outside [0, %d]",
                 who, row0, row1, img->h);
    if (row0 == row1) return CFOG_OK;

    ExtractArgs a{};
    const int R = p->gauss_radius;
    if (R >= 2 && R <= 4) {
        double sum = 0.0, tt[9];
        for (int t = -R; t <= R; ++t) {
            tt[t + R] = std::exp(-(double)(t * t) / (2.0 * (double)p->sigma * (double)p->sigma));
            sum += tt[t + R];
        }
        for (int t = 0; t <= 2 * R; ++t) a.taps[t] = (float)(tt[t] / sum);
    }
    for (int k = 0; k < p->m && k < 16; ++k) {
        const double th = (double)k * 3.14159265358979323846 / (double)p->m;
        a.cs[k] = (float)std::cos(th);
        a.sn[k] = (float)std::sin(th);
    }
    a.eps = p->eps;
    cudaStream_t st = as_stream(stream);
    switch (p->m) {
        case 6: return dispatch_radius<6>(R, p->orientation, img, out, a, row0, row1, st);
        case 8: return dispatch_radius<8>(R, p->orientation, img, out, a, row0, row1, st);
        case 9: return dispatch_radius<9>(R, p->orientation, img, out, a, row0, row1, st);
        case 12: return dispatch_radius<12>(R, p->orientation, img, out, a, row0, row1, st);
    }
    set_error("%s: m = %d not compiled (6, 8, 9, 12)", who, p->m);
    return CFOG_E_UNSUPPORTED;
}

}  // namespace
}  // namespace cfog

extern "C" cfog_status cfog_extract(const cfog_image *img, const cfog_params *p,
                                    const cfog_features *out, void *stream) {
    CFOG_TRACE("cfog_extract");
    return cfog::extract_impl(img, p, out, 0, img ? img->h : 0, stream, "cfog_extract");
}

extern "C" cfog_status cfog_extract_rows(const cfog_image *img, const cfog_params *p,
                                         const cfog_features *out, int32_t row0, int32_t row1,
                                         void *stream) {
    CFOG_TRACE("cfog_extract_rows");
    return cfog::extract_impl(img, p, out, row0, row1, stream, "cfog_extract_rows");
}
