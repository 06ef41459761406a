// K2: block-based Harris feature-point detection (Sec. IV).
//
// One CTA per grid cell.  The cell's chip is walked in 32 x 32 sub-tiles;
// each sub-tile stages the image plus a 5-pixel halo in shared memory (loaded
// into registers while the previous sub-tile is processed), forms
// the structure-tensor products of the [-1,0,1] gradients, smooths them with a
// separable 9-tap Gaussian (sigma 1.5) and evaluates det - 0.04 tr^2.  Every
// thread keeps its own k best pixels; k rounds of a block-wide arg-max then
// pick the chip's k best (ties: smaller y, then smaller x).
#include "cfog_internal.cuh"

#include <cfloat>
#include <cmath>
#include <cstdint>

namespace cfog {
namespace {

constexpr int HT = 32;            // sub-tile side (outputs)
constexpr int HR = 4;             // Gaussian radius
constexpr int HG = HT + 2 * HR;   // gradient-region side (40)
constexpr int HI = HG + 2;        // image-tile side (42)
constexpr int HNT = 256;
constexpr int KMAX = 8;
constexpr float KAPPA = 0.04f;

struct HarrisTaps {
    float w[2 * HR + 1];
};

__device__ __forceinline__ int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

struct Cand {
    float v;
    int y, x;
};

// a ranks before b: larger response, then smaller y, then smaller x
__device__ __forceinline__ bool better(const Cand &a, const Cand &b) {
    if (a.v != b.v) return a.v > b.v;
    if (a.y != b.y) return a.y < b.y;
    return a.x < b.x;
}

__device__ __forceinline__ void cell_chip(int h, int w, int gx, int gy, int chip, int margin, int gj,
                                          int gi, int &y0, int &y1, int &x0, int &x1) {
    const long long ih = h - 2 * margin, iw = w - 2 * margin;
    const int cy0 = margin + (int)(gj * ih / gy), cy1 = margin + (int)((gj + 1) * ih / gy);
    const int cx0 = margin + (int)(gi * iw / gx), cx1 = margin + (int)((gi + 1) * iw / gx);
    if (chip > 0) {
        const int cy = (cy0 + cy1) / 2, cx = (cx0 + cx1) / 2;
        const int a = cy - chip / 2, b = cx - chip / 2;
        y0 = max(a, cy0);
        y1 = min(a + chip, cy1);
        x0 = max(b, cx0);
        x1 = min(b + chip, cx1);
    } else {
        y0 = cy0;
        y1 = cy1;
        x0 = cx0;
        x1 = cx1;
    }
}

template <typename TIn>
__global__ void __launch_bounds__(HNT, 3)
harris_blockmax_kernel(const TIn *__restrict__ img, int h, int w, int64_t pitch, int grid_x,
                       int grid_y, int k, int chip, int margin, cfog_point *__restrict__ out,
                       const HarrisTaps taps) {
    __shared__ float tile[HI * HI];
    __shared__ float prod[3][HG * HG];
    __shared__ float hp[3][HG * HT];
    __shared__ Cand wbest[HNT / 32];
    __shared__ int wowner[HNT / 32];
    __shared__ int winner;

    const int tid = threadIdx.x;
    const int gi = blockIdx.x, gj = blockIdx.y;
    int y0, y1, x0, x1;
    cell_chip(h, w, grid_x, grid_y, chip, margin, gj, gi, y0, y1, x0, x1);

    Cand best[KMAX];
#pragma unroll
    for (int s = 0; s < KMAX; ++s) best[s] = Cand{-FLT_MAX, INT_MAX, INT_MAX};

    // The image tile of the next sub-tile is loaded into registers while the
    // current one is processed (PF values per thread).
    constexpr int PF = (HI * HI + HNT - 1) / HNT;
    float pf[PF];
    auto load_tile = [&](int sy, int sx) {
        const int oy = sy - HR - 1, ox = sx - HR - 1;
#pragma unroll
        for (int u = 0; u < PF; ++u) {
            const int i = tid + u * HNT;
            const int ty = i / HI, tx = i - ty * HI;
            const int yy = clampi(oy + ty, 0, h - 1), xx = clampi(ox + tx, 0, w - 1);
            pf[u] = i < HI * HI ? static_cast<float>(__ldg(img + (int64_t)yy * pitch + xx)) : 0.f;
        }
    };
    if (y0 < y1 && x0 < x1) load_tile(y0, x0);
    for (int sy = y0; sy < y1; sy += HT) {
        for (int sx = x0; sx < x1; sx += HT) {
            const int oy = sy - HR - 1, ox = sx - HR - 1;
#pragma unroll
            for (int u = 0; u < PF; ++u)
                if (tid + u * HNT < HI * HI) tile[tid + u * HNT] = pf[u];
            __syncthreads();
            {
                int nsy = sy, nsx = sx + HT;
                if (nsx >= x1) {
                    nsx = x0;
                    nsy += HT;
                }
                if (nsy < y1) load_tile(nsy, nsx);
            }
            for (int i = tid; i < HG * HG; i += HNT) {
                const int j = i / HG, c = i - j * HG;
                const int cy = clampi(sy - HR + j, 0, h - 1), cx = clampi(sx - HR + c, 0, w - 1);
                const int ty = cy - oy, tx = cx - ox;
                const int yu = clampi(cy - 1, 0, h - 1) - oy, yd = clampi(cy + 1, 0, h - 1) - oy;
                const int xl = clampi(cx - 1, 0, w - 1) - ox, xr = clampi(cx + 1, 0, w - 1) - ox;
                const float gxv = tile[ty * HI + xr] - tile[ty * HI + xl];
                const float gyv = tile[yd * HI + tx] - tile[yu * HI + tx];
                prod[0][i] = gxv * gxv;
                prod[1][i] = gyv * gyv;
                prod[2][i] = gxv * gyv;
            }
            __syncthreads();
            for (int i = tid; i < 3 * HG * HT; i += HNT) {
                const int q = i / (HG * HT), rem = i - q * (HG * HT);
                const int j = rem / HT, c = rem - j * HT;
                const float *src = &prod[q][j * HG + c];
                float acc = 0.f;
#pragma unroll
                for (int t = 0; t <= 2 * HR; ++t) acc = fmaf(taps.w[t], src[t], acc);
                hp[q][rem] = acc;
            }
            __syncthreads();
            {
                const int c = tid % HT;
                const int rg = tid / HT;   // 8 groups of 4 rows
#pragma unroll
                for (int i = 0; i < HT / (HNT / HT); ++i) {
                    const int row = rg * (HT / (HNT / HT)) + i;
                    float a = 0.f, b = 0.f, cc = 0.f;
#pragma unroll
                    for (int t = 0; t <= 2 * HR; ++t) {
                        a = fmaf(taps.w[t], hp[0][(row + t) * HT + c], a);
                        b = fmaf(taps.w[t], hp[1][(row + t) * HT + c], b);
                        cc = fmaf(taps.w[t], hp[2][(row + t) * HT + c], cc);
                    }
                    const float tr = a + b;
                    const float resp = (a * b - cc * cc) - KAPPA * tr * tr;
                    const int y = sy + row, x = sx + c;
                    if (y < y1 && x < x1) {
                        Cand cnd{resp, y, x};
                        // insert into the sorted local list (k <= KMAX)
#pragma unroll
                        for (int s = 0; s < KMAX; ++s) {
                            if (s < k && better(cnd, best[s])) {
                                Cand t = best[s];
                                best[s] = cnd;
                                cnd = t;
                            }
                        }
                    }
                }
            }
            __syncthreads();
        }
    }

    // k rounds of block arg-max; the owner of each winner pops it
    int ptr = 0;
    const int lane = tid & 31, warp = tid >> 5;
    for (int s = 0; s < k; ++s) {
        Cand c = Cand{-FLT_MAX, INT_MAX, INT_MAX};
#pragma unroll
        for (int u = 0; u < KMAX; ++u)
            if (u == ptr) c = best[u];
        int owner = tid;
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            Cand o;
            o.v = __shfl_down_sync(0xffffffffu, c.v, off);
            o.y = __shfl_down_sync(0xffffffffu, c.y, off);
            o.x = __shfl_down_sync(0xffffffffu, c.x, off);
            const int oo = __shfl_down_sync(0xffffffffu, owner, off);
            if (better(o, c)) {
                c = o;
                owner = oo;
            }
        }
        if (lane == 0) {
            wbest[warp] = c;
            wowner[warp] = owner;
        }
        __syncthreads();
        if (tid == 0) {
            Cand b = wbest[0];
            int bo = wowner[0];
            for (int u = 1; u < HNT / 32; ++u)
                if (better(wbest[u], b)) {
                    b = wbest[u];
                    bo = wowner[u];
                }
            const int idx = ((gj * grid_x) + gi) * k + s;
            if (b.y == INT_MAX) {
                out[idx] = cfog_point{-1, -1};
                winner = -1;
            } else {
                out[idx] = cfog_point{b.x, b.y};
                winner = bo;
            }
        }
        __syncthreads();
        if (winner == tid) ++ptr;
        __syncthreads();
    }
}

}  // namespace
}  // namespace cfog

extern "C" cfog_status cfog_detect_cps(const cfog_image *img, int32_t grid_x, int32_t grid_y,
                                       int32_t k, int32_t chip, int32_t margin, cfog_point *out_dev,
                                       void *stream) {
    CFOG_TRACE("cfog_detect_cps");
    using namespace cfog;
    CFOG_REQUIRE(img && img->data && out_dev, "cfog_detect_cps: null pointer");
    CFOG_REQUIRE(img->h > 0 && img->w > 0 && img->pitch >= img->w, "cfog_detect_cps: bad image");
    CFOG_REQUIRE(img->dtype == CFOG_DTYPE_F32 || img->dtype == CFOG_DTYPE_U16,
                 "cfog_detect_cps: unknown dtype %d", img->dtype);
    CFOG_REQUIRE(grid_x >= 1 && grid_y >= 1 && grid_x <= 65535 && grid_y <= 65535,
                 "cfog_detect_cps: bad grid %dx%d", grid_x, grid_y);
    CFOG_REQUIRE(k >= 1 && k <= KMAX, "cfog_detect_cps: k = %d outside [1, %d]", k, KMAX);
    CFOG_REQUIRE(margin >= 0 && 2 * margin < img->h && 2 * margin < img->w,
                 "cfog_detect_cps: margin %d leaves no interior", margin);
    const int ih = img->h - 2 * margin, iw = img->w - 2 * margin;
    CFOG_REQUIRE(grid_y <= ih && grid_x <= iw, "cfog_detect_cps: more cells than pixels");
    const int cell_h = (ih + grid_y - 1) / grid_y, cell_w = (iw + grid_x - 1) / grid_x;
    const int ch = chip > 0 ? (chip < cell_h ? chip : cell_h) : cell_h;
    const int cw = chip > 0 ? (chip < cell_w ? chip : cell_w) : cell_w;
    CFOG_REQUIRE(ch <= 256 && cw <= 256, "cfog_detect_cps: chip %dx%d exceeds 256x256", ch, cw);

    HarrisTaps taps{};
    const double sigma = 1.5;
    double sum = 0.0, tt[2 * HR + 1];
    for (int t = -HR; t <= HR; ++t) {
        tt[t + HR] = std::exp(-(double)(t * t) / (2.0 * sigma * sigma));
        sum += tt[t + HR];
    }
    for (int t = 0; t <= 2 * HR; ++t) taps.w[t] = (float)(tt[t] / sum);

    dim3 grid(grid_x, grid_y);
    cudaStream_t st = as_stream(stream);
    if (img->dtype == CFOG_DTYPE_F32)
        harris_blockmax_kernel<float><<<grid, HNT, 0, st>>>(
            static_cast<const float *>(img->data), img->h, img->w, img->pitch, grid_x, grid_y, k,
            chip, margin, out_dev, taps);
    else
        harris_blockmax_kernel<uint16_t><<<grid, HNT, 0, st>>>(
            static_cast<const uint16_t *>(img->data), img->h, img->w, img->pitch, grid_x, grid_y,
            k, chip, margin, out_dev, taps);
    return check_launch("cfog_detect_cps: launch");
}
