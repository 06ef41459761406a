// K8: least-squares affine mapping model in FP64 (Sec. IV, the geometric
// mapping model by least squares, affine case).
//
// One CTA reduces the normal equations of  x' = a0 + a1 x + a2 y  and
// y' = b0 + b1 x + b2 y  over the CPs whose status is OK, with a fixed
// per-thread stride and a fixed reduction tree (deterministic), then thread 0
// solves the two 3 x 3 systems by Cholesky.
#include "cfog_internal.cuh"

#include <cmath>

namespace cfog {
namespace {

constexpr int AT = 256;
constexpr int NS = 12;   // 1, x, y, xx, xy, yy, x', x x', y x', y', x y', y y'

__global__ void __launch_bounds__(AT) affine_ls_kernel(const cfog_point *__restrict__ cps,
                                                       const cfog_match_result *__restrict__ res,
                                                       int n, double *__restrict__ work) {
    __shared__ double part[NS][AT / 32];
    double s[NS];
#pragma unroll
    for (int i = 0; i < NS; ++i) s[i] = 0.0;
    for (int i = threadIdx.x; i < n; i += AT) {
        const cfog_match_result rr = res[i];
        if (rr.status != CFOG_CP_OK) continue;
        const double x = cps[i].x, y = cps[i].y;
        const double xp = x + (double)rr.sub_dx, yp = y + (double)rr.sub_dy;
        s[0] += 1.0;
        s[1] += x;
        s[2] += y;
        s[3] += x * x;
        s[4] += x * y;
        s[5] += y * y;
        s[6] += xp;
        s[7] += x * xp;
        s[8] += y * xp;
        s[9] += yp;
        s[10] += x * yp;
        s[11] += y * yp;
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int i = 0; i < NS; ++i) {
        double v = s[i];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) part[i][warp] = v;
    }
    __syncthreads();
    if (threadIdx.x != 0) return;
    double t[NS];
    for (int i = 0; i < NS; ++i) {
        double v = 0.0;
        for (int w = 0; w < AT / 32; ++w) v += part[i][w];
        t[i] = v;
    }
    // normal matrix M (symmetric 3x3) and right-hand sides
    const double M[3][3] = {{t[0], t[1], t[2]}, {t[1], t[3], t[4]}, {t[2], t[4], t[5]}};
    const double bx[3] = {t[6], t[7], t[8]}, by[3] = {t[9], t[10], t[11]};
    double Lc[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
    double scale = fmax(fabs(M[0][0]), fmax(fabs(M[1][1]), fabs(M[2][2])));
    bool ok = scale > 0.0;
    for (int i = 0; i < 3 && ok; ++i) {
        for (int j = 0; j <= i; ++j) {
            double acc = M[i][j];
            for (int k = 0; k < j; ++k) acc -= Lc[i][k] * Lc[j][k];
            if (i == j) {
                if (!(acc > 1e-12 * scale)) {
                    ok = false;
                    break;
                }
                Lc[i][i] = sqrt(acc);
            } else {
                Lc[i][j] = acc / Lc[j][j];
            }
        }
    }
    double sol[6] = {0, 0, 0, 0, 0, 0};
    if (ok) {
        for (int rhs = 0; rhs < 2; ++rhs) {
            const double *b = rhs ? by : bx;
            double z[3], x[3];
            for (int i = 0; i < 3; ++i) {
                double acc = b[i];
                for (int k = 0; k < i; ++k) acc -= Lc[i][k] * z[k];
                z[i] = acc / Lc[i][i];
            }
            for (int i = 2; i >= 0; --i) {
                double acc = z[i];
                for (int k = i + 1; k < 3; ++k) acc -= Lc[k][i] * x[k];
                x[i] = acc / Lc[i][i];
            }
            for (int i = 0; i < 3; ++i) sol[rhs * 3 + i] = x[i];
        }
    }
    for (int i = 0; i < 6; ++i) work[i] = sol[i];
    work[6] = ok ? 1.0 : 0.0;
    work[7] = t[0];
}

}  // namespace
}  // namespace cfog

extern "C" cfog_status cfog_fit_affine(const cfog_point *cps_dev, const cfog_match_result *res_dev,
                                       int32_t n, double *work_dev, double *out6, void *stream) {
    CFOG_TRACE("cfog_fit_affine");
    using namespace cfog;
    CFOG_REQUIRE(cps_dev && res_dev && work_dev && out6, "cfog_fit_affine: null pointer");
    CFOG_REQUIRE(n >= 0, "cfog_fit_affine: n = %d < 0", n);
    cudaStream_t st = as_stream(stream);
    affine_ls_kernel<<<1, AT, 0, st>>>(cps_dev, res_dev, n, work_dev);
    cfog_status s = check_launch("cfog_fit_affine: launch");
    if (s != CFOG_OK) return s;
    double host[8];
    s = check_cuda(cudaMemcpyAsync(host, work_dev, sizeof(host), cudaMemcpyDeviceToHost, st),
                   "cfog_fit_affine: copy");
    if (s != CFOG_OK) return s;
    s = check_cuda(cudaStreamSynchronize(st), "cfog_fit_affine: synchronize");
    if (s != CFOG_OK) return s;
    if (host[6] != 1.0) {
        set_error("cfog_fit_affine: singular normal equations (%g CPs with status OK)", host[7]);
        return CFOG_E_INVAL;
    }
    for (int i = 0; i < 6; ++i) out6[i] = host[i];
    return CFOG_OK;
}
