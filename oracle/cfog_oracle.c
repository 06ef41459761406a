/*
 * FP64 CPU oracle for CFOG template matching (Ye et al., "Fast and Robust
 * Matching for Multimodal Remote Sensing Image Registration", arXiv 1808.06194).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, obviously correct
 * statement of what the GPU path computes.  Only the tests, the smoke check and
 * the benchmark's CPU-baseline leg may load it.  It shares no code, header,
 * table or constant with the CUDA library and includes nothing from it.
 *
 * Every step follows the paper's definitions in their order:
 *   gradients            Sec. III-F (1-D filters [-1,0,1] and its transpose)
 *   oriented channels    Eq. 2 (abs of the directional derivative), or the
 *                        first scheme of Sec. III-F / Fig. 7 (magnitude shared
 *                        between the two nearest orientation bins)
 *   3-D smoothing        Sec. III-F (2-D Gaussian in x,y, [1,2,1] along Z)
 *   L2 normalisation     Sec. III-C (HOG); the CFOG chain of Fig. 9
 *   SSD surface          Eq. 3, brute force over every shift
 *   argmin               Eq. 4
 *   sub-pixel            Sec. V-B (local quadratic polynomial fit)
 *   Harris detection     Sec. IV (block-based Harris, k best per grid chip)
 *   affine LS            Sec. IV (least-squares mapping model, affine case)
 *   pixel-wise HOG       Sec. III-C (FHOG: 2x2 cells x 9 orientation bins per
 *                        pixel, trilinear interpolation, L2 normalisation)
 *   TIN rectification    Sec. IV (piecewise linear model: one affine map per
 *                        triangle of a TIN over the CPs, bilinear resampling)
 *   outlier rejection    Sec. IV (iterative LS fit of a polynomial model,
 *                        dropping the largest residual until RMSE < threshold)
 *
 * Readings where the paper is silent are marked "Reading:".
 * Feature volumes are planar: plane k of an h x w image at out[k*h*w + y*w + x].
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

static int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

/* Sec. III-F: gx, gy by the 1-D filters [-1,0,1] and [-1,0,1]^T.
 * gx(y,x) = I(y,x+1) - I(y,x-1); gy(y,x) = I(y+1,x) - I(y-1,x); y grows downward.
 * Reading: borders replicate the edge pixel. */
void orc_gradients(const double *img, int h, int w, double *gx, double *gy) {
    for (int y = 0; y < h; ++y) {
        for (int x = 0; x < w; ++x) {
            int xl = clampi(x - 1, 0, w - 1), xr = clampi(x + 1, 0, w - 1);
            int yu = clampi(y - 1, 0, h - 1), yd = clampi(y + 1, 0, h - 1);
            gx[(size_t)y * w + x] = img[(size_t)y * w + xr] - img[(size_t)y * w + xl];
            gy[(size_t)y * w + x] = img[(size_t)yd * w + x] - img[(size_t)yu * w + x];
        }
    }
}

/* Eq. 2: g_theta = abs(cos(theta) gx + sin(theta) gy) for m orientations
 * theta_k = k*pi/m, k = 0..m-1, covering [0, 180) degrees. */
void orc_channels(const double *gx, const double *gy, int h, int w, int m, double *g) {
    size_t hw = (size_t)h * w;
    for (int k = 0; k < m; ++k) {
        double th = (double)k * M_PI / (double)m;
        double c = cos(th), s = sin(th);
        for (size_t p = 0; p < hw; ++p) g[k * hw + p] = fabs(c * gx[p] + s * gy[p]);
    }
}

/* Sampled Gaussian exp(-t^2 / (2 sigma^2)), t = -R..R, normalised to sum 1.
 * Reading: R = ceil(3 sigma) unless given. */
void orc_gauss_taps(double sigma, int R, double *taps) {
    double sum = 0.0;
    for (int t = -R; t <= R; ++t) {
        taps[t + R] = exp(-(double)(t * t) / (2.0 * sigma * sigma));
        sum += taps[t + R];
    }
    for (int t = 0; t < 2 * R + 1; ++t) taps[t] /= sum;
}

/* Sec. III-F: 2-D Gaussian in X and Y applied to every channel, as a
 * horizontal pass followed by a vertical pass; replicate borders. */
void orc_smooth_xy(const double *in, int m, int h, int w, double sigma, int R, double *out) {
    double *taps = (double *)malloc(sizeof(double) * (2 * R + 1));
    double *tmp = (double *)malloc(sizeof(double) * (size_t)h * w);
    orc_gauss_taps(sigma, R, taps);
    size_t hw = (size_t)h * w;
    for (int k = 0; k < m; ++k) {
        const double *src = in + k * hw;
        double *dst = out + k * hw;
        for (int y = 0; y < h; ++y)
            for (int x = 0; x < w; ++x) {
                double acc = 0.0;
                for (int t = -R; t <= R; ++t)
                    acc += taps[t + R] * src[(size_t)y * w + clampi(x + t, 0, w - 1)];
                tmp[(size_t)y * w + x] = acc;
            }
        for (int y = 0; y < h; ++y)
            for (int x = 0; x < w; ++x) {
                double acc = 0.0;
                for (int t = -R; t <= R; ++t)
                    acc += taps[t + R] * tmp[(size_t)clampi(y + t, 0, h - 1) * w + x];
                dst[(size_t)y * w + x] = acc;
            }
    }
    free(tmp);
    free(taps);
}

/* Sec. III-F: the [1,2,1]^T kernel along the orientation (Z) direction.
 * Reading: circular in k (orientation is periodic over 180 degrees), and the
 * kernel is normalised to [1,2,1]/4. */
void orc_smooth_z(const double *in, int m, int h, int w, double *out) {
    size_t hw = (size_t)h * w;
    for (int k = 0; k < m; ++k) {
        int km = (k + m - 1) % m, kp = (k + 1) % m;
        for (size_t p = 0; p < hw; ++p)
            out[k * hw + p] = 0.25 * (in[km * hw + p] + 2.0 * in[k * hw + p] + in[kp * hw + p]);
    }
}

/* Per-pixel L2 normalisation of the m-vector: D_k = h_k / (||h||_2 + eps).
 * Also returns ||D||^2 per pixel. */
void orc_normalize(const double *in, int m, int h, int w, double eps, double *out, double *sqnorm) {
    size_t hw = (size_t)h * w;
    for (size_t p = 0; p < hw; ++p) {
        double ss = 0.0;
        for (int k = 0; k < m; ++k) ss += in[k * hw + p] * in[k * hw + p];
        double inv = 1.0 / (sqrt(ss) + eps);
        double dd = 0.0;
        for (int k = 0; k < m; ++k) {
            double d = in[k * hw + p] * inv;
            out[k * hw + p] = d;
            dd += d * d;
        }
        if (sqnorm) sqnorm[p] = dd;
    }
}

/* The CFOG chain (Fig. 9): gradients -> channels -> 2-D Gaussian -> Z kernel
 * -> L2 normalisation.  out: m planes of h x w; sqnorm: h x w (nullable). */
/* Sec. III-F, first scheme (Fig. 7): the gradient magnitude sqrt(gx^2 + gy^2)
 * is shared between the two orientation bins next to the gradient's
 * orientation in [0, 180) degrees, each weighted by one minus its distance to
 * the orientation in bin widths (the weight falls as the distance grows).
 * Reading: the bins are centred on theta_k = k*pi/m (the grid of Eq. 2) and
 * wrap around at 180 degrees; the orientation is atan2(gy, gx) folded into
 * [0, pi), which treats a gradient and its opposite alike, as abs does in Eq. 2. */
void orc_channels_binned(const double *gx, const double *gy, int h, int w, int m, double *g) {
    size_t hw = (size_t)h * w;
    for (size_t i = 0; i < hw * (size_t)m; ++i) g[i] = 0.0;
    for (size_t p = 0; p < hw; ++p) {
        double mag = sqrt(gx[p] * gx[p] + gy[p] * gy[p]);
        if (mag == 0.0) continue;
        double phi = atan2(gy[p], gx[p]);
        if (phi < 0.0) phi += M_PI;
        if (phi >= M_PI) phi -= M_PI;
        double t = phi / (M_PI / (double)m);   /* position in bin widths */
        int k0 = (int)floor(t);
        double frac = t - (double)k0;
        k0 %= m;
        int k1 = (k0 + 1) % m;
        g[(size_t)k0 * hw + p] += mag * (1.0 - frac);
        g[(size_t)k1 * hw + p] += mag * frac;
    }
}

/* CFOG with the orientation scheme chosen: 0 = Eq. 2, 1 = binned (Fig. 7). */
void orc_cfog_scheme(const double *img, int h, int w, int m, double sigma, int R, double eps,
                     int scheme, double *out, double *sqnorm) {
    size_t hw = (size_t)h * w;
    double *gx = (double *)malloc(sizeof(double) * hw);
    double *gy = (double *)malloc(sizeof(double) * hw);
    double *g = (double *)malloc(sizeof(double) * hw * m);
    double *s = (double *)malloc(sizeof(double) * hw * m);
    orc_gradients(img, h, w, gx, gy);
    if (scheme == 1)
        orc_channels_binned(gx, gy, h, w, m, g);
    else
        orc_channels(gx, gy, h, w, m, g);
    orc_smooth_xy(g, m, h, w, sigma, R, s);
    orc_smooth_z(s, m, h, w, g);
    orc_normalize(g, m, h, w, eps, out, sqnorm);
    free(gx);
    free(gy);
    free(g);
    free(s);
}

void orc_cfog(const double *img, int h, int w, int m, double sigma, int R, double eps,
              double *out, double *sqnorm) {
    size_t hw = (size_t)h * w;
    double *gx = (double *)malloc(sizeof(double) * hw);
    double *gy = (double *)malloc(sizeof(double) * hw);
    double *g = (double *)malloc(sizeof(double) * hw * m);
    double *s = (double *)malloc(sizeof(double) * hw * m);
    orc_gradients(img, h, w, gx, gy);
    orc_channels(gx, gy, h, w, m, g);
    orc_smooth_xy(g, m, h, w, sigma, R, s);
    orc_smooth_z(s, m, h, w, g);
    orc_normalize(g, m, h, w, eps, out, sqnorm);
    free(gx);
    free(gy);
    free(g);
    free(s);
}

/* ------------------------------------------------------------------------ */
/* Matching                                                                  */
/* ------------------------------------------------------------------------ */

/* Eq. 3, brute force.  Template window of the CP p = (px, py): pixels p + t
 * with t in [-floor(N/2), N-1-floor(N/2)]^2 (reading for even N: the centre is
 * index floor(N/2)).  For every shift v in [-r, r]^2,
 *     S(v) = sum_x sum_k (D_ref(x,k) - D_sen(x + q + v, k))^2
 * where q = (qx, qy) is the predicted search-region centre (Sec. IV, search
 * region from georeferencing).  Summed in FP64, row-major x, then k.
 * S is (2r+1)^2 doubles, row-major in (dy, dx).  Also E(v) = sum T^2 + sum over
 * the shifted window of ||D_sen||^2 (the energy scale used for tolerances).
 * Returns 0, or 1 when any needed pixel lies outside either image (no padding). */
int orc_ssd_surface(const double *dref, int hr, int wr, const double *dsen, int hs, int ws, int m,
                    int px, int py, int N, int r, int qx, int qy, double *S, double *E) {
    int t0 = N / 2;
    int ry0 = py - t0, rx0 = px - t0;
    if (ry0 < 0 || rx0 < 0 || ry0 + N > hr || rx0 + N > wr) return 1;
    int sy0 = py + qy - t0 - r, sx0 = px + qx - t0 - r;
    if (sy0 < 0 || sx0 < 0 || sy0 + N + 2 * r > hs || sx0 + N + 2 * r > ws) return 1;
    size_t hwr = (size_t)hr * wr, hws = (size_t)hs * ws;
    double tt = 0.0;
    for (int ty = 0; ty < N; ++ty)
        for (int tx = 0; tx < N; ++tx)
            for (int k = 0; k < m; ++k) {
                double a = dref[k * hwr + (size_t)(ry0 + ty) * wr + (rx0 + tx)];
                tt += a * a;
            }
    int L = 2 * r + 1;
    for (int dy = -r; dy <= r; ++dy)
        for (int dx = -r; dx <= r; ++dx) {
            double acc = 0.0, bb = 0.0;
            for (int ty = 0; ty < N; ++ty)
                for (int tx = 0; tx < N; ++tx) {
                    size_t ro = (size_t)(ry0 + ty) * wr + (rx0 + tx);
                    size_t so = (size_t)(py + qy - t0 + ty + dy) * ws + (px + qx - t0 + tx + dx);
                    for (int k = 0; k < m; ++k) {
                        double a = dref[k * hwr + ro];
                        double b = dsen[k * hws + so];
                        acc += (a - b) * (a - b);
                        bb += b * b;
                    }
                }
            S[(dy + r) * L + (dx + r)] = acc;
            if (E) E[(dy + r) * L + (dx + r)] = tt + bb;
        }
    return 0;
}

/* Solve the n x n system A z = b in place (Gaussian elimination, partial
 * pivoting).  Returns 0, or 1 if singular (a pivot below 1e-12 of the largest
 * entry). */
static int solve_dense(double *A, double *b, int n) {
    double scale = 0.0;
    for (int i = 0; i < n * n; ++i) scale = fabs(A[i]) > scale ? fabs(A[i]) : scale;
    for (int c = 0; c < n; ++c) {
        int piv = c;
        for (int i = c + 1; i < n; ++i)
            if (fabs(A[i * n + c]) > fabs(A[piv * n + c])) piv = i;
        if (!(fabs(A[piv * n + c]) > 1e-12 * scale)) return 1;
        if (piv != c) {
            for (int j = 0; j < n; ++j) {
                double t = A[c * n + j];
                A[c * n + j] = A[piv * n + j];
                A[piv * n + j] = t;
            }
            double t = b[c];
            b[c] = b[piv];
            b[piv] = t;
        }
        for (int i = c + 1; i < n; ++i) {
            double f = A[i * n + c] / A[c * n + c];
            for (int j = c; j < n; ++j) A[i * n + j] -= f * A[c * n + j];
            b[i] -= f * b[c];
        }
    }
    for (int i = n - 1; i >= 0; --i) {
        double acc = b[i];
        for (int j = i + 1; j < n; ++j) acc -= A[i * n + j] * b[j];
        b[i] = acc / A[i * n + i];
    }
    return 0;
}

/* Sec. V-B: sub-pixel position from a local quadratic polynomial.
 * Reading: least-squares fit of f = a + b x + c y + d x^2 + e xy + g y^2 to the
 * 3x3 neighbourhood S9 (row-major, x = dx in {-1,0,1}, y = dy), solved from the
 * normal equations; the stationary point is the offset.  When the Hessian is
 * not positive definite or the offset leaves [-1,1]^2, separable 1-D parabolas
 * are used instead, each clamped to [-0.5, 0.5] (0 when not convex).
 * Returns 0 for the full fit, 1 for the fallback. */
int orc_subpixel(const double *S9, double *ddx, double *ddy) {
    double M[36], rhs[6];
    memset(M, 0, sizeof(M));
    memset(rhs, 0, sizeof(rhs));
    for (int j = 0; j < 3; ++j)
        for (int i = 0; i < 3; ++i) {
            double x = i - 1, y = j - 1;
            double phi[6] = {1.0, x, y, x * x, x * y, y * y};
            for (int u = 0; u < 6; ++u) {
                rhs[u] += phi[u] * S9[j * 3 + i];
                for (int v = 0; v < 6; ++v) M[u * 6 + v] += phi[u] * phi[v];
            }
        }
    if (solve_dense(M, rhs, 6) == 0) {
        double b = rhs[1], c = rhs[2], d = rhs[3], e = rhs[4], g = rhs[5];
        double h11 = 2.0 * d, h12 = e, h22 = 2.0 * g;
        double det = h11 * h22 - h12 * h12;
        if (h11 > 0.0 && det > 0.0) {
            double ox = -(h22 * b - h12 * c) / det;
            double oy = -(-h12 * b + h11 * c) / det;
            if (fabs(ox) <= 1.0 && fabs(oy) <= 1.0) {
                *ddx = ox;
                *ddy = oy;
                return 0;
            }
        }
    }
    double sxm = S9[3], sx0 = S9[4], sxp = S9[5];
    double sym = S9[1], syp = S9[7];
    double denx = sxm - 2.0 * sx0 + sxp, deny = sym - 2.0 * sx0 + syp;
    double ox = denx > 0.0 ? (sxm - sxp) / (2.0 * denx) : 0.0;
    double oy = deny > 0.0 ? (sym - syp) / (2.0 * deny) : 0.0;
    *ddx = ox < -0.5 ? -0.5 : (ox > 0.5 ? 0.5 : ox);
    *ddy = oy < -0.5 ? -0.5 : (oy > 0.5 ? 0.5 : oy);
    return 1;
}

/* Eq. 4 plus sub-pixel refinement for one CP.
 * out_i[4] = {dx, dy, status, fallback}; out_d[6] = {sub_dx, sub_dy, ssd,
 * E(v*), second-best S, relative top-2 gap (S2 - S1) / E(v*)}.
 * dx, dy and sub_* are the total offsets q + v (+ delta) from the CP.
 * Tie-break: the lexicographically smallest (dy, dx) among equal minima.
 * Status: 0 OK, 1 out of bounds, 2 peak on the window edge (delta = 0). */
void orc_match_one(const double *dref, int hr, int wr, const double *dsen, int hs, int ws, int m,
                   int px, int py, int N, int r, int qx, int qy, int *out_i, double *out_d,
                   double *surface /* nullable, (2r+1)^2 */) {
    int L = 2 * r + 1;
    double *S = (double *)malloc(sizeof(double) * L * L);
    double *E = (double *)malloc(sizeof(double) * L * L);
    int st = orc_ssd_surface(dref, hr, wr, dsen, hs, ws, m, px, py, N, r, qx, qy, S, E);
    out_i[3] = 0;
    if (st) {
        out_i[0] = qx;
        out_i[1] = qy;
        out_i[2] = 1;
        for (int i = 0; i < 6; ++i) out_d[i] = 0.0;
        out_d[0] = qx;
        out_d[1] = qy;
        out_d[2] = INFINITY;
        free(S);
        free(E);
        return;
    }
    int best = 0;
    for (int i = 1; i < L * L; ++i)
        if (S[i] < S[best]) best = i;
    double second = INFINITY;
    for (int i = 0; i < L * L; ++i)
        if (i != best && S[i] < second) second = S[i];
    int by = best / L - r, bx = best % L - r;
    double ddx = 0.0, ddy = 0.0;
    int status = 0;
    if (bx == -r || bx == r || by == -r || by == r) {
        status = 2;
    } else {
        double S9[9];
        for (int j = -1; j <= 1; ++j)
            for (int i = -1; i <= 1; ++i) S9[(j + 1) * 3 + (i + 1)] = S[(by + r + j) * L + (bx + r + i)];
        out_i[3] = orc_subpixel(S9, &ddx, &ddy);
    }
    out_i[0] = qx + bx;
    out_i[1] = qy + by;
    out_i[2] = status;
    out_d[0] = qx + bx + ddx;
    out_d[1] = qy + by + ddy;
    out_d[2] = S[best];
    out_d[3] = E[best];
    out_d[4] = second;
    out_d[5] = (second - S[best]) / (E[best] > 0.0 ? E[best] : 1.0);
    if (surface) memcpy(surface, S, sizeof(double) * L * L);
    free(S);
    free(E);
}

/* Many CPs; features shared.  Arrays of length n; prior (qx, qy) nullable.
 * Parallel over CPs when built with OpenMP (each CP is independent). */
void orc_match_many(const double *dref, int hr, int wr, const double *dsen, int hs, int ws, int m,
                    int n, const int *px, const int *py, const int *N, const int *r,
                    const int *qx, const int *qy, int *out_i, double *out_d) {
#pragma omp parallel for schedule(dynamic, 1)
    for (int i = 0; i < n; ++i)
        orc_match_one(dref, hr, wr, dsen, hs, ws, m, px[i], py[i], N[i], r[i], qx ? qx[i] : 0,
                      qy ? qy[i] : 0, out_i + 4 * i, out_d + 6 * i, NULL);
}

/* ------------------------------------------------------------------------ */
/* Block-based Harris detection (Sec. IV)                                    */
/* ------------------------------------------------------------------------ */

/* Harris response det(M) - kappa tr(M)^2 with M the structure tensor of the
 * gradients above, each entry smoothed by a Gaussian of sigma, radius R.
 * Reading: sigma = 1.5, R = 4, kappa = 0.04; replicate borders. */
void orc_harris(const double *img, int h, int w, double sigma, int R, double kappa, double *resp) {
    size_t hw = (size_t)h * w;
    double *gx = (double *)malloc(sizeof(double) * hw);
    double *gy = (double *)malloc(sizeof(double) * hw);
    double *prod = (double *)malloc(sizeof(double) * hw * 3);
    double *sm = (double *)malloc(sizeof(double) * hw * 3);
    orc_gradients(img, h, w, gx, gy);
    for (size_t p = 0; p < hw; ++p) {
        prod[p] = gx[p] * gx[p];
        prod[hw + p] = gy[p] * gy[p];
        prod[2 * hw + p] = gx[p] * gy[p];
    }
    orc_smooth_xy(prod, 3, h, w, sigma, R, sm);
    for (size_t p = 0; p < hw; ++p) {
        double a = sm[p], b = sm[hw + p], c = sm[2 * hw + p];
        resp[p] = (a * b - c * c) - kappa * (a + b) * (a + b);
    }
    free(gx);
    free(gy);
    free(prod);
    free(sm);
}

/* Chip of grid cell (gi, gj): the interior box [margin, h-margin) x
 * [margin, w-margin) is cut into grid_y x grid_x cells; the chip is a
 * chip x chip window centred on the cell centre, clipped to the cell
 * (chip <= 0: the whole cell).  Writes [y0, y1) x [x0, x1). */
void orc_cell_chip(int h, int w, int grid_x, int grid_y, int chip, int margin, int gj, int gi,
                   int *y0, int *y1, int *x0, int *x1) {
    int ih = h - 2 * margin, iw = w - 2 * margin;
    int cy0 = margin + (int)((long long)gj * ih / grid_y);
    int cy1 = margin + (int)((long long)(gj + 1) * ih / grid_y);
    int cx0 = margin + (int)((long long)gi * iw / grid_x);
    int cx1 = margin + (int)((long long)(gi + 1) * iw / grid_x);
    if (chip > 0) {
        int cy = (cy0 + cy1) / 2, cx = (cx0 + cx1) / 2;
        int a = cy - chip / 2, b = cx - chip / 2;
        *y0 = a > cy0 ? a : cy0;
        *y1 = a + chip < cy1 ? a + chip : cy1;
        *x0 = b > cx0 ? b : cx0;
        *x1 = b + chip < cx1 ? b + chip : cx1;
    } else {
        *y0 = cy0;
        *y1 = cy1;
        *x0 = cx0;
        *x1 = cx1;
    }
}

/* k largest responses per chip (ties: lowest (y, x) first).  Output CP j*grid_x*k
 * + i*k + s for cell (j, i), rank s.  Returns the number written. */
int orc_detect(const double *resp, int h, int w, int grid_x, int grid_y, int k, int chip, int margin,
               int *xs, int *ys) {
    int cnt = 0;
    for (int gj = 0; gj < grid_y; ++gj)
        for (int gi = 0; gi < grid_x; ++gi) {
            int y0, y1, x0, x1;
            orc_cell_chip(h, w, grid_x, grid_y, chip, margin, gj, gi, &y0, &y1, &x0, &x1);
            for (int s = 0; s < k; ++s) {
                int by = -1, bx = -1;
                double bv = -INFINITY;
                for (int y = y0; y < y1; ++y)
                    for (int x = x0; x < x1; ++x) {
                        int taken = 0;
                        for (int u = 0; u < s; ++u)
                            if (xs[cnt - s + u] == x && ys[cnt - s + u] == y) taken = 1;
                        if (taken) continue;
                        double v = resp[(size_t)y * w + x];
                        if (v > bv) {
                            bv = v;
                            by = y;
                            bx = x;
                        }
                    }
                xs[cnt] = bx;
                ys[cnt] = by;
                ++cnt;
            }
        }
    return cnt;
}

/* ------------------------------------------------------------------------ */
/* Least-squares affine model (Sec. IV, the mapping model by least squares)   */
/* ------------------------------------------------------------------------ */

/* Fit xs' = a0 + a1 x + a2 y and ys' = b0 + b1 x + b2 y over CPs with
 * valid[i] != 0, in FP64 from the normal equations.  out6 = {a0,a1,a2,b0,b1,b2}.
 * Returns 0, or 1 if the system is singular (fewer than 3 independent CPs). */
int orc_affine_ls(const double *x, const double *y, const double *xp, const double *yp,
                  const int *valid, int n, double *out6) {
    double M[9] = {0}, bx[3] = {0}, by[3] = {0};
    for (int i = 0; i < n; ++i) {
        if (valid && !valid[i]) continue;
        double phi[3] = {1.0, x[i], y[i]};
        for (int u = 0; u < 3; ++u) {
            bx[u] += phi[u] * xp[i];
            by[u] += phi[u] * yp[i];
            for (int v = 0; v < 3; ++v) M[u * 3 + v] += phi[u] * phi[v];
        }
    }
    double M2[9];
    memcpy(M2, M, sizeof(M));
    if (solve_dense(M, bx, 3)) return 1;
    if (solve_dense(M2, by, 3)) return 1;
    for (int u = 0; u < 3; ++u) {
        out6[u] = bx[u];
        out6[3 + u] = by[u];
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Outlier rejection (Sec. IV): fit, measure, drop the worst CP, repeat        */
/* ------------------------------------------------------------------------ */

/* Number of monomials x^i y^j with i + j <= degree. */
int orc_poly_terms(int degree) { return (degree + 1) * (degree + 2) / 2; }

/* Monomials of total degree <= `degree` in the order
 * 1, u, v, u^2, uv, v^2, u^3, u^2 v, u v^2, v^3 (graded, u powers first). */
static void poly_basis(double u, double v, int degree, double *phi) {
    int t = 0;
    for (int d = 0; d <= degree; ++d)
        for (int j = 0; j <= d; ++j) {
            double a = 1.0;
            for (int e = 0; e < d - j; ++e) a *= u;
            for (int e = 0; e < j; ++e) a *= v;
            phi[t++] = a;
        }
}

/* One least-squares fit of xs' and ys' over the CPs with keep[i] != 0, from the
 * normal equations.  Returns 1 if the system is singular. */
static int poly_fit(const double *u, const double *v, const double *xp, const double *yp,
                    const int *keep, int n, int degree, double *coef) {
    const int T = orc_poly_terms(degree);
    double M[100], M2[100], bx[10], by[10], phi[10];
    memset(M, 0, sizeof(M));
    memset(bx, 0, sizeof(bx));
    memset(by, 0, sizeof(by));
    for (int i = 0; i < n; ++i) {
        if (!keep[i]) continue;
        poly_basis(u[i], v[i], degree, phi);
        for (int a = 0; a < T; ++a) {
            bx[a] += phi[a] * xp[i];
            by[a] += phi[a] * yp[i];
            for (int b = 0; b < T; ++b) M[a * T + b] += phi[a] * phi[b];
        }
    }
    memcpy(M2, M, sizeof(M));
    if (solve_dense(M, bx, T)) return 1;
    if (solve_dense(M2, by, T)) return 1;
    for (int a = 0; a < T; ++a) {
        coef[a] = bx[a];
        coef[10 + a] = by[a];
    }
    return 0;
}

/* Squared residual e_i^2 of CP i under coef (distance to the model's prediction). */
static double poly_resid2(double u, double v, double xp, double yp, int degree, const double *coef) {
    const int T = orc_poly_terms(degree);
    double phi[10], px = 0.0, py = 0.0;
    poly_basis(u, v, degree, phi);
    for (int a = 0; a < T; ++a) {
        px += coef[a] * phi[a];
        py += coef[10 + a] * phi[a];
    }
    return (xp - px) * (xp - px) + (yp - py) * (yp - py);
}

/* Sec. IV: (1) fit the mapping model to all CPs; (2) compute residuals and the
 * RMSE, drop the CP with the largest residual; (3) repeat until the RMSE is
 * below the threshold.  The model is the polynomial of total degree `degree`
 * (the paper's system: cubic) mapping (x, y) to (xp, yp).
 *
 * Reading: the monomials are taken in normalised coordinates u = (x - cx)/s,
 * v = (y - cy)/s, with (cx, cy) the centre of the bounding box of the valid CPs
 * and s the larger half-side (1 when 0).  Polynomials of degree <= d are closed
 * under this change of variables, so the fitted mapping is the same; only the
 * conditioning of the normal equations changes.
 * Reading: residual = Euclidean distance between (xp, yp) and the prediction,
 * RMSE = sqrt(mean of squared residuals over the kept CPs); ties of the largest
 * residual go to the lowest index.
 * Reading: the loop also stops when one more removal would leave fewer than
 * max(min_keep, terms) CPs (status 1), and a removal that would make the normal
 * equations singular is undone (status 2).  A singular first fit gives status 2,
 * rmse = -1 and zero coefficients.
 *
 * Outputs: keep[n] (1 = kept), order[n_removed] (indices in removal order),
 * coef[20] (x' coefficients, then y' at offset 10), norm3 = {cx, cy, s},
 * *rmse, *n_removed, *n_fits.  Returns the status (0: RMSE < threshold). */
int orc_reject_outliers(const double *x, const double *y, const double *xp, const double *yp,
                        const int *valid, int n, int degree, double thr, int min_keep, int *keep,
                        int *order, int *n_removed, double *coef, double *rmse, double *norm3,
                        int *n_fits) {
    const int T = orc_poly_terms(degree);
    double xmin = INFINITY, xmax = -INFINITY, ymin = INFINITY, ymax = -INFINITY;
    int kept = 0;
    for (int i = 0; i < n; ++i) {
        keep[i] = valid ? (valid[i] != 0) : 1;
        if (!keep[i]) continue;
        ++kept;
        xmin = fmin(xmin, x[i]);
        xmax = fmax(xmax, x[i]);
        ymin = fmin(ymin, y[i]);
        ymax = fmax(ymax, y[i]);
    }
    double cx = 0.0, cy = 0.0, s = 1.0;
    if (kept > 0) {
        cx = 0.5 * (xmin + xmax);
        cy = 0.5 * (ymin + ymax);
        s = fmax(0.5 * (xmax - xmin), 0.5 * (ymax - ymin));
        if (!(s > 0.0)) s = 1.0;
    }
    norm3[0] = cx;
    norm3[1] = cy;
    norm3[2] = s;
    double *u = (double *)malloc(sizeof(double) * (n > 0 ? n : 1));
    double *v = (double *)malloc(sizeof(double) * (n > 0 ? n : 1));
    for (int i = 0; i < n; ++i) {
        u[i] = (x[i] - cx) / s;
        v[i] = (y[i] - cy) / s;
    }
    for (int a = 0; a < 20; ++a) coef[a] = 0.0;
    *n_removed = 0;
    *n_fits = 0;
    *rmse = -1.0;
    int status = 2;
    double c[20];
    ++*n_fits;
    if (kept == 0 || poly_fit(u, v, xp, yp, keep, n, degree, c)) goto done;
    const int floor_n = min_keep > T ? min_keep : T;
    for (;;) {
        double sum = 0.0, worst = -1.0;
        int wi = -1;
        for (int i = 0; i < n; ++i) {
            if (!keep[i]) continue;
            const double e2 = poly_resid2(u[i], v[i], xp[i], yp[i], degree, c);
            sum += e2;
            if (e2 > worst) {
                worst = e2;
                wi = i;
            }
        }
        const double r = sqrt(sum / (double)kept);
        memcpy(coef, c, sizeof(c));
        *rmse = r;
        if (wi < 0 || !isfinite(r)) {
            break;   /* non-finite residuals cannot be ranked: status 2 */
        }
        if (r < thr) {
            status = 0;
            break;
        }
        if (kept - 1 < floor_n) {
            status = 1;
            break;
        }
        keep[wi] = 0;
        ++*n_fits;
        if (poly_fit(u, v, xp, yp, keep, n, degree, c)) {
            keep[wi] = 1;   /* undo: the kept set stays fittable */
            status = 2;
            break;
        }
        order[(*n_removed)++] = wi;
        --kept;
    }
done:
    free(u);
    free(v);
    return status;
}

/* ------------------------------------------------------------------------ */
/* Pixel-wise HOG (Sec. III-C, the FHOG descriptor of the framework)           */
/* ------------------------------------------------------------------------ */

/* Sec. III-C: at every pixel, a block centred on it of 2 x 2 cells, gradient
 * orientations in [0, 180) degrees quantised into 9 bins; each block pixel
 * adds its gradient magnitude to the histogram bins next to its position and
 * orientation by trilinear interpolation; the 36 bins are L2-normalised.
 * Readings:
 *   - cells are `cell` pixels wide (8, the usual HOG cell); the two cell
 *     centres along an axis lie at -cell/2 and +cell/2 from the pixel, and the
 *     block covers offsets -cell..cell, so it is symmetric about the pixel;
 *   - spatial weight of a block pixel for a cell: 1 - |offset - centre| / cell
 *     per axis, zero when negative (bilinear between the two cell centres);
 *   - orientation weight: the first scheme of Sec. III-F, bins centred on
 *     k*pi/9 wrapping at pi (see orc_channels_binned);
 *   - gradients by [-1,0,1] with replicate borders, block pixels outside the
 *     image replicate the edge pixel (as in the CFOG chain);
 *   - D = h / (||h||_2 + eps).
 * Output: 36 planes, plane (cy*2 + cx)*9 + k for cell row cy, cell column cx
 * (0 = the cell at -cell/2), bin k; sqnorm = ||D||^2 per pixel. */
void orc_fhog(const double *img, int h, int w, int cell, double eps, double *out, double *sqnorm) {
    const int m = 9;
    size_t hw = (size_t)h * w;
    double *gx = (double *)malloc(sizeof(double) * hw);
    double *gy = (double *)malloc(sizeof(double) * hw);
    double *mag = (double *)malloc(sizeof(double) * hw);
    double *frac = (double *)malloc(sizeof(double) * hw);
    int *bin = (int *)malloc(sizeof(int) * hw);
    orc_gradients(img, h, w, gx, gy);
    for (size_t p = 0; p < hw; ++p) {
        mag[p] = sqrt(gx[p] * gx[p] + gy[p] * gy[p]);
        double phi = atan2(gy[p], gx[p]);
        if (phi < 0.0) phi += M_PI;
        if (phi >= M_PI) phi -= M_PI;
        double t = phi / (M_PI / (double)m);
        int k0 = (int)floor(t);
        frac[p] = t - (double)k0;
        bin[p] = k0 % m;
    }
    const double half = 0.5 * (double)cell;
#pragma omp parallel for schedule(dynamic, 4)
    for (int y = 0; y < h; ++y) {
        for (int x = 0; x < w; ++x) {
            double hist[36];
            for (int i = 0; i < 36; ++i) hist[i] = 0.0;
            for (int dy = -cell; dy <= cell; ++dy) {
                const int qy = clampi(y + dy, 0, h - 1);
                for (int dx = -cell; dx <= cell; ++dx) {
                    const int qx = clampi(x + dx, 0, w - 1);
                    const size_t q = (size_t)qy * w + qx;
                    if (mag[q] == 0.0) continue;
                    for (int cy = 0; cy < 2; ++cy) {
                        const double wy = 1.0 - fabs((double)dy - (cy ? half : -half)) / (double)cell;
                        if (wy <= 0.0) continue;
                        for (int cx = 0; cx < 2; ++cx) {
                            const double wx = 1.0 - fabs((double)dx - (cx ? half : -half)) / (double)cell;
                            if (wx <= 0.0) continue;
                            const double v = mag[q] * wx * wy;
                            const int base = (cy * 2 + cx) * m;
                            hist[base + bin[q]] += v * (1.0 - frac[q]);
                            hist[base + (bin[q] + 1) % m] += v * frac[q];
                        }
                    }
                }
            }
            double ss = 0.0;
            for (int i = 0; i < 36; ++i) ss += hist[i] * hist[i];
            const double inv = 1.0 / (sqrt(ss) + eps);
            double dd = 0.0;
            for (int i = 0; i < 36; ++i) {
                const double d = hist[i] * inv;
                out[(size_t)i * hw + (size_t)y * w + x] = d;
                dd += d * d;
            }
            sqnorm[(size_t)y * w + x] = dd;
        }
    }
    free(gx);
    free(gy);
    free(mag);
    free(frac);
    free(bin);
}

/* ------------------------------------------------------------------------ */
/* Piecewise-linear rectification on a TIN (Sec. IV, image rectification)      */
/* ------------------------------------------------------------------------ */

static int64_t orient_i(int ax, int ay, int bx, int by, int qx, int qy) {
    return ((int64_t)bx - ax) * ((int64_t)qy - ay) - ((int64_t)by - ay) * ((int64_t)qx - ax);
}

/* Sec. IV: the image is divided into triangles; in each, the affine
 * transformation fixed by its three CP correspondences maps the reference
 * grid into the sensed image, which is resampled there.  Triangle t has
 * reference vertices (rx, ry)[tris[3t + k]] and sensed vertices (su, sv)[..].
 * Readings: a reference pixel (x, y) belongs to a triangle when it is inside
 * or on an edge (exact integer orientation tests); among several, the lowest
 * triangle index; the affine map is evaluated as the barycentric combination
 * of the sensed vertices; the sensed image is interpolated bilinearly, inside
 * 0 <= u <= w-1, 0 <= v <= h-1, else `nodata`; pixels in no triangle get
 * `nodata`.  Degenerate or clockwise triangles cover nothing. */
void orc_tin_rectify(const double *sen, int sh, int sw, const int *rx, const int *ry, const double *su,
                     const double *sv, const int *tris, int n_tris, int oh, int ow, double nodata,
                     double *out) {
#pragma omp parallel for schedule(dynamic, 4)
    for (int y = 0; y < oh; ++y) {
        for (int x = 0; x < ow; ++x) {
            double val = nodata;
            for (int t = 0; t < n_tris; ++t) {
                const int a = tris[3 * t], b = tris[3 * t + 1], c = tris[3 * t + 2];
                const int64_t area = orient_i(rx[a], ry[a], rx[b], ry[b], rx[c], ry[c]);
                if (area <= 0) continue;
                const int64_t la = orient_i(rx[b], ry[b], rx[c], ry[c], x, y);
                const int64_t lb = orient_i(rx[c], ry[c], rx[a], ry[a], x, y);
                const int64_t lc = orient_i(rx[a], ry[a], rx[b], ry[b], x, y);
                if (la < 0 || lb < 0 || lc < 0) continue;
                const double wa = (double)la / (double)area, wb = (double)lb / (double)area,
                             wc = (double)lc / (double)area;
                const double u = wa * su[a] + wb * su[b] + wc * su[c];
                const double v = wa * sv[a] + wb * sv[b] + wc * sv[c];
                if (u >= 0.0 && v >= 0.0 && u <= (double)(sw - 1) && v <= (double)(sh - 1)) {
                    const int iu = (int)floor(u), iv = (int)floor(v);
                    const int iu1 = iu + 1 < sw ? iu + 1 : sw - 1, iv1 = iv + 1 < sh ? iv + 1 : sh - 1;
                    const double fu = u - iu, fv = v - iv;
                    const double top = (1.0 - fu) * sen[(size_t)iv * sw + iu] + fu * sen[(size_t)iv * sw + iu1];
                    const double bot = (1.0 - fu) * sen[(size_t)iv1 * sw + iu] + fu * sen[(size_t)iv1 * sw + iu1];
                    val = (1.0 - fv) * top + fv * bot;
                }
                break;
            }
            out[(size_t)y * ow + x] = val;
        }
    }
}
