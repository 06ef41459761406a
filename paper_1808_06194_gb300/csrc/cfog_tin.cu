// Image rectification with a piecewise-linear model on a triangulated
// irregular network (Sec. IV, "Image rectification"): the kept CPs of the
// reference image are triangulated (Delaunay, on the host), each triangle
// carries the affine map fixed by its three CP correspondences, and every
// pixel of the reference grid is filled from the sensed image at the point its
// triangle's map gives (bilinear interpolation).
//
// Host part: Delaunay triangulation with exact predicates (CP positions are
// integers): take the points by their squared distance from a seed point,
// join each, as a new hull vertex, to the hull edges it sees, and restore the
// empty-circle property after every insertion by edge flips (Lawson).
//
// Device part (K11): one kernel bins the triangles into 64 x 64 pixel tiles
// by their bounding boxes and prepares each triangle's map; the rectify
// kernel takes one 64 x 64 tile per CTA, loads the tile's triangles into shared
// memory, finds each pixel's triangle by exact integer edge tests and samples
// the sensed image.
#include "cfog_internal.cuh"

#include <algorithm>
#include <climits>
#include <cmath>
#include <cstdint>
#include <utility>
#include <vector>

namespace cfog {
namespace {

// ---------------------------------------------------------------- host --
struct HTri {
    int v[3];   // counter-clockwise
    int n[3];   // neighbour across the edge opposite v[i]; -1 on the hull
};

inline int64_t orient2(const cfog_point &a, const cfog_point &b, const cfog_point &c) {
    return ((int64_t)b.x - a.x) * ((int64_t)c.y - a.y) - ((int64_t)b.y - a.y) * ((int64_t)c.x - a.x);
}

// > 0 when d lies inside the circle through the counter-clockwise a, b, c.
// Exact sign: the determinant in 128-bit integers.
inline int incircle_exact(const cfog_point &a, const cfog_point &b, const cfog_point &c,
                          const cfog_point &d) {
    const __int128 adx = (int64_t)a.x - d.x, ady = (int64_t)a.y - d.y;
    const __int128 bdx = (int64_t)b.x - d.x, bdy = (int64_t)b.y - d.y;
    const __int128 cdx = (int64_t)c.x - d.x, cdy = (int64_t)c.y - d.y;
    const __int128 al = adx * adx + ady * ady, bl = bdx * bdx + bdy * bdy, cl = cdx * cdx + cdy * cdy;
    const __int128 det = al * (bdx * cdy - bdy * cdx) - bl * (adx * cdy - ady * cdx) +
                         cl * (adx * bdy - ady * bdx);
    return det > 0 ? 1 : (det < 0 ? -1 : 0);
}

// The same sign through a floating-point filter (Shewchuk, "Adaptive precision
// floating-point arithmetic and fast robust geometric predicates", 1997): the
// determinant in double precision is trusted when it exceeds 1e-14 times the
// permanent of its terms (about nine times the published error bound of this
// evaluation order); otherwise the exact integer determinant decides.  The
// coordinate differences (below 2^28) are exact in double precision.
inline int incircle_sign(const cfog_point &a, const cfog_point &b, const cfog_point &c,
                         const cfog_point &d) {
    const double adx = (double)a.x - d.x, ady = (double)a.y - d.y;
    const double bdx = (double)b.x - d.x, bdy = (double)b.y - d.y;
    const double cdx = (double)c.x - d.x, cdy = (double)c.y - d.y;
    const double bdxcdy = bdx * cdy, cdxbdy = cdx * bdy;
    const double cdxady = cdx * ady, adxcdy = adx * cdy;
    const double adxbdy = adx * bdy, bdxady = bdx * ady;
    const double al = adx * adx + ady * ady, bl = bdx * bdx + bdy * bdy, cl = cdx * cdx + cdy * cdy;
    const double det = al * (bdxcdy - cdxbdy) + bl * (cdxady - adxcdy) + cl * (adxbdy - bdxady);
    const double perm = (std::fabs(bdxcdy) + std::fabs(cdxbdy)) * al +
                        (std::fabs(cdxady) + std::fabs(adxcdy)) * bl +
                        (std::fabs(adxbdy) + std::fabs(bdxady)) * cl;
    const double err = 1e-14 * perm;
    if (det > err) return 1;
    if (det < -err) return -1;
    return incircle_exact(a, b, c, d);
}

struct Delaunay {
    const cfog_point *P;
    std::vector<HTri> T;
    std::vector<int> hnext, hprev;   // counter-clockwise hull, by vertex
    std::vector<int> htri;           // triangle owning hull edge (v, hnext[v])
    std::vector<int> stack;          // flip work list, reused across insertions

    int local(int t, int vtx) const {
        for (int i = 0; i < 3; ++i)
            if (T[t].v[i] == vtx) return i;
        return -1;
    }
    int across(int t, int nb) const {
        for (int i = 0; i < 3; ++i)
            if (T[t].n[i] == nb) return i;
        return -1;
    }
    // Point the neighbour across edge i of t back at t (or record the hull edge).
    void relink(int t, int i) {
        const int u = T[t].n[i];
        const int a = T[t].v[(i + 1) % 3], b = T[t].v[(i + 2) % 3];
        if (u < 0) {
            htri[a] = t;   // hull edge a -> b
            return;
        }
        for (int j = 0; j < 3; ++j) {
            const int ua = T[u].v[(j + 1) % 3], ub = T[u].v[(j + 2) % 3];
            if (ua == b && ub == a) {
                T[u].n[j] = t;
                return;
            }
        }
    }
    int add(int a, int b, int c) {
        HTri h;
        h.v[0] = a;
        h.v[1] = b;
        h.v[2] = c;
        h.n[0] = h.n[1] = h.n[2] = -1;
        T.push_back(h);
        return (int)T.size() - 1;
    }
    // Restore the empty-circle property across the edge opposite p in t.
    void legalize(int t, int p) {
        stack.clear();
        stack.push_back(t);
        while (!stack.empty()) {
            const int x = stack.back();
            stack.pop_back();
            const int i = local(x, p);
            if (i < 0) continue;
            const int u = T[x].n[i];
            if (u < 0) continue;
            const int j = across(u, x);
            const int q = T[u].v[j];
            const int a = T[x].v[(i + 1) % 3], b = T[x].v[(i + 2) % 3];
            if (incircle_sign(P[p], P[a], P[b], P[q]) <= 0) continue;
            // u holds the edge as b -> a: u = (q, b, a) counter-clockwise from q.
            // Flip edge a-b to p-q: x = (p, a, q), u = (p, q, b).
            const int n_bp = T[x].n[(i + 1) % 3];   // across b-p (opposite a in x)
            const int n_pa = T[x].n[(i + 2) % 3];   // across p-a (opposite b in x)
            const int n_aq = T[u].n[(j + 1) % 3];   // across a-q (opposite b in u)
            const int n_qb = T[u].n[(j + 2) % 3];   // across q-b (opposite a in u)
            T[x].v[0] = p; T[x].v[1] = a; T[x].v[2] = q;
            T[x].n[0] = n_aq;
            T[x].n[1] = u;
            T[x].n[2] = n_pa;
            T[u].v[0] = p; T[u].v[1] = q; T[u].v[2] = b;
            T[u].n[0] = n_qb;
            T[u].n[1] = n_bp;
            T[u].n[2] = x;
            // only the edges a-q (now in x) and b-p (now in u) changed triangles
            relink(x, 0);
            relink(u, 1);
            stack.push_back(x);
            stack.push_back(u);
        }
    }
};

// Delaunay triangulation of the distinct points s (any order), as indices
// into P, counter-clockwise.  Radial sweep: the points are taken by their exact
// squared distance from a seed point o (ties: their order in s), so every
// point lies on or outside a circle about o that holds all earlier points and
// is therefore strictly outside their convex hull.  It is joined to the hull
// edges it sees, and edge flips restore the empty-circle property (Lawson).
// The seed triangle is o, the nearest point and the first point of the order
// not collinear with those two.  Returns {} when all points are collinear or
// (never expected) when a point sees no hull edge.
std::vector<HTri> triangulate(const cfog_point *P, const std::vector<int> &s, int npts_total) {
    const int n = (int)s.size();
    if (n < 3) return {};
    // o: the point nearest the centre of the bounding box (exact, ties: first)
    int64_t x0 = P[s[0]].x, x1 = x0, y0 = P[s[0]].y, y1 = y0;
    for (int i : s) {
        x0 = std::min<int64_t>(x0, P[i].x);
        x1 = std::max<int64_t>(x1, P[i].x);
        y0 = std::min<int64_t>(y0, P[i].y);
        y1 = std::max<int64_t>(y1, P[i].y);
    }
    // twice the centre, to stay in integers
    const int64_t cx2 = x0 + x1, cy2 = y0 + y1;
    int o = s[0];
    int64_t best = INT64_MAX;
    for (int i : s) {
        const int64_t dx = 2 * (int64_t)P[i].x - cx2, dy = 2 * (int64_t)P[i].y - cy2;
        const int64_t d = dx * dx + dy * dy;
        if (d < best) {
            best = d;
            o = i;
        }
    }
    // the other points by squared distance from o
    std::vector<std::pair<int64_t, int>> ord;
    ord.reserve(n - 1);
    for (int k = 0; k < n; ++k) {
        const int i = s[k];
        if (i == o) continue;
        const int64_t dx = (int64_t)P[i].x - P[o].x, dy = (int64_t)P[i].y - P[o].y;
        ord.push_back({dx * dx + dy * dy, k});
    }
    std::sort(ord.begin(), ord.end());
    const int a1 = s[ord[0].second];
    size_t j2 = 1;
    while (j2 < ord.size() && orient2(P[o], P[a1], P[s[ord[j2].second]]) == 0) ++j2;
    if (j2 == ord.size()) return {};   // all collinear
    const int a2 = s[ord[j2].second];

    Delaunay D;
    D.P = P;
    D.hnext.assign(npts_total, -1);
    D.hprev.assign(npts_total, -1);
    D.htri.assign(npts_total, -1);
    D.T.reserve(2 * (size_t)n);
    int va = o, vb = a1, vc = a2;
    if (orient2(P[va], P[vb], P[vc]) < 0) std::swap(vb, vc);
    const int t0 = D.add(va, vb, vc);
    auto link = [&](int u, int v) {
        D.hnext[u] = v;
        D.hprev[v] = u;
    };
    link(va, vb);
    link(vb, vc);
    link(vc, va);
    for (int k = 0; k < 3; ++k) D.htri[D.T[t0].v[(k + 1) % 3]] = t0;

    // hull vertices bucketed by the pseudo-angle of their direction from o,
    // to start the search for a visible edge near the new point
    const int nh = std::max(16, (int)std::ceil(std::sqrt((double)n)));
    std::vector<int> hash(nh, -1);
    auto key = [&](int v) {
        const double dx = (double)P[v].x - P[o].x, dy = (double)P[v].y - P[o].y;
        const double q = dx / (std::fabs(dx) + std::fabs(dy));
        const double ang = (dy > 0 ? 3.0 - q : 1.0 + q) / 4.0;   // in [0, 1)
        const int k = (int)(ang * nh);
        return k < 0 ? 0 : (k >= nh ? nh - 1 : k);
    };
    hash[key(va)] = va;
    hash[key(vb)] = vb;
    hash[key(vc)] = vc;

    std::vector<int> made;   // the triangles of one insertion, reused
    for (size_t m = 1; m < ord.size(); ++m) {
        if (m == j2) continue;
        const int p = s[ord[m].second];
        // a hull vertex near p's direction, then forward to a visible edge
        const int kp = key(p);
        int start = -1;
        for (int u = 0; u < nh && start < 0; ++u) {
            const int v = hash[(kp + u) % nh];
            if (v >= 0 && D.hnext[v] >= 0) start = v;
        }
        if (start < 0) return {};
        int e = start;
        while (orient2(P[e], P[D.hnext[e]], P[p]) >= 0) {
            e = D.hnext[e];
            if (e == start) return {};   // p sees no hull edge
        }
        int lo = e, hi = D.hnext[e];
        while (orient2(P[D.hprev[lo]], P[lo], P[p]) < 0) lo = D.hprev[lo];
        while (orient2(P[hi], P[D.hnext[hi]], P[p]) < 0) hi = D.hnext[hi];
        // new triangles (b, a, p) on each visible edge a -> b from lo to hi
        made.clear();
        int prev = -1;
        for (int a = lo; a != hi; a = D.hnext[a]) {
            const int b = D.hnext[a];
            const int ot = D.htri[a];
            const int t = D.add(b, a, p);
            D.T[t].n[2] = ot;   // opposite p: edge b -> a
            D.relink(t, 2);
            if (prev >= 0) {
                D.T[t].n[0] = prev;   // opposite b: edge a -> p
                D.T[prev].n[1] = t;   // opposite a': edge p -> b'
            }
            made.push_back(t);
            prev = t;
        }
        // hull: lo -> p -> hi
        for (int a = D.hnext[lo]; a != hi;) {
            const int nx = D.hnext[a];
            D.hnext[a] = D.hprev[a] = -1;
            a = nx;
        }
        link(lo, p);
        link(p, hi);
        for (int t : made)
            for (int k = 0; k < 3; ++k)
                if (D.T[t].n[k] < 0) D.htri[D.T[t].v[(k + 1) % 3]] = t;
        for (int t : made) D.legalize(t, p);
        hash[kp] = p;
        hash[key(lo)] = lo;
        hash[key(hi)] = hi;
    }
    return D.T;
}

}  // namespace
}  // namespace cfog

namespace cfog {
namespace {

// ---------------------------------------------------------------- device --
constexpr int TT = 64;        // output tile side (pixels)
constexpr int TNT = 256;      // threads per rectify CTA
constexpr int TCAP = 64;      // triangles listed per tile

// One triangle of the TIN: reference vertices (integers, counter-clockwise in
// the sense of orient2 > 0) and the affine map to the sensed image,
// s = s_a + J (q - a), with s_a split into an integer and a fraction so that
// the FP32 evaluation keeps the fraction's precision far from the origin.
struct TinTri {
    int ax, ay, bx, by, cx, cy;
    int iu0, iv0;
    float fu0, fv0;
    float j00, j01, j10, j11;
    int ok;
    int small;   // vertex extent <= 16384: the edge tests fit in 32-bit integers
};

struct TinWork {
    TinTri *tri;
    int *count;   // per tile
    int *list;    // TCAP per tile
    int tiles_x, tiles_y;
};

__device__ __forceinline__ long long orient_d(int ax, int ay, int bx, int by, int qx, int qy) {
    return (long long)(bx - ax) * (long long)(qy - ay) - (long long)(by - ay) * (long long)(qx - ax);
}

__device__ __forceinline__ int orient_s(int ax, int ay, int bx, int by, int qx, int qy) {
    return (bx - ax) * (qy - ay) - (by - ay) * (qx - ax);
}

__device__ __forceinline__ bool tri_contains64(const TinTri &t, int x, int y) {
    return orient_d(t.ax, t.ay, t.bx, t.by, x, y) >= 0 && orient_d(t.bx, t.by, t.cx, t.cy, x, y) >= 0 &&
           orient_d(t.cx, t.cy, t.ax, t.ay, x, y) >= 0;
}

// Inside or on an edge, for a pixel of a tile the triangle's bounding box
// touches.  For a triangle of extent <= 16384 every difference is then below
// 16384 + 32 in magnitude, so each product and the difference of two stay
// below 2^30 and the 32-bit test is exact.
__device__ __forceinline__ bool tri_contains(const TinTri &t, int x, int y) {
    if (t.small)
        return orient_s(t.ax, t.ay, t.bx, t.by, x, y) >= 0 && orient_s(t.bx, t.by, t.cx, t.cy, x, y) >= 0 &&
               orient_s(t.cx, t.cy, t.ax, t.ay, x, y) >= 0;
    return orient_d(t.ax, t.ay, t.bx, t.by, x, y) >= 0 && orient_d(t.bx, t.by, t.cx, t.cy, x, y) >= 0 &&
           orient_d(t.cx, t.cy, t.ax, t.ay, x, y) >= 0;
}

// Per triangle: the affine map in FP64, then its index into the list of every
// output tile its bounding box touches.
__global__ void tin_setup_kernel(const cfog_point *__restrict__ cps, const cfog_match_result *__restrict__ res,
                                 const int32_t *__restrict__ tris, int n_tris, int n_cps, int out_h,
                                 int out_w, TinWork wk) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n_tris) return;
    TinTri T{};
    const int ia = tris[3 * t], ib = tris[3 * t + 1], ic = tris[3 * t + 2];
    T.ok = 0;
    if (ia < 0 || ib < 0 || ic < 0 || ia >= n_cps || ib >= n_cps || ic >= n_cps) {
        wk.tri[t] = T;
        return;
    }
    T.ax = cps[ia].x; T.ay = cps[ia].y;
    T.bx = cps[ib].x; T.by = cps[ib].y;
    T.cx = cps[ic].x; T.cy = cps[ic].y;
    const long long area2 = orient_d(T.ax, T.ay, T.bx, T.by, T.cx, T.cy);
    if (area2 <= 0) {   // degenerate or clockwise: contains nothing
        wk.tri[t] = T;
        return;
    }
    // sensed positions of the vertices
    const double ua = T.ax + (double)res[ia].sub_dx, va = T.ay + (double)res[ia].sub_dy;
    const double ub = T.bx + (double)res[ib].sub_dx, vb = T.by + (double)res[ib].sub_dy;
    const double uc = T.cx + (double)res[ic].sub_dx, vc = T.cy + (double)res[ic].sub_dy;
    // J = [s_b - s_a, s_c - s_a] [b - a, c - a]^-1
    const double e1x = T.bx - T.ax, e1y = T.by - T.ay, e2x = T.cx - T.ax, e2y = T.cy - T.ay;
    const double det = (double)area2;   // e1x*e2y - e1y*e2x
    const double i00 = e2y / det, i01 = -e2x / det, i10 = -e1y / det, i11 = e1x / det;
    const double du1 = ub - ua, dv1 = vb - va, du2 = uc - ua, dv2 = vc - va;
    T.j00 = (float)(du1 * i00 + du2 * i10);
    T.j01 = (float)(du1 * i01 + du2 * i11);
    T.j10 = (float)(dv1 * i00 + dv2 * i10);
    T.j11 = (float)(dv1 * i01 + dv2 * i11);
    const double fu = floor(ua), fv = floor(va);
    T.iu0 = (int)fu;
    T.iv0 = (int)fv;
    T.fu0 = (float)(ua - fu);
    T.fv0 = (float)(va - fv);
    T.ok = 1;
    const int ext = max(max(T.ax, max(T.bx, T.cx)) - min(T.ax, min(T.bx, T.cx)),
                        max(T.ay, max(T.by, T.cy)) - min(T.ay, min(T.by, T.cy)));
    T.small = ext <= 16384 ? 1 : 0;
    wk.tri[t] = T;
    const int x0 = max(0, min(T.ax, min(T.bx, T.cx))), x1 = min(out_w - 1, max(T.ax, max(T.bx, T.cx)));
    const int y0 = max(0, min(T.ay, min(T.by, T.cy))), y1 = min(out_h - 1, max(T.ay, max(T.by, T.cy)));
    if (x0 > x1 || y0 > y1) return;
    for (int ty = y0 / TT; ty <= y1 / TT; ++ty)
        for (int tx = x0 / TT; tx <= x1 / TT; ++tx) {
            const int tile = ty * wk.tiles_x + tx;
            const int slot = atomicAdd(wk.count + tile, 1);
            if (slot < TCAP) wk.list[(size_t)tile * TCAP + slot] = t;
        }
}

template <typename T>
__device__ __forceinline__ float px_at(const T *img, int64_t pitch, int y, int x) {
    return static_cast<float>(__ldg(img + (int64_t)y * pitch + x));
}

// One CTA per output tile: the tile's triangles in shared memory; every
// pixel takes the lowest-index triangle that contains it (exact edge tests),
// maps itself into the sensed image and samples it bilinearly.  Pixels in no
// triangle, or mapped outside the sensed image, get `nodata`.  A tile whose
// list overflowed tests every triangle instead.
template <typename TIn>
__global__ void __launch_bounds__(TNT) tin_rectify_kernel(const TIn *__restrict__ sen, int sh, int sw,
                                                          int64_t spitch, TinWork wk, int n_tris,
                                                          int out_h, int out_w, float nodata,
                                                          float *__restrict__ out, int64_t opitch) {
    __shared__ TinTri st[TCAP];
    __shared__ int sidx[TCAP];
    __shared__ int raw[TCAP];
    __shared__ int4 sedge0[TCAP], sedgea[TCAP], sedgeb[TCAP];   // e0 (+ kind), a, b per edge
    const int tile = blockIdx.x;
    const int tx0 = (tile % wk.tiles_x) * TT, ty0 = (tile / wk.tiles_x) * TT;
    const int cnt = wk.count[tile];
    const bool listed = cnt <= TCAP;
    const int nl = listed ? cnt : 0;
    if (threadIdx.x < nl) raw[threadIdx.x] = wk.list[(size_t)tile * TCAP + threadIdx.x];
    __syncthreads();
    // the list in ascending triangle order (its rank among distinct indices),
    // so the first triangle that contains a pixel is the lowest-index one
    if (threadIdx.x < nl) {
        const int t = raw[threadIdx.x];
        int rank = 0;
        for (int i = 0; i < nl; ++i) rank += raw[i] < t;
        sidx[rank] = t;
        const TinTri T = wk.tri[t];
        st[rank] = T;
        // edge functions relative to the tile origin: E(x0 + i, y0 + j) =
        // e0 + a i + b j for each directed edge P -> Q (a = -(Qy - Py),
        // b = Qx - Px).  e0 is exact in 64 bits and clamped to +-2^30; for a
        // triangle of extent <= 16384 and i, j < TT, |a i + b j| < 2^21, so
        // the 32-bit sum keeps every sign that matters.
        const int px[3] = {T.ax, T.bx, T.cx}, py[3] = {T.ay, T.by, T.cy};
        int4 e;
        int ea[3], eb[3], e0[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const int P = k, Q = (k + 1) % 3;
            ea[k] = -(py[Q] - py[P]);
            eb[k] = px[Q] - px[P];
            const long long v = orient_d(px[P], py[P], px[Q], py[Q], tx0, ty0);
            e0[k] = (int)(v > (1LL << 30) ? (1LL << 30) : (v < -(1LL << 30) ? -(1LL << 30) : v));
        }
        e = make_int4(e0[0], e0[1], e0[2], (T.ok && T.small) ? 1 : (T.ok ? 2 : 0));
        sedge0[rank] = e;
        sedgea[rank] = make_int4(ea[0], ea[1], ea[2], 0);
        sedgeb[rank] = make_int4(eb[0], eb[1], eb[2], 0);
    }
    __syncthreads();
    const int c = threadIdx.x % TT;
    for (int r = threadIdx.x / TT; r < TT; r += TNT / TT) {
        const int x = tx0 + c, y = ty0 + r;
        if (x >= out_w || y >= out_h) continue;
        int best = INT_MAX;
        TinTri T{};
        if (listed) {
            const int li = x - tx0, lj = y - ty0;
            for (int i = 0; i < nl; ++i) {
                const int4 e0 = sedge0[i];
                if (e0.w == 0) continue;
                bool in;
                if (e0.w == 1) {
                    const int4 a = sedgea[i], b = sedgeb[i];
                    in = e0.x + a.x * li + b.x * lj >= 0 && e0.y + a.y * li + b.y * lj >= 0 &&
                         e0.z + a.z * li + b.z * lj >= 0;
                } else {
                    in = tri_contains64(st[i], x, y);
                }
                if (in) {
                    best = sidx[i];
                    T = st[i];
                    break;
                }
            }
        } else {
            for (int t = 0; t < n_tris; ++t) {
                const TinTri U = wk.tri[t];
                if (U.ok && tri_contains64(U, x, y)) {
                    best = t;
                    T = U;
                    break;
                }
            }
        }
        float v = nodata;
        if (best != INT_MAX) {
            const float dx = (float)(x - T.ax), dy = (float)(y - T.ay);
            const float du = T.fu0 + fmaf(T.j00, dx, T.j01 * dy);
            const float dv = T.fv0 + fmaf(T.j10, dx, T.j11 * dy);
            const bool finite = fabsf(du) < 16777216.f && fabsf(dv) < 16777216.f;   // also rejects NaN
            const float fdu = finite ? floorf(du) : 0.f, fdv = finite ? floorf(dv) : 0.f;
            const int iu = T.iu0 + (int)fdu, iv = T.iv0 + (int)fdv;
            const float wu = du - fdu, wv = dv - fdv;
            // inside the sensed image: 0 <= u <= w-1, 0 <= v <= h-1
            const bool in = finite && iu >= 0 && iv >= 0 && (iu < sw - 1 || (iu == sw - 1 && wu == 0.f)) &&
                            (iv < sh - 1 || (iv == sh - 1 && wv == 0.f));
            if (in) {
                const int iu1 = min(iu + 1, sw - 1), iv1 = min(iv + 1, sh - 1);
                const float p00 = px_at(sen, spitch, iv, iu), p01 = px_at(sen, spitch, iv, iu1);
                const float p10 = px_at(sen, spitch, iv1, iu), p11 = px_at(sen, spitch, iv1, iu1);
                const float top = fmaf(wu, p01 - p00, p00), bot = fmaf(wu, p11 - p10, p10);
                v = fmaf(wv, bot - top, top);
            }
        }
        out[(int64_t)y * opitch + x] = v;
    }
}

size_t align256(size_t b) { return (b + 255) / 256 * 256; }

void tin_layout(int32_t n_tris, int32_t out_h, int32_t out_w, size_t *tri_b, size_t *cnt_b, size_t *list_b,
                int *tiles_x, int *tiles_y) {
    *tiles_x = (out_w + TT - 1) / TT;
    *tiles_y = (out_h + TT - 1) / TT;
    const size_t tiles = (size_t)*tiles_x * (size_t)*tiles_y;
    *tri_b = align256((size_t)(n_tris > 0 ? n_tris : 1) * sizeof(TinTri));
    *cnt_b = align256(tiles * sizeof(int));
    *list_b = align256(tiles * TCAP * sizeof(int));
}

}  // namespace
}  // namespace cfog

extern "C" size_t cfog_tin_workspace_bytes(int32_t n_tris, int32_t out_h, int32_t out_w) {
    if (n_tris < 0 || out_h <= 0 || out_w <= 0) return 0;
    size_t a, b, c;
    int tx, ty;
    cfog::tin_layout(n_tris, out_h, out_w, &a, &b, &c, &tx, &ty);
    return a + b + c;
}

extern "C" cfog_status cfog_tin_rectify(const cfog_image *sen, const cfog_point *cps_dev,
                                        const cfog_match_result *res_dev, int32_t n_cps,
                                        const int32_t *tris_dev, int32_t n_tris, int32_t out_h,
                                        int32_t out_w, float nodata, float *out_dev, int64_t out_pitch,
                                        void *work_dev, size_t work_bytes, void *stream) {
    CFOG_TRACE("cfog_tin_rectify");
    using namespace cfog;
    const char *who = "cfog_tin_rectify";
    CFOG_REQUIRE(sen && sen->data, "%s: null sensed image", who);
    CFOG_REQUIRE(sen->h > 0 && sen->w > 0 && sen->pitch >= sen->w, "%s: bad sensed image", who);
    CFOG_REQUIRE(sen->dtype == CFOG_DTYPE_F32 || sen->dtype == CFOG_DTYPE_U16, "%s: unknown dtype %d",
                 who, sen->dtype);
    CFOG_REQUIRE(out_h > 0 && out_w > 0 && out_pitch >= out_w && out_dev, "%s: bad output %dx%d", who,
                 out_h, out_w);
    CFOG_REQUIRE(n_tris >= 0 && n_cps >= 0, "%s: negative counts", who);
    CFOG_REQUIRE(n_tris == 0 || (cps_dev && res_dev && tris_dev), "%s: null CP or triangle array", who);
    CFOG_REQUIRE(work_dev && reinterpret_cast<uintptr_t>(work_dev) % 256 == 0,
                 "%s: workspace null or not 256-byte aligned", who);
    size_t tri_b, cnt_b, list_b;
    TinWork wk;
    tin_layout(n_tris, out_h, out_w, &tri_b, &cnt_b, &list_b, &wk.tiles_x, &wk.tiles_y);
    if (work_bytes < tri_b + cnt_b + list_b) {
        set_error("%s: workspace of %zu bytes, %zu needed", who, work_bytes, tri_b + cnt_b + list_b);
        return CFOG_E_NOMEM;
    }
    unsigned char *w8 = static_cast<unsigned char *>(work_dev);
    wk.tri = reinterpret_cast<TinTri *>(w8);
    wk.count = reinterpret_cast<int *>(w8 + tri_b);
    wk.list = reinterpret_cast<int *>(w8 + tri_b + cnt_b);
    cudaStream_t st = as_stream(stream);
    cfog_status s = check_cuda(cudaMemsetAsync(wk.count, 0, cnt_b, st), "cfog_tin_rectify: clear counts");
    if (s != CFOG_OK) return s;
    if (n_tris > 0) {
        tin_setup_kernel<<<(n_tris + 127) / 128, 128, 0, st>>>(cps_dev, res_dev, tris_dev, n_tris, n_cps,
                                                              out_h, out_w, wk);
        s = check_launch("cfog_tin_rectify: setup launch");
        if (s != CFOG_OK) return s;
    }
    const int tiles = wk.tiles_x * wk.tiles_y;
    if (sen->dtype == CFOG_DTYPE_F32)
        tin_rectify_kernel<float><<<tiles, TNT, 0, st>>>(static_cast<const float *>(sen->data), sen->h,
                                                          sen->w, sen->pitch, wk, n_tris, out_h, out_w,
                                                          nodata, out_dev, out_pitch);
    else
        tin_rectify_kernel<uint16_t><<<tiles, TNT, 0, st>>>(static_cast<const uint16_t *>(sen->data),
                                                             sen->h, sen->w, sen->pitch, wk, n_tris, out_h,
                                                             out_w, nodata, out_dev, out_pitch);
    return check_launch("cfog_tin_rectify: launch");
}

extern "C" cfog_status cfog_tin_delaunay(const cfog_point *pts, int32_t n, const uint8_t *keep,
                                         int32_t *tris, int32_t cap, int32_t *n_tris) {
    CFOG_TRACE("cfog_tin_delaunay");
    using namespace cfog;
    CFOG_REQUIRE(n >= 0, "cfog_tin_delaunay: n = %d < 0", n);
    CFOG_REQUIRE(n_tris, "cfog_tin_delaunay: n_tris is NULL");
    CFOG_REQUIRE(n == 0 || pts, "cfog_tin_delaunay: pts is NULL");
    std::vector<int> idx;
    idx.reserve(n);
    for (int i = 0; i < n; ++i) {
        if (keep && !keep[i]) continue;
        CFOG_REQUIRE(std::abs(pts[i].x) <= (1 << 26) && std::abs(pts[i].y) <= (1 << 26),
                     "cfog_tin_delaunay: point %d outside +-2^26", i);
        idx.push_back(i);
    }
    std::stable_sort(idx.begin(), idx.end(), [&](int a, int b) {
        return pts[a].x != pts[b].x ? pts[a].x < pts[b].x : pts[a].y < pts[b].y;
    });
    std::vector<int> s;   // distinct points, the first (lowest index) of equal ones
    for (int i : idx)
        if (s.empty() || pts[s.back()].x != pts[i].x || pts[s.back()].y != pts[i].y) s.push_back(i);
    const std::vector<HTri> T = triangulate(pts, s, n);
    if (T.empty() && s.size() >= 3) {
        bool collinear = true;
        for (size_t i = 2; i < s.size() && collinear; ++i) collinear = orient2(pts[s[0]], pts[s[1]], pts[s[i]]) == 0;
        if (!collinear) {
            set_error("cfog_tin_delaunay: internal error in the sweep");
            return CFOG_E_INVAL;
        }
    }
    *n_tris = (int32_t)T.size();
    if ((int64_t)T.size() > cap || (!tris && !T.empty())) {
        set_error("cfog_tin_delaunay: %zu triangles, room for %d", T.size(), cap);
        return CFOG_E_NOMEM;
    }
    for (size_t t = 0; t < T.size(); ++t)
        for (int k = 0; k < 3; ++k) tris[3 * t + k] = T[t].v[k];
    return CFOG_OK;
}
