"""Pins for the oracle's piecewise-linear rectification on a TIN (Sec. IV) and
host checks of the library's Delaunay triangulation."""
import numpy as np
import pytest
from scipy.spatial import Delaunay

NODATA = -7.0


def _cps(seed, n=40, h=120, w=150, margin=6):
    rng = np.random.default_rng(seed)
    pts = np.unique(rng.integers([margin, margin], [w - margin, h - margin], (n, 2)), axis=0)
    return pts.astype(np.int32)


def test_identity_map_reproduces_the_image_inside_the_hull(orc):
    rng = np.random.default_rng(1)
    sen = rng.random((120, 150)) * 100
    pts = _cps(2)
    tris = Delaunay(pts.astype(float)).simplices
    out = orc.tin_rectify(sen, pts, pts.astype(float), tris, 120, 150, NODATA)
    yy, xx = np.mgrid[0:120, 0:150]
    inside = Delaunay(pts.astype(float)).find_simplex(np.stack([xx.ravel(), yy.ravel()], 1)) >= 0
    inside = inside.reshape(120, 150)
    np.testing.assert_allclose(out[inside], sen[inside], atol=1e-9)
    # scipy's point location may differ only on hull edges (the oracle counts edges in)
    assert np.all(out[~inside] == NODATA) or np.sum(out[~inside] != NODATA) < 0.02 * (~inside).sum()


def test_global_affine_on_a_linear_image_is_exact(orc):
    yy, xx = np.mgrid[0:200, 0:220].astype(np.float64)
    sen = 0.7 * xx - 0.3 * yy + 5.0            # bilinear interpolation of a plane is exact
    A = np.array([[0.98, 0.05, 6.5], [-0.04, 1.01, 3.25]])
    pts = _cps(3, n=60, h=150, w=160, margin=8)
    uv = pts @ A[:, :2].T + A[:, 2]
    tris = Delaunay(pts.astype(float)).simplices
    out = orc.tin_rectify(sen, pts, uv, tris, 150, 160, NODATA)
    qy, qx = np.mgrid[0:150, 0:160].astype(np.float64)
    u = A[0, 0] * qx + A[0, 1] * qy + A[0, 2]
    v = A[1, 0] * qx + A[1, 1] * qy + A[1, 2]
    ok = out != NODATA
    assert ok.sum() > 0.5 * ok.size
    np.testing.assert_allclose(out[ok], (0.7 * u - 0.3 * v + 5.0)[ok], atol=1e-9)


def test_neighbouring_triangles_agree_on_shared_edges(orc):
    """A pixel on an edge shared by two triangles maps to the same sensed point
    through either triangle (the model is continuous)."""
    rng = np.random.default_rng(4)
    yy, xx = np.mgrid[0:100, 0:100].astype(np.float64)
    sen = 0.5 * xx + 0.25 * yy
    pts = np.array([[10, 10], [90, 10], [10, 90], [90, 90]], dtype=np.int32)
    uv = pts + rng.normal(0, 2.0, pts.shape)
    t1 = np.array([[0, 1, 3], [0, 3, 2]])        # diagonal 0-3 shared
    t2 = t1[::-1]
    o1 = orc.tin_rectify(sen, pts, uv, t1, 100, 100, NODATA)
    o2 = orc.tin_rectify(sen, pts, uv, t2, 100, 100, NODATA)
    d = np.arange(10, 91)
    np.testing.assert_allclose(o1[d, d], o2[d, d], atol=1e-9)   # the diagonal
    off = np.ones((100, 100), bool)
    off[d, d] = False
    np.testing.assert_array_equal(o1[off], o2[off])


def test_degenerate_and_clockwise_triangles_cover_nothing(orc):
    sen = np.ones((20, 20))
    pts = np.array([[2, 2], [15, 2], [2, 15], [8, 8]], dtype=np.int32)
    cw = np.array([[0, 2, 1]])                   # clockwise in the orientation convention
    flat = np.array([[0, 3, 3]])
    for t in (cw, flat):
        out = orc.tin_rectify(sen, pts, pts.astype(float), t, 20, 20, NODATA)
        assert np.all(out == NODATA)


# ------------------------------------------------ library triangulation (host) --

def _lib_tris(pts, keep=None):
    from paper_1808_06194_gb300 import api, build
    build.build()
    return api.tin_delaunay(pts, keep)


def _canon(T):
    return sorted(tuple(sorted(t)) for t in np.asarray(T).tolist())


def _incircle_det(tri_pts, q):
    """Exact incircle determinants of the points q against the circle through
    the counter-clockwise triangle tri_pts (int64: coordinates below 2^13)."""
    a, b, c = (np.asarray(v, np.int64) for v in tri_pts)
    q = np.asarray(q, np.int64)
    ad, bd, cd = a - q, b - q, c - q
    al = (ad * ad).sum(1)
    bl = (bd * bd).sum(1)
    cl = (cd * cd).sum(1)
    return (al * (bd[:, 0] * cd[:, 1] - bd[:, 1] * cd[:, 0])
            - bl * (ad[:, 0] * cd[:, 1] - ad[:, 1] * cd[:, 0])
            + cl * (ad[:, 0] * bd[:, 1] - ad[:, 1] * bd[:, 0]))


def _assert_delaunay_as_scipy(pts, T, S):
    """T is a Delaunay triangulation of pts equal to scipy's S wherever the
    triangulation is unique: the same triangle count, every circumcircle of T
    empty (exact), and every triangle in which T and S differ has a fourth
    point exactly on its circumcircle (there either diagonal is Delaunay)."""
    assert len(T) == len(S)
    pts = np.asarray(pts, np.int64)
    assert np.abs(pts).max() < 2 ** 13
    for t in T:
        d = _incircle_det(pts[t], pts)
        d[t] = 0
        assert (d <= 0).all()
    for t in set(_canon(T)) ^ set(_canon(S)):
        t = list(t)
        a, b, c = pts[t]
        if (b[0] - a[0]) * (c[1] - a[1]) - (b[1] - a[1]) * (c[0] - a[0]) < 0:
            t = [t[0], t[2], t[1]]
        d = _incircle_det(pts[t], pts)
        d[t] = 1
        assert (d == 0).any()


@pytest.mark.parametrize("seed,n", [(0, 3), (1, 30), (2, 300), (3, 2000)])
def test_library_delaunay_equals_scipy(seed, n):
    rng = np.random.default_rng(seed)
    pts = np.unique(rng.integers(0, 5000, (n, 2)), axis=0)
    rng.shuffle(pts)
    T = _lib_tris(pts)
    _assert_delaunay_as_scipy(pts, T, Delaunay(pts.astype(float)).simplices)
    a, b, c = pts[T[:, 0]], pts[T[:, 1]], pts[T[:, 2]]
    orient = (b[:, 0] - a[:, 0]) * (c[:, 1] - a[:, 1]) - (b[:, 1] - a[:, 1]) * (c[:, 0] - a[:, 0])
    assert np.all(orient > 0)


def test_library_delaunay_keep_duplicates_and_collinear():
    rng = np.random.default_rng(5)
    g = (np.stack(np.meshgrid(np.arange(30), np.arange(30)), -1).reshape(-1, 2) * 64
         + rng.integers(0, 40, (900, 2)))
    keep = rng.random(900) > 0.2
    T = _lib_tris(g, keep)
    sub = np.nonzero(keep)[0]
    assert set(np.unique(T)) <= set(sub.tolist())
    local = {v: i for i, v in enumerate(sub.tolist())}
    T_local = np.vectorize(local.get)(T)
    _assert_delaunay_as_scipy(g[sub], T_local, Delaunay(g[sub].astype(float)).simplices)
    dup = np.array([[0, 0], [10, 0], [0, 10], [0, 0], [10, 0]])
    T = _lib_tris(dup)
    assert _canon(T) == [(0, 1, 2)]
    assert len(_lib_tris(np.array([[0, 0], [1, 1], [2, 2], [5, 5]]))) == 0
    T = _lib_tris(np.array([[0, 0], [1, 0], [2, 0], [3, 0], [1, 5]]))
    assert len(T) == 3


def test_delaunay_check_rejects_a_flipped_edge():
    """The comparison above is not vacuous: flipping one interior edge whose
    quadrilateral is not co-circular breaks the empty circle and is caught."""
    rng = np.random.default_rng(11)
    pts = np.unique(rng.integers(0, 3000, (60, 2)), axis=0)
    S = Delaunay(pts.astype(float))
    T = S.simplices.copy()
    for i in range(len(T)):
        for k in range(3):
            j = S.neighbors[i, k]
            if j < 0:
                continue
            a, b = [v for v in T[i] if v != T[i][k]]
            q = [v for v in T[j] if v not in (a, b)][0]
            p = T[i][k]
            quad = [p, a, q, b]
            P4 = pts[quad].astype(np.int64)
            cross = lambda o, u, v: (u[0] - o[0]) * (v[1] - o[1]) - (u[1] - o[1]) * (v[0] - o[0])
            convex = all(cross(P4[m], P4[(m + 1) % 4], P4[(m + 2) % 4]) > 0 for m in range(4)) or \
                all(cross(P4[m], P4[(m + 1) % 4], P4[(m + 2) % 4]) < 0 for m in range(4))
            if not convex:
                continue
            bad = T.copy()
            bad[i] = [p, a, q]
            bad[j] = [p, q, b]
            t_ccw = np.array([t if ((pts[t[1]][0] - pts[t[0]][0]) * (pts[t[2]][1] - pts[t[0]][1])
                                    - (pts[t[1]][1] - pts[t[0]][1]) * (pts[t[2]][0] - pts[t[0]][0])) > 0
                              else t[[0, 2, 1]] for t in bad])
            with pytest.raises(AssertionError):
                _assert_delaunay_as_scipy(pts, t_ccw, S.simplices)
            return
    pytest.fail("no flippable interior edge found")


@pytest.mark.parametrize("seed", range(24))
def test_library_delaunay_stress(seed):
    """Uniform, clustered, jittered-grid (many co-circular quadruples) and
    collinear-run point sets: a Delaunay triangulation equal to scipy's
    wherever it is unique."""
    rng = np.random.default_rng(100 + seed)
    kind = seed % 4
    n = int(rng.integers(20, 400))
    if kind == 0:
        pts = rng.integers(0, 8000, (n, 2))
    elif kind == 1:
        centres = rng.integers(500, 7500, (5, 2))
        pts = centres[rng.integers(0, 5, n)] + rng.integers(-60, 60, (n, 2))
    elif kind == 2:
        pts = rng.integers(0, 20, (n, 2)) * 40 + rng.integers(-1, 2, (n, 2))
    else:
        t = rng.integers(0, 300, n)
        line = rng.integers(0, 3, n)
        pts = np.stack([t * 7 + line * 1000, t * 3 + line * 11], 1)
        pts[: n // 10] = rng.integers(0, 3000, (n // 10, 2))
    pts = np.unique(pts, axis=0)
    rng.shuffle(pts)
    T = _lib_tris(pts)
    _assert_delaunay_as_scipy(pts, T, Delaunay(pts.astype(float)).simplices)


def test_library_delaunay_full_coordinate_range():
    """CPs anywhere in the supported range +-2^26: counter-clockwise triangles,
    the triangle count of the hull, and every circumcircle empty (exact, in
    Python integers)."""
    rng = np.random.default_rng(77)
    pts = np.unique(rng.integers(-(1 << 26), 1 << 26, (150, 2)), axis=0)
    T = _lib_tris(pts)
    P = [tuple(int(v) for v in p) for p in pts]
    hull = Delaunay(pts.astype(float)).convex_hull
    assert len(T) == 2 * len(P) - len(hull) - 2
    for t in T.tolist():
        a, b, c = (P[i] for i in t)
        assert (b[0] - a[0]) * (c[1] - a[1]) - (b[1] - a[1]) * (c[0] - a[0]) > 0
        for i, q in enumerate(P):
            if i in t:
                continue
            ad = (a[0] - q[0], a[1] - q[1])
            bd = (b[0] - q[0], b[1] - q[1])
            cd = (c[0] - q[0], c[1] - q[1])
            det = ((ad[0] ** 2 + ad[1] ** 2) * (bd[0] * cd[1] - bd[1] * cd[0])
                   - (bd[0] ** 2 + bd[1] ** 2) * (ad[0] * cd[1] - ad[1] * cd[0])
                   + (cd[0] ** 2 + cd[1] ** 2) * (ad[0] * bd[1] - ad[1] * bd[0]))
            assert det <= 0
