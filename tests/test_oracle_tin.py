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


@pytest.mark.parametrize("seed,n", [(0, 3), (1, 30), (2, 300), (3, 2000)])
def test_library_delaunay_equals_scipy(seed, n):
    rng = np.random.default_rng(seed)
    pts = np.unique(rng.integers(0, 5000, (n, 2)), axis=0)
    rng.shuffle(pts)
    T = _lib_tris(pts)
    assert _canon(T) == _canon(Delaunay(pts.astype(float)).simplices)
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
    assert _canon(T) == _canon(sub[Delaunay(g[sub].astype(float)).simplices])
    dup = np.array([[0, 0], [10, 0], [0, 10], [0, 0], [10, 0]])
    T = _lib_tris(dup)
    assert _canon(T) == [(0, 1, 2)]
    assert len(_lib_tris(np.array([[0, 0], [1, 1], [2, 2], [5, 5]]))) == 0
    T = _lib_tris(np.array([[0, 0], [1, 0], [2, 0], [3, 0], [1, 5]]))
    assert len(T) == 3
