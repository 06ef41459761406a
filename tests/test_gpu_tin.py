"""TIN rectification on the GPU (Sec. IV) against the FP64 oracle."""
import numpy as np
import pytest
from scipy.spatial import Delaunay

import oracle
import synth
from tests._util import cuda_or_skip, to_dev

pytestmark = pytest.mark.gpu

NODATA = -1.0


def _setup(seed, n, sh, sw, oh, ow, shift=(3.5, -2.25), jitter=1.5):
    rng = np.random.default_rng(seed)
    pts = np.unique(rng.integers([4, 4], [ow - 4, oh - 4], (n, 2)), axis=0).astype(np.int32)
    res = np.zeros(len(pts), dtype=synth.RESULT_DTYPE)
    res["sub_dx"] = (shift[0] + rng.normal(0, jitter, len(pts))).astype(np.float32)
    res["sub_dy"] = (shift[1] + rng.normal(0, jitter, len(pts))).astype(np.float32)
    sen_xy = pts + np.stack([res["sub_dx"], res["sub_dy"]], 1).astype(np.float64)
    return pts, res, sen_xy


def _run(torch, P, sen, pts, res, tris, oh, ow, **kw):
    c = torch.from_numpy(pts).cuda()
    r = torch.from_numpy(res.view(np.int32).reshape(-1, 6)).cuda()
    t = torch.from_numpy(np.ascontiguousarray(tris, dtype=np.int32)).cuda()
    out = P.cfog_tin_rectify(to_dev(torch, sen), c, r, t, oh, ow, NODATA, **kw)
    torch.cuda.synchronize()
    return out.cpu().numpy().astype(np.float64)


def _compare(g, o, sen, pts, sen_xy, tris, rng_val):
    valid_g, valid_o = g != NODATA, o != NODATA
    both = valid_g & valid_o
    assert both.sum() > 0
    # FP32 maps against FP64: values within 1e-4 of the image range
    assert np.abs(g[both] - o[both]).max() <= 1e-4 * rng_val
    # validity may differ only where the sensed point sits on the image border
    assert (valid_g != valid_o).sum() <= 2e-3 * g.size


@pytest.mark.parametrize("dtype", [np.float32, np.uint16])
def test_tin_rectify_parity(dtype):
    torch, P = cuda_or_skip()
    rng = np.random.default_rng(11)
    sen = (synth.rect_texture(rng, 210, 250) * (16 if dtype == np.uint16 else 1)).astype(dtype)
    pts, res, sen_xy = _setup(12, 70, 210, 250, 200, 240)
    tris = Delaunay(pts.astype(float)).simplices
    g = _run(torch, P, sen, pts, res, tris, 200, 240)
    o = oracle.tin_rectify(sen.astype(np.float64), pts, sen_xy, tris, 200, 240, NODATA)
    _compare(g, o, sen, pts, sen_xy, tris, float(sen.max()) - float(sen.min()))


def test_tin_rectify_library_triangulation_and_overflowing_tiles():
    """Dense CPs (more triangles than a tile lists) and the library's own
    triangulation, equal as a set to scipy's."""
    torch, P = cuda_or_skip()
    rng = np.random.default_rng(13)
    sen = synth.rect_texture(rng, 130, 140).astype(np.float32)
    pts, res, sen_xy = _setup(14, 900, 130, 140, 128, 136, jitter=0.4)
    tris = P.tin_delaunay(pts)
    # integer CPs this dense have co-circular quadruples, so the Delaunay TIN is
    # not unique: check that it is one (no point strictly inside any
    # circumcircle, as many triangles as any triangulation of the hull has)
    ref = Delaunay(pts.astype(float))
    n_hull = len(ref.convex_hull)
    assert len(tris) == len(ref.simplices) == 2 * len(pts) - n_hull - 2
    a, b, c = (pts[tris[:, k]].astype(np.int64) for k in range(3))
    for q in pts.astype(np.int64):
        ad, bd, cd = a - q, b - q, c - q
        la, lb, lc = (ad ** 2).sum(1), (bd ** 2).sum(1), (cd ** 2).sum(1)
        det = (la * (bd[:, 0] * cd[:, 1] - bd[:, 1] * cd[:, 0]) - lb * (ad[:, 0] * cd[:, 1] - ad[:, 1] * cd[:, 0])
               + lc * (ad[:, 0] * bd[:, 1] - ad[:, 1] * bd[:, 0]))
        assert det.max() <= 0
    g = _run(torch, P, sen, pts, res, tris, 128, 136)
    o = oracle.tin_rectify(sen.astype(np.float64), pts, sen_xy, tris, 128, 136, NODATA)
    _compare(g, o, sen, pts, sen_xy, tris, float(sen.max() - sen.min()))


def test_tin_rectify_edges_cases():
    """No triangles, an output larger than the TIN, degenerate triangles, and
    two calls in a row on one workspace give the same result."""
    torch, P = cuda_or_skip()
    sen = np.arange(40 * 50, dtype=np.float32).reshape(40, 50)
    pts = np.array([[5, 5], [40, 6], [6, 30], [30, 30]], dtype=np.int32)
    res = np.zeros(4, dtype=synth.RESULT_DTYPE)
    g = _run(torch, P, sen, pts, res, np.zeros((0, 3), np.int32), 40, 50)
    assert np.all(g == NODATA)
    tris = np.array([[0, 1, 3], [0, 3, 2], [0, 0, 1], [0, 2, 1]], dtype=np.int32)
    ws = P.tin_workspace(4, 70, 90)
    g1 = _run(torch, P, sen, pts, res, tris, 70, 90, workspace=ws)
    g2 = _run(torch, P, sen, pts, res, tris, 70, 90, workspace=ws)
    np.testing.assert_array_equal(g1, g2)
    o = oracle.tin_rectify(sen.astype(np.float64), pts, pts.astype(float), tris, 70, 90, NODATA)
    np.testing.assert_allclose(g1, o, atol=1e-3)
    assert np.all(g1[45:, :] == NODATA)
