"""Pixel-wise HOG (Sec. III-C) on the GPU against the FP64 oracle, and the
matcher on 36-channel HOG volumes (the framework's descriptor generality)."""
import numpy as np
import pytest

import oracle
import synth
from tests._util import CFOG_ATOL, check_match_parity, cuda_or_skip, gpu_results, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch, P = cuda_or_skip()
    oracle.build()
    return torch, P


def _gpu_fhog(torch, P, img, cell=8):
    f = P.cfog_extract_fhog(to_dev(torch, img), cell)
    torch.cuda.synchronize()
    return f, f.volume().cpu().numpy().astype(np.float64), f.sq().cpu().numpy().astype(np.float64)


@pytest.mark.parametrize("h,w,cell", [(1, 1, 8), (5, 70, 8), (33, 65, 8), (70, 45, 8), (131, 97, 8),
                                      (40, 50, 4)])
def test_fhog_parity_shapes(env, h, w, cell):
    torch, P = env
    rng = np.random.default_rng(h * 11 + w)
    img = (rng.random((h, w)) * 255).astype(np.float32)
    _, dg, sg = _gpu_fhog(torch, P, img, cell)
    do, so = oracle.fhog(img, cell)
    assert dg.shape == (36, h, w)
    assert np.abs(dg - do).max() <= CFOG_ATOL
    assert np.abs(sg - so).max() <= 4 * CFOG_ATOL


def test_fhog_uint16_and_constant(env):
    torch, P = env
    rng = np.random.default_rng(9)
    img = (synth.rect_texture(rng, 90, 120) * 16).astype(np.uint16)
    _, dg, _ = _gpu_fhog(torch, P, img)
    do, _ = oracle.fhog(img.astype(np.float64))
    assert np.abs(dg - do).max() <= CFOG_ATOL
    _, dg, sg = _gpu_fhog(torch, P, np.full((30, 40), 7.0, np.float32))
    assert (dg == 0).all() and (sg == 0).all()


def test_fhog_full_size_sampled(env):
    """2048^2 image: sampled pixels against the oracle on a crop around each
    (the descriptor depends on a (2*cell+3)^2 neighbourhood only)."""
    torch, P = env
    pair = synth.batched_pair(1, 2048)
    _, dg, _ = _gpu_fhog(torch, P, pair.A)
    rng = np.random.default_rng(4)
    ys = np.concatenate([[0, 2047, 5], rng.integers(0, 2048, 9)])
    xs = np.concatenate([[0, 2047, 2040], rng.integers(0, 2048, 9)])
    for y, x in zip(ys, xs):
        y0, x0 = max(0, y - 12), max(0, x - 12)
        y1, x1 = min(2048, y + 13), min(2048, x + 13)
        crop = pair.A[y0:y1, x0:x1]
        do, _ = oracle.fhog(crop)
        # a crop edge that is not an image edge would change the replicated
        # pixels, so the crops extend 12 px beyond every block
        np.testing.assert_allclose(dg[:, y, x], do[:, y - y0, x - x0], atol=CFOG_ATOL)


def test_matching_on_fhog_volumes(env):
    """The matcher with m = 36 on GPU HOG volumes equals the oracle matcher on
    the oracle's HOG volumes (batched launch, mixed N and r)."""
    torch, P = env
    pair = synth.tiny_pair(7)
    fa, dga, _ = _gpu_fhog(torch, P, pair.A)
    fb, dgb, _ = _gpu_fhog(torch, P, pair.B)
    doa, _ = oracle.fhog(pair.A)
    dob, _ = oracle.fhog(pair.B)
    assert np.abs(dga - doa).max() <= CFOG_ATOL and np.abs(dgb - dob).max() <= CFOG_ATOL
    pts = np.array([[128, 128], [100, 140], [150, 110], [90, 90]], dtype=np.int32)
    N = np.array([64, 48, 40, 33], dtype=np.int32)
    r = np.array([12, 9, 16, 5], dtype=np.int32)
    cps = torch.from_numpy(pts).cuda()
    tm = torch.from_numpy(N).cuda()
    rd = torch.from_numpy(r).cuda()
    res = P.cfog_match_batched(P.job_table([(fa, fb)]), 1, cps, tm, rd, 64, 16, m=36)
    torch.cuda.synchronize()
    g = gpu_results(P, res)
    o = oracle.match_many(doa, dob, pts[:, 0], pts[:, 1], N, r)
    check_match_parity(g, o)
