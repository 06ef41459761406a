"""GPU parity on the workloads the benchmark and the configurations run, each
against the FP64 oracle on the same inputs (Sec. III-G, Eq. 3-9; Sec. IV):

* the headline step at full size (2048^2 pair, 1024 Harris CPs, mixed N and
  r) through the batched persistent launch in the variant the benchmark
  times, every CP compared with the oracle's brute force;
* the plain one-CTA-per-CP path against the batched path on the same CPs:
  the same integer offsets except at the oracle's near-ties, and the same
  ground-truth accuracy;
* the map-like precision pair (6 levels, 1-px boundary lines, N(0, 10^2)
  noise) on a crop with N 96 and r 20: full SSD surfaces of the FP32 FFT
  path within 1e-4 of E(v) and of the BF16 tensor-core path within 1e-2,
  peaks against the oracle for both;
* the 12-bit uint16 pair with the SAR-like log-speckle remap, 0.3 degree
  rotation and a georeferenced search prior: integer and sub-pixel offsets.
"""
import numpy as np
import pytest

import oracle
import synth
from tests._util import SUBPIX_ATOL, TIE_REL, check_match_parity, cuda_or_skip, to_dev

pytestmark = pytest.mark.gpu

SIZE, GRID, MARGIN = 2048, 32, 100
TMPL_SIZES, RMIN, RMAX = (48, 64, 96, 128), 8, 20
BF16_REL = 1e-2   # BF16 surface error relative to E(v), before re-scoring


def _unpack(res):
    res = np.asarray(res)
    f = res.view(np.float32)
    return {"dx": res[:, 0], "dy": res[:, 1], "sub_dx": f[:, 2], "sub_dy": f[:, 3],
            "ssd": f[:, 4], "status": res[:, 5]}


@pytest.fixture(scope="module")
def headline():
    """The benchmark's step: features, Harris CPs, per-CP (N, r) and the
    oracle's results for every CP."""
    torch, P = cuda_or_skip()
    oracle.build()
    pair = synth.batched_pair(1, SIZE)
    tm, rd = synth.random_cp_params(101, GRID * GRID, TMPL_SIZES, RMIN, RMAX)
    A, B = to_dev(torch, pair.A), to_dev(torch, pair.B)
    fa, fb = P.cfog_extract(A), P.cfog_extract(B)
    cps = P.cfog_detect_cps(A, GRID, GRID, 1, 0, MARGIN)
    torch.cuda.synchronize()
    pts = cps.cpu().numpy()
    da, _ = oracle.cfog(pair.A)
    db, _ = oracle.cfog(pair.B)
    o = oracle.match_many(da, db, pts[:, 0], pts[:, 1], tm, rd)
    return dict(torch=torch, P=P, pair=pair, tm=tm, rd=rd, fa=fa, fb=fb, cps=cps, pts=pts, o=o)


def _batched(h, variant, precision=0):
    torch, P = h["torch"], h["P"]
    jobs = P.job_table([(h["fa"], h["fb"])])
    res = P.cfog_match_batched(jobs, 1, h["cps"], torch.from_numpy(h["tm"]).cuda(),
                               torch.from_numpy(h["rd"]).cuda(), max(TMPL_SIZES), RMAX,
                               variant=variant, precision=precision)
    torch.cuda.synchronize()
    return _unpack(res.cpu().numpy())


@pytest.mark.parametrize("variant", [0, 2])
def test_headline_batched_every_cp_against_oracle(headline, variant):
    """All 1024 CPs of the full-size step, through the persistent launch
    (library default and the two-CTA-per-SM variant the benchmark picks)."""
    g = _batched(headline, variant)
    p = check_match_parity(g, headline["o"])
    assert p.n_inb == GRID * GRID
    assert p.n_ok >= GRID * GRID - p.n_tie


def test_plain_path_equals_batched_path_accuracy(headline):
    """Same accuracy: the plain path (cfog_match, one CTA per CP, the kernel a
    one-CP-per-launch caller runs) and the batched path agree on every
    integer offset except where the oracle itself has a near-tie; sub-pixel
    offsets agree within the parity tolerance; ground-truth accuracy is the
    same up to those near-ties."""
    h = headline
    torch, P = h["torch"], h["P"]
    plain = P.cfog_match(h["fa"], h["fb"], h["cps"], torch.from_numpy(h["tm"]).cuda(),
                         torch.from_numpy(h["rd"]).cuda(), max(TMPL_SIZES), RMAX)
    torch.cuda.synchronize()
    gp = _unpack(plain.cpu().numpy())
    gb = _batched(h, 2)
    check_match_parity(gp, h["o"])
    tie = h["o"]["gap_rel"] < TIE_REL
    same = (gp["dx"] == gb["dx"]) & (gp["dy"] == gb["dy"])
    assert (same | tie).all()
    both = same & (gp["status"] == 0) & (gb["status"] == 0)
    np.testing.assert_allclose(gp["sub_dx"][both], gb["sub_dx"][both], atol=SUBPIX_ATOL, rtol=0)
    np.testing.assert_allclose(gp["sub_dy"][both], gb["sub_dy"][both], atol=SUBPIX_ATOL, rtol=0)
    ty, tx = h["pair"].truth(h["pts"][:, 1], h["pts"][:, 0])

    def correct(g):
        ok = g["status"] == 0
        return ok & (np.hypot(g["sub_dx"] - tx, g["sub_dy"] - ty) < 1.5)

    assert abs(int(correct(gp).sum()) - int(correct(gb).sum())) <= int((~same).sum())


@pytest.fixture(scope="module")
def precision_crop():
    torch, P = cuda_or_skip()
    oracle.build()
    pair = synth.precision_pair(2, 4096)
    c0, side = 1664, 768
    A = np.ascontiguousarray(pair.A[c0:c0 + side, c0:c0 + side])
    B = np.ascontiguousarray(pair.B[c0:c0 + side, c0:c0 + side])
    dA, dB = to_dev(torch, A), to_dev(torch, B)
    fa, fb = P.cfog_extract(dA), P.cfog_extract(dB)
    margin = 48 + 20 + 17
    cps = P.cfog_detect_cps(dA, 8, 8, 1, 0, margin)
    torch.cuda.synchronize()
    pts = cps.cpu().numpy()
    da, _ = oracle.cfog(A)
    db, _ = oracle.cfog(B)
    n = pts.shape[0]
    N = np.full(n, 96, np.int32)
    r = np.full(n, 20, np.int32)
    o = oracle.match_many(da, db, pts[:, 0], pts[:, 1], N, r)
    return dict(torch=torch, P=P, fa=fa, fb=fb, cps=cps, pts=pts, da=da, db=db, N=N, r=r, o=o)


@pytest.mark.parametrize("precision,rel", [(0, 1e-4), (1, BF16_REL)])
def test_precision_pair_surfaces_and_peaks(precision_crop, precision, rel):
    h = precision_crop
    torch, P = h["torch"], h["P"]
    n = h["pts"].shape[0]
    tm = torch.from_numpy(h["N"]).cuda()
    rd = torch.from_numpy(h["r"]).cuda()
    surf = torch.full((n, 41 * 41), float("nan"), device="cuda")
    res = P.cfog_match(h["fa"], h["fb"], h["cps"], tm, rd, 96, 20, precision=precision,
                       surface=surf)
    torch.cuda.synchronize()
    g = _unpack(res.cpu().numpy())
    p = check_match_parity(g, h["o"])
    assert p.n_inb == n and p.n_ok >= n - p.n_tie
    S_g = surf.cpu().numpy().reshape(n, 41, 41).astype(np.float64)
    worst = 0.0
    for i in range(n):
        S_o, E = oracle.ssd_surface(h["da"], h["db"], int(h["pts"][i, 0]), int(h["pts"][i, 1]),
                                    96, 20)
        worst = max(worst, float((np.abs(S_g[i] - S_o) / E).max()))
    assert worst <= rel, worst
    # the batched launch gives the same peaks for the same precision
    jobs = P.job_table([(h["fa"], h["fb"])])
    gb = _unpack(P.cfog_match_batched(jobs, 1, h["cps"], tm, rd, 96, 20,
                                      precision=precision).cpu().numpy())
    check_match_parity(gb, h["o"])


def test_large_scene_pair_with_georeference_prior():
    """The uint16 log-speckle pair rotated 0.3 degrees, CPs searched around a
    georeferenced prior with up to 3 px error (Sec. IV)."""
    torch, P = cuda_or_skip()
    oracle.build()
    from paper_1808_06194_gb300 import scene
    pair = synth.large_scene_pair(4, size=2048)
    dA, dB = to_dev(torch, pair.A), to_dev(torch, pair.B)
    fa, fb = P.cfog_extract(dA), P.cfog_extract(dB)
    cps = P.cfog_detect_cps(dA, 12, 12, 1, 0, 48 + 16 + 16)
    torch.cuda.synchronize()
    pts = cps.cpu().numpy()
    prior = scene.georeference_prior(pair.field, 3, 11)
    qx, qy = prior(pts[:, 0].astype(np.float64), pts[:, 1].astype(np.float64))
    n = pts.shape[0]
    N = np.full(n, 96, np.int32)
    r = np.full(n, 16, np.int32)
    pr = torch.from_numpy(np.stack([qx, qy], 1).astype(np.int32)).cuda()
    jobs = P.job_table([(fa, fb)])
    g = _unpack(P.cfog_match_batched(jobs, 1, cps, torch.from_numpy(N).cuda(),
                                     torch.from_numpy(r).cuda(), 96, 16, prior=pr).cpu().numpy())
    da, _ = oracle.cfog(pair.A.astype(np.float64))
    db, _ = oracle.cfog(pair.B.astype(np.float64))
    o = oracle.match_many(da, db, pts[:, 0], pts[:, 1], N, r, qx, qy)
    p = check_match_parity(g, o)
    assert p.n_inb >= n - 2 and p.n_ok >= p.n_inb - p.n_tie
    # the prior centres the search: most matches land near the truth
    ty, tx = pair.truth(pts[:, 1], pts[:, 0])
    ok = g["status"] == 0
    assert (np.hypot(g["sub_dx"][ok] - tx[ok], g["sub_dy"][ok] - ty[ok]) < 1.5).mean() > 0.8
