"""GPU parity: every kernel through the C ABI against the FP64 oracle."""
import numpy as np
import pytest

import oracle
import synth
from tests._util import (CFOG_ATOL, SURF_REL, check_match_parity, cuda_or_skip, gpu_results,
                         to_dev)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch, P = cuda_or_skip()
    oracle.build()
    return torch, P


def _gpu_cfog(torch, P, img, **kw):
    p = P.params(**kw) if kw else None
    f = P.cfog_extract(to_dev(torch, img), p)
    torch.cuda.synchronize()
    return f, f.volume().cpu().numpy().astype(np.float64), f.sq().cpu().numpy().astype(np.float64)


# ------------------------------------------------------------------ CFOG --

def test_cfog_parity_tiny_pair(env):
    torch, P = env
    pair = synth.tiny_pair(0)
    for img in (pair.A, pair.B):
        _, dg, sg = _gpu_cfog(torch, P, img)
        do, so = oracle.cfog(img)
        assert np.abs(dg - do).max() <= CFOG_ATOL
        assert np.abs(sg - so).max() <= 4 * CFOG_ATOL


@pytest.mark.parametrize("h,w", [(1, 1), (2, 3), (5, 70), (33, 65), (64, 64), (65, 129), (131, 97)])
def test_cfog_parity_shapes_and_tails(env, h, w):
    torch, P = env
    rng = np.random.default_rng(h * 1000 + w)
    img = (rng.random((h, w)) * 255).astype(np.float32)
    _, dg, _ = _gpu_cfog(torch, P, img)
    do, _ = oracle.cfog(img)
    assert np.abs(dg - do).max() <= CFOG_ATOL


def test_cfog_parity_uint16_and_params(env):
    torch, P = env
    rng = np.random.default_rng(3)
    img = rng.integers(0, 4096, size=(150, 203)).astype(np.uint16)
    _, dg, _ = _gpu_cfog(torch, P, img)
    do, _ = oracle.cfog(img.astype(np.float64))
    assert np.abs(dg - do).max() <= CFOG_ATOL
    _, dg, _ = _gpu_cfog(torch, P, img, m=8, sigma=0.6, eps=1e-6, gauss_radius=2)
    do, _ = oracle.cfog(img.astype(np.float64), m=8, sigma=0.6, R=2)
    assert np.abs(dg - do).max() <= CFOG_ATOL


@pytest.mark.parametrize("h,w,m", [(1, 1, 9), (5, 70, 9), (33, 65, 8), (131, 97, 9), (64, 64, 12),
                                   (70, 45, 6)])
def test_cfog_binned_orientation_parity(env, h, w, m):
    """Orientation scheme 1 (Fig. 7): magnitude shared between the two nearest bins."""
    torch, P = env
    rng = np.random.default_rng(h * 7 + w * 3 + m)
    img = (rng.random((h, w)) * 255).astype(np.float32)
    _, dg, sg = _gpu_cfog(torch, P, img, m=m, orientation=P._lib.CFOG_ORIENT_BINS)
    do, so = oracle.cfog(img, m=m, scheme=1)
    assert np.abs(dg - do).max() <= CFOG_ATOL
    assert np.abs(sg - so).max() <= 4 * CFOG_ATOL


def test_cfog_binned_uint16_and_matching(env):
    """Binned features of a u16 pair, then the matcher on them equals the oracle
    matcher on the oracle's binned features."""
    torch, P = env
    pair = synth.tiny_pair(5)
    A = np.clip(np.rint(pair.A * 16), 0, 4095).astype(np.uint16)
    B = np.clip(np.rint(pair.B * 16), 0, 4095).astype(np.uint16)
    fa, dga, _ = _gpu_cfog(torch, P, A, orientation=P._lib.CFOG_ORIENT_BINS)
    fb, dgb, _ = _gpu_cfog(torch, P, B, orientation=P._lib.CFOG_ORIENT_BINS)
    doa, _ = oracle.cfog(A.astype(np.float64), scheme=1)
    dob, _ = oracle.cfog(B.astype(np.float64), scheme=1)
    assert np.abs(dga - doa).max() <= CFOG_ATOL and np.abs(dgb - dob).max() <= CFOG_ATOL
    pts = np.array([[128, 128], [100, 140], [150, 110]], dtype=np.int32)
    n = len(pts)
    cps = torch.from_numpy(pts).cuda()
    tm = torch.full((n,), 64, dtype=torch.int32, device="cuda")
    rd = torch.full((n,), 12, dtype=torch.int32, device="cuda")
    res = P.cfog_match(fa, fb, cps, tm, rd, 64, 12)
    torch.cuda.synchronize()
    g = gpu_results(P, res)
    o = oracle.match_many(doa, dob, pts[:, 0], pts[:, 1], np.full(n, 64), np.full(n, 12))
    check_match_parity(g, o)


def test_cfog_constant_image_is_zero(env):
    torch, P = env
    _, dg, sg = _gpu_cfog(torch, P, np.full((40, 70), 9.0, np.float32))
    assert (dg == 0).all() and (sg == 0).all()


# ---------------------------------------------------------------- Harris --

def _check_harris(pts, resp, grid_x, grid_y, k, chip, margin):
    h, w = resp.shape
    ox, oy = oracle.detect(resp, grid_x, grid_y, k, chip, margin)
    n_exact = 0
    for c in range(grid_x * grid_y):
        gj, gi = divmod(c, grid_x)
        y0, y1, x0, x1 = oracle.cell_chip(h, w, grid_x, grid_y, chip, margin, gj, gi)
        sub = resp[y0:y1, x0:x1]
        scale = np.abs(sub).max() + 1e-30
        for s in range(k):
            i = c * k + s
            gx, gy = pts[i]
            assert y0 <= gy < y1 and x0 <= gx < x1
            if (gx, gy) == (ox[i], oy[i]):
                n_exact += 1
                continue
            # a different pixel is valid only as a near-tie of the oracle's choice
            assert abs(resp[gy, gx] - resp[oy[i], ox[i]]) <= 1e-5 * scale
    return n_exact


def test_harris_parity_tiny(env):
    torch, P = env
    A = synth.tiny_pair(0).A
    resp = oracle.harris(A)
    for (gx, gy, k, chip, margin) in [(4, 4, 2, 40, 20), (5, 3, 1, 0, 0), (8, 8, 3, 0, 9)]:
        pts = P.cfog_detect_cps(to_dev(torch, A), gx, gy, k, chip, margin).cpu().numpy()
        n = _check_harris(pts, resp, gx, gy, k, chip, margin)
        assert n >= 0.9 * gx * gy * k


def test_harris_uint16_and_large_chip(env):
    torch, P = env
    rng = np.random.default_rng(5)
    A = (synth.rect_texture(rng, 600, 520) * 16).astype(np.uint16)
    resp = oracle.harris(A.astype(np.float64))
    pts = P.cfog_detect_cps(to_dev(torch, A), 3, 3, 2, 0, 10).cpu().numpy()
    _check_harris(pts, resp, 3, 3, 2, 0, 10)   # cells of 193 x 166 pixels
    with pytest.raises(P.CfogError):            # a 290-pixel chip exceeds the limit
        P.cfog_detect_cps(to_dev(torch, A), 2, 2, 2, 0, 10)


# -------------------------------------------------------------- matching --

def _match(torch, P, fr, fs, px, py, N, r, qx=None, qy=None, rmax=None, surface=False, nmax=None):
    n = len(px)
    cps = torch.tensor(np.stack([px, py], 1).astype(np.int32), device="cuda")
    tm = torch.tensor(np.asarray(N, np.int32), device="cuda")
    rd = torch.tensor(np.asarray(r, np.int32), device="cuda")
    prior = None
    if qx is not None:
        prior = torch.tensor(np.stack([qx, qy], 1).astype(np.int32), device="cuda")
    rmax = int(np.max(r)) if rmax is None else rmax
    nmax = int(np.max(N)) if nmax is None else nmax
    surf = None
    if surface:
        surf = torch.full((n, (2 * rmax + 1) ** 2), float("nan"), device="cuda")
    res = P.cfog_match(fr, fs, cps, tm, rd, nmax, rmax, prior, surface=surf)
    torch.cuda.synchronize()
    out = gpu_results(P, res)
    out["raw"] = res.cpu().numpy()
    if surface:
        out["surface"] = surf.cpu().numpy().reshape(n, 2 * rmax + 1, 2 * rmax + 1)
    return out


def test_match_parity_tiny_config(env):
    torch, P = env
    pair = synth.tiny_pair(0)
    fr, _, _ = _gpu_cfog(torch, P, pair.A)
    fs, _, _ = _gpu_cfog(torch, P, pair.B)
    dr, _ = oracle.cfog(pair.A)
    ds, _ = oracle.cfog(pair.B)
    g = _match(torch, P, fr, fs, [128], [128], [64], [16], surface=True)
    o = oracle.match_one(dr, ds, 128, 128, 64, 16, want_surface=True)
    od = {k: np.array([v]) for k, v in o.items() if k != "surface"}
    assert check_match_parity(g, od, max_tie=0).n_ok == 1
    S_o = o["surface"]
    _, E = oracle.ssd_surface(dr, ds, 128, 128, 64, 16)
    assert np.abs(g["surface"][0] - S_o).max() <= SURF_REL * E.min()


def _mixed_cps(rng, h, w, n, sizes, radii, prior=3):
    N = rng.choice(sizes, n).astype(np.int32)
    r = rng.choice(radii, n).astype(np.int32)
    px = rng.integers(0, w, n).astype(np.int32)
    py = rng.integers(0, h, n).astype(np.int32)
    qx = rng.integers(-prior, prior + 1, n).astype(np.int32)
    qy = rng.integers(-prior, prior + 1, n).astype(np.int32)
    return px, py, N, r, qx, qy


def test_match_parity_mixed_classes(env):
    torch, P = env
    pair = synth.batched_pair(7, size=384)
    fr, _, _ = _gpu_cfog(torch, P, pair.A)
    fs, _, _ = _gpu_cfog(torch, P, pair.B)
    dr, _ = oracle.cfog(pair.A)
    ds, _ = oracle.cfog(pair.B)
    rng = np.random.default_rng(11)
    px, py, N, r, qx, qy = _mixed_cps(rng, 384, 384, 48, [8, 9, 16, 33, 48, 64, 100],
                                      [1, 2, 5, 8, 13, 20])
    g = _match(torch, P, fr, fs, px, py, N, r, qx, qy, surface=True)
    o = oracle.match_many(dr, ds, px, py, N, r, qx, qy)
    n_ok = check_match_parity(g, o).n_ok
    assert (o["status"] == 1).any() and n_ok >= 10
    # full surfaces of the in-bounds CPs
    for i in np.nonzero(o["status"] != 1)[0]:
        ri = int(r[i])
        S_o, E = oracle.ssd_surface(dr, ds, int(px[i]), int(py[i]), int(N[i]), ri, int(qx[i]),
                                    int(qy[i]))
        c = g["surface"].shape[1] // 2
        S_g = g["surface"][i, c - ri:c + ri + 1, c - ri:c + ri + 1]
        assert (np.abs(S_g - S_o) <= SURF_REL * E).all()


def test_match_batch_invariance(env):
    torch, P = env
    pair = synth.batched_pair(8, size=320)
    fr, _, _ = _gpu_cfog(torch, P, pair.A)
    fs, _, _ = _gpu_cfog(torch, P, pair.B)
    rng = np.random.default_rng(12)
    px, py, N, r, qx, qy = _mixed_cps(rng, 320, 320, 24, [16, 48, 64, 96], [3, 8, 20])
    batch = _match(torch, P, fr, fs, px, py, N, r, qx, qy, rmax=32, nmax=128)["raw"]
    for i in range(len(px)):
        one = _match(torch, P, fr, fs, px[i:i + 1], py[i:i + 1], N[i:i + 1], r[i:i + 1],
                     qx[i:i + 1], qy[i:i + 1], rmax=20, nmax=96)["raw"]
        np.testing.assert_array_equal(one[0], batch[i])


def test_match_exact_shift_and_extremes(env):
    torch, P = env
    rng = np.random.default_rng(13)
    base = synth.rect_texture(rng, 400, 400).astype(np.float32)
    shifted = np.roll(base, (7, -5), axis=(0, 1))
    fr, _, _ = _gpu_cfog(torch, P, base)
    fs, _, _ = _gpu_cfog(torch, P, shifted)
    dr, _ = oracle.cfog(base)
    ds, _ = oracle.cfog(shifted)
    # N = 256 with a small radius (blocked plan), r = 32 with a small template,
    # odd N, a peak on the window edge (true shift outside [-r, r])
    px = np.array([200, 200, 190, 201, 150], np.int32)
    py = np.array([200, 195, 210, 199, 150], np.int32)
    N = np.array([256, 8, 33, 64, 48], np.int32)
    r = np.array([8, 32, 9, 12, 4], np.int32)
    g = _match(torch, P, fr, fs, px, py, N, r)
    o = oracle.match_many(dr, ds, px, py, N, r)
    check_match_parity(g, o)
    for i in range(4):
        assert (g["dy"][i], g["dx"][i]) == (7, -5)
        assert g["ssd"][i] <= 1e-3 * o["E"][i]
    assert g["status"][4] == 2 and o["status"][4] == 2


@pytest.mark.parametrize("precision", [0, 1])
def test_match_degenerate_classes(env, precision):
    """Degenerate (N, r) through both precisions: a 1-pixel template, a
    single-lag window (r = 0: the only lag is on the window edge), odd
    windows (the BF16 path's two-row steps end on a zero row), and the radii
    either side of the BF16 path's two-rows-per-MMA limit (2r+1 = 63 and 65).
    Offsets and statuses equal the oracle's; the SSD at the chosen lag is
    within the FP32 surface tolerance."""
    torch, P = env
    rng = np.random.default_rng(61)
    base = rng.normal(100.0, 30.0, (160, 160)).astype(np.float32)
    shifted = np.roll(base, (1, -1), axis=(0, 1))
    fr, _, _ = _gpu_cfog(torch, P, base)
    fs, _, _ = _gpu_cfog(torch, P, shifted)
    dr, _ = oracle.cfog(base)
    ds, _ = oracle.cfog(shifted)
    N = np.array([1, 1, 2, 3, 17, 16, 16, 3], np.int32)
    r = np.array([0, 1, 1, 0, 0, 31, 32, 2], np.int32)
    px = np.full(len(N), 80, np.int32) + np.arange(len(N), dtype=np.int32)
    py = np.full(len(N), 80, np.int32) - np.arange(len(N), dtype=np.int32)
    if precision == 0:
        g = _match(torch, P, fr, fs, px, py, N, r)
    else:
        g = _match_prec(torch, P, fr, fs, px, py, N, r, 1, nmax=32, rmax=32)
    o = oracle.match_many(dr, ds, px, py, N, r)
    check_match_parity(g, o)
    same = (g["dx"] == o["dx"]) & (g["dy"] == o["dy"])   # all but exempted near ties
    np.testing.assert_array_equal(g["status"][same], o["status"][same])
    # r = 0: one lag, on the window edge, no sub-pixel fit
    zero = r == 0
    assert (g["status"][zero] == 2).all() and (g["dx"][zero] == 0).all() and (g["dy"][zero] == 0).all()
    for i in range(len(N)):
        S_o, E = oracle.ssd_surface(dr, ds, int(px[i]), int(py[i]), int(N[i]), int(r[i]))
        iy, ix = int(g["dy"][i]) + int(r[i]), int(g["dx"][i]) + int(r[i])
        assert abs(float(g["ssd"][i]) - S_o[iy, ix]) <= SURF_REL * E[iy, ix]


def test_match_all_out_of_bounds(env):
    torch, P = env
    f, _, _ = _gpu_cfog(torch, P, np.zeros((50, 50), np.float32))
    g = _match(torch, P, f, f, [2, 49, 25], [25, 25, 0], [16, 16, 16], [4, 4, 4])
    assert (g["status"] == 1).all()
    assert np.isinf(g["ssd"]).all()


def test_fit_affine_matches_oracle(env):
    torch, P = env
    rng = np.random.default_rng(14)
    n = 500
    cps = rng.integers(0, 4000, (n, 2)).astype(np.int32)
    res = np.zeros((n, 6), np.int32)
    sub = np.stack([1.5 + 0.001 * cps[:, 0] - 0.002 * cps[:, 1] + rng.normal(0, 0.2, n),
                    -2.0 + 0.0005 * cps[:, 0] + rng.normal(0, 0.2, n)], 1).astype(np.float32)
    res.view(np.float32)[:, 2:4] = sub
    res[:, 5] = (rng.random(n) < 0.8).astype(np.int32) * 2  # 0 OK, 2 EDGE (ignored)
    got = P.cfog_fit_affine(torch.tensor(cps, device="cuda"), torch.tensor(res, device="cuda"))
    v = (res[:, 5] == 0).astype(np.int32)
    x, y = cps[:, 0].astype(np.float64), cps[:, 1].astype(np.float64)
    exp = oracle.affine_ls(x, y, x + sub[:, 0].astype(np.float64), y + sub[:, 1].astype(np.float64),
                           v)
    np.testing.assert_allclose(got, exp, rtol=1e-9, atol=1e-7)


def test_fit_affine_singular_raises(env):
    torch, P = env
    cps = torch.tensor([[10, 10], [20, 20]], dtype=torch.int32, device="cuda")
    res = torch.zeros((2, 6), dtype=torch.int32, device="cuda")
    with pytest.raises(P.CfogError):
        P.cfog_fit_affine(cps, res)


def test_full_size_batched_workload_sampled(env):
    """The benchmark's workload at full size (2048^2 pair, 1024 Harris CPs, mixed
    N and r, one launch): every CP checked by properties, a seeded sample of CPs
    against the oracle's brute force."""
    torch, P = env
    size, grid, margin = 2048, 32, 100
    pair = synth.batched_pair(1, size)
    tm, rd = synth.random_cp_params(101, grid * grid, (48, 64, 96, 128), 8, 20)
    A, B = to_dev(torch, pair.A), to_dev(torch, pair.B)
    fa, fb = P.cfog_extract(A), P.cfog_extract(B)
    cps = P.cfog_detect_cps(A, grid, grid, 1, 0, margin)
    res = P.cfog_match(fa, fb, cps, torch.from_numpy(tm).cuda(), torch.from_numpy(rd).cuda(),
                       128, 20)
    torch.cuda.synchronize()
    g = gpu_results(P, res)
    pts = cps.cpu().numpy()
    # properties of every CP
    assert set(np.unique(g["status"])) <= {0, 2}
    edge = (np.abs(g["dx"]) == rd) | (np.abs(g["dy"]) == rd)
    np.testing.assert_array_equal(edge, g["status"] == 2)
    ok = g["status"] == 0
    assert (np.abs(g["sub_dx"][ok] - g["dx"][ok]) <= 1.0).all()
    assert (np.abs(g["sub_dy"][ok] - g["dy"][ok]) <= 1.0).all()
    assert (g["ssd"] >= -1e-3 * tm.astype(np.float64) ** 2).all()
    # sampled brute force
    rng = np.random.default_rng(2024)
    idx = np.sort(rng.choice(grid * grid, 24, replace=False))
    da, _ = oracle.cfog(pair.A)
    db, _ = oracle.cfog(pair.B)
    o = oracle.match_many(da, db, pts[idx, 0], pts[idx, 1], tm[idx], rd[idx])
    assert check_match_parity({k: v[idx] for k, v in g.items()}, o).n_ok >= 20


# ------------------------------------------------------- batched matching --

def _batched(torch, P, pairs, job_of_cp, px, py, N, r, variant, nmax=128, rmax=20, prior=None):
    jobs = P.job_table(pairs)
    cps = torch.tensor(np.stack([px, py], 1).astype(np.int32), device="cuda")
    tm = torch.tensor(np.asarray(N, np.int32), device="cuda")
    rd = torch.tensor(np.asarray(r, np.int32), device="cuda")
    jo = None if job_of_cp is None else torch.tensor(np.asarray(job_of_cp, np.int32), device="cuda")
    pr = None if prior is None else torch.tensor(np.asarray(prior, np.int32), device="cuda")
    res = P.cfog_match_batched(jobs, len(pairs), cps, tm, rd, nmax, rmax, 9, job_of_cp=jo,
                               prior=pr, variant=variant)
    torch.cuda.synchronize()
    return res.cpu().numpy()


@pytest.mark.parametrize("precision,variant", [(0, 1), (0, 2), (0, 3), (0, 4), (1, 0)])
def test_batched_degenerate_classes(env, precision, variant):
    """Degenerate (N, r) in one persistent launch (FFT planes of 2 x 2 and up,
    single-lag windows): every CP equals the oracle and, bitwise, the same CP
    matched alone in its own launch."""
    torch, P = env
    rng = np.random.default_rng(62)
    base = rng.normal(100.0, 30.0, (160, 160)).astype(np.float32)
    shifted = np.roll(base, (1, -1), axis=(0, 1))
    fr, _, _ = _gpu_cfog(torch, P, base)
    fs, _, _ = _gpu_cfog(torch, P, shifted)
    dr, _ = oracle.cfog(base)
    ds, _ = oracle.cfog(shifted)
    N = np.array([1, 1, 2, 3, 17, 8, 9, 2], np.int32)
    r = np.array([0, 1, 1, 0, 0, 2, 9, 3], np.int32)
    n = len(N)
    px = (60 + 5 * np.arange(n)).astype(np.int32)
    py = (100 - 4 * np.arange(n)).astype(np.int32)

    def run(sel):
        jobs = P.job_table([(fr, fs)])
        cps = torch.tensor(np.stack([px[sel], py[sel]], 1), device="cuda")
        out = P.cfog_match_batched(jobs, 1, cps, torch.tensor(N[sel], device="cuda"),
                                   torch.tensor(r[sel], device="cuda"), 32, 16,
                                   precision=precision, variant=variant)
        torch.cuda.synchronize()
        return out.cpu().numpy()

    res = run(slice(None))
    f = res.view(np.float32)
    g = {"dx": res[:, 0], "dy": res[:, 1], "sub_dx": f[:, 2], "sub_dy": f[:, 3], "ssd": f[:, 4],
         "status": res[:, 5]}
    o = oracle.match_many(dr, ds, px, py, N, r)
    check_match_parity(g, o)
    assert (g["status"][r == 0] == 2).all()
    for i in range(n):
        np.testing.assert_array_equal(run(slice(i, i + 1))[0], res[i])


@pytest.mark.parametrize("variant", [1, 2, 3, 4])
def test_batched_multi_job_parity_and_invariance(env, variant):
    """Two jobs interleaved in one persistent launch: every CP equals the oracle
    and, bitwise, the same CP matched alone in its own launch."""
    torch, P = env
    pairs_np = [synth.batched_pair(21, size=320), synth.batched_pair(22, size=288)]
    feats = [(_gpu_cfog(torch, P, p.A)[0], _gpu_cfog(torch, P, p.B)[0]) for p in pairs_np]
    orc = [(oracle.cfog(p.A)[0], oracle.cfog(p.B)[0]) for p in pairs_np]
    rng = np.random.default_rng(31)
    n = 40
    job = rng.integers(0, 2, n).astype(np.int32)
    px = rng.integers(40, 250, n).astype(np.int32)
    py = rng.integers(40, 250, n).astype(np.int32)
    N = rng.choice([16, 48, 64, 96, 128], n).astype(np.int32)
    r = rng.choice([4, 9, 16, 20], n).astype(np.int32)
    q = rng.integers(-2, 3, (n, 2)).astype(np.int32)
    res = _batched(torch, P, feats, job, px, py, N, r, variant, prior=q)
    g = {k: v for k, v in zip(["dx", "dy"], [res[:, 0], res[:, 1]])}
    g.update({"sub_dx": res.view(np.float32)[:, 2], "sub_dy": res.view(np.float32)[:, 3],
              "ssd": res.view(np.float32)[:, 4], "status": res[:, 5]})
    for j in range(2):
        sel = job == j
        o = oracle.match_many(orc[j][0], orc[j][1], px[sel], py[sel], N[sel], r[sel],
                              q[sel, 0], q[sel, 1])
        check_match_parity({k: v[sel] for k, v in g.items()}, o)
    for i in range(0, n, 7):
        alone = _batched(torch, P, [feats[job[i]]], None, px[i:i + 1], py[i:i + 1], N[i:i + 1],
                         r[i:i + 1], variant, prior=q[i:i + 1])
        np.testing.assert_array_equal(alone[0], res[i])


def test_batched_wide_equals_single_launch_kernel(env):
    torch, P = env
    pair = synth.batched_pair(23, size=300)
    fr, _, _ = _gpu_cfog(torch, P, pair.A)
    fs, _, _ = _gpu_cfog(torch, P, pair.B)
    rng = np.random.default_rng(32)
    px, py, N, r, qx, qy = _mixed_cps(rng, 300, 300, 30, [16, 48, 64, 96], [3, 8, 20])
    single = _match(torch, P, fr, fs, px, py, N, r, qx, qy, rmax=20, nmax=128)["raw"]
    batched = _batched(torch, P, [(fr, fs)], None, px, py, N, r, 1,
                       prior=np.stack([qx, qy], 1))
    np.testing.assert_array_equal(single, batched)


def test_batched_bad_job_index_is_oob(env):
    torch, P = env
    pair = synth.batched_pair(24, size=256)
    fr, _, _ = _gpu_cfog(torch, P, pair.A)
    fs, _, _ = _gpu_cfog(torch, P, pair.B)
    res = _batched(torch, P, [(fr, fs)], [0, 1, -1], [128, 128, 128], [128, 128, 128],
                   [48, 48, 48], [8, 8, 8], 1)
    assert res[0, 5] != 1 and res[1, 5] == 1 and res[2, 5] == 1


def test_batched_workspace_too_small(env):
    torch, P = env
    f = P.alloc_features(64, 64)
    jobs = P.job_table([(f, f)])
    cps = torch.zeros((10, 2), dtype=torch.int32, device="cuda")
    t = torch.full((10,), 16, dtype=torch.int32, device="cuda")
    ws = torch.empty(64, dtype=torch.uint8, device="cuda")
    with pytest.raises(P.CfogError) as e:
        P.cfog_match_batched(jobs, 1, cps, t, t, 16, 16, workspace=ws)
    assert e.value.status == 3


# ------------------------------------------------ BF16 tensor-core variant --

def _match_prec(torch, P, fr, fs, px, py, N, r, precision, qx=None, qy=None, nmax=128, rmax=32):
    n = len(px)
    cps = torch.tensor(np.stack([px, py], 1).astype(np.int32), device="cuda")
    tm = torch.tensor(np.asarray(N, np.int32), device="cuda")
    rd = torch.tensor(np.asarray(r, np.int32), device="cuda")
    prior = None
    if qx is not None:
        prior = torch.tensor(np.stack([qx, qy], 1).astype(np.int32), device="cuda")
    surf = torch.full((n, (2 * rmax + 1) ** 2), float("nan"), device="cuda")
    res = P.cfog_match(fr, fs, cps, tm, rd, nmax, rmax, prior, precision=precision, surface=surf)
    torch.cuda.synchronize()
    out = gpu_results(P, res)
    out["raw"] = res.cpu().numpy()
    out["surface"] = surf.cpu().numpy().reshape(n, 2 * rmax + 1, 2 * rmax + 1)
    return out


def test_bf16_direct_single_cp(env):
    """One CP: BF16 surface within 1e-2 of E(v); re-scored peak equals the oracle's."""
    torch, P = env
    pair = synth.tiny_pair(0)
    fr, _, _ = _gpu_cfog(torch, P, pair.A)
    fs, _, _ = _gpu_cfog(torch, P, pair.B)
    dr, _ = oracle.cfog(pair.A)
    ds, _ = oracle.cfog(pair.B)
    g = _match_prec(torch, P, fr, fs, [128], [128], [64], [16], 1, nmax=64, rmax=16)
    o = oracle.match_one(dr, ds, 128, 128, 64, 16)
    assert check_match_parity(g, {k: np.array([v]) for k, v in o.items()}, max_tie=0).n_ok == 1
    S_o, E = oracle.ssd_surface(dr, ds, 128, 128, 64, 16)
    assert (np.abs(g["surface"][0] - S_o) <= 1e-2 * E).all()


def test_bf16_direct_mixed_classes(env):
    torch, P = env
    pair = synth.batched_pair(9, size=352)
    fr, _, _ = _gpu_cfog(torch, P, pair.A)
    fs, _, _ = _gpu_cfog(torch, P, pair.B)
    dr, _ = oracle.cfog(pair.A)
    ds, _ = oracle.cfog(pair.B)
    rng = np.random.default_rng(33)
    px, py, N, r, qx, qy = _mixed_cps(rng, 352, 352, 40, [8, 16, 33, 48, 64, 96, 128],
                                      [1, 2, 5, 8, 13, 20, 32])
    g = _match_prec(torch, P, fr, fs, px, py, N, r, 1, qx, qy)
    o = oracle.match_many(dr, ds, px, py, N, r, qx, qy)
    n_ok = check_match_parity(g, o).n_ok
    assert n_ok >= 8
    c = g["surface"].shape[1] // 2
    for i in np.nonzero(o["status"] != 1)[0]:
        ri = int(r[i])
        S_o, E = oracle.ssd_surface(dr, ds, int(px[i]), int(py[i]), int(N[i]), ri, int(qx[i]),
                                    int(qy[i]))
        S_g = g["surface"][i, c - ri:c + ri + 1, c - ri:c + ri + 1]
        assert (np.abs(S_g - S_o) <= 1e-2 * E).all()


def _bf16_ops_bytes(N, r):
    """Operand-region bytes of the BF16 kernel for one (N, r): the shared memory
    the FP32 re-scoring may stage into (B operand + BF16 window with its zero
    row and tail + three im2col slots of four window rows, or the ||D||^2
    window with its box-sum rows, rounded to 128 B).  Two window rows share an MMA when 2r+1 <= 64."""
    L, W = 2 * r + 1, N + 2 * r
    J = 2 if L <= 64 else 1
    Nx, Ng = -(-N // 16) * 16, -(-(L + J - 1) // 16) * 16
    CA, JB, Wp = (Nx + 128 // J) // 8, W + Ng - 1, -(-W // 8) * 8
    wb = -(-((W + 1) * Wp * 2 + (4 * CA + 4) * 4) // 16) * 16
    ops = (Nx // 8) * JB * 16 + wb + 3 * 4 * CA * 128
    ops = max(ops, (W * W + W * L) * 4)
    return -(-ops // 128) * 128


def test_bf16_rescoring_spread_candidates(env):
    """Unrelated noise images: the BF16 top-8 lags scatter over the search
    window, so for some CPs the bounding box of their windows does not fit
    beside the template and the FP32 re-scoring stages the whole window.  The
    re-scored SSD at the chosen lag equals the oracle's (Eq. 3) within the FP32
    surface tolerance, and the chosen lag is a near-minimum of the oracle
    surface within the BF16 nomination error."""
    torch, P = env
    rng = np.random.default_rng(41)
    A = rng.normal(128.0, 40.0, (256, 256)).astype(np.float32)
    B = rng.normal(128.0, 40.0, (256, 256)).astype(np.float32)
    fr, _, _ = _gpu_cfog(torch, P, A)
    fs, _, _ = _gpu_cfog(torch, P, B)
    dr, _ = oracle.cfog(A)
    ds, _ = oracle.cfog(B)
    N, r = 96, 20
    grid = np.array([70, 110, 150, 186])   # 4 x 4 CPs, every window inside the image
    px, py = (v.ravel() for v in np.meshgrid(grid, grid))
    n = len(px)
    g = _match_prec(torch, P, fr, fs, px, py, np.full(n, N), np.full(n, r), 1, nmax=N, rmax=r)
    L = 2 * r + 1
    spread_path = 0
    for i in range(n):
        S_o, E = oracle.ssd_surface(dr, ds, int(px[i]), int(py[i]), N, r)
        iy, ix = int(g["dy"][i]) + r, int(g["dx"][i]) + r
        assert abs(float(g["ssd"][i]) - S_o[iy, ix]) <= SURF_REL * E[iy, ix]
        assert S_o[iy, ix] - S_o.min() <= 2e-2 * E.max()
        # the kernel's candidate set: 8 smallest BF16 scores (ties: lower
        # index) plus the 3 x 3 neighbourhood of the smallest
        flat = g["surface"][i].reshape(-1)
        top = list(np.argsort(flat, kind="stable")[:8])
        by, bx = divmod(int(top[0]), L)
        for j in (-1, 0, 1):
            for k in (-1, 0, 1):
                if 0 <= by + j < L and 0 <= bx + k < L:
                    top.append((by + j) * L + bx + k)
        ys, xs = np.divmod(np.array(top), L)
        uh, uw = N + ys.max() - ys.min(), N + xs.max() - xs.min()
        spread_path += (uh * uw + N * N) * 4 > _bf16_ops_bytes(N, r)
    assert spread_path >= 1, "no CP exercised the whole-window re-scoring"


def test_bf16_batched_equals_single(env):
    torch, P = env
    pair = synth.batched_pair(10, size=300)
    fr, _, _ = _gpu_cfog(torch, P, pair.A)
    fs, _, _ = _gpu_cfog(torch, P, pair.B)
    rng = np.random.default_rng(34)
    px, py, N, r, qx, qy = _mixed_cps(rng, 300, 300, 20, [32, 64, 96], [4, 12, 20])
    single = _match_prec(torch, P, fr, fs, px, py, N, r, 1, qx, qy, nmax=96, rmax=20)["raw"]
    jobs = P.job_table([(fr, fs)])
    cps = torch.tensor(np.stack([px, py], 1).astype(np.int32), device="cuda")
    res = P.cfog_match_batched(jobs, 1, cps, torch.tensor(N, device="cuda"),
                               torch.tensor(r, device="cuda"), 96, 20,
                               prior=torch.tensor(np.stack([qx, qy], 1), device="cuda"),
                               precision=1)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(res.cpu().numpy(), single)
