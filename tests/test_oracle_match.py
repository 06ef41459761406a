"""Pins for the oracle's matcher (Eq. 3-9, Sec. V-B), Harris detection and
least-squares fit (Sec. IV)."""
import numpy as np
import pytest
from scipy import ndimage


def _vol(seed, m=4, h=48, w=50):
    rng = np.random.default_rng(seed)
    return rng.random((m, h, w))


def _fft_ssd(dref, dsen, px, py, N, r, qx, qy):
    """Independent statement of the SSD surface through the FFT (Eq. 5, 8, 9):
    S(v) = sum T^2 + sum_window ||D_sen||^2 - 2 * corr(v), with the correlation
    taken by numpy FFTs of the zero-padded template and search window."""
    t0 = N // 2
    T = dref[:, py - t0:py - t0 + N, px - t0:px - t0 + N]
    y0, x0 = py + qy - t0 - r, px + qx - t0 - r
    Wn = N + 2 * r
    Wd = dsen[:, y0:y0 + Wn, x0:x0 + Wn]
    P = Wn
    Tf = np.fft.fft2(T, s=(P, P))
    Wf = np.fft.fft2(Wd, s=(P, P))
    corr = np.real(np.fft.ifft2((np.conj(Tf) * Wf).sum(0)))[:2 * r + 1, :2 * r + 1]
    ones = np.zeros((P, P))
    ones[:N, :N] = 1.0
    box = np.real(np.fft.ifft2(np.conj(np.fft.fft2(ones)) * np.fft.fft2((Wd ** 2).sum(0))))
    box = box[:2 * r + 1, :2 * r + 1]
    return (T ** 2).sum() + box - 2 * corr


@pytest.mark.parametrize("N,r,qx,qy", [(8, 3, 0, 0), (9, 4, 2, -3), (12, 5, -4, 1)])
def test_bruteforce_ssd_equals_fft_ssd(orc, N, r, qx, qy):
    dref, dsen = _vol(10), _vol(11)
    S, E = orc.ssd_surface(dref, dsen, 24, 23, N, r, qx, qy)
    ref = _fft_ssd(dref, dsen, 24, 23, N, r, qx, qy)
    np.testing.assert_allclose(S, ref, rtol=1e-10, atol=1e-10 * E.max())


def test_ssd_sign_convention_and_energy(orc):
    dref, dsen = _vol(12), _vol(13)
    N, r = 7, 3
    S, E = orc.ssd_surface(dref, dsen, 20, 21, N, r, 1, 2)
    # one entry by hand: v = (dy, dx) = (-2, 1)
    t0 = N // 2
    T = dref[:, 21 - t0:21 - t0 + N, 20 - t0:20 - t0 + N]
    Wv = dsen[:, 21 + 2 - 2 - t0:21 + 2 - 2 - t0 + N, 20 + 1 + 1 - t0:20 + 1 + 1 - t0 + N]
    assert S[-2 + r, 1 + r] == pytest.approx(((T - Wv) ** 2).sum(), rel=1e-13)
    assert E[-2 + r, 1 + r] == pytest.approx((T ** 2).sum() + (Wv ** 2).sum(), rel=1e-13)


@pytest.mark.parametrize("shift", [(0, 0), (3, -2), (-5, 4), (6, 6)])
def test_exact_shift_recovered_with_zero_ssd(orc, shift):
    rng = np.random.default_rng(14)
    img = ndimage.gaussian_filter(rng.normal(0, 40, (96, 96)), 1.2)
    dref, _ = orc.cfog(img)
    dsen, _ = orc.cfog(np.roll(img, shift, axis=(0, 1)))
    res = orc.match_one(dref, dsen, 48, 47, 24, 8)
    assert (res["dy"], res["dx"]) == shift
    assert res["ssd"] == 0.0
    assert res["status"] == 0
    # the 3x3 least-squares quadratic does not interpolate: small bias only
    assert res["sub_dx"] == pytest.approx(shift[1], abs=0.05)
    assert res["sub_dy"] == pytest.approx(shift[0], abs=0.05)


def test_prior_offset_is_added(orc):
    rng = np.random.default_rng(15)
    img = ndimage.gaussian_filter(rng.normal(0, 40, (96, 96)), 1.2)
    dref, _ = orc.cfog(img)
    dsen, _ = orc.cfog(np.roll(img, (9, -11), axis=(0, 1)))
    res = orc.match_one(dref, dsen, 50, 45, 20, 4, qx=-10, qy=7)
    assert (res["dy"], res["dx"]) == (9, -11)


def test_out_of_bounds_status(orc):
    d = _vol(16)
    assert orc.ssd_surface(d, d, 3, 20, 8, 2) is None           # template leaves ref
    assert orc.ssd_surface(d, d, 10, 20, 8, 7) is None          # window leaves sen
    assert orc.ssd_surface(d, d, 11, 20, 8, 7) is not None      # exactly fits
    res = orc.match_one(d, d, 3, 20, 8, 2)
    assert res["status"] == 1


def test_tie_break_smallest_dy_then_dx(orc):
    # the first minimum in row-major (dy, dx) order wins
    d = np.zeros((2, 40, 40))
    res = orc.match_one(d, d, 20, 20, 6, 3)
    assert (res["dy"], res["dx"]) == (-3, -3)
    assert res["status"] == 2  # on the window edge


@pytest.mark.parametrize("x0,y0,cross", [(0.0, 0.0, 0.0), (0.31, -0.22, 0.0),
                                         (-0.45, 0.4, 0.3), (0.8, -0.9, -0.2)])
def test_subpixel_recovers_quadratic_minimum(orc, x0, y0, cross):
    xs, ys = np.meshgrid([-1.0, 0.0, 1.0], [-1.0, 0.0, 1.0])
    A = np.array([[2.0, cross], [cross, 1.5]])
    dx, dy = xs - x0, ys - y0
    S = A[0, 0] * dx * dx + 2 * A[0, 1] * dx * dy + A[1, 1] * dy * dy + 5.0
    ox, oy, fb = orc.subpixel(S)
    assert fb == 0
    assert ox == pytest.approx(x0, abs=1e-12)
    assert oy == pytest.approx(y0, abs=1e-12)


def test_subpixel_fallback_for_saddle(orc):
    xs, ys = np.meshgrid([-1.0, 0.0, 1.0], [-1.0, 0.0, 1.0])
    S = xs ** 2 - 0.5 * ys ** 2 + 0.2 * xs
    ox, oy, fb = orc.subpixel(S)
    assert fb == 1
    assert ox == pytest.approx(-0.1, abs=1e-12)   # 1-D parabola in x
    assert oy == 0.0                               # not convex in y


def test_subpixel_on_smooth_shift_ground_truth(orc):
    """A Fourier-shifted smooth image: the fit lands within 0.15 px of truth."""
    rng = np.random.default_rng(17)
    img = ndimage.gaussian_filter(rng.normal(0, 40, (128, 128)), 3.0)
    fy, fx = np.meshgrid(np.fft.fftfreq(128), np.fft.fftfreq(128), indexing="ij")
    sy, sx = 2.3, -1.6
    sh = np.real(np.fft.ifft2(np.fft.fft2(img) * np.exp(-2j * np.pi * (fy * sy + fx * sx))))
    dref, _ = orc.cfog(img)
    dsen, _ = orc.cfog(sh)
    res = orc.match_one(dref, dsen, 64, 64, 48, 5)
    assert abs(res["sub_dx"] - sx) < 0.15 and abs(res["sub_dy"] - sy) < 0.15


def test_match_many_equals_match_one(orc):
    rng = np.random.default_rng(18)
    img = ndimage.gaussian_filter(rng.normal(0, 40, (80, 80)), 1.2)
    dref, _ = orc.cfog(img)
    dsen, _ = orc.cfog(np.roll(img, (2, 1), axis=(0, 1)) + rng.normal(0, 2, (80, 80)))
    px = np.array([30, 40, 50], np.int32)
    py = np.array([35, 40, 45], np.int32)
    N = np.array([16, 20, 12], np.int32)
    r = np.array([4, 5, 6], np.int32)
    many = orc.match_many(dref, dsen, px, py, N, r)
    for i in range(3):
        one = orc.match_one(dref, dsen, int(px[i]), int(py[i]), int(N[i]), int(r[i]))
        assert many["dx"][i] == one["dx"] and many["dy"][i] == one["dy"]
        assert many["ssd"][i] == one["ssd"] and many["sub_dx"][i] == one["sub_dx"]


# ---------------------------------------------------------------- Harris --

def test_harris_matches_scipy_statement(orc):
    rng = np.random.default_rng(19)
    img = ndimage.gaussian_filter(rng.normal(0, 30, (33, 37)), 1.0)
    R = orc.harris(img, 1.5, 4, 0.04)
    gx = ndimage.correlate1d(img, [-1.0, 0.0, 1.0], axis=1, mode="nearest")
    gy = ndimage.correlate1d(img, [-1.0, 0.0, 1.0], axis=0, mode="nearest")

    def g(a):  # radius int(truncate * sigma + 0.5) = 4
        return ndimage.gaussian_filter(a, 1.5, truncate=4.0 / 1.5, mode="nearest")

    a, b, c = g(gx * gx), g(gy * gy), g(gx * gy)
    np.testing.assert_allclose(R, a * b - c * c - 0.04 * (a + b) ** 2, rtol=1e-10,
                               atol=1e-10 * np.abs(R).max())


def test_harris_single_corner(orc):
    img = np.zeros((40, 40))
    img[20:, 20:] = 100.0
    R = orc.harris(img)
    y, x = np.unravel_index(np.argmax(R), R.shape)
    assert abs(y - 19.5) <= 1.0 and abs(x - 19.5) <= 1.0
    # an edge is not a corner: along the straight edge the response is negative
    assert R[30, 20] < 0 and R[20, 30] < 0


def test_detect_equals_bruteforce_argmax(orc):
    rng = np.random.default_rng(20)
    resp = rng.random((64, 80))
    xs, ys = orc.detect(resp, 4, 3, k=2, chip=0, margin=5)
    assert len(xs) == 24
    h, w = resp.shape
    for gj in range(3):
        for gi in range(4):
            y0, y1, x0, x1 = orc.cell_chip(h, w, 4, 3, 0, 5, gj, gi)
            sub = resp[y0:y1, x0:x1]
            order = np.argsort(-sub, axis=None, kind="stable")[:2]
            for s in range(2):
                yy, xx = np.unravel_index(order[s], sub.shape)
                i = (gj * 4 + gi) * 2 + s
                assert (ys[i], xs[i]) == (yy + y0, xx + x0)


def test_cell_chip_centred_and_clipped(orc):
    y0, y1, x0, x1 = orc.cell_chip(1000, 1000, 4, 4, 60, 100, 1, 2)
    # interior 800 -> cells of 200; cell (1, 2): y [300,500), x [500,700)
    assert (y0, y1, x0, x1) == (370, 430, 570, 630)
    assert orc.cell_chip(1000, 1000, 4, 4, 0, 100, 1, 2) == (300, 500, 500, 700)


# ------------------------------------------------------------ affine LS --

def test_affine_exact_recovery(orc):
    rng = np.random.default_rng(21)
    x, y = rng.uniform(0, 1000, 50), rng.uniform(0, 1000, 50)
    p = [3.5, 1.001, -0.004, -7.25, 0.003, 0.9995]
    xp = p[0] + p[1] * x + p[2] * y
    yp = p[3] + p[4] * x + p[5] * y
    np.testing.assert_allclose(orc.affine_ls(x, y, xp, yp), p, rtol=1e-9, atol=1e-9)


def test_affine_matches_lstsq_with_mask(orc):
    rng = np.random.default_rng(22)
    x, y = rng.uniform(0, 500, 40), rng.uniform(0, 500, 40)
    xp = 2 + x + rng.normal(0, 0.5, 40)
    yp = -1 + y + 0.01 * x + rng.normal(0, 0.5, 40)
    valid = (rng.random(40) > 0.3).astype(np.int32)
    got = orc.affine_ls(x, y, xp, yp, valid)
    v = valid.astype(bool)
    A = np.stack([np.ones(v.sum()), x[v], y[v]], 1)
    ex = np.linalg.lstsq(A, xp[v], rcond=None)[0]
    ey = np.linalg.lstsq(A, yp[v], rcond=None)[0]
    np.testing.assert_allclose(got, np.concatenate([ex, ey]), rtol=1e-9, atol=1e-9)
    assert orc.affine_ls(x[:2], y[:2], xp[:2], yp[:2]) is None
