"""Pins for the oracle's CFOG (Sec. III-F, Eq. 2, Fig. 9): each step against an
independent library routine, and the whole chain against invariants and
closed forms that a dropped term, a wrong sign, index or transposition breaks."""
import json
import os

import numpy as np
import pytest
from scipy import ndimage

HERE = os.path.dirname(os.path.abspath(__file__))


def _img(seed, h=40, w=52):
    rng = np.random.default_rng(seed)
    return ndimage.gaussian_filter(rng.normal(0, 50, (h, w)), 1.0) + 100.0


def test_paper_defaults_fixture(orc):
    with open(os.path.join(HERE, "golden", "paper_defaults.json")) as f:
        g = json.load(f)
    assert orc.DEFAULTS["m"] == g["cfog_m"]["value"]
    assert orc.DEFAULTS["sigma"] == g["cfog_sigma"]["value"]


def test_gradients_match_scipy_correlate(orc):
    img = _img(0)
    gx, gy = orc.gradients(img)
    ex = ndimage.correlate1d(img, [-1.0, 0.0, 1.0], axis=1, mode="nearest")
    ey = ndimage.correlate1d(img, [-1.0, 0.0, 1.0], axis=0, mode="nearest")
    np.testing.assert_allclose(gx, ex, rtol=0, atol=1e-12)
    np.testing.assert_allclose(gy, ey, rtol=0, atol=1e-12)


def test_channels_special_orientations(orc):
    rng = np.random.default_rng(1)
    gx = rng.normal(size=(7, 9))
    gy = rng.normal(size=(7, 9))
    g = orc.channels(gx, gy, m=8)
    # theta_0 = 0 -> |gx|; theta_4 = pi/2 -> |gy|; theta_2 = pi/4 -> |gx+gy|/sqrt2
    np.testing.assert_allclose(g[0], np.abs(gx), atol=1e-15)
    np.testing.assert_allclose(g[4], np.abs(gy), atol=1e-15)
    np.testing.assert_allclose(g[2], np.abs(gx + gy) / np.sqrt(2.0), atol=1e-14)
    # theta_6 = 3pi/4 -> |gy - gx|/sqrt2
    np.testing.assert_allclose(g[6], np.abs(gy - gx) / np.sqrt(2.0), atol=1e-14)
    # a unit gradient at angle phi peaks in the nearest bin mod pi
    for phi in np.linspace(0.01, 2 * np.pi - 0.01, 23):
        gg = orc.channels(np.full((1, 1), np.cos(phi)), np.full((1, 1), np.sin(phi)), m=9)
        k = int(np.argmax(gg[:, 0, 0]))
        d = abs(((phi % np.pi) - k * np.pi / 9 + np.pi / 2) % np.pi - np.pi / 2)
        assert d <= np.pi / 18 + 1e-12
        assert gg[:, 0, 0].max() == pytest.approx(abs(np.cos(phi - k * np.pi / 9)))


def test_gauss_taps_sum_and_shape(orc):
    t = orc.gauss_taps(0.8, 3)
    assert t.sum() == pytest.approx(1.0, abs=1e-15)
    np.testing.assert_allclose(t, t[::-1], atol=0)
    assert np.all(np.diff(t[:4]) > 0)


def test_smooth_xy_matches_scipy_gaussian(orc):
    rng = np.random.default_rng(2)
    vol = rng.random((3, 30, 41))
    out = orc.smooth_xy(vol, 0.8, 3)
    # scipy radius = int(truncate * sigma + 0.5) = 3 for truncate = 3.75
    ref = ndimage.gaussian_filter(vol, sigma=(0.0, 0.8, 0.8), truncate=3.75, mode="nearest")
    np.testing.assert_allclose(out, ref, rtol=0, atol=1e-13)


def test_smooth_xy_equals_bruteforce_2d(orc):
    rng = np.random.default_rng(3)
    vol = rng.random((1, 13, 17))
    out = orc.smooth_xy(vol, 1.1, 2)
    t = np.exp(-np.arange(-2, 3) ** 2 / (2 * 1.1 ** 2))
    k2 = np.outer(t, t) / np.outer(t, t).sum()
    ref = ndimage.correlate(vol[0], k2, mode="nearest")
    np.testing.assert_allclose(out[0], ref, atol=1e-13)


def test_smooth_z_matches_scipy_wrap(orc):
    rng = np.random.default_rng(4)
    vol = rng.random((9, 5, 6))
    out = orc.smooth_z(vol)
    ref = ndimage.correlate1d(vol, [0.25, 0.5, 0.25], axis=0, mode="wrap")
    np.testing.assert_allclose(out, ref, atol=1e-15)


def test_normalize_unit_and_zero(orc):
    rng = np.random.default_rng(5)
    vol = rng.random((9, 4, 5))
    vol[:, 0, 0] = 0.0
    d, sq = orc.normalize(vol, 1e-6)
    n = np.sqrt((vol ** 2).sum(0))
    assert np.all(d >= 0)
    assert np.all(d[:, 0, 0] == 0) and sq[0, 0] == 0
    np.testing.assert_allclose(np.sqrt(sq)[n > 1e-3], 1.0, atol=1e-5)
    np.testing.assert_allclose(sq, (d ** 2).sum(0), atol=1e-15)


def test_cfog_constant_image_is_zero(orc):
    d, sq = orc.cfog(np.full((20, 24), 77.0))
    assert np.all(d == 0) and np.all(sq == 0)


def test_cfog_nonneg_unit_norm(orc):
    d, sq = orc.cfog(_img(6))
    assert np.all(d >= 0)
    np.testing.assert_allclose(sq, 1.0, atol=1e-6)


@pytest.mark.parametrize("a,b", [(3.0, 5.0), (-1.0, 255.0), (-0.37, -12.0)])
def test_cfog_affine_intensity_invariance(orc, a, b):
    img = _img(7)
    d0, _ = orc.cfog(img, eps=0.0)
    d1, _ = orc.cfog(a * img + b, eps=0.0)
    np.testing.assert_allclose(d1, d0, atol=1e-12)


def test_cfog_horizontal_flip_permutes_channels(orc):
    img = _img(8)
    m = 9
    d0, _ = orc.cfog(img, m=m)
    d1, _ = orc.cfog(img[:, ::-1], m=m)
    perm = [(m - k) % m for k in range(m)]
    np.testing.assert_allclose(d1, d0[perm][:, :, ::-1], atol=1e-12)


def test_cfog_transpose_permutes_channels_even_m(orc):
    img = _img(9)
    m = 8
    d0, _ = orc.cfog(img, m=m)
    d1, _ = orc.cfog(img.T, m=m)
    perm = [(m // 2 - k) % m for k in range(m)]
    np.testing.assert_allclose(d1, d0[perm].transpose(0, 2, 1), atol=1e-12)


def test_cfog_linear_ramp_closed_form(orc):
    a, b = 1.7, -0.6
    yy, xx = np.mgrid[0:30, 0:30].astype(np.float64)
    d, _ = orc.cfog(a * xx + b * yy, m=9, eps=0.0)
    th = np.arange(9) * np.pi / 9
    g = 2.0 * np.abs(a * np.cos(th) + b * np.sin(th))
    hz = (np.roll(g, 1) + 2 * g + np.roll(g, -1)) / 4
    expect = hz / np.linalg.norm(hz)
    interior = d[:, 5:-5, 5:-5].reshape(9, -1)
    np.testing.assert_allclose(interior, expect[:, None].repeat(interior.shape[1], 1), atol=1e-13)


def test_cfog_without_z_kernel_would_fail_ramp(orc):
    """Sanity: the ramp check is sensitive to the Z kernel (a dropped term)."""
    th = np.arange(9) * np.pi / 9
    g = 2.0 * np.abs(1.7 * np.cos(th) - 0.6 * np.sin(th))
    hz = (np.roll(g, 1) + 2 * g + np.roll(g, -1)) / 4
    assert np.abs(g / np.linalg.norm(g) - hz / np.linalg.norm(hz)).max() > 1e-2


# ------------------------------------------- orientation scheme 1 (Fig. 7) --

def _tri_weights(phi, m):
    """Triangular-kernel statement of the binned channels: weight of bin k is
    max(0, 1 - circular distance from phi to k*pi/m in bin widths)."""
    t = phi / (np.pi / m)
    k = np.arange(m)
    d = np.abs(t[..., None] - k)
    d = np.minimum(d, m - d)
    return np.maximum(0.0, 1.0 - d)


def test_binned_channels_centres_halfway_and_wrap(orc):
    m = 9
    mag = 3.5
    th = np.arange(m) * np.pi / m
    # gradients exactly on bin centres, and their opposites
    gx = np.concatenate([mag * np.cos(th), -mag * np.cos(th)])[None, :]
    gy = np.concatenate([mag * np.sin(th), -mag * np.sin(th)])[None, :]
    g = orc.channels_binned(gx, gy, m)[:, 0, :]
    expect = np.concatenate([np.eye(m), np.eye(m)], axis=1) * mag
    np.testing.assert_allclose(g, expect, atol=1e-12)
    # halfway between bins k and k+1, including the wrap from bin m-1 to bin 0
    half = th + 0.5 * np.pi / m
    g = orc.channels_binned((mag * np.cos(half))[None, :], (mag * np.sin(half))[None, :], m)[:, 0, :]
    expect = 0.5 * mag * (np.eye(m) + np.roll(np.eye(m), 1, axis=0))
    np.testing.assert_allclose(g, expect, atol=1e-12)


def test_binned_channels_equal_triangular_kernel(orc):
    rng = np.random.default_rng(21)
    gx = rng.normal(size=(13, 17))
    gy = rng.normal(size=(13, 17))
    gx[0, 0] = gy[0, 0] = 0.0
    for m in (6, 8, 9, 12):
        g = orc.channels_binned(gx, gy, m)
        phi = np.mod(np.arctan2(gy, gx), np.pi)
        expect = (np.hypot(gx, gy)[..., None] * _tri_weights(phi, m)).transpose(2, 0, 1)
        np.testing.assert_allclose(g, expect, atol=1e-12)
        np.testing.assert_allclose(g.sum(0), np.hypot(gx, gy), atol=1e-12)   # weights sum to one


def test_binned_cfog_ramp_closed_form(orc):
    a, b = 1.7, -0.6
    m = 9
    yy, xx = np.mgrid[0:30, 0:30].astype(np.float64)
    d, _ = orc.cfog(a * xx + b * yy, m=m, eps=0.0, scheme=1)
    g = 2.0 * np.hypot(a, b) * _tri_weights(np.mod(np.arctan2(b, a), np.pi), m)
    hz = (np.roll(g, 1) + 2 * g + np.roll(g, -1)) / 4
    expect = hz / np.linalg.norm(hz)
    interior = d[:, 5:-5, 5:-5].reshape(m, -1)
    np.testing.assert_allclose(interior, expect[:, None].repeat(interior.shape[1], 1), atol=1e-13)


@pytest.mark.parametrize("a,b", [(3.0, 5.0), (-1.0, 255.0)])
def test_binned_cfog_affine_intensity_invariance(orc, a, b):
    img = _img(17)
    d0, _ = orc.cfog(img, eps=0.0, scheme=1)
    d1, _ = orc.cfog(a * img + b, eps=0.0, scheme=1)
    np.testing.assert_allclose(d1, d0, atol=1e-12)


def test_binned_cfog_flip_and_transpose_permutations(orc):
    img = _img(18)
    m = 8
    d0, sq = orc.cfog(img, m=m, scheme=1)
    assert np.all(d0 >= 0)
    np.testing.assert_allclose(sq, 1.0, atol=1e-6)
    d1, _ = orc.cfog(img[:, ::-1], m=m, scheme=1)
    np.testing.assert_allclose(d1, d0[[(m - k) % m for k in range(m)]][:, :, ::-1], atol=1e-12)
    d2, _ = orc.cfog(img.T, m=m, scheme=1)
    np.testing.assert_allclose(d2, d0[[(m // 2 - k) % m for k in range(m)]].transpose(0, 2, 1),
                               atol=1e-12)
