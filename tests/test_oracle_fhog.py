"""Pins for the oracle's pixel-wise HOG (Sec. III-C): 2 x 2 cells x 9
orientation bins around every pixel, trilinear interpolation, L2 norm."""
import numpy as np
import pytest
from scipy import ndimage


def _img(seed, h=40, w=44):
    rng = np.random.default_rng(seed)
    return ndimage.gaussian_filter(rng.random((h, w)) * 255.0, 1.0)


def _cell_weights(cell):
    """Spatial weight of block offsets -cell..cell for the cell centred at
    -cell/2 (index 0) and +cell/2 (index 1): 1 - |d - c| / cell, clipped at 0."""
    d = np.arange(-cell, cell + 1, dtype=np.float64)
    return [np.maximum(0.0, 1.0 - np.abs(d - c) / cell) for c in (-cell / 2, cell / 2)]


def _separable_statement(orc, img, cell, eps=1e-6):
    """FHOG as a separable correlation of the binned channels with the cell
    weight kernels (edge pixels replicated), then the L2 norm."""
    gx, gy = orc.gradients(img)
    g = orc.channels_binned(gx, gy, 9)
    wk = _cell_weights(cell)
    hist = np.empty((36,) + img.shape)
    for cy in range(2):
        for cx in range(2):
            for k in range(9):
                t = ndimage.correlate1d(g[k], wk[cx], axis=1, mode="nearest")
                hist[(cy * 2 + cx) * 9 + k] = ndimage.correlate1d(t, wk[cy], axis=0, mode="nearest")
    nrm = np.sqrt((hist ** 2).sum(0))
    return hist / (nrm + eps)


@pytest.mark.parametrize("cell", [8, 4])
def test_fhog_equals_separable_triangular_statement(orc, cell):
    img = _img(31)
    d, sq = orc.fhog(img, cell)
    np.testing.assert_allclose(d, _separable_statement(orc, img, cell), atol=1e-12)
    np.testing.assert_allclose(sq, (d ** 2).sum(0), atol=1e-12)


def test_fhog_ramp_closed_form(orc):
    a, b = 1.3, 0.7
    yy, xx = np.mgrid[0:40, 0:40].astype(np.float64)
    d, _ = orc.fhog(a * xx + b * yy, 8, eps=0.0)
    # interior: constant gradient (2a, 2b), every block pixel in one orientation
    phi = np.arctan2(2 * b, 2 * a) % np.pi
    t = phi / (np.pi / 9)
    k0 = int(np.floor(t))
    f = t - k0
    hv = np.zeros(9)
    hv[k0 % 9] += 1 - f
    hv[(k0 + 1) % 9] += f
    v = np.tile(hv, 4)            # the four cells see the same weights in total
    v /= np.linalg.norm(v)
    inner = d[:, 10:-10, 10:-10].reshape(36, -1)
    np.testing.assert_allclose(inner, v[:, None].repeat(inner.shape[1], 1), atol=1e-13)


def test_fhog_constant_nonneg_unit(orc):
    d, sq = orc.fhog(np.full((20, 25), 40.0), 8)
    assert np.all(d == 0) and np.all(sq == 0)
    d, sq = orc.fhog(_img(32), 8)
    assert np.all(d >= 0)
    np.testing.assert_allclose(sq, 1.0, atol=1e-6)


@pytest.mark.parametrize("a,b", [(2.0, 7.0), (-1.0, 255.0)])
def test_fhog_affine_intensity_invariance(orc, a, b):
    img = _img(33)
    d0, _ = orc.fhog(img, 8, eps=0.0)
    d1, _ = orc.fhog(a * img + b, 8, eps=0.0)
    np.testing.assert_allclose(d1, d0, atol=1e-12)


def test_fhog_flips_permute_cells_and_bins(orc):
    img = _img(34)
    d0, _ = orc.fhog(img, 8)
    binmap = [(9 - k) % 9 for k in range(9)]
    def perm(swap_x, swap_y):
        idx = []
        for cy in range(2):
            for cx in range(2):
                sy, sx = (1 - cy if swap_y else cy), (1 - cx if swap_x else cx)
                idx += [(sy * 2 + sx) * 9 + binmap[k] for k in range(9)]
        return idx
    d1, _ = orc.fhog(img[:, ::-1], 8)
    np.testing.assert_allclose(d1, d0[perm(True, False)][:, :, ::-1], atol=1e-12)
    d2, _ = orc.fhog(img[::-1, :], 8)
    np.testing.assert_allclose(d2, d0[perm(False, True)][:, ::-1, :], atol=1e-12)
