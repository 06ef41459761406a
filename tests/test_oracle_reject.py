"""Pins for the oracle's outlier rejection (Sec. IV): iterative least-squares
fitting of a polynomial mapping model, dropping the CP with the largest
residual until the RMSE falls below the threshold."""
import numpy as np
import pytest

import synth


def _xy(cps, res):
    x = cps[:, 0].astype(np.float64)
    y = cps[:, 1].astype(np.float64)
    return x, y, x + res["sub_dx"].astype(np.float64), y + res["sub_dy"].astype(np.float64)


def _lstsq_fit(x, y, xp, yp, degree):
    """Independent LS fit: numpy.linalg.lstsq on monomials of x/1000, y/1000
    (another centre and scale than the oracle's).  Returns the predictor."""
    def vander(xx, yy):
        a, b = xx / 1000.0, yy / 1000.0
        return np.stack([a ** i * b ** j for i in range(degree + 1) for j in range(degree + 1 - i)], -1)
    V = vander(x, y)
    cx = np.linalg.lstsq(V, xp, rcond=None)[0]
    cy = np.linalg.lstsq(V, yp, rcond=None)[0]
    return lambda xx, yy: (vander(xx, yy) @ cx, vander(xx, yy) @ cy)


def _resid2(pred, x, y, xp, yp):
    px, py = pred(x, y)
    return (xp - px) ** 2 + (yp - py) ** 2


def test_terms(orc):
    assert [orc.poly_terms(d) for d in (1, 2, 3)] == [3, 6, 10]


def test_exact_cubic_is_kept_whole(orc):
    cps, res, info = synth.cp_set(40, 300, noise=0.0, outlier_frac=0.0, bad_status_frac=0.0)
    x, y, xp, yp = _xy(cps, res)
    out = orc.reject_outliers(x, y, xp, yp, degree=3, thr=1e-3)
    assert out["status"] == 0 and out["keep"].all() and len(out["order"]) == 0
    assert out["n_fits"] == 1 and out["rmse"] < 1e-5    # float32 offsets
    fx, fy = info["field"](x, y)
    px, py = orc.poly_predict(out["coef"], out["norm"], x, y, 3)
    np.testing.assert_allclose(px, x + fx + 7.0, atol=1e-5)
    np.testing.assert_allclose(py, y + fy - 4.0, atol=1e-5)


@pytest.mark.parametrize("degree", [1, 2, 3])
def test_single_fit_matches_lstsq_in_another_basis(orc, degree):
    cps, res, _ = synth.cp_set(41, 250, field="sine", outlier_frac=0.0, bad_status_frac=0.0)
    x, y, xp, yp = _xy(cps, res)
    out = orc.reject_outliers(x, y, xp, yp, degree=degree, thr=np.inf)
    assert out["status"] == 0 and out["n_fits"] == 1
    pred = _lstsq_fit(x, y, xp, yp, degree)
    gx, gy = pred(x, y)
    px, py = orc.poly_predict(out["coef"], out["norm"], x, y, degree)
    np.testing.assert_allclose(px, gx, atol=1e-8)
    np.testing.assert_allclose(py, gy, atol=1e-8)
    r2 = _resid2(pred, x, y, xp, yp)
    assert out["rmse"] == pytest.approx(np.sqrt(r2.mean()), rel=1e-9)


@pytest.mark.parametrize("degree,field,thr", [(3, "cubic", 0.3), (3, "sine", 0.8), (2, "sine", 1.2),
                                              (1, "cubic", 4.0)])
def test_every_removal_replayed_with_lstsq(orc, degree, field, thr):
    """Step by step: each removed CP is the largest residual of a fresh LS fit
    of the CPs kept so far, each earlier RMSE is >= thr, the final one < thr."""
    cps, res, _ = synth.cp_set(42, 220, field=field, outlier_frac=0.06)
    x, y, xp, yp = _xy(cps, res)
    valid = (res["status"] == 0).astype(np.int32)
    out = orc.reject_outliers(x, y, xp, yp, valid, degree=degree, thr=thr)
    assert out["status"] == 0
    keep = valid.astype(bool).copy()
    for idx in out["order"]:
        pred = _lstsq_fit(x[keep], y[keep], xp[keep], yp[keep], degree)
        r2 = np.where(keep, _resid2(pred, x, y, xp, yp), -1.0)
        assert np.sqrt(r2[keep].mean()) >= thr
        top = np.sort(r2)[-2:]
        assert int(np.argmax(r2)) == idx or top[1] - top[0] < 1e-9 * top[1]
        keep[idx] = False
    np.testing.assert_array_equal(out["keep"], keep)
    pred = _lstsq_fit(x[keep], y[keep], xp[keep], yp[keep], degree)
    final = np.sqrt(_resid2(pred, x, y, xp, yp)[keep].mean())
    assert final < thr
    assert out["rmse"] == pytest.approx(final, rel=1e-8)
    assert out["n_fits"] == len(out["order"]) + 1


def test_planted_outliers_removed_largest_first(orc):
    cps, res, info = synth.cp_set(43, 400, noise=0.05, outlier_frac=0.03, outlier_min=8.0,
                                  outlier_step=3.0)
    x, y, xp, yp = _xy(cps, res)
    valid = (res["status"] == 0).astype(np.int32)
    out = orc.reject_outliers(x, y, xp, yp, valid, degree=3, thr=0.2)
    assert out["status"] == 0
    planted = sorted(info["outliers"].tolist(), key=lambda i: -info["outlier_mags"][i])
    assert out["order"].tolist() == planted
    assert out["keep"].sum() == valid.sum() - len(planted)


def test_min_keep_floor(orc):
    cps, res, _ = synth.cp_set(44, 80, field="sine", bad_status_frac=0.0)
    x, y, xp, yp = _xy(cps, res)
    out = orc.reject_outliers(x, y, xp, yp, degree=3, thr=0.0, min_keep=50)
    assert out["status"] == 1 and out["keep"].sum() == 50 and len(out["order"]) == 30
    out = orc.reject_outliers(x, y, xp, yp, degree=2, thr=0.0, min_keep=0)
    assert out["status"] == 1 and out["keep"].sum() == 6


def test_degenerate_sets(orc):
    x = np.arange(20, dtype=np.float64) * 10.0
    y = 3.0 * x + 5.0                       # collinear: the y monomials are dependent
    out = orc.reject_outliers(x, y, x + 1.0, y - 2.0, degree=1, thr=1.0)
    assert out["status"] == 2 and out["rmse"] == -1.0 and out["keep"].all()
    out = orc.reject_outliers(x, y, x, y, valid=np.zeros(20, np.int32), degree=3, thr=1.0)
    assert out["status"] == 2 and not out["keep"].any()
    out = orc.reject_outliers(x[:5], x[:5] ** 0.5, x[:5], x[:5], degree=3, thr=1.0)   # 5 < 10 terms
    assert out["status"] == 2


def test_translation_invariance(orc):
    cps, res, _ = synth.cp_set(45, 200, field="sine", outlier_frac=0.05)
    x, y, xp, yp = _xy(cps, res)
    valid = (res["status"] == 0).astype(np.int32)
    a = orc.reject_outliers(x, y, xp, yp, valid, degree=3, thr=0.5)
    b = orc.reject_outliers(x + 1000.0, y - 512.0, xp + 1000.0, yp - 512.0, valid, degree=3, thr=0.5)
    assert a["order"].tolist() == b["order"].tolist()
    assert b["rmse"] == pytest.approx(a["rmse"], rel=1e-9)


def test_degree1_equals_affine_ls(orc):
    cps, res, _ = synth.cp_set(46, 150, field="sine")
    x, y, xp, yp = _xy(cps, res)
    valid = (res["status"] == 0).astype(np.int32)
    out = orc.reject_outliers(x, y, xp, yp, valid, degree=1, thr=np.inf)
    a = orc.affine_ls(x, y, xp, yp, valid)
    px, py = orc.poly_predict(out["coef"], out["norm"], x, y, 1)
    np.testing.assert_allclose(px, a[0] + a[1] * x + a[2] * y, atol=1e-8)
    np.testing.assert_allclose(py, a[3] + a[4] * x + a[5] * y, atol=1e-8)
