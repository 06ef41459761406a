"""Outlier rejection on the GPU (Sec. IV) against the FP64 oracle: removal
order, kept set, RMSE and the fitted model, for single and batched jobs."""
import ctypes

import numpy as np
import pytest

import oracle
import synth
from tests._util import cuda_or_skip

pytestmark = pytest.mark.gpu

RMSE_REL = 1e-5        # GPU residuals: FP32 change of the model on FP64 first-fit residuals
PRED_ATOL = 1e-6       # model predictions at the CPs, pixels
RESID_ATOL = 1e-4      # squared-residual slack when several removals are correct


def _dev(torch, cps, res):
    c = torch.from_numpy(np.ascontiguousarray(cps)).cuda()
    r = torch.from_numpy(np.ascontiguousarray(res).view(np.int32).reshape(-1, 6)).cuda()
    return c, r


def _xy(cps, res):
    x = cps[:, 0].astype(np.float64)
    y = cps[:, 1].astype(np.float64)
    return x, y, x + res["sub_dx"].astype(np.float64), y + res["sub_dy"].astype(np.float64)


def _oracle(cps, res, degree, thr, min_keep=0):
    x, y, xp, yp = _xy(cps, res)
    return oracle.reject_outliers(x, y, xp, yp, (res["status"] == 0).astype(np.int32), degree,
                                  thr, min_keep)


def _check_job(P, model, keep, order, cps, res, degree, thr, min_keep=0, exact_order=True):
    o = _oracle(cps, res, degree, thr, min_keep)
    x, y, xp, yp = _xy(cps, res)
    assert model["status"] == o["status"]
    assert model["n_valid"] == int((res["status"] == 0).sum())
    assert model["terms"] == oracle.poly_terms(degree)
    assert tuple(model["norm"]) == tuple(o["norm"])
    if o["status"] == 2 and o["n_fits"] == 1:
        assert model["rmse"] == -1.0 and model["n_removed"] == 0
        np.testing.assert_array_equal(keep.astype(bool), res["status"] == 0)
        return o
    if exact_order:
        assert order[:model["n_removed"]].tolist() == o["order"].tolist()
        np.testing.assert_array_equal(keep.astype(bool), o["keep"])
        assert model["n_fits"] == o["n_fits"]
        assert model["rmse"] == pytest.approx(o["rmse"], rel=RMSE_REL)
        coef = np.array(model["coef"])
        gx, gy = oracle.poly_predict(coef, model["norm"], x, y, degree)
        ox, oy = oracle.poly_predict(o["coef"], o["norm"], x, y, degree)
        np.testing.assert_allclose(gx, ox, atol=PRED_ATOL)
        np.testing.assert_allclose(gy, oy, atol=PRED_ATOL)
    else:
        _check_valid_sequence(model, keep, order, cps, res, degree, thr)
    return o


def _check_valid_sequence(model, keep, order, cps, res, degree, thr):
    """Several removal sequences are correct when residuals nearly tie: replay
    the GPU's sequence with the oracle's fit and check each step."""
    x, y, xp, yp = _xy(cps, res)
    cur = (res["status"] == 0).copy()
    for idx in order[:model["n_removed"]]:
        o = oracle.reject_outliers(x, y, xp, yp, cur.astype(np.int32), degree, np.inf)
        px, py = oracle.poly_predict(o["coef"], o["norm"], x, y, degree)
        e2 = np.where(cur, (xp - px) ** 2 + (yp - py) ** 2, -1.0)
        assert np.sqrt(e2[cur].mean()) >= thr * (1 - RMSE_REL)
        assert cur[idx] and e2[idx] >= e2.max() - RESID_ATOL
        cur[idx] = False
    np.testing.assert_array_equal(keep.astype(bool), cur)
    o = oracle.reject_outliers(x, y, xp, yp, cur.astype(np.int32), degree, np.inf)
    assert model["rmse"] == pytest.approx(o["rmse"], rel=RMSE_REL)
    if model["status"] == 0:
        assert model["rmse"] < thr


def _run(torch, P, cps, res, degree, thr, min_keep=0, job_start=None):
    c, r = _dev(torch, cps, res)
    keep, order, models = P.cfog_reject_outliers(c, r, job_start, degree, thr, min_keep)
    torch.cuda.synchronize()
    return keep.cpu().numpy(), order.cpu().numpy(), P.unpack_models(models)


@pytest.mark.parametrize("n,seed", [(400, 50), (1500, 51)])
def test_cubic_with_planted_outliers(n, seed):
    torch, P = cuda_or_skip()
    cps, res, info = synth.cp_set(seed, n, noise=0.05, outlier_frac=0.05)
    keep, order, models = _run(torch, P, cps, res, 3, 0.25)
    o = _check_job(P, models[0], keep, order, cps, res, 3, 0.25)
    assert set(o["order"].tolist()) <= set(info["outliers"].tolist())
    assert len(o["order"]) >= len(info["outliers"]) - 2


@pytest.mark.parametrize("degree,field,thr", [(1, "sine", 2.0), (2, "sine", 1.5), (3, "sine", 1.0),
                                              (2, "cubic", 3.0)])
def test_lower_degree_and_smooth_fields(degree, field, thr):
    torch, P = cuda_or_skip()
    cps, res, _ = synth.cp_set(52 + degree, 600, field=field, outlier_frac=0.04)
    keep, order, models = _run(torch, P, cps, res, degree, thr)
    _check_job(P, models[0], keep, order, cps, res, degree, thr, exact_order=False)


def test_min_keep_floor_and_zero_threshold():
    torch, P = cuda_or_skip()
    cps, res, _ = synth.cp_set(56, 120, field="sine", bad_status_frac=0.0)
    keep, order, models = _run(torch, P, cps, res, 3, 0.0, min_keep=90)
    assert models[0]["status"] == 1 and models[0]["n_kept"] == 90 and keep.sum() == 90
    _check_job(P, models[0], keep, order, cps, res, 3, 0.0, 90, exact_order=False)


def test_batched_jobs_equal_single_jobs():
    """Jobs of mixed sizes in one launch, including an empty job, a job with no
    valid CP and a degenerate (collinear) job."""
    torch, P = cuda_or_skip()
    sets = [synth.cp_set(60, 700, noise=0.05), synth.cp_set(61, 0), synth.cp_set(62, 40),
            synth.cp_set(63, 2500, noise=0.05, outlier_frac=0.08), synth.cp_set(64, 30)]
    cps = [s[0] for s in sets]
    res = [s[1].copy() for s in sets]
    res[2]["status"][:] = 1                                   # no valid CP
    cps[4][:, 1] = cps[4][:, 0] // 2 + 100                    # collinear CPs
    job_start = np.concatenate([[0], np.cumsum([len(c) for c in cps])]).tolist()
    allc = np.concatenate(cps).astype(np.int32)
    allr = np.concatenate(res)
    keep, order, models = _run(torch, P, allc, allr, 3, 0.25, job_start=job_start)
    assert len(models) == 5
    for j in range(5):
        a, b = job_start[j], job_start[j + 1]
        m = models[j]
        if b == a:
            assert m["n_valid"] == 0 and m["status"] == 2
            continue
        ordj = order[a:b] - a
        o = _check_job(P, m, keep[a:b], ordj, cps[j], res[j], 3, 0.25)
        if j == 2 or j == 4:
            assert o["status"] == 2 and m["status"] == 2
    # the same job alone gives the same bytes
    k1, o1, m1 = _run(torch, P, cps[3], res[3], 3, 0.25)
    np.testing.assert_array_equal(k1, keep[job_start[3]:job_start[4]])
    assert m1[0] == models[3]


def test_deterministic_and_full_size():
    """10 000 CPs (the large-scene CP count) with 5 % gross mismatches; two runs
    give identical bytes."""
    torch, P = cuda_or_skip()
    cps, res, info = synth.cp_set(65, 10000, size=20000, noise=0.1, outlier_frac=0.05,
                                  outlier_min=5.0, outlier_step=0.5)
    c, r = _dev(torch, cps, res)
    outs = []
    for _ in range(2):
        keep, order, models = P.cfog_reject_outliers(c, r, None, 3, 0.3)
        torch.cuda.synchronize()
        outs.append((keep.cpu().numpy(), order.cpu().numpy(), models.cpu().numpy()))
    for a, b in zip(outs[0], outs[1]):
        np.testing.assert_array_equal(a, b)
    keep, order, raw = outs[0]
    m = P.unpack_models(torch.from_numpy(raw))[0]
    o = _check_job(P, m, keep, order, cps, res, 3, 0.3)
    assert set(o["order"].tolist()) <= set(info["outliers"].tolist())
    assert len(o["order"]) >= 0.95 * len(info["outliers"])
    assert ctypes.sizeof(P._lib.cfog_poly_model) == raw.shape[1]
