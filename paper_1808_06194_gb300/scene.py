"""Large-scene registration: band streaming, CFOG, CPs, batched matching and
the FP64 affine fit (the partition strategy and system of Sec. IV).

The reference and sensed images stay in pinned host memory and are streamed
to the device in row bands on a copy stream; as soon as a band and the first
rows of the next one are resident, `cfog_extract_rows` computes that band's
CFOG rows on the compute stream, exactly as a whole-image extraction would.
Block-based Harris CPs are detected on the reference image, each CP gets the
search-centre prior of the georeference model (Sec. IV: the search region is
predicted from georeferencing), all CPs are matched in one batched launch (or,
for comparison, one launch per CP), `cfog_fit_affine` estimates the affine
mapping model in FP64, and `cfog_reject_outliers` runs the system's outlier
rejection (Sec. IV: cubic polynomial model, drop the largest residual until
the RMSE is below the threshold).
"""
from __future__ import annotations

import time

import numpy as np

from . import _lib as L
from . import api


def register_scene(ref, sen, prior_fn, grid, tmpl=96, radius=16, band=2048, batched=True,
                   precision=L.CFOG_PREC_FP32_FFT, device="cuda", reject_degree=3,
                   reject_rmse=1.0, rectify=False, nodata=0.0, autotune=True):
    """Register a large pair held in pinned host tensors (uint16 or float32).

    prior_fn(xs, ys) -> (qx, qy): integer search-centre offsets per CP.
    grid: CP grid side (grid x grid cells, one CP each).
    reject_degree, reject_rmse: model degree and RMSE threshold (pixels) of
    the outlier rejection (Sec. IV: cubic, 1 px).
    rectify: also resample the sensed image onto the reference grid with the
    piecewise-linear model on the Delaunay TIN of the kept CPs (Sec. IV).
    autotune: apply (or first measure and cache) the autotuner's variant and
    plan for the class (tmpl, radius) before matching.
    Returns a dict with CPs, results, the affine model, the rejection outcome
    (kept mask, removal order, polynomial model), the rectified image when
    asked for, and stage timings (ms).
    """
    import torch
    dev = torch.device(device)
    if autotune and batched:
        from . import autotune as at
        at.ensure([(tmpl, radius)], 9, tmpl, radius, precision, device=dev)
    h, w = ref.shape
    s_copy = torch.cuda.Stream(dev)
    s_comp = torch.cuda.current_stream(dev)
    ev = lambda: torch.cuda.Event(enable_timing=True)  # noqa: E731
    t = {"start": ev(), "features": ev(), "cps": ev(), "matched": ev(), "rejected": ev()}
    ref_d = torch.empty((h, w), dtype=ref.dtype, device=dev)
    sen_d = torch.empty((h, w), dtype=sen.dtype, device=dev)
    fr = api.alloc_features(h, w, 9, dev)
    fs = api.alloc_features(h, w, 9, dev)
    nb = (h + band - 1) // band
    halo = 4
    t["start"].record(s_comp)
    s_copy.wait_stream(s_comp)
    arrived = []
    with torch.cuda.stream(s_copy):
        for b in range(nb):
            y0, y1 = b * band, min(h, (b + 1) * band)
            ref_d[y0:y1].copy_(ref[y0:y1], non_blocking=True)
            sen_d[y0:y1].copy_(sen[y0:y1], non_blocking=True)
            e = torch.cuda.Event()
            e.record(s_copy)
            arrived.append(e)
    for b in range(nb):
        y0, y1 = b * band, min(h, (b + 1) * band)
        s_comp.wait_event(arrived[b])
        if y1 + halo < h and b + 1 < nb:
            s_comp.wait_event(arrived[b + 1])
        api.cfog_extract_rows(ref_d, y0, y1, fr, stream=s_comp)
        api.cfog_extract_rows(sen_d, y0, y1, fs, stream=s_comp)
    t["features"].record(s_comp)
    margin = tmpl // 2 + radius + 16
    cps = api.cfog_detect_cps(ref_d, grid, grid, 1, 0, margin, stream=s_comp)
    t["cps"].record(s_comp)
    pts = cps.cpu().numpy()          # host prior model needs the CP positions
    qx, qy = prior_fn(pts[:, 0].astype(np.float64), pts[:, 1].astype(np.float64))
    prior = torch.from_numpy(np.stack([qx, qy], 1).astype(np.int32)).to(dev)
    n = pts.shape[0]
    tm = torch.full((n,), tmpl, dtype=torch.int32, device=dev)
    rd = torch.full((n,), radius, dtype=torch.int32, device=dev)
    t_match0 = ev()
    t_match0.record(s_comp)
    if batched:
        res = api.cfog_match_batched(api.job_table([(fr, fs)], dev), 1, cps, tm, rd, tmpl, radius,
                                     prior=prior, precision=precision, stream=s_comp)
    else:
        res = torch.empty((n, 6), dtype=torch.int32, device=dev)
        for i in range(n):
            api.cfog_match(fr, fs, cps[i:i + 1], tm[i:i + 1], rd[i:i + 1], tmpl, radius,
                           prior[i:i + 1], precision=precision, out=res[i:i + 1], stream=s_comp)
    t["matched"].record(s_comp)
    keep, order, models = api.cfog_reject_outliers(cps, res, None, reject_degree, reject_rmse,
                                                   stream=s_comp)
    t["rejected"].record(s_comp)
    t0 = time.perf_counter()
    model = api.cfog_fit_affine(cps, res, stream=s_comp)
    fit_ms = (time.perf_counter() - t0) * 1e3
    torch.cuda.synchronize()
    times = {"stream_and_cfog_ms": t["start"].elapsed_time(t["features"]),
             "harris_ms": t["features"].elapsed_time(t["cps"]),
             "match_ms": t_match0.elapsed_time(t["matched"]),
             "reject_ms": t["matched"].elapsed_time(t["rejected"]), "fit_wall_ms": fit_ms}
    rect = None
    if rectify:
        t1 = time.perf_counter()
        tris = api.tin_delaunay(pts, keep.cpu().numpy())
        tri_ms = (time.perf_counter() - t1) * 1e3
        tris_d = torch.from_numpy(tris).to(dev)
        ws = api.tin_workspace(len(tris), h, w, dev)
        rect = torch.empty((h, w), dtype=torch.float32, device=dev)
        e0, e1 = ev(), ev()
        e0.record(s_comp)
        api.cfog_tin_rectify(sen_d, cps, res, tris_d, h, w, nodata, out=rect, workspace=ws, stream=s_comp)
        e1.record(s_comp)
        torch.cuda.synchronize()
        times["delaunay_host_ms"] = tri_ms
        times["rectify_ms"] = e0.elapsed_time(e1)
        times["n_triangles"] = int(len(tris))
    m = api.unpack_models(models)[0]
    n_rm = m["n_removed"]
    return {"cps": pts, "results": res.cpu().numpy(), "affine": np.array(model),
            "keep": keep.cpu().numpy().astype(bool), "removed": order[:n_rm].cpu().numpy(),
            "poly_model": m, "rectified": rect,
            "n": n, "times": times, "features": (fr, fs), "images": (ref_d, sen_d)}


def georeference_prior(field, error_px, seed):
    """Prior of a georeferenced pair: the true displacement at each CP plus a
    seeded error of at most `error_px` pixels per axis, rounded (Sec. IV uses
    the georeferencing information to predict the search region)."""
    def prior(xs, ys):
        dy, dx = field(ys, xs)
        rng = np.random.default_rng(seed)
        ex = rng.integers(-error_px, error_px + 1, xs.shape[0])
        ey = rng.integers(-error_px, error_px + 1, xs.shape[0])
        return np.rint(dx).astype(np.int32) + ex, np.rint(dy).astype(np.int32) + ey
    return prior
