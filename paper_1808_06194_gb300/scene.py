"""Large-scene registration: band streaming, CFOG, CPs, batched matching and
the FP64 affine fit (the partition strategy and system of Sec. IV).

The reference and sensed images stay in pinned host memory and are streamed
to the device in row bands on a copy stream.  Block-based Harris CPs are
detected on the reference image and each CP gets the search-centre prior of
the georeference model (Sec. IV: the search region is predicted from
georeferencing).  The scene is then processed band by band (the partition
strategy of Sec. IV): each CP belongs to the band of its row, the band's CFOG
is computed for the rows its CPs' templates and windows reach plus the
filters' 4-row halo (those rows equal the whole-image CFOG exactly), and the
band's CPs are matched in one batched launch (or, for comparison, one launch
per CP) on band coordinates.  Only one band-sized pair of feature volumes
is held on the device, however tall the scene.  `cfog_fit_affine` then
estimates the affine mapping model in FP64, and `cfog_reject_outliers` runs
the system's outlier rejection (Sec. IV: cubic polynomial model, drop the
largest residual until the RMSE is below the threshold).
"""
from __future__ import annotations

import dataclasses
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
    band: rows per band.  The images are streamed to the device in bands on
    a copy stream; CFOG is computed band by band, each band with the margin of
    rows its CPs' templates and search windows reach (plus the 4-row halo of
    the filters), into one band-sized pair of feature buffers, so device
    memory for features does not grow with the scene's height.
    reject_degree, reject_rmse: model degree and RMSE threshold (pixels) of
    the outlier rejection (Sec. IV: cubic, 1 px).
    rectify: also resample the sensed image onto the reference grid with the
    piecewise-linear model on the Delaunay TIN of the kept CPs (Sec. IV).
    autotune: apply (or first measure and cache) the autotuner's variant and
    plan for the class (tmpl, radius) before matching.
    Returns a dict with CPs, results, the affine model, the rejection outcome
    (kept mask, removal order, polynomial model), the rectified image when
    asked for, stage timings (ms) and the feature bytes held on the device.
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
    t = {"start": ev(), "resident": ev(), "cps": ev(), "bands": ev(), "rejected": ev()}
    ref_d = torch.empty((h, w), dtype=ref.dtype, device=dev)
    sen_d = torch.empty((h, w), dtype=sen.dtype, device=dev)
    halo = 4
    t["start"].record(s_comp)
    s_copy.wait_stream(s_comp)
    with torch.cuda.stream(s_copy):
        for y0 in range(0, h, band):
            y1 = min(h, y0 + band)
            ref_d[y0:y1].copy_(ref[y0:y1], non_blocking=True)
            sen_d[y0:y1].copy_(sen[y0:y1], non_blocking=True)
    s_comp.wait_stream(s_copy)
    t["resident"].record(s_comp)
    margin = tmpl // 2 + radius + 16
    cps = api.cfog_detect_cps(ref_d, grid, grid, 1, 0, margin, stream=s_comp)
    t["cps"].record(s_comp)
    pts = cps.cpu().numpy()          # host prior model needs the CP positions
    qx, qy = prior_fn(pts[:, 0].astype(np.float64), pts[:, 1].astype(np.float64))
    qx, qy = np.asarray(qx, np.int32), np.asarray(qy, np.int32)
    n = pts.shape[0]

    # Rows each CP reads: its template [py - t0, py - t0 + N) in the reference
    # and its window [py + qy - t0 - r, ... + N + 2r) in the sensed image.  A
    # CP belongs to the band of its row; the band's feature rows reach as far
    # as its CPs need, and its CFOG view adds the filters' halo.
    t0 = tmpl // 2
    lo = np.minimum(pts[:, 1] - t0, pts[:, 1] + qy - t0 - radius)
    hi = np.maximum(pts[:, 1] - t0 + tmpl, pts[:, 1] + qy - t0 - radius + tmpl + 2 * radius)
    bands = []
    for y0 in range(0, h, band):
        sel = np.nonzero((pts[:, 1] >= y0) & (pts[:, 1] < min(h, y0 + band)))[0]
        if sel.size == 0:
            continue
        v0 = max(0, int(lo[sel].min()) - halo)
        v1 = min(h, int(hi[sel].max()) + halo)
        bands.append((sel, v0, v1))
    hmax = max((v1 - v0 for _, v0, v1 in bands), default=1)
    # one band-sized pair of feature volumes: every band's CFOG and matching
    # run on the compute stream in order, so the next band's CFOG overwrites
    # it only after the previous band's matching has read it
    bufs = [(api.alloc_features(hmax, w, 9, dev), api.alloc_features(hmax, w, 9, dev))]
    feat_bytes = sum(f.nbytes for pair in bufs for f in pair)

    res = torch.empty((n, 6), dtype=torch.int32, device=dev)
    tm_all = torch.full((n,), tmpl, dtype=torch.int32, device=dev)
    rd_all = torch.full((n,), radius, dtype=torch.int32, device=dev)
    cfog_evs, match_evs = [], []
    for bi, (sel, v0, v1) in enumerate(bands):
        fr_buf, fs_buf = bufs[bi % len(bufs)]
        hv = v1 - v0
        fr = dataclasses.replace(fr_buf, h=hv)
        fs = dataclasses.replace(fs_buf, h=hv)
        e0, e1, e2 = ev(), ev(), ev()
        e0.record(s_comp)
        api.cfog_extract(ref_d[v0:v1], out=fr, stream=s_comp)
        api.cfog_extract(sen_d[v0:v1], out=fs, stream=s_comp)
        e1.record(s_comp)
        m = sel.size
        band_pts = pts[sel].copy()
        band_pts[:, 1] -= v0
        cps_b = torch.from_numpy(band_pts.astype(np.int32)).to(dev)
        pr_b = torch.from_numpy(np.stack([qx[sel], qy[sel]], 1).astype(np.int32)).to(dev)
        out_b = torch.empty((m, 6), dtype=torch.int32, device=dev)
        if batched:
            jt = api.job_table([(fr, fs)], dev)
            api.cfog_match_batched(jt, 1, cps_b, tm_all[:m], rd_all[:m], tmpl, radius,
                                   prior=pr_b, precision=precision, out=out_b, stream=s_comp)
        else:
            for i in range(m):
                api.cfog_match(fr, fs, cps_b[i:i + 1], tm_all[i:i + 1], rd_all[i:i + 1], tmpl,
                               radius, pr_b[i:i + 1], precision=precision, out=out_b[i:i + 1],
                               stream=s_comp)
        e2.record(s_comp)
        res[torch.from_numpy(sel).to(dev)] = out_b
        cfog_evs.append((e0, e1))
        match_evs.append((e1, e2))
    t["bands"].record(s_comp)
    keep, order, models = api.cfog_reject_outliers(cps, res, None, reject_degree, reject_rmse,
                                                   stream=s_comp)
    t["rejected"].record(s_comp)
    w0 = time.perf_counter()
    model = api.cfog_fit_affine(cps, res, stream=s_comp)
    fit_ms = (time.perf_counter() - w0) * 1e3
    torch.cuda.synchronize()
    cfog_ms = sum(a.elapsed_time(b) for a, b in cfog_evs)
    match_ms = sum(a.elapsed_time(b) for a, b in match_evs)
    times = {"upload_ms": t["start"].elapsed_time(t["resident"]),
             "harris_ms": t["resident"].elapsed_time(t["cps"]),
             "bands_ms": t["cps"].elapsed_time(t["bands"]),
             "cfog_ms": cfog_ms, "match_ms": match_ms, "n_bands": len(bands),
             "stream_and_cfog_ms": t["start"].elapsed_time(t["resident"]) + cfog_ms,
             "reject_ms": t["bands"].elapsed_time(t["rejected"]), "fit_wall_ms": fit_ms}
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
            "poly_model": m, "rectified": rect, "n": n, "times": times,
            "feature_bytes": feat_bytes, "images": (ref_d, sen_d)}


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
