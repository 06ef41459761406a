"""Autotuner of the FFT matcher: kernel variant and per-class FFT plans
picked by measurement on the GPU at hand, cached as JSON.

Sec. III-G computes the SSD of Eq. 3 by FFT correlation (Eq. 8-9).  How fast
one control point (CP) is matched depends on the FFT size and the template
blocking chosen for its class (N, r), and on which kernel variant runs the
batch (threads per CTA, CTAs per SM, where the accumulator lives).  The
library plans every class with an integer cost model; this module replaces
the model's guesses by timings:

1. the variants (WIDE, PAIR, TRIO, PAIRT) are timed on a batch that mixes the
   caller's classes; the fastest becomes the AUTO variant of that launch class
   (cfog_match_set_auto_variant);
2. for the chosen variant, each class's six best plans by the cost model
   (cfog_plan_candidates) are timed on a batch of that class alone; a plan
   that beats the model's own choice by more than the noise margin is
   recorded (cfog_match_set_plan);
3. the mix is timed again with the tuned plans; if it is not faster, the plans
   are dropped;
4. every other class of the list records the cost model's own plan, so the
   kernels read each class's plan from the table instead of searching.

Timings use synthetic feature volumes larger than L2 (their values do not
change the work) and CUDA events around single launches.  The outcome is
stored in a JSON cache keyed by GPU name, compute capability, a hash of the
library build, m, the launch bounds (tmpl_max, radius_max), precision and the
class list, so a later process applies it without timing anything
(`ensure`).  The cache file is $CFOG_TUNE_CACHE, else
$XDG_CACHE_HOME/cfog/autotune.json, else ~/.cache/cfog/autotune.json.
"""
from __future__ import annotations

import ctypes
import json
import os
import statistics
import tempfile
import time

import numpy as np

from . import _lib as L

FORMAT = 2
NOISE = 0.03         # a tuned plan must beat the model's plan by 3 %
FEATURE_SIDE = 2048  # synthetic volumes: 2 x 2048^2 x (m + 1) x 4 B > L2


def cache_path():
    p = os.environ.get("CFOG_TUNE_CACHE")
    if p:
        return p
    base = os.environ.get("XDG_CACHE_HOME") or os.path.join(os.path.expanduser("~"), ".cache")
    return os.path.join(base, "cfog", "autotune.json")


def device_key(name, cc, build):
    return f"{name}|sm{cc[0]}{cc[1]}|libcfog-{build}"


def class_key(m, tmpl_max, radius_max, precision, classes):
    cl = ",".join(f"{int(n)}x{int(r)}" for n, r in sorted(set(map(tuple, classes))))
    return f"m{m}|tmax{tmpl_max}|rmax{radius_max}|prec{precision}|{cl}"


def load_cache(path=None):
    path = path or cache_path()
    try:
        with open(path) as f:
            data = json.load(f)
    except (OSError, ValueError):
        return {"format": FORMAT, "entries": {}}
    if data.get("format") != FORMAT or not isinstance(data.get("entries"), dict):
        return {"format": FORMAT, "entries": {}}
    return data


def save_cache(data, path=None):
    """Write the cache atomically (a temporary file renamed over the old one)."""
    path = path or cache_path()
    d = os.path.dirname(path) or "."
    os.makedirs(d, exist_ok=True)
    fd, tmp = tempfile.mkstemp(prefix=".autotune.", dir=d)
    with os.fdopen(fd, "w") as f:
        json.dump(data, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def apply(entry, m, tmpl_max, radius_max, precision, lib=None):
    """Record a tuning outcome in the library: the AUTO variant of the launch
    class and the tuned plan of each class."""
    lib = lib or L.lib()
    v = int(entry["variant"])
    L.check(lib.cfog_match_set_auto_variant(m, tmpl_max, radius_max, precision, v),
            "cfog_match_set_auto_variant")
    for table in ("plans", "model_plans"):
        for cls, code in entry.get(table, {}).items():
            n, r = (int(x) for x in cls.split("x"))
            L.check(lib.cfog_match_set_plan(v, m, n, r, int(code)), "cfog_match_set_plan")


def candidates(n, r, m, variant, k=4, lib=None):
    """The k best plans of class (n, r) by the library's cost model:
    list of dicts with the code and the plan fields."""
    lib = lib or L.lib()
    out = (ctypes.c_int32 * (9 * k))()
    cnt = ctypes.c_int32()
    L.check(lib.cfog_plan_candidates(n, r, m, variant, k, out, ctypes.byref(cnt)),
            "cfog_plan_candidates")
    keys = ["code", "nb_y", "nb_x", "P_y", "P_x", "b_y", "b_x", "stages", "smem"]
    return [dict(zip(keys, list(out[9 * i:9 * i + 9]))) for i in range(cnt.value)]


class _Bench:
    """Synthetic features and CP batches for timing launches."""

    def __init__(self, torch, api, dev, m, tmpl_max, radius_max, seed=0):
        self.torch, self.api, self.dev = torch, api, dev
        side = FEATURE_SIDE
        g = torch.Generator(device=dev)
        g.manual_seed(seed)
        self.fa = api.alloc_features(side, side, m, dev)
        self.fb = api.alloc_features(side, side, m, dev)
        for f in (self.fa, self.fb):
            f.data.uniform_(0.0, 1.0 / np.sqrt(m), generator=g)
            f.sqnorm.uniform_(0.0, 1.0, generator=g)
        self.jobs = api.job_table([(self.fa, self.fb)], dev)
        self.side, self.m = side, m
        self.tmpl_max, self.radius_max = tmpl_max, radius_max
        self.rng = np.random.default_rng(seed)
        self.n_sm = torch.cuda.get_device_properties(dev).multi_processor_count

    def batch(self, classes, n):
        margin = self.tmpl_max // 2 + self.radius_max + 2
        idx = self.rng.integers(0, len(classes), n)
        cl = np.asarray(classes, np.int32)[idx]
        pts = self.rng.integers(margin, self.side - margin, (n, 2)).astype(np.int32)
        t = self.torch
        return (t.from_numpy(pts).to(self.dev), t.from_numpy(cl[:, 0].copy()).to(self.dev),
                t.from_numpy(cl[:, 1].copy()).to(self.dev))

    def time(self, b, variant, precision=0, reps=3):
        """Median event time (ms) of one batched launch, after one untimed launch."""
        t = self.torch
        cps, tm, rd = b
        n = cps.shape[0]
        out = t.empty((n, 6), dtype=t.int32, device=self.dev)
        ws = self.api.match_workspace(n, self.dev)
        ts = []
        for k in range(reps + 1):
            a, e = t.cuda.Event(enable_timing=True), t.cuda.Event(enable_timing=True)
            a.record()
            self.api.cfog_match_batched(self.jobs, 1, cps, tm, rd, self.tmpl_max, self.radius_max,
                                        self.m, precision=precision, variant=variant, out=out,
                                        workspace=ws)
            e.record()
            t.cuda.synchronize()
            if k:
                ts.append(a.elapsed_time(e))
        return statistics.median(ts)


def tune(classes, m=9, tmpl_max=None, radius_max=None, precision=L.CFOG_PREC_FP32_FFT,
         device="cuda", variants=(1, 2, 3, 4), k_plans=6, reps=3, mix_cps=1024, seed=0):
    """Time variants and plans for `classes` [(N, r), ...]; record the outcome
    in the library and return it (JSON-serialisable)."""
    import torch
    from . import api
    classes = sorted(set((int(n), int(r)) for n, r in classes))
    tmpl_max = tmpl_max or max(n for n, _ in classes)
    radius_max = radius_max or max(r for _, r in classes)
    dev = torch.device(device)
    lib = L.lib()
    t0 = time.perf_counter()
    entry = {"classes": [f"{n}x{r}" for n, r in classes], "plans": {}}
    if precision != L.CFOG_PREC_FP32_FFT:
        entry.update(variant=L.CFOG_MATCH_VARIANT_WIDE, note="BF16 path has one kernel")
        return entry
    B = _Bench(torch, api, dev, m, tmpl_max, radius_max, seed)
    # forget earlier choices for these classes so the model's plans are timed
    for v in variants:
        for n, r in classes:
            L.check(lib.cfog_match_set_plan(v, m, n, r, -1), "cfog_match_set_plan")
    mix = B.batch(classes, mix_cps)
    vms = {int(v): B.time(mix, v, reps=reps) for v in variants}
    best_v = min(vms, key=vms.get)
    entry["variants_ms"] = {str(v): t for v, t in vms.items()}
    entry["variant"] = best_v
    # per-class plans of the chosen variant
    per_class = 2 * B.n_sm * 2
    timed = {}
    for n, r in classes:
        cands = candidates(n, r, m, best_v, k_plans, lib)
        if len(cands) < 2:
            continue
        b = B.batch([(n, r)], per_class)
        ts = []
        for c in cands:
            L.check(lib.cfog_match_set_plan(best_v, m, n, r, c["code"]), "cfog_match_set_plan")
            ts.append(B.time(b, best_v, reps=reps))
        L.check(lib.cfog_match_set_plan(best_v, m, n, r, -1), "cfog_match_set_plan")
        j = int(np.argmin(ts))
        timed[f"{n}x{r}"] = {"ms": ts, "plans": [[c["P_y"], c["P_x"], c["nb_y"], c["nb_x"]]
                                                  for c in cands]}
        if j > 0 and ts[j] < (1.0 - NOISE) * ts[0]:
            entry["plans"][f"{n}x{r}"] = cands[j]["code"]
    entry["class_ms"] = timed
    if entry["plans"]:
        for cls, code in entry["plans"].items():
            nn, rr = (int(x) for x in cls.split("x"))
            L.check(lib.cfog_match_set_plan(best_v, m, nn, rr, code), "cfog_match_set_plan")
        tuned_ms = B.time(mix, best_v, reps=reps)
        entry["mix_ms_tuned"] = tuned_ms
        if tuned_ms >= vms[best_v]:
            for cls in entry["plans"]:
                nn, rr = (int(x) for x in cls.split("x"))
                L.check(lib.cfog_match_set_plan(best_v, m, nn, rr, -1), "cfog_match_set_plan")
            entry["plans_dropped"] = entry.pop("plans")
            entry["plans"] = {}
    # every class gets a table entry: the timed winner, else the cost model's
    # own plan (the same plan the kernel's search would find), so a launch
    # reads each class's plan from the table instead of searching for it
    entry["model_plans"] = {}
    for n, r in classes:
        key = f"{n}x{r}"
        if key not in entry["plans"]:
            cands = candidates(n, r, m, best_v, 1, lib)
            if cands:
                entry["model_plans"][key] = cands[0]["code"]
    for cls, code in entry["model_plans"].items():
        nn, rr = (int(x) for x in cls.split("x"))
        L.check(lib.cfog_match_set_plan(best_v, m, nn, rr, code), "cfog_match_set_plan")
    entry["mix_ms_model"] = vms[best_v]
    entry["tune_s"] = time.perf_counter() - t0
    L.check(lib.cfog_match_set_auto_variant(m, tmpl_max, radius_max, precision, best_v),
            "cfog_match_set_auto_variant")
    return entry


def ensure(classes, m=9, tmpl_max=None, radius_max=None, precision=L.CFOG_PREC_FP32_FFT,
           device="cuda", path=None, retune=False):
    """Apply the cached tuning of this GPU and launch class, tuning (and
    caching) first when there is none.  Returns the entry, with "source"
    "cache" or "tuned"."""
    import torch
    classes = sorted(set((int(n), int(r)) for n, r in classes))
    tmpl_max = tmpl_max or max(n for n, _ in classes)
    radius_max = radius_max or max(r for _, r in classes)
    dev = torch.device(device)
    props = torch.cuda.get_device_properties(dev)
    dkey = device_key(props.name, (props.major, props.minor), L.lib_fingerprint())
    ckey = class_key(m, tmpl_max, radius_max, precision, classes)
    data = load_cache(path)
    entry = data["entries"].get(dkey, {}).get(ckey)
    if entry is not None and not retune:
        with torch.cuda.device(dev):
            apply(entry, m, tmpl_max, radius_max, precision)
        return dict(entry, source="cache")
    with torch.cuda.device(dev):
        entry = tune(classes, m, tmpl_max, radius_max, precision, device=dev)
    data = load_cache(path)   # another process may have written meanwhile
    data["entries"].setdefault(dkey, {})[ckey] = entry
    save_cache(data, path)
    return dict(entry, source="tuned")
