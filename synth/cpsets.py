"""Seeded synthetic control-point sets for the outlier-rejection step.

A set is what the matcher hands to the rejection step: CP positions p in the
reference image and match results whose sub-pixel offsets d place p + d in
the sensed image.  The truth mapping is a smooth field: a cubic polynomial, or
the sum of sinusoids used by the batched image pairs.  A fraction of the CPs
are gross mismatches: their offsets are moved by distinct, well-separated
amounts, as clouds or shadows do in the paper's scenes.  A few CPs carry a
non-OK status.  Nothing here fits, solves or ranks anything.
"""
from __future__ import annotations

import numpy as np

# cfog_match_result as a numpy record (24 bytes, the C ABI layout)
RESULT_DTYPE = np.dtype([("dx", "<i4"), ("dy", "<i4"), ("sub_dx", "<f4"), ("sub_dy", "<f4"),
                         ("ssd", "<f4"), ("status", "<i4")])


def _cubic_field(rng, size, amp):
    """A random cubic displacement field with |d| of order `amp` pixels."""
    c = rng.normal(0.0, 1.0, (2, 10)) * amp

    def field(x, y):
        u = x / size * 2.0 - 1.0
        v = y / size * 2.0 - 1.0
        mons = np.stack([np.ones_like(u), u, v, u * u, u * v, v * v,
                         u ** 3, u * u * v, u * v * v, v ** 3])
        return np.tensordot(c[0], mons, 1), np.tensordot(c[1], mons, 1)
    return field


def _sine_field(rng, size, amp):
    """Two sinusoids per axis with at most 2 cycles per image side."""
    pars = [(rng.uniform(0.3, 1.0) * amp / 2, rng.uniform(0, 2), rng.uniform(0, 2),
             rng.uniform(0, 2 * np.pi)) for _ in range(4)]

    def field(x, y):
        out = []
        for ax in range(2):
            acc = 0.0
            for a, f, g, ph in pars[2 * ax:2 * ax + 2]:
                acc = acc + a * np.sin(2 * np.pi * (f * x + g * y) / size + ph)
            out.append(acc)
        return out[0], out[1]
    return field


def cp_set(seed, n, size=4096, field="cubic", amp=6.0, shift=(7.0, -4.0), noise=0.15,
           outlier_frac=0.05, outlier_min=6.0, outlier_step=1.5, bad_status_frac=0.02):
    """CP positions (int32 [n, 2]), match results (RESULT_DTYPE [n]) and truth.

    Outliers get offset errors of distinct sizes outlier_min + k * outlier_step
    (k = 0, 1, ...) in random directions, so that no two are near a tie.
    Returns (cps, res, info) with info = {"outliers": indices, "bad": indices,
    "field": callable(x, y) -> (dx, dy)}.
    """
    rng = np.random.default_rng(seed)
    margin = size // 16
    cps = rng.integers(margin, size - margin, (n, 2)).astype(np.int32)
    fld = (_cubic_field if field == "cubic" else _sine_field)(rng, size, amp)
    x = cps[:, 0].astype(np.float64)
    y = cps[:, 1].astype(np.float64)
    dx, dy = fld(x, y)
    dx = dx + shift[0] + rng.normal(0.0, noise, n)
    dy = dy + shift[1] + rng.normal(0.0, noise, n)
    n_out = int(round(outlier_frac * n))
    out_idx = rng.choice(n, n_out, replace=False) if n_out else np.zeros(0, dtype=np.int64)
    mags = outlier_min + outlier_step * rng.permutation(n_out)
    ang = rng.uniform(0, 2 * np.pi, n_out)
    dx[out_idx] += mags * np.cos(ang)
    dy[out_idx] += mags * np.sin(ang)
    res = np.zeros(n, dtype=RESULT_DTYPE)
    res["sub_dx"] = dx.astype(np.float32)
    res["sub_dy"] = dy.astype(np.float32)
    res["dx"] = np.rint(dx).astype(np.int32)
    res["dy"] = np.rint(dy).astype(np.int32)
    res["ssd"] = rng.uniform(0, 100, n).astype(np.float32)
    rest = np.setdiff1d(np.arange(n), out_idx)
    n_bad = int(round(bad_status_frac * n))
    bad = rng.choice(rest, n_bad, replace=False) if n_bad else np.zeros(0, dtype=np.int64)
    res["status"][bad] = rng.choice([1, 2], n_bad)
    return cps, res, {"outliers": np.sort(out_idx), "outlier_mags": dict(zip(out_idx.tolist(), mags)),
                      "bad": np.sort(bad), "field": fld}
