"""Synthetic multimodal image pairs (seeded, numpy + scipy only).

Recipes (all draws from ``numpy.random.default_rng(seed)``):

* ``rect_texture``: additive axis-aligned rectangles (corners uniform, side
  lengths uniform in {8..64}, intensity U[0,255]) plus white noise
  N(0, 20^2) blurred by a Gaussian of sigma 1.5, min-max rescaled to [0,255].
  The rectangle count scales with area (40 per 256x256).
* ``tiny_pair``: 256x256; B = 255*(1-(A/255)^0.5) times Gamma(4, 1/4)
  speckle, circularly shifted by an integer (dx, dy) in U{-8..8}.
* ``batched_pair``: as tiny, 2048x2048, but B is also warped by a smooth
  field (two random low-frequency sines per axis, |u| <= 6 px) on top of a
  global integer shift in U{-10..10}; bilinear resampling.
* ``precision_pair``: 4096x4096 geometry as batched, B a map-like rendering
  of A (6 quantisation levels, level boundaries drawn as 1-px lines of value
  0, additive N(0, 10^2) noise).
* ``serving_jobs``: a Poisson stream of job descriptions; pair sizes
  log-uniform in [512, 8192], float32 or uint16 input, one CP per 64x64
  block, template in {64, 96}, radius in {10..20}.
* ``large_scene_pair``: uint16 12-bit pair, log-normal intensity; B is a
  SAR-like log-speckled remap of A rotated by 0.3 degrees and shifted.

Ground truth: the displacement ``d(p)`` such that B(p + d) shows the same
scene point as A(p).  The generators hold none of the matching method's
arithmetic.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np
from scipy import ndimage


@dataclasses.dataclass
class Pair:
    A: np.ndarray          # reference image (float32 or uint16), H x W
    B: np.ndarray          # sensed image, same size
    shift: tuple           # global integer shift (dy, dx)
    field: object = None   # callable (ys, xs) -> (dy, dx) arrays, or None
    meta: dict = dataclasses.field(default_factory=dict)

    def truth(self, ys, xs):
        """Ground-truth displacement (dy, dx) at reference pixels (ys, xs)."""
        ys = np.asarray(ys, dtype=np.float64)
        xs = np.asarray(xs, dtype=np.float64)
        if self.field is None:
            return (np.full(ys.shape, float(self.shift[0])),
                    np.full(xs.shape, float(self.shift[1])))
        return self.field(ys, xs)


def rect_texture(rng, h, w, n_rect=None, noise_sigma=20.0, blur=1.5, dtype=np.float64):
    """Sum of random rectangles plus blurred white noise, rescaled to [0,255]."""
    if n_rect is None:
        n_rect = max(1, int(round(40 * (h * w) / (256 * 256))))
    acc = np.zeros((h + 1, w + 1), dtype=dtype)
    y0 = rng.integers(0, h, size=n_rect)
    x0 = rng.integers(0, w, size=n_rect)
    sh = rng.integers(8, 65, size=n_rect)
    sw = rng.integers(8, 65, size=n_rect)
    val = rng.uniform(0.0, 255.0, size=n_rect)
    y1 = np.minimum(y0 + sh, h)
    x1 = np.minimum(x0 + sw, w)
    # 2-D difference array: +v at (y0,x0), -v at (y0,x1), (y1,x0), +v at (y1,x1)
    np.add.at(acc, (y0, x0), val)
    np.add.at(acc, (y0, x1), -val)
    np.add.at(acc, (y1, x0), -val)
    np.add.at(acc, (y1, x1), val)
    np.cumsum(acc, axis=0, out=acc)
    np.cumsum(acc, axis=1, out=acc)
    img = acc[:h, :w]
    noise = rng.normal(0.0, noise_sigma, size=(h, w)).astype(dtype, copy=False)
    img += ndimage.gaussian_filter(noise, blur, mode="wrap")
    del noise
    lo, hi = img.min(), img.max()
    img -= lo
    img *= img.dtype.type(255.0 / max(hi - lo, 1e-12))
    return img


def _remap_speckle(rng, A):
    """Nonlinear intensity remap with multiplicative Gamma(L=4) speckle."""
    B0 = 255.0 * (1.0 - np.power(np.clip(A, 0.0, 255.0) / 255.0, 0.5))
    return B0 * rng.gamma(4.0, 0.25, size=A.shape)


def _smooth_field(rng, h, w, amp_max=6.0):
    """Two random low-frequency sines per axis; |u| <= amp_max."""
    params = []
    for _axis in range(2):
        a = rng.uniform(0.0, amp_max / 2.0, size=2)
        f = rng.uniform(-2.0, 2.0, size=2)
        g = rng.uniform(-2.0, 2.0, size=2)
        ph = rng.uniform(0.0, 2.0 * math.pi, size=2)
        params.append((a, f, g, ph))

    def u(ys, xs):
        out = []
        for a, f, g, ph in params:
            val = np.zeros(np.broadcast(ys, xs).shape)
            for j in range(2):
                val = val + a[j] * np.sin(2.0 * math.pi * (f[j] * xs / w + g[j] * ys / h) + ph[j])
            out.append(val)
        return out[0], out[1]

    return u


def _warp(img, sy, sx, u):
    """B(y,x) = img(y - sy - uy(y,x), x - sx - ux(y,x)), bilinear, wrap."""
    h, w = img.shape
    yy, xx = np.meshgrid(np.arange(h, dtype=np.float64), np.arange(w, dtype=np.float64),
                         indexing="ij")
    uy, ux = u(yy, xx)
    coords = np.stack([yy - sy - uy, xx - sx - ux])
    return ndimage.map_coordinates(img, coords, order=1, mode="grid-wrap")


def tiny_pair(seed=0, size=256):
    rng = np.random.default_rng(seed)
    A = rect_texture(rng, size, size, n_rect=40)
    B = _remap_speckle(rng, A)
    dy, dx = (int(v) for v in rng.integers(-8, 9, size=2))
    B = np.roll(B, (dy, dx), axis=(0, 1))
    return Pair(A.astype(np.float32), B.astype(np.float32), (dy, dx), None,
                {"config": "tiny", "size": size})


def batched_pair(seed=1, size=2048, render="speckle"):
    rng = np.random.default_rng(seed)
    A = rect_texture(rng, size, size)
    if render == "speckle":
        B0 = _remap_speckle(rng, A)
    else:
        B0 = _map_render(rng, A)
    sy, sx = (int(v) for v in rng.integers(-10, 11, size=2))
    u = _smooth_field(rng, size, size, 6.0)
    B = _warp(B0, sy, sx, u)

    def field(ys, xs):
        uy, ux = u(ys, xs)
        return sy + uy, sx + ux

    return Pair(A.astype(np.float32), B.astype(np.float32), (sy, sx), field,
                {"config": "batched", "size": size, "render": render})


def _map_render(rng, A, levels=6, noise=10.0):
    """Map-like rendering: quantised levels with 1-px boundary lines, plus noise."""
    qs = np.quantile(A, np.linspace(0.0, 1.0, levels + 1)[1:-1])
    lab = np.digitize(A, qs)
    out = (lab.astype(np.float64) + 0.5) * (255.0 / levels)
    edge = np.zeros(A.shape, dtype=bool)
    edge[:, :-1] |= lab[:, :-1] != lab[:, 1:]
    edge[:-1, :] |= lab[:-1, :] != lab[1:, :]
    out[edge] = 0.0
    return out + rng.normal(0.0, noise, size=A.shape)


def precision_pair(seed=2, size=4096):
    return batched_pair(seed, size, render="map")


def random_cp_params(seed, n, sizes=(48, 64, 96, 128), rmin=8, rmax=20):
    """Per-CP template sizes (uniform over ``sizes``) and radii (U{rmin..rmax})."""
    rng = np.random.default_rng(seed)
    tmpl = rng.choice(np.asarray(sizes, dtype=np.int32), size=n)
    rad = rng.integers(rmin, rmax + 1, size=n).astype(np.int32)
    return tmpl.astype(np.int32), rad


def serving_jobs(seed=3, duration_s=60.0, rate=200.0, smin=512, smax=8192, align=16):
    """Poisson stream of job descriptions (no pixels; see ``job_pair``)."""
    rng = np.random.default_rng(seed)
    t = 0.0
    jobs = []
    while True:
        t += rng.exponential(1.0 / rate)
        if t > duration_s:
            break
        side = math.exp(rng.uniform(math.log(smin), math.log(smax)))
        side = max(smin, int(side) // align * align)
        jobs.append({
            "t": t,
            "size": side,
            "dtype": "u16" if rng.random() < 0.5 else "f32",
            "tmpl": int(rng.choice([64, 96])),
            "radius": int(rng.integers(10, 21)),
            "seed": int(rng.integers(0, 2**31 - 1)),
        })
    return jobs


def job_pair(job, base=None):
    """Pixels for one serving job: a crop of a shared base texture (speckled B).

    Cropping a shared base keeps host-side generation cheap for a stream of
    thousands of jobs while every job still has its own shift and speckle.
    """
    rng = np.random.default_rng(job["seed"])
    s = job["size"]
    if base is None or base.shape[0] < s + 32:
        base = rect_texture(rng, s + 32, s + 32)
    oy, ox = (int(v) for v in rng.integers(0, base.shape[0] - s + 1, size=2))
    A = base[oy:oy + s, ox:ox + s]
    B = np.roll(_remap_speckle(rng, A), tuple(int(v) for v in rng.integers(-6, 7, size=2)),
                axis=(0, 1))
    if job["dtype"] == "u16":
        A = np.clip(np.rint(A * 16.0), 0, 4095).astype(np.uint16)
        B = np.clip(np.rint(B * 16.0), 0, 4095).astype(np.uint16)
    else:
        A = A.astype(np.float32)
        B = B.astype(np.float32)
    return A, B


def large_scene_pair(seed=4, size=20000, angle_deg=0.3, band=1024):
    """12-bit uint16 pair: log-normal intensity; B is a SAR-like log-speckled remap
    of A, rotated by ``angle_deg`` about the centre and shifted by <= 10 px.
    Generated in float32 row bands so that a 20000^2 pair fits in host memory."""
    rng = np.random.default_rng(seed)
    tex = rect_texture(rng, size, size, dtype=np.float32)
    A = np.empty((size, size), dtype=np.float32)
    Bl = np.empty((size, size), dtype=np.float32)
    norm = np.float32(4095.0 / np.log1p(4095.0 * 4.0))
    for y0 in range(0, size, band):
        y1 = min(size, y0 + band)
        a = np.exp(rng.normal(6.0, 0.6, size=(y1 - y0, size))).astype(np.float32)
        a *= tex[y0:y1] / np.float32(255.0)
        np.clip(a, 0.0, 4095.0, out=a)
        A[y0:y1] = a
        g = rng.gamma(4.0, 0.25, size=(y1 - y0, size)).astype(np.float32)
        Bl[y0:y1] = np.minimum(np.log1p(a * g) * norm, np.float32(4095.0))
    del tex
    sy, sx = (int(v) for v in rng.integers(-10, 11, size=2))
    th = math.radians(angle_deg)
    c = (size - 1) / 2.0

    def field(ys, xs):
        # B(p + d) = Bl(p): p + d = R(p - c) + c + s
        ry = math.cos(th) * (ys - c) + math.sin(th) * (xs - c) + c + sy
        rx = -math.sin(th) * (ys - c) + math.cos(th) * (xs - c) + c + sx
        return ry - ys, rx - xs

    B = np.empty((size, size), dtype=np.uint16)
    xx = np.arange(size, dtype=np.float64)
    for y0 in range(0, size, band):
        y1 = min(size, y0 + band)
        yy = np.arange(y0, y1, dtype=np.float64)[:, None]
        # inverse map: source = R^T (q - c - s) + c
        qy, qx = yy - c - sy, xx[None, :] - c - sx
        src_y = math.cos(th) * qy - math.sin(th) * qx + c
        src_x = math.sin(th) * qy + math.cos(th) * qx + c
        lo = max(0, int(np.floor(src_y.min())) - 2)
        hi = min(size, int(np.ceil(src_y.max())) + 3)
        v = ndimage.map_coordinates(Bl[lo:hi], np.stack([src_y - lo, src_x]), order=1,
                                    mode="nearest")
        B[y0:y1] = np.clip(np.rint(v), 0, 4095).astype(np.uint16)
    del Bl
    A16 = np.clip(np.rint(A), 0, 4095).astype(np.uint16)
    return Pair(A16, B, (sy, sx), field, {"config": "large", "size": size,
                                          "angle_deg": angle_deg})


def make_pair(config_id, seed=None, **kw):
    seed = config_id if seed is None else seed
    if config_id == 0:
        return tiny_pair(seed, **kw)
    if config_id == 1:
        return batched_pair(seed, **kw)
    if config_id == 2:
        return precision_pair(seed, **kw)
    if config_id == 4:
        return large_scene_pair(seed, **kw)
    raise ValueError(f"no pair generator for config {config_id}")
