"""ctypes wrapper around the FP64 C oracle (test infrastructure only).

The shared object is compiled from ``cfog_oracle.c`` with the host compiler
into ``oracle/_build/`` on first use (or by ``build()``).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "cfog_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_SO = os.path.join(_OUT_DIR, "libcfog_oracle.so")
_lock = threading.Lock()
_lib = None

# Paper defaults: m = 9, sigma = 0.8 (Sec. V-C); R = ceil(3 sigma) and
# eps = 1e-6 are readings.  Harris: sigma 1.5, R 4, kappa 0.04 (readings).
DEFAULTS = {"m": 9, "sigma": 0.8, "radius": 3, "eps": 1e-6,
            "harris_sigma": 1.5, "harris_radius": 4, "harris_kappa": 0.04}


def build(force=False):
    """Compile the oracle into oracle/_build/libcfog_oracle.so."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if (not force and os.path.exists(_SO)
            and os.path.getmtime(_SO) >= os.path.getmtime(_SRC)):
        return _SO
    tmp = _SO + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-std=c11", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _SO)
    return _SO


def lib():
    global _lib
    with _lock:
        if _lib is None:
            _lib = ctypes.CDLL(build())
            _declare(_lib)
    return _lib


_D = ctypes.POINTER(ctypes.c_double)
_I = ctypes.POINTER(ctypes.c_int)
_i = ctypes.c_int
_d = ctypes.c_double


def _declare(L):
    L.orc_gradients.argtypes = [_D, _i, _i, _D, _D]
    L.orc_channels.argtypes = [_D, _D, _i, _i, _i, _D]
    L.orc_gauss_taps.argtypes = [_d, _i, _D]
    L.orc_smooth_xy.argtypes = [_D, _i, _i, _i, _d, _i, _D]
    L.orc_smooth_z.argtypes = [_D, _i, _i, _i, _D]
    L.orc_normalize.argtypes = [_D, _i, _i, _i, _d, _D, _D]
    L.orc_cfog.argtypes = [_D, _i, _i, _i, _d, _i, _d, _D, _D]
    L.orc_cfog_scheme.argtypes = [_D, _i, _i, _i, _d, _i, _d, _i, _D, _D]
    L.orc_channels_binned.argtypes = [_D, _D, _i, _i, _i, _D]
    L.orc_fhog.argtypes = [_D, _i, _i, _i, _d, _D, _D]
    L.orc_tin_rectify.argtypes = [_D, _i, _i, _I, _I, _D, _D, _I, _i, _i, _i, _d, _D]
    L.orc_ssd_surface.argtypes = [_D, _i, _i, _D, _i, _i, _i, _i, _i, _i, _i, _i, _i, _D, _D]
    L.orc_ssd_surface.restype = _i
    L.orc_subpixel.argtypes = [_D, _D, _D]
    L.orc_subpixel.restype = _i
    L.orc_match_one.argtypes = [_D, _i, _i, _D, _i, _i, _i, _i, _i, _i, _i, _i, _i, _I, _D, _D]
    L.orc_match_many.argtypes = [_D, _i, _i, _D, _i, _i, _i, _i, _I, _I, _I, _I, _I, _I, _I, _D]
    L.orc_harris.argtypes = [_D, _i, _i, _d, _i, _d, _D]
    L.orc_cell_chip.argtypes = [_i, _i, _i, _i, _i, _i, _i, _i, _I, _I, _I, _I]
    L.orc_detect.argtypes = [_D, _i, _i, _i, _i, _i, _i, _i, _I, _I]
    L.orc_detect.restype = _i
    L.orc_affine_ls.argtypes = [_D, _D, _D, _D, _I, _i, _D]
    L.orc_affine_ls.restype = _i
    L.orc_poly_terms.argtypes = [_i]
    L.orc_poly_terms.restype = _i
    L.orc_reject_outliers.argtypes = [_D, _D, _D, _D, _I, _i, _i, _d, _i, _I, _I, _I, _D, _D, _D,
                                      _I]
    L.orc_reject_outliers.restype = _i


def _dp(a):
    return a.ctypes.data_as(_D)


def _ip(a):
    return a.ctypes.data_as(_I)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def gradients(img):
    img = _f64(img)
    h, w = img.shape
    gx = np.empty_like(img)
    gy = np.empty_like(img)
    lib().orc_gradients(_dp(img), h, w, _dp(gx), _dp(gy))
    return gx, gy


def channels(gx, gy, m=9):
    gx, gy = _f64(gx), _f64(gy)
    h, w = gx.shape
    g = np.empty((m, h, w))
    lib().orc_channels(_dp(gx), _dp(gy), h, w, m, _dp(g))
    return g


def gauss_taps(sigma, R):
    t = np.empty(2 * R + 1)
    lib().orc_gauss_taps(sigma, R, _dp(t))
    return t


def smooth_xy(vol, sigma=0.8, R=3):
    vol = _f64(vol)
    m, h, w = vol.shape
    out = np.empty_like(vol)
    lib().orc_smooth_xy(_dp(vol), m, h, w, sigma, R, _dp(out))
    return out


def smooth_z(vol):
    vol = _f64(vol)
    m, h, w = vol.shape
    out = np.empty_like(vol)
    lib().orc_smooth_z(_dp(vol), m, h, w, _dp(out))
    return out


def normalize(vol, eps=1e-6):
    vol = _f64(vol)
    m, h, w = vol.shape
    out = np.empty_like(vol)
    sq = np.empty((h, w))
    lib().orc_normalize(_dp(vol), m, h, w, eps, _dp(out), _dp(sq))
    return out, sq


def cfog(img, m=9, sigma=0.8, R=3, eps=1e-6, scheme=0):
    """CFOG volume (m, h, w) and per-pixel ||D||^2 (h, w), FP64.
    scheme 0: channels of Eq. 2; scheme 1: binned orientations (Fig. 7)."""
    img = _f64(img)
    h, w = img.shape
    out = np.empty((m, h, w))
    sq = np.empty((h, w))
    if scheme:
        lib().orc_cfog_scheme(_dp(img), h, w, m, sigma, R, eps, int(scheme), _dp(out), _dp(sq))
    else:
        lib().orc_cfog(_dp(img), h, w, m, sigma, R, eps, _dp(out), _dp(sq))
    return out, sq


def channels_binned(gx, gy, m=9):
    """Oriented channels of the first scheme (Fig. 7): magnitude split between
    the two nearest of m bins centred on k*pi/m."""
    gx, gy = _f64(gx), _f64(gy)
    h, w = gx.shape
    g = np.empty((m, h, w))
    lib().orc_channels_binned(_dp(gx), _dp(gy), h, w, m, _dp(g))
    return g


def ssd_surface(dref, dsen, px, py, N, r, qx=0, qy=0):
    """Brute-force SSD surface S (2r+1, 2r+1) [dy, dx] and energies E; None if OOB."""
    dref, dsen = _f64(dref), _f64(dsen)
    m, hr, wr = dref.shape
    _, hs, ws = dsen.shape
    L = 2 * r + 1
    S = np.empty((L, L))
    E = np.empty((L, L))
    st = lib().orc_ssd_surface(_dp(dref), hr, wr, _dp(dsen), hs, ws, m, px, py, N, r, qx, qy,
                               _dp(S), _dp(E))
    return None if st else (S, E)


def subpixel(S9):
    S9 = _f64(np.asarray(S9).reshape(9))
    dx = ctypes.c_double()
    dy = ctypes.c_double()
    fb = lib().orc_subpixel(_dp(S9), ctypes.byref(dx), ctypes.byref(dy))
    return dx.value, dy.value, fb


def match_one(dref, dsen, px, py, N, r, qx=0, qy=0, want_surface=False):
    dref, dsen = _f64(dref), _f64(dsen)
    m, hr, wr = dref.shape
    _, hs, ws = dsen.shape
    oi = np.zeros(4, dtype=np.int32)
    od = np.zeros(6)
    L = 2 * r + 1
    surf = np.full((L, L), np.nan) if want_surface else None
    lib().orc_match_one(_dp(dref), hr, wr, _dp(dsen), hs, ws, m, px, py, N, r, qx, qy, _ip(oi),
                        _dp(od), _dp(surf) if want_surface else None)
    res = {"dx": int(oi[0]), "dy": int(oi[1]), "status": int(oi[2]), "fallback": int(oi[3]),
           "sub_dx": od[0], "sub_dy": od[1], "ssd": od[2], "E": od[3], "second": od[4],
           "gap_rel": od[5]}
    if want_surface:
        res["surface"] = surf
    return res


def match_many(dref, dsen, px, py, N, r, qx=None, qy=None):
    """Arrays of per-CP results: dict of numpy arrays (see match_one)."""
    dref, dsen = _f64(dref), _f64(dsen)
    m, hr, wr = dref.shape
    _, hs, ws = dsen.shape
    px, py, N, r = _i32(px), _i32(py), _i32(N), _i32(r)
    n = px.shape[0]
    qx = _i32(qx) if qx is not None else None
    qy = _i32(qy) if qy is not None else None
    oi = np.zeros((n, 4), dtype=np.int32)
    od = np.zeros((n, 6))
    lib().orc_match_many(_dp(dref), hr, wr, _dp(dsen), hs, ws, m, n, _ip(px), _ip(py), _ip(N),
                         _ip(r), _ip(qx) if qx is not None else None,
                         _ip(qy) if qy is not None else None, _ip(oi), _dp(od))
    return {"dx": oi[:, 0], "dy": oi[:, 1], "status": oi[:, 2], "fallback": oi[:, 3],
            "sub_dx": od[:, 0], "sub_dy": od[:, 1], "ssd": od[:, 2], "E": od[:, 3],
            "second": od[:, 4], "gap_rel": od[:, 5]}


def harris(img, sigma=1.5, R=4, kappa=0.04):
    img = _f64(img)
    h, w = img.shape
    out = np.empty_like(img)
    lib().orc_harris(_dp(img), h, w, sigma, R, kappa, _dp(out))
    return out


def cell_chip(h, w, grid_x, grid_y, chip, margin, gj, gi):
    v = [ctypes.c_int() for _ in range(4)]
    lib().orc_cell_chip(h, w, grid_x, grid_y, chip, margin, gj, gi,
                        *(ctypes.byref(x) for x in v))
    return tuple(x.value for x in v)  # y0, y1, x0, x1


def detect(resp, grid_x, grid_y, k=1, chip=0, margin=0):
    """Top-k Harris pixels per grid chip: arrays (xs, ys) of grid_y*grid_x*k."""
    resp = _f64(resp)
    h, w = resp.shape
    n = grid_x * grid_y * k
    xs = np.zeros(n, dtype=np.int32)
    ys = np.zeros(n, dtype=np.int32)
    cnt = lib().orc_detect(_dp(resp), h, w, grid_x, grid_y, k, chip, margin, _ip(xs), _ip(ys))
    return xs[:cnt], ys[:cnt]


def affine_ls(x, y, xp, yp, valid=None):
    x, y, xp, yp = _f64(x), _f64(y), _f64(xp), _f64(yp)
    n = x.shape[0]
    v = _i32(valid) if valid is not None else None
    out = np.zeros(6)
    st = lib().orc_affine_ls(_dp(x), _dp(y), _dp(xp), _dp(yp), _ip(v) if v is not None else None,
                             n, _dp(out))
    return None if st else out


def poly_terms(degree):
    return lib().orc_poly_terms(int(degree))


def reject_outliers(x, y, xp, yp, valid=None, degree=3, thr=1.0, min_keep=0):
    """Sec. IV outlier rejection; returns a dict (status, keep, order, coef[2, T],
    rmse, norm = (cx, cy, s), n_fits)."""
    x, y, xp, yp = _f64(x), _f64(y), _f64(xp), _f64(yp)
    n = x.shape[0]
    v = _i32(valid) if valid is not None else None
    keep = np.zeros(max(n, 1), dtype=np.int32)
    order = np.zeros(max(n, 1), dtype=np.int32)
    nrem = np.zeros(1, dtype=np.int32)
    nfit = np.zeros(1, dtype=np.int32)
    coef = np.zeros(20)
    rmse = np.zeros(1)
    norm = np.zeros(3)
    st = lib().orc_reject_outliers(_dp(x), _dp(y), _dp(xp), _dp(yp),
                                   _ip(v) if v is not None else None, n, int(degree), float(thr),
                                   int(min_keep), _ip(keep), _ip(order), _ip(nrem), _dp(coef),
                                   _dp(rmse), _dp(norm), _ip(nfit))
    T = poly_terms(degree)
    return {"status": int(st), "keep": keep[:n].astype(bool), "order": order[:int(nrem[0])].copy(),
            "coef": np.stack([coef[:T], coef[10:10 + T]]), "rmse": float(rmse[0]),
            "norm": tuple(norm), "n_fits": int(nfit[0])}


def poly_predict(coef, norm, x, y, degree=3):
    """Model prediction (x', y') of the fitted polynomial at reference points (x, y)."""
    cx, cy, s = norm
    u = (np.asarray(x, dtype=np.float64) - cx) / s
    v = (np.asarray(y, dtype=np.float64) - cy) / s
    cols = [u ** (d - j) * v ** j for d in range(degree + 1) for j in range(d + 1)]
    Phi = np.stack(cols, axis=-1)
    return Phi @ coef[0], Phi @ coef[1]


def fhog(img, cell=8, eps=1e-6):
    """Pixel-wise HOG (Sec. III-C): 36 planes (2 x 2 cells x 9 bins) and ||D||^2, FP64."""
    img = _f64(img)
    h, w = img.shape
    out = np.empty((36, h, w))
    sq = np.empty((h, w))
    lib().orc_fhog(_dp(img), h, w, int(cell), float(eps), _dp(out), _dp(sq))
    return out, sq


def tin_rectify(sen, ref_xy, sen_xy, tris, out_h, out_w, nodata=0.0):
    """Piecewise-linear rectification (Sec. IV): ref_xy int [n, 2], sen_xy float
    [n, 2] (sensed positions of the CPs), tris int [t, 3]; returns (out_h, out_w)."""
    sen = _f64(sen)
    sh, sw = sen.shape
    rx, ry = _i32(np.asarray(ref_xy)[:, 0]), _i32(np.asarray(ref_xy)[:, 1])
    su, sv = _f64(np.asarray(sen_xy)[:, 0]), _f64(np.asarray(sen_xy)[:, 1])
    t = _i32(np.asarray(tris).reshape(-1))
    out = np.empty((out_h, out_w))
    lib().orc_tin_rectify(_dp(sen), sh, sw, _ip(rx), _ip(ry), _dp(su), _dp(sv), _ip(t),
                          len(t) // 3, out_h, out_w, float(nodata), _dp(out))
    return out
