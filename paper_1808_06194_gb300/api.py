"""Torch-facing wrappers over the C ABI (device memory and streams only).

Every function marshals torch tensors into the plain structs of
include/cfog.h and calls the library entry point of the same name; no
arithmetic of the method happens here.
"""
from __future__ import annotations

import ctypes
import dataclasses

import torch

from . import _lib as L


def _stream_ptr(stream):
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def params(m=9, sigma=0.8, eps=1e-6, gauss_radius=3, orientation=L.CFOG_ORIENT_EQ2):
    return L.cfog_params(m, sigma, eps, gauss_radius, orientation)


def default_params():
    p = L.cfog_params()
    L.check(L.lib().cfog_default_params(ctypes.byref(p)), "cfog_default_params")
    return p


def image_struct(img):
    """cfog_image for a 2-D CUDA tensor (float32 or uint16), rows contiguous."""
    if img.dim() != 2 or img.stride(1) != 1:
        raise ValueError("image must be a 2-D tensor with contiguous rows")
    if img.dtype == torch.float32:
        dt = L.CFOG_DTYPE_F32
    elif img.dtype == torch.uint16:
        dt = L.CFOG_DTYPE_U16
    else:
        raise TypeError(f"unsupported image dtype {img.dtype}")
    return L.cfog_image(img.data_ptr(), img.shape[0], img.shape[1], img.stride(0), dt)


@dataclasses.dataclass
class Features:
    """A CFOG volume: planar FP32 channels plus the ||D||^2 plane, on the device."""
    data: torch.Tensor      # flat float32, m * plane_pitch
    sqnorm: torch.Tensor    # flat float32, h * row_pitch
    m: int
    h: int
    w: int
    row_pitch: int
    plane_pitch: int

    def struct(self):
        return L.cfog_features(self.data.data_ptr(), self.sqnorm.data_ptr(), self.m, self.h,
                               self.w, self.row_pitch, self.plane_pitch)

    def volume(self):
        """(m, h, w) strided view of the channels."""
        return self.data.as_strided((self.m, self.h, self.w), (self.plane_pitch, self.row_pitch, 1))

    def sq(self):
        return self.sqnorm.as_strided((self.h, self.w), (self.row_pitch, 1))

    @property
    def nbytes(self):
        return (self.data.numel() + self.sqnorm.numel()) * 4


def feature_layout(h, w, m=9):
    rp = ctypes.c_int64()
    pp = ctypes.c_int64()
    nbytes = L.lib().cfog_feature_layout(h, w, m, ctypes.byref(rp), ctypes.byref(pp))
    if nbytes == 0:
        raise ValueError(f"bad feature layout request {h}x{w}x{m}")
    return rp.value, pp.value, nbytes


def alloc_features(h, w, m=9, device="cuda"):
    rp, pp, nbytes = feature_layout(h, w, m)
    data = torch.empty(nbytes // 4, dtype=torch.float32, device=device)
    sq = torch.empty(h * rp, dtype=torch.float32, device=device)
    return Features(data, sq, m, h, w, rp, pp)


def cfog_extract(img, p=None, out=None, stream=None):
    """CFOG of a device image (Sec. III-F); returns Features."""
    if p is None:
        p = default_params()
    if out is None:
        out = alloc_features(img.shape[0], img.shape[1], p.m, img.device)
    im = image_struct(img)
    f = out.struct()
    L.check(L.lib().cfog_extract(ctypes.byref(im), ctypes.byref(p), ctypes.byref(f),
                                 _stream_ptr(stream)), "cfog_extract")
    return out


def cfog_extract_fhog(img, cell=8, eps=1e-6, out=None, stream=None):
    """Pixel-wise HOG (Sec. III-C) of a device image: Features with m = 36."""
    if out is None:
        out = alloc_features(img.shape[0], img.shape[1], 36, img.device)
    im = image_struct(img)
    f = out.struct()
    L.check(L.lib().cfog_extract_fhog(ctypes.byref(im), int(cell), float(eps), ctypes.byref(f),
                                      _stream_ptr(stream)), "cfog_extract_fhog")
    return out


def cfog_extract_rows(img, row0, row1, out, p=None, stream=None):
    """CFOG of rows [row0, row1) of a device image into `out` (full-size Features)."""
    if p is None:
        p = default_params()
    im = image_struct(img)
    f = out.struct()
    L.check(L.lib().cfog_extract_rows(ctypes.byref(im), ctypes.byref(p), ctypes.byref(f), row0,
                                      row1, _stream_ptr(stream)), "cfog_extract_rows")
    return out


def cfog_detect_cps(img, grid_x, grid_y, k=1, chip=0, margin=0, out=None, stream=None):
    """Block-based Harris CPs (Sec. IV): int32 tensor (grid_y*grid_x*k, 2) of (x, y)."""
    n = grid_x * grid_y * k
    if out is None:
        out = torch.empty((n, 2), dtype=torch.int32, device=img.device)
    im = image_struct(img)
    L.check(L.lib().cfog_detect_cps(ctypes.byref(im), grid_x, grid_y, k, chip, margin, _ptr(out),
                                    _stream_ptr(stream)), "cfog_detect_cps")
    return out


def cfog_match(ref, sen, cps, tmpl, radius, tmpl_max, radius_max, prior=None,
               precision=L.CFOG_PREC_FP32_FFT, out=None, surface=None, stream=None):
    """Match CPs (Eq. 3-9): int32 tensor (n, 6) of cfog_match_result rows."""
    n = cps.shape[0]
    if out is None:
        out = torch.empty((n, 6), dtype=torch.int32, device=cps.device)
    rf, sf = ref.struct(), sen.struct()
    L.check(L.lib().cfog_match(ctypes.byref(rf), ctypes.byref(sf), _ptr(cps), n, _ptr(tmpl),
                               _ptr(radius), int(tmpl_max), int(radius_max), _ptr(prior),
                               precision, _ptr(out), _ptr(surface), _stream_ptr(stream)),
            "cfog_match")
    return out


def cfog_fit_affine(cps, res, work=None, stream=None):
    """FP64 affine LS fit (Sec. IV) over CPs with status OK; returns 6 floats."""
    if work is None:
        work = torch.empty(L.CFOG_AFFINE_WORK_DOUBLES, dtype=torch.float64, device=cps.device)
    out6 = (ctypes.c_double * 6)()
    L.check(L.lib().cfog_fit_affine(_ptr(cps), _ptr(res), cps.shape[0], _ptr(work), out6,
                                    _stream_ptr(stream)), "cfog_fit_affine")
    return [out6[i] for i in range(6)]


def reject_workspace(n_cps, n_jobs, device="cuda"):
    """Workspace tensor for cfog_reject_outliers (256-byte aligned by torch)."""
    nbytes = L.lib().cfog_reject_workspace_bytes(int(n_cps), int(n_jobs))
    return torch.empty(max(nbytes, 256), dtype=torch.uint8, device=device)


def cfog_reject_outliers(cps, res, job_start=None, degree=3, rmse_threshold=1.0, min_keep=0,
                         keep=None, order=None, models=None, workspace=None, stream=None):
    """Iterative outlier rejection with a polynomial model (Sec. IV), one CTA per job.

    job_start: host sequence of n_jobs + 1 offsets into cps/res (default: one job
    over all CPs).  Returns (keep uint8 [n], order int32 [n], models uint8
    [n_jobs, sizeof(cfog_poly_model)]); `unpack_models` reads the models.
    """
    n = cps.shape[0]
    if job_start is None:
        job_start = [0, n]
    js = (ctypes.c_int32 * len(job_start))(*[int(v) for v in job_start])
    n_jobs = len(job_start) - 1
    dev = cps.device
    if keep is None:
        keep = torch.zeros(n, dtype=torch.uint8, device=dev)
    if order is None:
        order = torch.full((n,), -1, dtype=torch.int32, device=dev)
    msz = ctypes.sizeof(L.cfog_poly_model)
    if models is None:
        models = torch.zeros((max(n_jobs, 1), msz), dtype=torch.uint8, device=dev)
    if workspace is None:
        workspace = reject_workspace(job_start[-1], n_jobs, dev)
    L.check(L.lib().cfog_reject_outliers(_ptr(cps), _ptr(res), js, n_jobs, int(degree),
                                         float(rmse_threshold), int(min_keep), _ptr(keep),
                                         _ptr(order), _ptr(models), _ptr(workspace),
                                         workspace.numel(), _stream_ptr(stream)),
            "cfog_reject_outliers")
    return keep, order, models


def unpack_models(models):
    """cfog_poly_model rows (uint8 tensor) -> list of dicts (copies to the host)."""
    raw = models.cpu().numpy().tobytes()
    msz = ctypes.sizeof(L.cfog_poly_model)
    out = []
    for j in range(len(raw) // msz):
        m = L.cfog_poly_model.from_buffer_copy(raw[j * msz:(j + 1) * msz])
        t = m.terms
        out.append({"status": m.status, "terms": t, "n_valid": m.n_valid, "n_kept": m.n_kept,
                    "n_removed": m.n_removed, "n_fits": m.n_fits, "rmse": m.rmse,
                    "norm": (m.cx, m.cy, m.scale),
                    "coef": [list(m.coef_x)[:t], list(m.coef_y)[:t]]})
    return out


def tin_delaunay(pts, keep=None):
    """Delaunay triangles (int32 [n_tris, 3], indices into pts) of the CPs pts
    (int array [n, 2] or a CPU tensor), keeping those with keep != 0; host only."""
    import numpy as np
    p = np.ascontiguousarray(np.asarray(pts.cpu() if hasattr(pts, "cpu") else pts, dtype=np.int32))
    n = p.shape[0]
    arr = (L.cfog_point * max(n, 1)).from_buffer_copy(p.tobytes() if n else bytes(8))
    kp = None
    if keep is not None:
        k = np.ascontiguousarray(np.asarray(keep.cpu() if hasattr(keep, "cpu") else keep, dtype=np.uint8))
        kp = (ctypes.c_uint8 * max(n, 1)).from_buffer_copy(k.tobytes() if n else bytes(1))
    cap = 2 * n + 4
    out = (ctypes.c_int32 * (3 * cap))()
    nt = ctypes.c_int32()
    L.check(L.lib().cfog_tin_delaunay(arr, n, kp, out, cap, ctypes.byref(nt)), "cfog_tin_delaunay")
    return np.frombuffer(bytes(out), dtype=np.int32)[:3 * nt.value].reshape(-1, 3).copy()


def tin_workspace(n_tris, out_h, out_w, device="cuda"):
    nbytes = L.lib().cfog_tin_workspace_bytes(int(n_tris), int(out_h), int(out_w))
    return torch.empty(max(nbytes, 256), dtype=torch.uint8, device=device)


def cfog_tin_rectify(sen, cps, res, tris, out_h, out_w, nodata=0.0, out=None, workspace=None,
                     stream=None):
    """Piecewise-linear rectification (Sec. IV) of a device sensed image onto an
    out_h x out_w reference grid over the triangles `tris` (device int32 [t, 3])."""
    n_tris = tris.shape[0]
    if out is None:
        out = torch.empty((out_h, out_w), dtype=torch.float32, device=sen.device)
    if workspace is None:
        workspace = tin_workspace(n_tris, out_h, out_w, sen.device)
    im = image_struct(sen)
    L.check(L.lib().cfog_tin_rectify(ctypes.byref(im), _ptr(cps), _ptr(res), cps.shape[0], _ptr(tris),
                                     n_tris, int(out_h), int(out_w), float(nodata), _ptr(out),
                                     out.stride(0), _ptr(workspace), workspace.numel(),
                                     _stream_ptr(stream)), "cfog_tin_rectify")
    return out


def cfog_plan_info(tmpl, radius, m=9, variant=L.CFOG_MATCH_VARIANT_AUTO):
    """FFT plan of a CP class: dict with blocks, FFT sizes, passes, smem bytes."""
    out = (ctypes.c_int32 * 8)()
    L.check(L.lib().cfog_plan_info(tmpl, radius, m, variant, out), "cfog_plan_info")
    keys = ["nb_y", "nb_x", "P_y", "P_x", "b_y", "b_x", "stages", "smem"]
    return dict(zip(keys, list(out)))


def resolve_variant(tmpl_max, radius_max, m=9, precision=L.CFOG_PREC_FP32_FFT,
                    variant=L.CFOG_MATCH_VARIANT_AUTO):
    """The matcher variant a batched launch of this class runs (AUTO resolved)."""
    if variant != L.CFOG_MATCH_VARIANT_AUTO:
        return int(variant)
    return int(L.lib().cfog_match_auto_variant(m, int(tmpl_max), int(radius_max), precision))


def job_table(pairs, device="cuda"):
    """Device array of cfog_job for a list of (ref Features, sen Features)."""
    arr = (L.cfog_job * len(pairs))()
    for i, (rf, sf) in enumerate(pairs):
        arr[i].ref = rf.struct()
        arr[i].sen = sf.struct()
    raw = bytes(arr)
    return torch.frombuffer(bytearray(raw), dtype=torch.uint8).to(device)


def match_workspace(n, device="cuda"):
    """Workspace tensor for cfog_match_batched (256-byte aligned by torch)."""
    nbytes = L.lib().cfog_match_workspace_bytes(n)
    return torch.empty(max(nbytes, 256), dtype=torch.uint8, device=device)


def cfog_match_batched(jobs, n_jobs, cps, tmpl, radius, tmpl_max, radius_max, m=9,
                       job_of_cp=None, prior=None, precision=L.CFOG_PREC_FP32_FFT,
                       variant=L.CFOG_MATCH_VARIANT_AUTO, out=None, workspace=None, stream=None):
    """Batched matching over a device job table in one persistent launch."""
    n = cps.shape[0]
    if out is None:
        out = torch.empty((n, 6), dtype=torch.int32, device=cps.device)
    if workspace is None:
        workspace = match_workspace(n, cps.device)
    L.check(L.lib().cfog_match_batched(_ptr(jobs), n_jobs, _ptr(job_of_cp), _ptr(cps), n,
                                       _ptr(tmpl), _ptr(radius), int(tmpl_max), int(radius_max),
                                       m, _ptr(prior), precision, variant, _ptr(out),
                                       _ptr(workspace), workspace.numel(), _stream_ptr(stream)),
            "cfog_match_batched")
    return out


def unpack_results(res):
    """Split (n, 6) int32 result rows into named tensors."""
    f = res.view(torch.float32)
    return {"dx": res[:, 0], "dy": res[:, 1], "sub_dx": f[:, 2], "sub_dy": f[:, 3],
            "ssd": f[:, 4], "status": res[:, 5]}
