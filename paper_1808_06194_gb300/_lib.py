"""ctypes binding of libcfog.so: the C ABI of include/cfog.h, same names.

Argument marshalling only: every step of the hot path runs in the CUDA
kernels of libcfog.so.  Loading fails loudly when the library is missing;
there is no fallback implementation.
"""
from __future__ import annotations

import ctypes
import os
import threading

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "_build", "libcfog.so")

CFOG_OK = 0
CFOG_E_INVAL = 1
CFOG_E_CUDA = 2
CFOG_E_NOMEM = 3
CFOG_E_TIMEOUT = 4
CFOG_E_UNSUPPORTED = 5
STATUS_NAMES = {0: "CFOG_OK", 1: "CFOG_E_INVAL", 2: "CFOG_E_CUDA", 3: "CFOG_E_NOMEM",
                4: "CFOG_E_TIMEOUT", 5: "CFOG_E_UNSUPPORTED"}

CFOG_CP_OK = 0
CFOG_CP_OOB = 1
CFOG_CP_EDGE_PEAK = 2
CFOG_CP_FLAT = 3
CFOG_CP_TIMEOUT = 4

CFOG_DTYPE_F32 = 0
CFOG_DTYPE_U16 = 1
CFOG_ORIENT_EQ2 = 0
CFOG_ORIENT_BINS = 1
CFOG_PREC_FP32_FFT = 0
CFOG_PREC_BF16_DIRECT = 1
CFOG_AFFINE_WORK_DOUBLES = 16
CFOG_MATCH_VARIANT_AUTO = 0
CFOG_MATCH_VARIANT_WIDE = 1
CFOG_MATCH_VARIANT_PAIR = 2
CFOG_MATCH_VARIANT_TRIO = 3
CFOG_MATCH_VARIANT_PAIRT = 4
CFOG_REJECT_OK = 0
CFOG_REJECT_MIN_KEEP = 1
CFOG_REJECT_SINGULAR = 2


class cfog_params(ctypes.Structure):
    _fields_ = [("m", ctypes.c_int32), ("sigma", ctypes.c_float), ("eps", ctypes.c_float),
                ("gauss_radius", ctypes.c_int32), ("orientation", ctypes.c_int32)]


class cfog_image(ctypes.Structure):
    _fields_ = [("data", ctypes.c_void_p), ("h", ctypes.c_int32), ("w", ctypes.c_int32),
                ("pitch", ctypes.c_int64), ("dtype", ctypes.c_int32)]


class cfog_features(ctypes.Structure):
    _fields_ = [("data", ctypes.c_void_p), ("sqnorm", ctypes.c_void_p), ("m", ctypes.c_int32),
                ("h", ctypes.c_int32), ("w", ctypes.c_int32), ("row_pitch", ctypes.c_int64),
                ("plane_pitch", ctypes.c_int64)]


class cfog_point(ctypes.Structure):
    _fields_ = [("x", ctypes.c_int32), ("y", ctypes.c_int32)]


class cfog_job(ctypes.Structure):
    _fields_ = [("ref", cfog_features), ("sen", cfog_features)]


class cfog_match_result(ctypes.Structure):
    _fields_ = [("dx", ctypes.c_int32), ("dy", ctypes.c_int32), ("sub_dx", ctypes.c_float),
                ("sub_dy", ctypes.c_float), ("ssd", ctypes.c_float), ("status", ctypes.c_int32)]


class cfog_poly_model(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("terms", ctypes.c_int32), ("n_valid", ctypes.c_int32),
                ("n_kept", ctypes.c_int32), ("n_removed", ctypes.c_int32), ("n_fits", ctypes.c_int32),
                ("rmse", ctypes.c_double), ("cx", ctypes.c_double), ("cy", ctypes.c_double),
                ("scale", ctypes.c_double), ("coef_x", ctypes.c_double * 10),
                ("coef_y", ctypes.c_double * 10)]


# name -> (restype, argtypes); every symbol include/cfog.h declares
_P = ctypes.c_void_p
_i32 = ctypes.c_int32
SIGNATURES = {
    "cfog_version": (ctypes.c_int32, []),
    "cfog_last_error": (ctypes.c_char_p, []),
    "cfog_default_params": (ctypes.c_int, [ctypes.POINTER(cfog_params)]),
    "cfog_feature_layout": (ctypes.c_size_t, [_i32, _i32, _i32, ctypes.POINTER(ctypes.c_int64),
                                              ctypes.POINTER(ctypes.c_int64)]),
    "cfog_extract": (ctypes.c_int, [ctypes.POINTER(cfog_image), ctypes.POINTER(cfog_params),
                                    ctypes.POINTER(cfog_features), _P]),
    "cfog_extract_rows": (ctypes.c_int, [ctypes.POINTER(cfog_image), ctypes.POINTER(cfog_params),
                                         ctypes.POINTER(cfog_features), _i32, _i32, _P]),
    "cfog_extract_fhog": (ctypes.c_int, [ctypes.POINTER(cfog_image), _i32, ctypes.c_float,
                                         ctypes.POINTER(cfog_features), _P]),
    "cfog_detect_cps": (ctypes.c_int, [ctypes.POINTER(cfog_image), _i32, _i32, _i32, _i32, _i32,
                                       _P, _P]),
    "cfog_match": (ctypes.c_int, [ctypes.POINTER(cfog_features), ctypes.POINTER(cfog_features),
                                  _P, _i32, _P, _P, _i32, _i32, _P, _i32, _P, _P, _P]),
    "cfog_fit_affine": (ctypes.c_int, [_P, _P, _i32, _P, ctypes.POINTER(ctypes.c_double), _P]),
    "cfog_plan_info": (ctypes.c_int, [_i32, _i32, _i32, _i32, ctypes.POINTER(ctypes.c_int32)]),
    "cfog_plan_candidates": (ctypes.c_int, [_i32, _i32, _i32, _i32, _i32, ctypes.POINTER(ctypes.c_int32),
                                            ctypes.POINTER(ctypes.c_int32)]),
    "cfog_match_set_plan": (ctypes.c_int, [_i32, _i32, _i32, _i32, _i32]),
    "cfog_match_set_auto_variant": (ctypes.c_int, [_i32, _i32, _i32, _i32, _i32]),
    "cfog_match_auto_variant": (ctypes.c_int32, [_i32, _i32, _i32, _i32]),
    "cfog_match_clear_tuning": (ctypes.c_int, []),
    "cfog_test_inject_wait_timeout": (ctypes.c_int, [_i32, ctypes.c_int64]),
    "cfog_probe_fp32_fma": (ctypes.c_int, [_i32, _i32, _i32, _P, ctypes.POINTER(ctypes.c_double), _P]),
    "cfog_tin_delaunay": (ctypes.c_int, [ctypes.POINTER(cfog_point), _i32, ctypes.POINTER(ctypes.c_uint8),
                                         ctypes.POINTER(ctypes.c_int32), _i32,
                                         ctypes.POINTER(ctypes.c_int32)]),
    "cfog_tin_workspace_bytes": (ctypes.c_size_t, [_i32, _i32, _i32]),
    "cfog_tin_rectify": (ctypes.c_int, [ctypes.POINTER(cfog_image), _P, _P, _i32, _P, _i32, _i32, _i32,
                                        ctypes.c_float, _P, ctypes.c_int64, _P, ctypes.c_size_t, _P]),
    "cfog_reject_workspace_bytes": (ctypes.c_size_t, [_i32, _i32]),
    "cfog_reject_outliers": (ctypes.c_int, [_P, _P, ctypes.POINTER(ctypes.c_int32), _i32, _i32,
                                            ctypes.c_double, _i32, _P, _P, _P, _P, ctypes.c_size_t,
                                            _P]),
    "cfog_match_workspace_bytes": (ctypes.c_size_t, [_i32]),
    "cfog_match_batched_noalloc_max_cps": (ctypes.c_int32, []),
    "cfog_match_batched_noalloc": (ctypes.c_int, [_P, _i32, _P, _P, _i32, _P, _P, _i32, _i32,
                                                  _i32, _P, _i32, _i32, _P, _P]),
    "cfog_match_batched": (ctypes.c_int, [_P, _i32, _P, _P, _i32, _P, _P, _i32, _i32, _i32, _P,
                                          _i32, _i32, _P, _P, ctypes.c_size_t, _P]),
}

_lock = threading.Lock()
_lib = None


class CfogError(RuntimeError):
    def __init__(self, status, where, msg):
        super().__init__(f"{where}: {STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


def lib():
    """Load libcfog.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(
                    f"libcfog.so not found at {LIB_PATH}; build it with "
                    "`python -m paper_1808_06194_gb300.build` (nvcc, sm_103a)")
            L = ctypes.CDLL(LIB_PATH)
            for name, (res, args) in SIGNATURES.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
    return _lib


_fingerprint = None


def lib_fingerprint():
    """Short hash of the loaded libcfog.so: tuning caches are tied to the exact build."""
    global _fingerprint
    if _fingerprint is None:
        import hashlib
        with open(LIB_PATH, "rb") as f:
            _fingerprint = hashlib.sha1(f.read()).hexdigest()[:12]
    return _fingerprint


def check(status, where):
    if status != CFOG_OK:
        msg = lib().cfog_last_error()
        raise CfogError(status, where, msg.decode() if msg else "")
    return status
