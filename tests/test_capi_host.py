"""Host-only checks of the C ABI: the library builds and loads, exports every
symbol include/cfog.h declares, and rejects bad arguments before any launch."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "cfog.h")


@pytest.fixture(scope="module")
def L():
    from paper_1808_06194_gb300 import build, _lib
    build.build()
    return _lib


def _declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(cfog_[a-z0-9_]+)\s*\(", text)))


def test_header_declares_expected_entry_points():
    names = _declared_functions()
    for n in ["cfog_extract", "cfog_detect_cps", "cfog_match", "cfog_match_batched",
              "cfog_match_workspace_bytes", "cfog_plan_info", "cfog_fit_affine",
              "cfog_last_error", "cfog_version", "cfog_default_params", "cfog_feature_layout"]:
        assert n in names


def test_library_exports_every_declared_symbol(L):
    lib = L.lib()
    for n in _declared_functions():
        assert hasattr(lib, n), n
        assert n in L.SIGNATURES, f"binding lacks {n}"


def test_struct_layout_matches_c_compiler(L, tmp_path):
    """Sizes and field offsets of the ctypes structs equal the C compiler's."""
    import subprocess
    structs = {"cfog_params": L.cfog_params, "cfog_image": L.cfog_image,
               "cfog_features": L.cfog_features, "cfog_point": L.cfog_point,
               "cfog_match_result": L.cfog_match_result}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "cfog.h"', "int main(void){"]
    structs["cfog_job"] = L.cfog_job
    structs["cfog_poly_model"] = L.cfog_poly_model
    for name, cls in structs.items():
        lines.append(f'printf("{name} %zu\\n", sizeof({name}));')
        for fname, _ in cls._fields_:
            lines.append(f'printf("{name}.{fname} %zu\\n", offsetof({name}, {fname}));')
    lines.append("return 0;}")
    src = tmp_path / "abi.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "abi"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                   check=True)
    got = dict(line.split() for line in subprocess.run([str(exe)], capture_output=True,
                                                        text=True, check=True).stdout.splitlines())
    for name, cls in structs.items():
        assert int(got[name]) == ctypes.sizeof(cls), name
        for fname, _ in cls._fields_:
            assert int(got[f"{name}.{fname}"]) == getattr(cls, fname).offset, (name, fname)
    assert ctypes.sizeof(L.cfog_match_result) == 24
    assert ctypes.sizeof(L.cfog_poly_model) == 216


def test_version_and_defaults(L):
    lib = L.lib()
    assert lib.cfog_version() == 1
    p = L.cfog_params()
    assert lib.cfog_default_params(ctypes.byref(p)) == L.CFOG_OK
    assert (p.m, round(p.sigma, 6), p.gauss_radius) == (9, 0.8, 3)
    assert p.orientation == L.CFOG_ORIENT_EQ2
    assert lib.cfog_default_params(None) == L.CFOG_E_INVAL
    assert b"NULL" in lib.cfog_last_error()


def test_feature_layout(L):
    lib = L.lib()
    rp, pp = ctypes.c_int64(), ctypes.c_int64()
    nb = lib.cfog_feature_layout(100, 77, 9, ctypes.byref(rp), ctypes.byref(pp))
    assert rp.value == 96 and pp.value == 96 * 100 and nb == 9 * 96 * 100 * 4
    assert lib.cfog_feature_layout(0, 5, 9, None, None) == 0


def test_argument_errors_before_launch(L):
    lib = L.lib()
    # null image
    assert lib.cfog_extract(None, None, None, None) == L.CFOG_E_INVAL
    im = L.cfog_image(0x1000, 10, 10, 10, L.CFOG_DTYPE_F32)
    # k out of range
    assert lib.cfog_detect_cps(ctypes.byref(im), 2, 2, 9, 0, 0, ctypes.c_void_p(0x1000),
                               None) == L.CFOG_E_INVAL
    assert b"k = 9" in lib.cfog_last_error()
    # margin leaves no interior
    assert lib.cfog_detect_cps(ctypes.byref(im), 2, 2, 1, 0, 5, ctypes.c_void_p(0x1000),
                               None) == L.CFOG_E_INVAL
    f = L.cfog_features(0x1000, 0x2000, 9, 10, 10, 32, 320)
    # n == 0 is a no-op
    assert lib.cfog_match(ctypes.byref(f), ctypes.byref(f), None, 0, None, None, 8, 1, None, 0,
                          None, None, None) == L.CFOG_OK
    # radius_max out of range
    p = ctypes.c_void_p(0x3000)
    assert lib.cfog_match(ctypes.byref(f), ctypes.byref(f), p, 1, p, p, 8, 33, None, 0, p, None,
                          None) == L.CFOG_E_INVAL
    # channel mismatch
    g = L.cfog_features(0x1000, 0x2000, 8, 10, 10, 32, 320)
    assert lib.cfog_match(ctypes.byref(f), ctypes.byref(g), p, 1, p, p, 8, 1, None, 0, p, None,
                          None) == L.CFOG_E_INVAL
    assert lib.cfog_fit_affine(None, None, 0, None, None, None) == L.CFOG_E_INVAL
    # orientation schemes: unknown -> INVAL, binned with R != 3 -> UNSUPPORTED
    fo = L.cfog_features(0x1000, 0x2000, 9, 10, 10, 32, 320)
    bad = L.cfog_params(9, 0.8, 1e-6, 3, 2)
    assert lib.cfog_extract(ctypes.byref(im), ctypes.byref(bad), ctypes.byref(fo), None) == L.CFOG_E_INVAL
    assert b"orientation" in lib.cfog_last_error()
    # pixel-wise HOG: 36 channels only, cells 4 and 8
    assert lib.cfog_extract_fhog(ctypes.byref(im), 8, 1e-6, ctypes.byref(fo), None) == L.CFOG_E_INVAL
    f36 = L.cfog_features(0x1000, 0x2000, 36, 10, 10, 32, 320)
    assert lib.cfog_extract_fhog(ctypes.byref(im), 5, 1e-6, ctypes.byref(f36), None) == L.CFOG_E_UNSUPPORTED
    assert lib.cfog_extract_fhog(None, 8, 1e-6, ctypes.byref(f36), None) == L.CFOG_E_INVAL
    r2 = L.cfog_params(9, 0.8, 1e-6, 2, L.CFOG_ORIENT_BINS)
    assert (lib.cfog_extract(ctypes.byref(im), ctypes.byref(r2), ctypes.byref(fo), None)
            == L.CFOG_E_UNSUPPORTED)


def test_batched_host_checks(L):
    lib = L.lib()
    assert lib.cfog_match_workspace_bytes(1000) >= 4000
    assert lib.cfog_match_workspace_bytes(-1) == 0
    p = ctypes.c_void_p(0x1000)
    # n == 0: nothing to do
    assert lib.cfog_match_batched(p, 1, None, None, 0, None, None, 16, 8, 9, None, 0, 0, None,
                                  None, 0, None) == L.CFOG_OK
    # workspace too small -> NOMEM before any launch
    assert lib.cfog_match_batched(p, 1, None, p, 10, p, p, 16, 8, 9, None, 0, 0, p, p, 8,
                                  None) == L.CFOG_E_NOMEM
    # misaligned workspace
    assert lib.cfog_match_batched(p, 1, None, p, 10, p, p, 16, 8, 9, None, 0, 0, p,
                                  ctypes.c_void_p(0x1004), 1 << 20, None) == L.CFOG_E_INVAL
    # unknown variant
    assert lib.cfog_match_batched(p, 1, None, p, 10, p, p, 16, 8, 9, None, 0, 5, p, p, 1 << 20,
                                  None) == L.CFOG_E_INVAL
    # BF16 direct precision: templates up to 128 only
    assert lib.cfog_match_batched(p, 1, None, p, 10, p, p, 200, 8, 9, None, 1, 0, p, p, 1 << 20,
                                  None) == L.CFOG_E_UNSUPPORTED
    assert b"128" in lib.cfog_last_error()
    out = (ctypes.c_int32 * 8)()
    assert lib.cfog_plan_info(96, 20, 9, 2, out) == L.CFOG_OK
    assert out[2] * out[3] <= 9216
    assert lib.cfog_plan_info(96, 20, 9, 1, out) == L.CFOG_OK
    assert out[2] * out[3] <= 16384
    assert lib.cfog_plan_info(96, 20, 9, 3, out) == L.CFOG_OK
    assert out[2] * out[3] <= 7680


def test_reject_host_checks(L):
    lib = L.lib()
    assert lib.cfog_reject_workspace_bytes(1000, 3) >= 16 * 1000 + 16
    assert lib.cfog_reject_workspace_bytes(-1, 1) == 0
    p = ctypes.c_void_p(0x1000)
    w = ctypes.c_void_p(0x10000)

    def call(js, degree=3, thr=1.0, min_keep=0, work=w, nbytes=1 << 20, models=p):
        arr = (ctypes.c_int32 * len(js))(*js)
        return lib.cfog_reject_outliers(p, p, arr, len(js) - 1, degree, thr, min_keep, p, None,
                                        models, work, nbytes, None)
    # n_jobs = 0: nothing to do
    assert lib.cfog_reject_outliers(None, None, None, 0, 3, 1.0, 0, None, None, None, None, 0,
                                    None) == L.CFOG_OK
    assert call([0, 10], degree=4) == L.CFOG_E_INVAL
    assert b"degree 4" in lib.cfog_last_error()
    assert call([0, 10], degree=0) == L.CFOG_E_INVAL
    assert call([0, 10], thr=-1.0) == L.CFOG_E_INVAL
    assert call([0, 10], thr=float("nan")) == L.CFOG_E_INVAL
    assert call([0, 10], min_keep=-2) == L.CFOG_E_INVAL
    assert call([0, 10, 5]) == L.CFOG_E_INVAL
    assert b"decreases" in lib.cfog_last_error()
    assert call([-1, 10]) == L.CFOG_E_INVAL
    assert call([0, 10], models=None) == L.CFOG_E_INVAL
    assert call([0, 1000], nbytes=64) == L.CFOG_E_NOMEM
    assert call([0, 10], work=ctypes.c_void_p(0x10008)) == L.CFOG_E_INVAL


def test_tin_host_checks(L):
    lib = L.lib()
    assert lib.cfog_tin_workspace_bytes(10, 100, 100) > 0
    assert lib.cfog_tin_workspace_bytes(-1, 100, 100) == 0
    im = L.cfog_image(0x1000, 10, 10, 10, L.CFOG_DTYPE_F32)
    p = ctypes.c_void_p(0x2000)
    w = ctypes.c_void_p(0x10000)
    # short workspace -> NOMEM, misaligned -> INVAL, null output -> INVAL
    assert lib.cfog_tin_rectify(ctypes.byref(im), p, p, 4, p, 2, 10, 10, 0.0, p, 10, w, 16,
                                None) == L.CFOG_E_NOMEM
    assert lib.cfog_tin_rectify(ctypes.byref(im), p, p, 4, p, 2, 10, 10, 0.0, p, 10,
                                ctypes.c_void_p(0x10004), 1 << 20, None) == L.CFOG_E_INVAL
    assert lib.cfog_tin_rectify(ctypes.byref(im), p, p, 4, p, 2, 10, 10, 0.0, None, 10, w, 1 << 20,
                                None) == L.CFOG_E_INVAL
    n = ctypes.c_int32()
    assert lib.cfog_tin_delaunay(None, 0, None, None, 0, ctypes.byref(n)) == L.CFOG_OK and n.value == 0


def test_missing_library_fails_loudly(monkeypatch):
    """The product path has no fallback: without libcfog.so every call raises."""
    from paper_1808_06194_gb300 import _lib
    monkeypatch.setattr(_lib, "LIB_PATH", os.path.join(ROOT, "no_such_dir", "libcfog.so"))
    monkeypatch.setattr(_lib, "_lib", None)
    with pytest.raises(RuntimeError, match="libcfog.so not found"):
        _lib.lib()
    with pytest.raises(RuntimeError, match="libcfog.so not found"):
        _lib.check(_lib.CFOG_E_INVAL, "probe")


def test_product_shares_no_code_with_the_oracle():
    """Neither the package nor its CUDA sources import, include or load
    anything under oracle/."""
    pkg = os.path.join(ROOT, "paper_1808_06194_gb300")
    seen = 0
    for dirpath, _, files in os.walk(pkg):
        if "_build" in dirpath or "__pycache__" in dirpath:
            continue
        for f in files:
            if not f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                continue
            text = open(os.path.join(dirpath, f)).read()
            seen += 1
            assert not re.search(r"^\s*(import|from)\s+oracle\b", text, re.M), f
            assert "cfog_oracle" not in text, f   # the oracle library and its C file
    assert seen >= 10


def test_failure_hook_validates_on_host(L):
    lib = L.lib()
    assert lib.cfog_test_inject_wait_timeout(-2, 5000) == L.CFOG_E_INVAL
    assert lib.cfog_test_inject_wait_timeout(0, 10) == L.CFOG_E_INVAL
    assert lib.cfog_test_inject_wait_timeout(0, 10**12) == L.CFOG_E_INVAL
    assert lib.cfog_test_inject_wait_timeout(-1, 1000) == L.CFOG_OK
