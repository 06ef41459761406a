"""Host checks of the autotuner's library calls and JSON cache (no GPU):
plan candidates are feasible, distinct and led by the cost model's plan;
invalid plan codes are rejected before any device work; the AUTO table and
the cache round-trip."""
import ctypes
import json

import pytest

from paper_1808_06194_gb300 import _lib as L
from paper_1808_06194_gb300 import autotune

MAXE = {1: 16384, 2: 9216, 3: 7680, 4: 9216}


@pytest.fixture(scope="module")
def lib():
    from paper_1808_06194_gb300 import build
    build.build()
    return L.lib()


def _plan_info(lib, n, r, m, v):
    out = (ctypes.c_int32 * 8)()
    return list(out) if lib.cfog_plan_info(n, r, m, v, out) == 0 else None


@pytest.mark.parametrize("variant", [1, 2, 3, 4])
@pytest.mark.parametrize("n,r", [(48, 8), (64, 14), (96, 20), (128, 20), (128, 8), (17, 3), (256, 32)])
def test_candidates_feasible_distinct_and_model_first(lib, variant, n, r):
    c = autotune.candidates(n, r, 9, variant, k=6, lib=lib)
    model = _plan_info(lib, n, r, 9, variant)
    if model is None:            # no plan fits this variant's plane bound
        assert c == []
        return
    assert 1 <= len(c) <= 6
    assert [c[0][k] for k in ("nb_y", "nb_x", "P_y", "P_x", "b_y", "b_x", "stages", "smem")] == \
        model
    seen = set()
    for p in c:
        assert p["P_y"] >= p["b_y"] + 2 * r and p["P_x"] >= p["b_x"] + 2 * r
        assert p["P_y"] * p["P_x"] <= MAXE[variant]
        assert p["nb_y"] * p["b_y"] >= n and p["nb_x"] * p["b_x"] >= n
        key = (p["nb_y"], p["nb_x"], p["P_y"], p["P_x"])
        assert key not in seen
        seen.add(key)


def test_set_plan_rejects_infeasible_codes(lib):
    assert lib.cfog_match_set_plan(2, 9, 64, 14, 999) == L.CFOG_E_INVAL
    assert lib.cfog_match_set_plan(5, 9, 64, 14, 0) == L.CFOG_E_INVAL
    assert lib.cfog_match_set_plan(2, 9, 300, 14, 0) == L.CFOG_E_INVAL
    # split l = 15 (4 x 4 blocks) of a 4-px template: blocks of 1 px, feasible;
    # a 1-px template cannot be cut into 4 blocks
    assert lib.cfog_match_set_plan(2, 9, 1, 2, 15 << 4) == L.CFOG_E_INVAL
    assert b"no feasible plan" in lib.cfog_last_error()


def test_auto_variant_table(lib):
    assert lib.cfog_match_auto_variant(9, 128, 20, 0) == L.CFOG_MATCH_VARIANT_WIDE
    assert lib.cfog_match_set_auto_variant(9, 128, 20, 0, 2) == 0
    try:
        assert lib.cfog_match_auto_variant(9, 128, 20, 0) == 2
        assert lib.cfog_match_auto_variant(9, 96, 20, 0) == L.CFOG_MATCH_VARIANT_WIDE
        assert lib.cfog_match_auto_variant(36, 128, 20, 0) == L.CFOG_MATCH_VARIANT_WIDE
    finally:
        assert lib.cfog_match_set_auto_variant(9, 128, 20, 0, 0) == 0
    assert lib.cfog_match_auto_variant(9, 128, 20, 0) == L.CFOG_MATCH_VARIANT_WIDE
    assert lib.cfog_match_set_auto_variant(9, 128, 20, 7, 2) == L.CFOG_E_INVAL


def test_cache_roundtrip_and_keys(tmp_path):
    path = str(tmp_path / "sub" / "tune.json")
    assert autotune.load_cache(path) == {"format": autotune.FORMAT, "entries": {}}
    k1 = autotune.class_key(9, 128, 20, 0, [(64, 8), (48, 9), (64, 8)])
    k2 = autotune.class_key(9, 128, 20, 0, [(48, 9), (64, 8)])
    assert k1 == k2
    dk = autotune.device_key("NVIDIA GB300", (10, 3), "abc123")
    data = {"format": autotune.FORMAT, "entries": {dk: {k1: {"variant": 2, "plans": {"64x8": 5}}}}}
    autotune.save_cache(data, path)
    assert autotune.load_cache(path) == data
    with open(path, "w") as f:
        json.dump({"format": -1, "entries": {}}, f)
    assert autotune.load_cache(path)["entries"] == {}
    with open(path, "w") as f:
        f.write("{not json")
    assert autotune.load_cache(path)["entries"] == {}


def test_apply_records_variant_and_plans():
    calls = []

    class Fake:
        def cfog_match_set_auto_variant(self, *a):
            calls.append(("auto",) + a)
            return 0

        def cfog_match_set_plan(self, *a):
            calls.append(("plan",) + a)
            return 0

    autotune.apply({"variant": 2, "plans": {"64x8": 17, "128x20": 3}, "model_plans": {"48x9": 5}},
                   9, 128, 20, 0, lib=Fake())
    assert calls[0] == ("auto", 9, 128, 20, 0, 2)
    assert sorted(calls[1:]) == [("plan", 2, 9, 48, 9, 5), ("plan", 2, 9, 64, 8, 17),
                                 ("plan", 2, 9, 128, 20, 3)]


def test_cache_path_from_environment(monkeypatch, tmp_path):
    monkeypatch.setenv("CFOG_TUNE_CACHE", str(tmp_path / "x.json"))
    assert autotune.cache_path() == str(tmp_path / "x.json")
    monkeypatch.delenv("CFOG_TUNE_CACHE")
    monkeypatch.setenv("XDG_CACHE_HOME", str(tmp_path))
    assert autotune.cache_path() == str(tmp_path / "cfog" / "autotune.json")
