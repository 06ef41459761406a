"""The autotuner on the GPU: it records the fastest measured variant as the
AUTO variant, a second process-level call is served from the JSON cache, and
every plan it may choose keeps the FFT path's parity with the oracle and its
batch invariance (Sec. III-G, Eq. 8-9 applied with other FFT sizes and
template blockings)."""
import numpy as np
import pytest

import oracle
import synth
from tests._util import check_match_parity, cuda_or_skip, to_dev

pytestmark = pytest.mark.gpu

CLASSES = [(48, 8), (64, 12), (96, 20), (128, 16)]


@pytest.fixture()
def clean_tuning():
    torch, P = cuda_or_skip()
    assert P.lib().cfog_match_clear_tuning() == 0
    yield torch, P
    assert P.lib().cfog_match_clear_tuning() == 0


def test_tuner_records_fastest_variant_and_caches(clean_tuning, tmp_path):
    torch, P = clean_tuning
    from paper_1808_06194_gb300 import autotune
    path = str(tmp_path / "tune.json")
    e1 = autotune.ensure(CLASSES, 9, 128, 20, 0, path=path)
    assert e1["source"] == "tuned"
    vms = {int(k): v for k, v in e1["variants_ms"].items()}
    assert e1["variant"] == min(vms, key=vms.get)
    assert P.lib().cfog_match_auto_variant(9, 128, 20, 0) == e1["variant"]
    assert P.resolve_variant(128, 20, 9, 0, 0) == e1["variant"]
    # every recorded plan is one of its class's timed candidates and was faster
    for cls, code in e1["plans"].items():
        n, r = (int(x) for x in cls.split("x"))
        codes = [c["code"] for c in autotune.candidates(n, r, 9, e1["variant"], 6)]
        assert code in codes[1:]
        ms = e1["class_ms"][cls]["ms"]
        assert ms[codes.index(code)] < ms[0]
    # every class has a table entry: tuned, or the cost model's own plan
    for n, r in CLASSES:
        cls = f"{n}x{r}"
        assert (cls in e1["plans"]) != (cls in e1["model_plans"])
        if cls in e1["model_plans"]:
            assert e1["model_plans"][cls] == autotune.candidates(n, r, 9, e1["variant"], 1)[0]["code"]
    assert P.lib().cfog_match_clear_tuning() == 0
    assert P.lib().cfog_match_auto_variant(9, 128, 20, 0) == 1
    e2 = autotune.ensure(CLASSES, 9, 128, 20, 0, path=path)
    assert e2["source"] == "cache" and e2["variant"] == e1["variant"]
    assert e2["plans"] == e1["plans"]
    assert P.lib().cfog_match_auto_variant(9, 128, 20, 0) == e1["variant"]


@pytest.mark.parametrize("variant", [1, 2])
def test_every_candidate_plan_keeps_parity_and_invariance(clean_tuning, variant):
    torch, P = clean_tuning
    from paper_1808_06194_gb300 import autotune
    pair = synth.batched_pair(51, size=384)
    fa, fb = P.cfog_extract(to_dev(torch, pair.A)), P.cfog_extract(to_dev(torch, pair.B))
    da, _ = oracle.cfog(pair.A)
    db, _ = oracle.cfog(pair.B)
    jobs = P.job_table([(fa, fb)])
    rng = np.random.default_rng(52)
    n = 24
    cls = np.array(CLASSES, np.int32)[rng.integers(0, len(CLASSES), n)]
    N, r = cls[:, 0].copy(), cls[:, 1].copy()
    px = rng.integers(90, 294, n).astype(np.int32)
    py = rng.integers(90, 294, n).astype(np.int32)
    o = oracle.match_many(da, db, px, py, N, r)
    cps = torch.tensor(np.stack([px, py], 1), device="cuda")
    tm, rd = torch.tensor(N, device="cuda"), torch.tensor(r, device="cuda")

    def run(sel=None):
        c, t, d = (cps, tm, rd) if sel is None else (cps[sel:sel + 1], tm[sel:sel + 1],
                                                     rd[sel:sel + 1])
        out = P.cfog_match_batched(jobs, 1, c, t, d, 128, 20, variant=variant)
        torch.cuda.synchronize()
        return out.cpu().numpy()

    def unpack(res):
        f = res.view(np.float32)
        return {"dx": res[:, 0], "dy": res[:, 1], "sub_dx": f[:, 2], "sub_dy": f[:, 3],
                "ssd": f[:, 4], "status": res[:, 5]}

    base = run()
    check_match_parity(unpack(base), o)
    cands = {c: autotune.candidates(c[0], c[1], 9, variant, 6) for c in CLASSES}
    for k in range(1, 6):
        changed = False
        for (cn, cr), cs in cands.items():
            code = cs[min(k, len(cs) - 1)]["code"]
            assert P.lib().cfog_match_set_plan(variant, 9, cn, cr, code) == 0
            changed = changed or len(cs) > 1
        got = run()
        check_match_parity(unpack(got), o)
        for i in range(0, n, 5):        # batch invariance under the tuned table
            np.testing.assert_array_equal(run(i)[0], got[i])
        if not changed:
            np.testing.assert_array_equal(got, base)
    # forgetting the plans restores the cost model's bytes
    for (cn, cr) in CLASSES:
        assert P.lib().cfog_match_set_plan(variant, 9, cn, cr, -1) == 0
    np.testing.assert_array_equal(run(), base)
