"""Failure detection of the BF16 tensor-core path without a GPU fault: a
host-set hook makes one CP wait on a barrier that nothing arrives at, with a
short cycle limit.  That CP must report CFOG_CP_TIMEOUT and every other CP of
the same launch (including later CPs of the same persistent CTA) must equal
the run without the hook, byte for byte, and the oracle (Eq. 3)."""
import numpy as np
import pytest

import oracle
import synth
from paper_1808_06194_gb300 import _lib as L
from tests._util import check_match_parity, cuda_or_skip, to_dev

pytestmark = pytest.mark.gpu


def _unpack(res):
    f = res.view(np.float32)
    return {"dx": res[:, 0], "dy": res[:, 1], "sub_dx": f[:, 2], "sub_dy": f[:, 3],
            "ssd": f[:, 4], "status": res[:, 5]}


@pytest.mark.parametrize("batched", [True, False])
def test_bf16_wait_timeout_is_reported_per_cp(batched):
    torch, P = cuda_or_skip()
    oracle.build()
    pair = synth.batched_pair(61, size=320)
    fa, fb = P.cfog_extract(to_dev(torch, pair.A)), P.cfog_extract(to_dev(torch, pair.B))
    rng = np.random.default_rng(62)
    n = 700 if batched else 12          # more CPs than CTA slots: CTAs take several
    N = rng.choice([16, 32, 48], n).astype(np.int32)
    r = rng.choice([4, 8, 12], n).astype(np.int32)
    px = rng.integers(60, 260, n).astype(np.int32)
    py = rng.integers(60, 260, n).astype(np.int32)
    cps = torch.tensor(np.stack([px, py], 1), device="cuda")
    tm, rd = torch.tensor(N, device="cuda"), torch.tensor(r, device="cuda")
    jobs = P.job_table([(fa, fb)])

    def run():
        if batched:
            out = P.cfog_match_batched(jobs, 1, cps, tm, rd, 48, 12, precision=1)
        else:
            out = P.cfog_match(fa, fb, cps, tm, rd, 48, 12, precision=1)
        torch.cuda.synchronize()
        return out.cpu().numpy()

    base = run()
    stall = [3, n // 2] if batched else [3]
    lib = P.lib()
    try:
        for s in stall:
            assert lib.cfog_test_inject_wait_timeout(s, 2_000_000) == 0   # about 1 ms
            got = run()
            assert got[s, 5] == L.CFOG_CP_TIMEOUT
            keep = np.arange(n) != s
            np.testing.assert_array_equal(got[keep], base[keep])
    finally:
        assert lib.cfog_test_inject_wait_timeout(-1, 1000) == 0
    np.testing.assert_array_equal(run(), base)
    sel = np.arange(0, n, max(1, n // 24))
    da, _ = oracle.cfog(pair.A)
    db, _ = oracle.cfog(pair.B)
    o = oracle.match_many(da, db, px[sel], py[sel], N[sel], r[sel])
    check_match_parity({k: v[sel] for k, v in _unpack(base).items()}, o)
