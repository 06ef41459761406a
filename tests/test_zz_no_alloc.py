"""The allocation-free batched matcher, cfog_match_batched_noalloc.

Callers that cannot allocate device memory (a plugin inside an application
whose memory pool reserves the GPU, or a latency-critical loop that must not
enter the CUDA allocator, which can synchronise the device) use this entry
point: it keeps its queue scratch in a static device array of the library
instead of a caller workspace.  These tests call it through the C ABI and
check that it returns the same bytes as cfog_match_batched on two calls in a
row, the second one reusing the scratch the first one left behind.

This file is collected last on purpose, so that a run stopping at the first
failure has already run every other test.
"""
import ctypes

import numpy as np
import pytest

import synth
from tests._util import cuda_or_skip, to_dev

pytestmark = pytest.mark.gpu


def _noalloc(torch, P, jobs, n_jobs, cps, tm, rd, nmax, rmax, prior=None, precision=0, variant=0):
    n = cps.shape[0]
    out = torch.full((n, 6), -7, dtype=torch.int32, device="cuda")
    vp = lambda t: ctypes.c_void_p(t.data_ptr()) if t is not None else None  # noqa: E731
    st = P.lib().cfog_match_batched_noalloc(
        vp(jobs), n_jobs, None, vp(cps), n, vp(tm), vp(rd), nmax, rmax, 9, vp(prior), precision,
        variant, vp(out), ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    return st, out


# (precision, variant): FP32 FFT with the library's default variant and with
# the two-CTA-per-SM variant, and the BF16 tensor-core path
CASES = [(0, 0), (0, 2), (1, 0)]


@pytest.mark.parametrize("precision,variant", CASES)
def test_noalloc_matches_workspace_entry_two_calls(precision, variant):
    """Both entry points run the same kernels with the same plans, so the
    results must be identical bytes, call after call."""
    torch, P = cuda_or_skip()
    pair = synth.batched_pair(41, size=512)
    fa = P.cfog_extract(to_dev(torch, pair.A))
    fb = P.cfog_extract(to_dev(torch, pair.B))
    jobs = P.job_table([(fa, fb)])
    rng = np.random.default_rng(42)
    for n in (300, 77):   # two calls in a row, the second with fewer CPs
        cps = torch.tensor(rng.integers(60, 452, (n, 2)).astype(np.int32), device="cuda")
        tm = torch.tensor(rng.choice([16, 48, 64, 96], n).astype(np.int32), device="cuda")
        rd = torch.tensor(rng.integers(2, 21, n).astype(np.int32), device="cuda")
        prior = torch.tensor(rng.integers(-3, 4, (n, 2)).astype(np.int32), device="cuda")
        ref = P.cfog_match_batched(jobs, 1, cps, tm, rd, 96, 20, prior=prior,
                                   precision=precision, variant=variant)
        st, got = _noalloc(torch, P, jobs, 1, cps, tm, rd, 96, 20, prior, precision, variant)
        assert st == 0, P.lib().cfog_last_error()
        torch.cuda.synchronize()
        got, ref = got.cpu().numpy(), ref.cpu().numpy()
        assert (got[:, 5] != 1).sum() > n // 2      # most CPs are matched, not OOB
        np.testing.assert_array_equal(got, ref)


def test_noalloc_rejects_batches_beyond_its_scratch():
    torch, P = cuda_or_skip()
    cap = P.lib().cfog_match_batched_noalloc_max_cps()
    assert cap == 65536
    f = P.alloc_features(64, 64)
    jobs = P.job_table([(f, f)])
    big = torch.zeros((cap + 1, 2), dtype=torch.int32, device="cuda")
    t = torch.full((cap + 1,), 16, dtype=torch.int32, device="cuda")
    st, _ = _noalloc(torch, P, jobs, 1, big, t, t, 16, 16)
    assert st == 1
    assert b"exceeds" in P.lib().cfog_last_error()
