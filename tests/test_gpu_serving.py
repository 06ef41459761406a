"""Serving loop on the GPU: continuous batching across jobs with HBM-budget
admission gives every job exactly the result it gets alone."""
import numpy as np
import pytest

import synth
from tests._util import cuda_or_skip

pytestmark = pytest.mark.gpu


def _jobs(serve):
    rng = np.random.default_rng(5)
    jobs = []
    for i, (size, dt, tm, r) in enumerate([(256, "f32", 48, 8), (384, "u16", 64, 12),
                                           (320, "f32", 64, 16), (448, "u16", 48, 10),
                                           (288, "f32", 48, 16), (512, "f32", 64, 8)]):
        p = synth.batched_pair(100 + i, size=size)
        A, B = p.A, p.B
        if dt == "u16":
            A = np.clip(np.rint(A * 16), 0, 4095).astype(np.uint16)
            B = np.clip(np.rint(B * 16), 0, 4095).astype(np.uint16)
        jobs.append(serve.Job(A, B, tmpl=tm, radius=r))
    return jobs


def _run(serve, jobs, budget):
    srv = serve.Server(hbm_budget=budget, ring=1 << 14, max_batch=200, max_jobs=8,
                       tmpl_max=64, radius_max=16)
    for j in jobs:
        srv.submit(j)
    srv.drain()
    return srv


def test_mix_equals_alone_and_budget_holds():
    torch, P = cuda_or_skip()
    from paper_1808_06194_gb300 import serve
    jobs = _jobs(serve)
    sizes = [serve.job_bytes(j) for j in jobs]
    budget = 2 * max(sizes) + min(sizes)     # forces jobs to wait for memory
    srv = _run(serve, jobs, budget)
    assert len(srv.finished) == len(jobs)
    assert srv.adm.peak <= budget and srv.adm.used == 0
    mixed = {j.key: j.results.copy() for j in srv.finished}   # keys in submission order
    for i, j in enumerate(_jobs(serve)):
        alone = _run(serve, [j], budget)
        np.testing.assert_array_equal(alone.finished[0].results, mixed[i])


def test_served_job_equals_direct_batched_call():
    torch, P = cuda_or_skip()
    from paper_1808_06194_gb300 import serve
    job = _jobs(serve)[2]
    srv = _run(serve, [job], 1 << 34)
    got = srv.finished[0].results
    A = torch.from_numpy(job.ref).cuda()
    B = torch.from_numpy(job.sen).cuda()
    fa, fb = P.cfog_extract(A), P.cfog_extract(B)
    gx, gy = job.grid()
    cps = P.cfog_detect_cps(A, gx, gy, 1, 0, job.margin)
    n = cps.shape[0]
    tm = torch.full((n,), job.tmpl, dtype=torch.int32, device="cuda")
    rd = torch.full((n,), job.radius, dtype=torch.int32, device="cuda")
    ref = P.cfog_match_batched(P.job_table([(fa, fb)]), 1, cps, tm, rd, 64, 16)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(got, ref.cpu().numpy())
    np.testing.assert_array_equal(srv.finished[0].cps, cps.cpu().numpy())
