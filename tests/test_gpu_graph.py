"""The batched step (CFOG of both images, Harris CPs, one persistent matching
launch) captured in a CUDA graph gives the same bytes as the eager calls."""
import numpy as np
import pytest

import synth
from tests._util import cuda_or_skip

pytestmark = pytest.mark.gpu


def test_graph_replay_equals_eager():
    torch, P = cuda_or_skip()
    dev = torch.device("cuda:0")
    pair = synth.batched_pair(1, 512)
    A = torch.from_numpy(pair.A).to(dev)
    B = torch.from_numpy(pair.B).to(dev)
    fa, fb = P.alloc_features(512, 512, 9, dev), P.alloc_features(512, 512, 9, dev)
    jobs = P.job_table([(fa, fb)], dev)
    n = 64
    tm_np, rd_np = synth.random_cp_params(5, n, (48, 64), 8, 16)
    tm, rd = torch.from_numpy(tm_np).to(dev), torch.from_numpy(rd_np).to(dev)
    cps = torch.empty((n, 2), dtype=torch.int32, device=dev)
    res = torch.empty((n, 6), dtype=torch.int32, device=dev)
    ws = P.match_workspace(n, dev)

    def step():
        P.cfog_extract(A, out=fa)
        P.cfog_extract(B, out=fb)
        P.cfog_detect_cps(A, 8, 8, 1, 0, 60, out=cps)
        P.cfog_match_batched(jobs, 1, cps, tm, rd, 64, 16, variant=P._lib.CFOG_MATCH_VARIANT_PAIR,
                             out=res, workspace=ws)

    step()
    torch.cuda.synchronize()
    eager = res.clone()
    eager_f = fa.volume().clone()
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream(dev)
    s.wait_stream(torch.cuda.current_stream(dev))
    with torch.cuda.stream(s):
        with torch.cuda.graph(g):
            step()
    res.zero_()
    fa.volume().zero_()
    for _ in range(2):
        g.replay()
    torch.cuda.synchronize()
    assert torch.equal(res, eager)
    assert torch.equal(fa.volume(), eager_f)
    assert int((res[:, 5] == 0).sum()) > n // 2
