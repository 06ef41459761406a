"""Large-scene path: band-wise CFOG equals whole-image CFOG bitwise, and the
streamed registration, which computes CFOG and matches band by band in
band-sized feature buffers, equals the one-shot library calls on whole-image
features byte for byte."""
import numpy as np
import pytest

import oracle
import synth
from tests._util import cuda_or_skip, to_dev

pytestmark = pytest.mark.gpu


def test_extract_rows_bands_equal_whole_image():
    torch, P = cuda_or_skip()
    rng = np.random.default_rng(3)
    img = rng.integers(0, 4096, size=(700, 300)).astype(np.uint16)
    d = to_dev(torch, img)
    whole = P.cfog_extract(d)
    banded = P.alloc_features(700, 300)
    for r0, r1 in [(0, 128), (128, 300), (300, 301), (301, 700)]:
        P.cfog_extract_rows(d, r0, r1, banded)
    torch.cuda.synchronize()
    assert torch.equal(whole.volume(), banded.volume())
    assert torch.equal(whole.sq(), banded.sq())
    with pytest.raises(P.CfogError):
        P.cfog_extract_rows(d, 10, 701, banded)


def test_scene_streamed_equals_direct_calls():
    torch, P = cuda_or_skip()
    from paper_1808_06194_gb300 import scene
    pair = synth.large_scene_pair(4, size=1536)
    ref = torch.from_numpy(pair.A.astype(np.int32)).to(torch.uint16).pin_memory()
    sen = torch.from_numpy(pair.B.astype(np.int32)).to(torch.uint16).pin_memory()
    prior = scene.georeference_prior(pair.field, 3, 11)
    out = scene.register_scene(ref, sen, prior, grid=6, tmpl=96, radius=16, band=512)
    # band-sized feature buffers: less than the two whole-scene volumes
    whole = 2 * P.alloc_features(1536, 1536).nbytes
    assert out["times"]["n_bands"] == 3 and out["feature_bytes"] < whole
    fr, fs = P.cfog_extract(ref.cuda()), P.cfog_extract(sen.cuda())
    cps = torch.from_numpy(out["cps"]).cuda()
    qx, qy = prior(out["cps"][:, 0].astype(np.float64), out["cps"][:, 1].astype(np.float64))
    pr = torch.from_numpy(np.stack([qx, qy], 1).astype(np.int32)).cuda()
    n = cps.shape[0]
    t = torch.full((n,), 96, dtype=torch.int32, device="cuda")
    r = torch.full((n,), 16, dtype=torch.int32, device="cuda")
    direct = P.cfog_match_batched(P.job_table([(fr, fs)]), 1, cps, t, r, 96, 16, prior=pr)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(out["results"], direct.cpu().numpy())
    # the FP64 affine fit equals the oracle's least squares on the same matches
    res = out["results"]
    ok = res[:, 5] == 0
    x, y = out["cps"][:, 0].astype(np.float64), out["cps"][:, 1].astype(np.float64)
    f = res.view(np.float32)
    exp = oracle.affine_ls(x, y, x + f[:, 2].astype(np.float64), y + f[:, 3].astype(np.float64),
                           ok.astype(np.int32))
    np.testing.assert_allclose(out["affine"], exp, rtol=1e-8, atol=1e-6)
