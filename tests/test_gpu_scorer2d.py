"""The paper's own 2-D learned scorer on the GPU (forward pass, binary32 on
the CUDA cores) against the oracle's binary64 network.

Tolerance: each output sums at most 144 products per layer over three
layers and the head in binary32 (fused multiply-adds); the relative error of
such a sum is below 2^-24 times the number of terms times the sum of the
magnitudes, about 1e-5 of the logits' scale here.  The test allows
2e-4 (1 + |logit|)."""
import numpy as np
import pytest

from paper_2210_14771_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def ca():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2210_14771_gb300.build import build
    build()
    from paper_2210_14771_gb300 import api
    h = api.ContentArea(0)
    yield h
    h.close()


@pytest.mark.parametrize("H,W", [(1080, 1920), (300, 200), (50, 37)])
def test_forward_matches_oracle(ca, orc, H, W):
    frame, _ = synth.frame(5, 0, H, W, "clipped" if W > 100 else "centred")
    ys = [1, 2, H // 3, H // 2, H - 4, H - 2]
    pairs = [orc.sc2_strip(frame, y) for y in ys]
    s7 = np.stack([p[0] for p in pairs])
    rows = np.stack([p[1] for p in pairs]).astype(np.int32)
    rng = np.random.default_rng(W)
    prm = (rng.standard_normal(orc.SC2_NPARAM) * 0.3).astype(np.float32)
    got = ca.scorer2d_forward(torch.from_numpy(s7).cuda(), torch.from_numpy(rows).cuda(), H,
                              torch.from_numpy(prm).cuda()).cpu().numpy()
    for i in range(len(ys)):
        want = orc.sc2_forward(s7[i], rows[i], H, prm)
        err = np.abs(got[i] - want) / (1.0 + np.abs(want))
        assert err.max() <= 2e-4, (i, float(err.max()))


def test_forward_arguments(ca):
    from paper_2210_14771_gb300 import _native as N
    lib = N.lib()
    assert lib.ca_scorer2d_forward(ca._h, None, None, 0, 64, 48, None, None, None) == 0
    assert lib.ca_scorer2d_forward(ca._h, None, None, 1, 64, 48, None, None, None) == 1
    assert lib.ca_scorer2d_forward(ca._h, None, None, 1, 0, 48, None, None, None) == 1
