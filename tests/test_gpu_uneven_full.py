"""The 64-image uneven workload at its full size (sides 96..320, C = 512, d = 32,
B = 64, radii 5..12, BF16 projection) in the launch configuration the benchmark
times: one qfca_score_batch per batch with the window-stage autotuner on,
replayed from a captured CUDA graph.

Every map is checked by properties that hold at any size (finite, within the
EMD's range [0, B - 1], the graph replay equal to the direct call bit for bit,
a clean device status).  The smallest image is checked against the FP64
oracle's whole pipeline (fit, projection, quantisation, window EMD): pixel
AUROC within 0.005 (the BF16 bound) and the score within 2e-3 relative on
average and 5e-3 at the worst pixel.  A CPU emulation of the BF16 operand
rounding on this image gives 1.2% bin flips (B = 64), 1.4e-4 and 4.2e-4."""
import numpy as np
import pytest
import torch

import oracle
from paper_2510_15602_gb300.metrics import auroc
from tests import uneven_inputs

pytestmark = pytest.mark.gpu

N_IMG, D, B = 64, 32, 64


@pytest.fixture(scope="module")
def q():
    from paper_2510_15602_gb300 import qfca
    assert torch.cuda.is_available()
    return qfca


def test_uneven_workload_full_size_graph_against_oracle(q):
    host = uneven_inputs.draw_all(N_IMG)
    Xs = [torch.from_numpy(x).cuda() for x, _, _ in host]
    rs = [r for _, _, r in host]
    ctx = q.Context()
    ctx.set_autotune(True)
    st = torch.cuda.Stream()
    scores = [torch.empty(x.shape[1], x.shape[2], dtype=torch.float32, device="cuda") for x in Xs]

    def run():
        q.score_batch(Xs, rs, D, B, "bf16", ctx=ctx, stream=st, scores=scores)

    with torch.cuda.stream(st):
        run()  # the autotuner measures the window tilings (outside capture)
    torch.cuda.synchronize()
    first = [s.clone() for s in scores]
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=st):
        run()
    for s in scores:
        s.fill_(-1.0)
    torch.cuda.synchronize()
    with torch.cuda.stream(st):
        g.replay()
    torch.cuda.synchronize()
    assert ctx.device_status() == 0
    for i, (a, b) in enumerate(zip(first, scores)):
        assert torch.equal(a, b), i
    for i, s in enumerate(scores):
        sn = s.cpu().numpy()
        assert np.isfinite(sn).all() and sn.min() >= 0.0 and sn.max() <= B - 1, i

    # the smallest image of the batch through the FP64 oracle
    i = min(range(N_IMG), key=lambda k: host[k][0].shape[1] * host[k][0].shape[2])
    X, mask, r = host[i]
    ref = oracle.pipeline(X, D, B, r)
    s, so = scores[i].cpu().numpy().astype(np.float64), ref["score"]
    assert np.abs(s - so).mean() <= 2e-3 * so.mean()
    assert np.abs(s - so).max() <= 5e-3 * so.max()
    assert abs(auroc(s, mask) - auroc(so, mask)) <= 0.005
