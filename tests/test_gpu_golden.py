"""The hand-worked cases of `tests/golden/hand_examples.json` through the C ABI on
the GPU: the PCA fit and projection (Sec. 3.3), quantisation and reference
histogram (Sec. 3.1), the window-EMD score (Sec. 3.1, Sec. 3), the paper's
association scoring (Sec. 3.1) and the median reference (Sec. 3.2).  Integer
results are compared exactly; maps within one FP32 rounding of the exact
fractions (the association map within its fixed-point bound, 2^-21 here)."""
import json
import pathlib
from fractions import Fraction

import numpy as np
import pytest
import torch

from tests.gpu_helpers import to_dev

pytestmark = pytest.mark.gpu

GOLD = json.loads((pathlib.Path(__file__).parent / "golden" / "hand_examples.json").read_text())


def frac(v):
    return np.array([float(Fraction(x)) for x in v], np.float64)


@pytest.fixture(scope="module")
def q():
    from paper_2510_15602_gb300 import qfca
    assert torch.cuda.is_available()
    return qfca


def dev_bins(q, qb):
    d, H, W = qb.shape
    bins = torch.zeros(d, H, q.bins_pitch(W), dtype=torch.uint8, device="cuda")
    bins[:, :, :W] = to_dev(qb)
    return bins


def test_pipeline_hand_on_gpu(q):
    g = GOLD["pipeline_1x4"]
    X = to_dev(np.array(g["X"], np.float32))
    mean, V, ev = q.fit_pca(X, g["d"])
    torch.cuda.synchronize()
    assert abs(ev.cpu().item() - 2.0) <= 1e-12
    np.testing.assert_allclose(mean.cpu().numpy(), [0.0, 0.0], atol=1e-15)
    np.testing.assert_allclose(V.cpu().numpy()[:, 0], [1.0, 0.0], atol=1e-12)
    basis = (torch.zeros(2, dtype=torch.float64, device="cuda"),
             torch.tensor([[1.0], [0.0]], dtype=torch.float64, device="cuda"))
    out = q.quantize(X, basis, g["B"], "f32", want_Y=True)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(out["Y"].cpu().numpy()[0, 0], np.array(g["Y"], np.float32))
    np.testing.assert_array_equal(out["bins"][0, 0, :4].cpu().numpy(), g["q"])
    np.testing.assert_array_equal(out["hist"].cpu().numpy()[0], g["R"])
    s = q.score(out["bins"], 4, g["B"], g["r"], out["hist"], 4)
    torch.cuda.synchronize()
    np.testing.assert_allclose(s.cpu().numpy()[0], frac(g["score"]), rtol=2.0 ** -23, atol=0)


def test_score_hand_on_gpu(q):
    g = GOLD["score_1x3"]
    qb = np.array(g["q"], np.uint8)
    R = torch.tensor([[1, 2]], dtype=torch.int32, device="cuda")
    s = q.score(dev_bins(q, qb), 3, g["B"], g["r"], R, 3)
    torch.cuda.synchronize()
    np.testing.assert_allclose(s.cpu().numpy()[0], frac(g["score"]), rtol=2.0 ** -23, atol=0)


def test_assoc_hand_on_gpu(q):
    g = GOLD["assoc_1x3"]
    qb = np.array(g["q"], np.uint8)
    R = torch.tensor([[1, 2]], dtype=torch.int32, device="cuda")
    s = q.score_assoc(dev_bins(q, qb), 3, g["B"], g["r"], R, 3, sigma_s=0.0)
    torch.cuda.synchronize()
    np.testing.assert_allclose(s.cpu().numpy()[0], frac(g["raw"]), rtol=0, atol=2.0 ** -21)


def test_median_reference_hand_on_gpu(q):
    g = GOLD["median_3x5"]
    qb = np.array(g["q"], np.uint8)
    R = q.median_reference(dev_bins(q, qb), 5, g["B"], g["r"])
    torch.cuda.synchronize()
    np.testing.assert_array_equal(R.cpu().numpy()[0], g["ref"])
