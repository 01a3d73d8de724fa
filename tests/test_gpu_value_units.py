"""GPU parity of the value-unit option (Sec. 3.1: Algorithm 1 charges each
transported amount at |Q_i - Q_j|, the distance of the quantized values; with
uniform bins that is |i - j| times the component's bin width (hi - lo) / B)
through the C ABI against the FP64 oracle's literal value-unit statements.

Tolerances: the plain EMD sums w_k D_k exactly-rounded in FP64 and rounds the
result once to FP32 (2^-23 relative, plus the oracle's FP64 rounding); the
paper's scoring keeps the bin-unit bound of its fixed-point errors
(4 * 2^-24 (B - 1) + 2^-(s+1), tests/test_gpu_assoc.py) scaled by the largest
bin width, plus FP32 rounding.  Components get deliberately different ranges.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2510_15602_gb300 import synth
from tests.gpu_helpers import to_dev
from tests.test_gpu_assoc import dev_bins, tol

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def q():
    from paper_2510_15602_gb300 import qfca
    assert torch.cuda.is_available()
    return qfca


def ranges(rng, d):
    lo = rng.uniform(-4.0, 2.0, d).astype(np.float32)
    hi = (lo + rng.uniform(0.05, 6.0, d)).astype(np.float32)
    return lo, hi


@pytest.mark.parametrize("d,H,W,B,r,seed", [(3, 37, 150, 16, 4, 0), (2, 33, 129, 32, 7, 1), (4, 40, 52, 64, 12, 2),
                                            (2, 1, 40, 16, 3, 3)])
def test_score_value_units_against_oracle(q, d, H, W, B, r, seed):
    rng = np.random.default_rng(seed)
    qb = synth.random_bins(rng, d, H, W, B)
    lo, hi = ranges(rng, d)
    R = oracle.ref_hist(qb, B)
    s_o, _, _ = oracle.score(qb, B, r, R, H * W, lo=lo.astype(np.float64), hi=hi.astype(np.float64))
    s_g = q.score(dev_bins(q, qb), W, B, r, to_dev(R.astype(np.int32)), H * W, lo=to_dev(lo), hi=to_dev(hi))
    torch.cuda.synchronize()
    np.testing.assert_allclose(s_g.cpu().numpy(), s_o, rtol=2.0 ** -22, atol=1e-30)
    # bin units are unchanged by the option's existence
    s_b, _, _ = oracle.score(qb, B, r, R, H * W)
    s_gb = q.score(dev_bins(q, qb), W, B, r, to_dev(R.astype(np.int32)), H * W)
    torch.cuda.synchronize()
    np.testing.assert_allclose(s_gb.cpu().numpy(), s_b, rtol=2.0 ** -23, atol=1e-12)


@pytest.mark.parametrize("d,H,W,B,r,seed", [(3, 37, 300, 16, 4, 4), (2, 33, 129, 32, 7, 5), (3, 40, 52, 64, 12, 6)])
def test_assoc_value_units_against_oracle(q, d, H, W, B, r, seed):
    rng = np.random.default_rng(seed)
    qb = synth.random_bins(rng, d, H, W, B)
    lo, hi = ranges(rng, d)
    R = oracle.ref_hist(qb, B)
    s_o, raw_o, comp_o = oracle.assoc(qb, B, r, R, H * W, sigma_s=1.0, lo=lo.astype(np.float64),
                                      hi=hi.astype(np.float64))
    s_g, raw_g, comp_g = q.score_assoc(dev_bins(q, qb), W, B, r, to_dev(R.astype(np.int32)), H * W, sigma_s=1.0,
                                       want_raw=True, want_comp=True, lo=to_dev(lo), hi=to_dev(hi))
    torch.cuda.synchronize()
    t = tol(B, r) * float(np.max((hi.astype(np.float64) - lo) / B))
    np.testing.assert_allclose(comp_g.cpu().numpy(), comp_o, rtol=2.0 ** -22, atol=t)
    np.testing.assert_allclose(raw_g.cpu().numpy(), raw_o, rtol=2.0 ** -21, atol=t)
    np.testing.assert_allclose(s_g.cpu().numpy(), s_o, rtol=2.0 ** -19, atol=t)


def test_value_units_hand_case_on_the_gpu(q):
    import json
    import pathlib
    from fractions import Fraction
    g = json.loads((pathlib.Path(__file__).parent / "golden" / "hand_examples.json").read_text())["value_units_1x3"]
    qb = np.array(g["q"], np.uint8)
    B, r = g["B"], g["r"]
    R = oracle.ref_hist(qb, B)
    lo = to_dev(np.array(g["lo"], np.float32))
    hi = to_dev(np.array(g["hi"], np.float32))
    s = q.score(dev_bins(q, qb), 3, B, r, to_dev(R.astype(np.int32)), 3, lo=lo, hi=hi)
    _, raw = q.score_assoc(dev_bins(q, qb), 3, B, r, to_dev(R.astype(np.int32)), 3, sigma_s=0.0, want_raw=True,
                           lo=lo, hi=hi)
    torch.cuda.synchronize()
    exp_s = [float(Fraction(x)) for x in g["score_value"]]
    exp_raw = [float(Fraction(x)) for x in g["assoc_raw_value"]]
    np.testing.assert_allclose(s.cpu().numpy()[0], exp_s, rtol=2.0 ** -23, atol=1e-7)
    np.testing.assert_allclose(raw.cpu().numpy()[0], exp_raw, rtol=2.0 ** -21, atol=tol(B, r) * 2.0)
