"""GPU parity of the median reference (arXiv 2510.15602, Sec. 3.2) through the
C ABI against the oracle: integer work, bit-exact; and the EMD / paper scoring
against it, bit-exact numerators and within the association bound."""
import numpy as np
import pytest
import torch

import oracle
from paper_2510_15602_gb300 import synth
from tests.gpu_helpers import to_dev

pytestmark = pytest.mark.gpu


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


@pytest.mark.parametrize("d,H,W,B,r,seed", [
    (3, 40, 300, 16, 4, 0),     # two strips of centres, ragged
    (2, 33, 65, 32, 7, 1),
    (2, 3, 5, 8, 1, 2),         # a single full window
    (2, 60, 9, 16, 4, 3),       # a single column of centres
    (2, 50, 70, 64, 12, 4),     # B = 64, r = 12
    (2, 20, 24, 255, 3, 5),     # maximum bin count
])
def test_median_reference_bit_exact(q, d, H, W, B, r, seed):
    rng = np.random.default_rng(400 + seed)
    qb = synth.random_bins(rng, d, H, W, B, smooth=(seed % 2 == 0))
    R_o = oracle.median_ref(qb, B, r)
    R_g = q.median_reference(dev_bins(q, qb), W, B, r).cpu().numpy().astype(np.uint32)
    np.testing.assert_array_equal(R_g, R_o)
    assert (R_g.sum(axis=1) == (2 * r + 1) ** 2).all()


def test_median_reference_clamps_and_batches(q):
    rng = np.random.default_rng(410)
    B = 10
    shapes = [(30, 41, 3), (25, 25, 5), (64, 33, 2)]
    bl, Ws, rs, ro = [], [], [], []
    for H, W, r in shapes:
        qb = synth.random_bins(rng, 3, H, W, 14, smooth=True)  # values up to 13 with B = 10
        bl.append(dev_bins(q, qb))
        Ws.append(W)
        rs.append(r)
        ro.append(oracle.median_ref(np.minimum(qb, B - 1), B, r))
    outs = q.median_reference_batch(bl, Ws, rs, B)
    for o, R in zip(outs, ro):
        np.testing.assert_array_equal(o.cpu().numpy().astype(np.uint32), R)


def test_scores_against_the_median_reference(q):
    # the full path of Table 3's median reference: reference -> plain EMD and the paper's scoring
    rng = np.random.default_rng(420)
    d, H, W, B, r = 4, 48, 72, 16, 4
    qb = synth.random_bins(rng, d, H, W, B, smooth=True)
    bins = dev_bins(q, qb)
    Rg = q.median_reference(bins, W, B, r)
    R = Rg.cpu().numpy().astype(np.uint32)
    T2 = (2 * r + 1) ** 2
    _, num_o, _ = oracle.score(qb, B, r, R, T2)
    _, num_g = q.score(bins, W, B, r, Rg, T2, want_numer=True)
    np.testing.assert_array_equal(num_g.cpu().numpy(), num_o)
    s_o, _, _ = oracle.assoc(qb, B, r, R, T2, sigma_s=1.0)
    s_g = q.score_assoc(bins, W, B, r, Rg, T2, sigma_s=1.0).cpu().numpy()
    np.testing.assert_allclose(s_g, s_o, rtol=2.0 ** -20, atol=4 * 2.0 ** -24 * (B - 1) + 2.0 ** -21)


def test_median_reference_full_size_batch_sampled(q):
    # the benchmark's launch: 16 images of 32 x 256 x 256 bins, B = 32, r = 7, one batched call.
    # Each component's reference depends on its own plane only, so sampled planes of the first
    # and last image are checked bit for bit against the oracle, and every row of every image
    # counts each of the (2r + 1)^2-pixel windows once
    n, d, H, W, B, r = 16, 32, 256, 256, 32, 7
    rng = np.random.default_rng(430)
    qbs = [synth.random_bins(rng, d, H, W, B, smooth=True) for _ in range(n)]
    outs = q.median_reference_batch([dev_bins(q, qb) for qb in qbs], [W] * n, [r] * n, B)
    torch.cuda.synchronize()
    for o in outs:
        assert (o.cpu().numpy().astype(np.int64).sum(axis=1) == (2 * r + 1) ** 2).all()
    planes = [0, 17, d - 1]
    for i in (0, n - 1):
        R_o = oracle.median_ref(np.ascontiguousarray(qbs[i][planes]), B, r)
        np.testing.assert_array_equal(outs[i].cpu().numpy().astype(np.uint32)[planes], R_o)


def test_median_reference_rejects_bad_arguments(q):
    bins = torch.zeros(1, 8, 16, dtype=torch.uint8, device="cuda")
    with pytest.raises(RuntimeError):
        q.median_reference(bins, 8, 8, 4)   # 8 x 8 has no full 9 x 9 window
    with pytest.raises(RuntimeError):
        q.median_reference(torch.zeros(1, 64, 64, dtype=torch.uint8, device="cuda"), 64, 255, 20)  # table too large


def test_median_reference_beyond_one_launch(q):
    rng = np.random.default_rng(430)
    B, n = 12, 70
    bl, Ws, rs, ro = [], [], [], []
    for i in range(n):
        r = int(rng.integers(1, 4))
        H, W = int(rng.integers(2 * r + 1, 30)), int(rng.integers(2 * r + 1, 40))
        qb = synth.random_bins(rng, 2, H, W, B, smooth=(i % 2 == 1))
        bl.append(dev_bins(q, qb))
        Ws.append(W)
        rs.append(r)
        if i in (0, 40, 64, 69):
            ro.append((i, oracle.median_ref(qb, B, r)))
    outs = q.median_reference_batch(bl, Ws, rs, B)
    for i, R in ro:
        np.testing.assert_array_equal(outs[i].cpu().numpy().astype(np.uint32), R)
