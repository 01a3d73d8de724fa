"""GPU parity of the paper's own scoring (Algorithm 1, error-to-pixel
association, component mean, Gaussian smoothing; arXiv 2510.15602 Sec. 3.1)
through the C ABI against the FP64 oracle.

Tolerance (derived from the kernel's arithmetic): each per-bin error E <= B-1
is formed as fl(fl(Enum) * fl(2^s / fl(n N_ref))) (at most four FP32 roundings,
<= 4 * 2^-24 * E) and rounded to the fixed point 2^-s, s = min(20,
floor(log2((2^32 - 1) / ((2r+1)^2 (B-1))))); every later sum is exact, so a
per-component map differs from the oracle by at most
    tol = 4 * 2^-24 * (B - 1) + 2^-(s+1)
plus one FP32 rounding of the result; the component mean keeps that bound and
the smoothing adds FP32 rounding of the weighted sums (<= 2^-20 relative).
"""
import math

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


def shift(B, r):
    return min(20, max(0, math.floor(math.log2((2 ** 32 - 1) / ((2 * r + 1) ** 2 * (B - 1))))))


def tol(B, r):
    return 4 * 2.0 ** -24 * (B - 1) + 2.0 ** -(shift(B, r) + 1)


def dev_bins(q, qb):
    d, H, W = qb.shape
    bins = torch.zeros(d, H, q.bins_pitch(W), dtype=torch.uint8, device="cuda")
    bins[:, :, :W] = to_dev(qb)
    return bins


def run(q, qb, B, r, R, Nref, sigma_s):
    d, H, W = qb.shape
    s, raw, comp = q.score_assoc(dev_bins(q, qb), W, B, r, to_dev(R.astype(np.int32)), Nref, sigma_s=sigma_s,
                                 want_raw=True, want_comp=True)
    torch.cuda.synchronize()
    return s.cpu().numpy(), raw.cpu().numpy(), comp.cpu().numpy()


def check(q, qb, B, r, sigma_s=1.0, Rmod=None):
    d, H, W = qb.shape
    qc = np.minimum(qb, B - 1)  # values >= B count as B-1
    R = oracle.ref_hist(qc, B) if Rmod is None else Rmod
    Nref = int(R[0].sum())
    s_o, raw_o, comp_o = oracle.assoc(qc, B, r, R, Nref, sigma_s=sigma_s)
    s_g, raw_g, comp_g = run(q, qb, B, r, R, Nref, sigma_s)
    t = tol(B, r)
    np.testing.assert_allclose(comp_g, comp_o, rtol=2.0 ** -23, atol=t)
    np.testing.assert_allclose(raw_g, raw_o, rtol=2.0 ** -22, atol=t)
    np.testing.assert_allclose(s_g, s_o, rtol=2.0 ** -20, atol=t)
    return s_g, raw_g


@pytest.mark.parametrize("d,H,W,B,r,seed", [
    (3, 37, 300, 16, 4, 0),     # two strips, ragged rows and columns
    (2, 33, 129, 32, 7, 1),
    (1, 5, 7, 8, 4, 2),         # window larger than the image
    (2, 1, 40, 16, 3, 3),       # a single row
    (2, 40, 1, 16, 3, 4),       # a single column
    (3, 40, 52, 64, 12, 5),     # B = 64, r = 12
    (2, 30, 33, 255, 2, 6),     # maximum bin count
])
def test_assoc_matches_oracle(q, d, H, W, B, r, seed):
    rng = np.random.default_rng(300 + seed)
    qb = synth.random_bins(rng, d, H, W, B, smooth=(seed % 2 == 0))
    check(q, qb, B, r)


def test_assoc_plain_128_c64_with_planted_square(q):
    # 128 x 128, d = 16, B = 16, r = 4: the small single-image workload
    rng = np.random.default_rng(41)
    qb = synth.random_bins(rng, 16, 128, 128, 16, smooth=True)
    qb[:, 50:62, 70:82] = np.minimum(qb[:, 50:62, 70:82].astype(np.int64) + 5, 15).astype(np.uint8)
    s_g, _ = check(q, qb, 16, 4)
    assert s_g[52:60, 72:80].mean() > 1.2 * s_g[:40].mean()  # the shifted square stands out


def test_assoc_wide_accumulator(q):
    # (B-1)(2r+1)^2 N_ref >= 2^32: the two-pointer walk runs in 64-bit integers
    rng = np.random.default_rng(42)
    B, r, H, W = 255, 12, 210, 200
    assert (B - 1) * (2 * r + 1) ** 2 * H * W >= 2 ** 32
    qb = synth.random_bins(rng, 1, H, W, B, smooth=True)
    check(q, qb, B, r)


def test_assoc_degenerate_maps_are_exactly_zero(q):
    rng = np.random.default_rng(43)
    qb = synth.random_bins(rng, 2, 17, 19, 8, smooth=False)
    s_g, raw_g = check(q, qb, 8, 20)  # every window is the whole image
    assert np.abs(raw_g).max() == 0.0 and np.abs(s_g).max() == 0.0
    qc = np.full((2, 23, 31), 5, np.uint8)
    s_g, raw_g = check(q, qc, 8, 3)
    assert np.abs(s_g).max() == 0.0


def test_assoc_bins_above_range_and_foreign_reference(q):
    rng = np.random.default_rng(44)
    qb = synth.random_bins(rng, 2, 29, 41, 20, smooth=True)  # values up to 19 with B = 12: clamped
    R = oracle.ref_hist(np.minimum(synth.random_bins(rng, 2, 40, 40, 12, smooth=False), 11), 12)
    check(q, qb, 12, 3, Rmod=R)  # a reference of another size (N_ref = 1600)


def test_assoc_no_smoothing_returns_raw(q):
    rng = np.random.default_rng(45)
    qb = synth.random_bins(rng, 2, 20, 26, 16, smooth=True)
    s_g, raw_g = check(q, qb, 16, 2, sigma_s=0.0)
    np.testing.assert_array_equal(s_g, raw_g)
    check(q, qb, 16, 2, sigma_s=2.5)


def test_assoc_batch_equals_single_calls(q):
    rng = np.random.default_rng(46)
    B, d = 32, 4
    shapes = [(40, 75, 5), (64, 64, 7), (23, 130, 9)]
    bl, Rs, Ws, rs, tot = [], [], [], [], []
    for H, W, r in shapes:
        qb = synth.random_bins(rng, d, H, W, B, smooth=True)
        R = oracle.ref_hist(qb, B)
        bl.append(dev_bins(q, qb))
        Rs.append(to_dev(R.astype(np.int32)))
        Ws.append(W)
        rs.append(r)
        tot.append(H * W)
    outs = q.score_assoc_batch(bl, Ws, rs, B, Rs, tot, sigma_s=1.0)
    for b, W, r, R, n, o in zip(bl, Ws, rs, Rs, tot, outs):
        single = q.score_assoc(b, W, B, r, R, n, sigma_s=1.0)
        torch.testing.assert_close(o, single, rtol=0, atol=0)


def test_assoc_full_size_256_c32(q):
    # one image at the batch workload's per-image size: 256 x 256, d = 32, B = 32, r = 7
    rng = np.random.default_rng(47)
    qb = synth.random_bins(rng, 32, 256, 256, 32, smooth=True)
    check(q, qb, 32, 7)


def test_assoc_full_size_batch_equals_single_calls(q):
    # the benchmark's launch: 16 images of 32 x 256 x 256 bins, B = 32, r = 7, each image's own
    # global histogram as reference, one batched call; images 0, 7 and 15 equal the single-image
    # call (itself checked against the oracle at this size above) bit for bit
    n, d, H, W, B, r = 16, 32, 256, 256, 32, 7
    rng = np.random.default_rng(49)
    qbs = [synth.random_bins(rng, d, H, W, B, smooth=True) for _ in range(n)]
    bl = [dev_bins(q, qb) for qb in qbs]
    Rs = [to_dev(oracle.ref_hist(qb, B).astype(np.int32)) for qb in qbs]
    outs = q.score_assoc_batch(bl, [W] * n, [r] * n, B, Rs, [H * W] * n, sigma_s=1.0)
    for i in (0, 7, n - 1):
        single = q.score_assoc(bl[i], W, B, r, Rs[i], H * W, sigma_s=1.0)
        torch.testing.assert_close(outs[i], single, rtol=0, atol=0)


def test_assoc_rejects_bad_arguments(q):
    bins = torch.zeros(1, 8, 16, dtype=torch.uint8, device="cuda")
    R = torch.zeros(1, 8, dtype=torch.int32, device="cuda")
    R[0, 0] = 64
    with pytest.raises(RuntimeError):
        q.score_assoc(bins, 8, 8, 1, R, 64, sigma_s=5.0)
    with pytest.raises(RuntimeError):
        q.score_assoc(bins, 8, 255, 40, R, 64)  # 2r > 56 with B > 128
    with pytest.raises(RuntimeError):
        q.score_assoc(bins, 8, 8, 0, R, 64)


def test_assoc_batch_beyond_one_launch(q):
    # more than 64 images: several launches per stage, results equal single calls
    rng = np.random.default_rng(48)
    B, d, n = 16, 2, 70
    bl, Rs, Ws, rs, tot = [], [], [], [], []
    for i in range(n):
        H, W, r = int(rng.integers(6, 30)), int(rng.integers(6, 40)), int(rng.integers(1, 5))
        qb = synth.random_bins(rng, d, H, W, B, smooth=(i % 2 == 0))
        bl.append(dev_bins(q, qb))
        Rs.append(to_dev(oracle.ref_hist(qb, B).astype(np.int32)))
        Ws.append(W)
        rs.append(r)
        tot.append(H * W)
    outs = q.score_assoc_batch(bl, Ws, rs, B, Rs, tot, sigma_s=1.0)
    for i in (0, 33, 64, 69):
        single = q.score_assoc(bl[i], Ws[i], B, rs[i], Rs[i], tot[i], sigma_s=1.0)
        torch.testing.assert_close(outs[i], single, rtol=0, atol=0)
