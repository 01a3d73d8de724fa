"""Pins of the oracle's Algorithm 1, error-to-pixel association and final blur
(arXiv 2510.15602, Sec. 3.1 and the supplement's correctness proof) against
facts fixed independently of the oracle's code: the scalar W1 closed form,
scipy's 1-D Wasserstein distance, the supplement's sort-and-match statement by
brute force, the 2N-1 step bound, and scipy's Gaussian filter in the interior.
CPU only."""
import numpy as np
import pytest

import oracle

scipy_stats = pytest.importorskip("scipy.stats")
scipy_ndimage = pytest.importorskip("scipy.ndimage")


def cdf_numerator(P, R, Nloc, Nref):
    # W1 closed form of the supplement, bin units: sum_b |cumP_b N_ref - cumR_b N_loc|
    return int(np.abs(np.cumsum(P) * Nref - np.cumsum(R) * Nloc).sum())


def sort_and_match(P, R, Nloc, Nref):
    """FCA on quantized values by brute force (supplement, proof of Algorithm 1):
    both samples at the common mass (every local value repeated N_ref times,
    every reference value N_loc times), sorted, matched by rank; the error of a
    local element is its distance to the matched reference element.  Returns the
    summed error of the elements of each local bin."""
    B = len(P)
    X = np.repeat(np.arange(B), np.asarray(P) * Nref)
    Y = np.repeat(np.arange(B), np.asarray(R) * Nloc)
    assert len(X) == len(Y)
    err = np.abs(np.sort(X) - np.sort(Y))
    return np.array([int(err[X == b].sum()) for b in range(B)], np.int64)  # X is already sorted


@pytest.mark.parametrize("seed", range(6))
def test_alg1_sum_is_the_scalar_emd(seed):
    rng = np.random.default_rng(seed)
    B = int(rng.integers(2, 40))
    P = rng.integers(0, 12, B) * (rng.random(B) < 0.6)
    if P.sum() == 0:
        P[0] = 1
    R = rng.integers(0, 50, B)
    R[rng.integers(0, B)] += 1
    Nloc, Nref = int(P.sum()), int(R.sum())
    En, steps = oracle.alg1(P, R)
    assert (En >= 0).all()
    assert int(En.sum()) == cdf_numerator(P, R, Nloc, Nref)
    w = scipy_stats.wasserstein_distance(np.arange(B), np.arange(B), P, R)
    assert En.sum() / (Nloc * Nref) == pytest.approx(w, rel=1e-12, abs=1e-12)
    assert 1 <= steps <= 2 * B - 1


@pytest.mark.parametrize("seed", range(8))
def test_alg1_equals_sort_and_match_by_rank(seed):
    rng = np.random.default_rng(100 + seed)
    B = int(rng.integers(2, 7))
    P = rng.integers(0, 4, B)
    if P.sum() == 0:
        P[-1] = 2
    R = rng.integers(0, 5, B)
    if R.sum() == 0:
        R[0] = 3
    Nloc, Nref = int(P.sum()), int(R.sum())
    En, _ = oracle.alg1(P, R)
    np.testing.assert_array_equal(En, sort_and_match(P, R, Nloc, Nref))


def test_alg1_special_cases():
    # identical shapes transport nothing
    R = np.array([3, 0, 6, 9, 3])
    En, _ = oracle.alg1(2 * R // 3, R)
    assert (En == 0).all()
    # point masses: the whole error sits on the patch's bin, |a - b| per unit mass
    for a, b in [(0, 4), (4, 0), (2, 2), (1, 3)]:
        P = np.zeros(5, np.int64)
        P[a] = 9
        R = np.zeros(5, np.int64)
        R[b] = 25
        En, steps = oracle.alg1(P, R)
        assert En[a] == 9 * 25 * abs(a - b) and En.sum() == En[a]
        assert steps <= 2 * 5 - 1
    # the bound is reached: with equal bins every tie moves the reference pointer
    # first and the emptied patch bin costs one more step, ending at i = B - 1, j = B
    P = np.ones(6, np.int64)
    En, steps = oracle.alg1(P, 2 * P)
    assert steps == 2 * 6 - 1 and (En == 0).all()


def assoc_scatter(q, B, r, R, Nref):
    """The association written in scatter form, with per-bin errors from the
    sort-and-match brute force: every window spreads the error of each of its
    bins onto the pixels of that bin; each pixel divides by the number of
    windows that contain it."""
    d, H, W = q.shape
    comp = np.zeros((d, H, W))
    for k in range(d):
        acc = np.zeros((H, W))
        cnt = np.zeros((H, W))
        for py in range(H):
            for px in range(W):
                ys, xs = slice(max(0, py - r), min(H, py + r + 1)), slice(max(0, px - r), min(W, px + r + 1))
                win = q[k, ys, xs]
                P = np.bincount(win.ravel(), minlength=B)
                Nloc = win.size
                En = sort_and_match(P, R[k], Nloc, Nref)
                E = np.where(P > 0, En / np.maximum(P * Nref, 1), 0.0)
                acc[ys, xs] += E[win]
                cnt[ys, xs] += 1
        comp[k] = acc / cnt
    return comp


@pytest.mark.parametrize("seed,B,r", [(0, 4, 1), (1, 5, 2), (2, 3, 1)])
def test_assoc_against_scatter_form_8x8(seed, B, r):
    rng = np.random.default_rng(200 + seed)
    q = rng.integers(0, B, (2, 8, 8)).astype(np.uint8)
    q[1, 2:5, 3:6] = B - 1  # a planted block
    R = oracle.ref_hist(q, B)
    s, raw, comp = oracle.assoc(q, B, r, R, 64, sigma_s=0.0)
    ref = assoc_scatter(q, B, r, R.astype(np.int64), 64)
    np.testing.assert_allclose(comp, ref, rtol=1e-13, atol=1e-13)
    np.testing.assert_allclose(raw, ref.mean(axis=0), rtol=1e-13, atol=1e-13)
    np.testing.assert_array_equal(s, raw)


def test_assoc_degenerate_cases_are_zero():
    rng = np.random.default_rng(7)
    q = rng.integers(0, 6, (2, 7, 9)).astype(np.uint8)
    R = oracle.ref_hist(q, 6)
    # a window covering the whole image is the reference itself
    s, raw, _ = oracle.assoc(q, 6, 9, R, 63, sigma_s=1.0)
    assert np.abs(raw).max() == 0.0 and np.abs(s).max() == 0.0
    # constant planes
    qc = np.full((2, 7, 9), 3, np.uint8)
    s, raw, _ = oracle.assoc(qc, 6, 2, oracle.ref_hist(qc, 6), 63, sigma_s=1.0)
    assert np.abs(s).max() == 0.0


def test_assoc_anomaly_scores_higher():
    rng = np.random.default_rng(3)
    B = 8
    q = rng.integers(2, 6, (1, 24, 24)).astype(np.uint8)
    q[0, 10:14, 10:14] = 7
    R = oracle.ref_hist(q, B)
    s, _, _ = oracle.assoc(q, B, 3, R, 24 * 24, sigma_s=1.0)
    inside = s[10:14, 10:14].mean()
    far = np.concatenate([s[:4].ravel(), s[-4:].ravel()]).mean()
    assert inside > 3 * far


def test_blur_against_scipy_interior_and_constant_at_border():
    rng = np.random.default_rng(11)
    a = rng.random((20, 23))
    for sigma in (1.0, 1.5):
        out = oracle.blur(a, sigma)
        R4 = int(np.ceil(4 * sigma))
        ref = scipy_ndimage.gaussian_filter(a, sigma, truncate=R4 / sigma, mode="constant")
        np.testing.assert_allclose(out[R4:-R4, R4:-R4], ref[R4:-R4, R4:-R4], rtol=1e-12, atol=1e-14)
    c = np.full((9, 7), 2.5)
    np.testing.assert_allclose(oracle.blur(c, 1.0), c, rtol=1e-15)
    # border renormalisation: a corner delta keeps its weight share of the clipped kernel
    dlt = np.zeros((12, 12))
    dlt[0, 0] = 1.0
    g = np.exp(-np.arange(5) ** 2 / 2.0)
    np.testing.assert_allclose(oracle.blur(dlt, 1.0)[0, 0], (1 / g.sum()) ** 2, rtol=1e-14)
    np.testing.assert_array_equal(oracle.blur(a, 0.0), a)
