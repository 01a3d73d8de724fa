"""Pins of the oracle's median reference (arXiv 2510.15602, Sec. 3.2): the
per-rank median over patches is the reference that minimises the summed
Wasserstein distance to all patches -- checked by exhaustive search over every
reference on tiny cases, with the distance from the oracle's independent W1
(the CDF-difference score numerators), and by closed-form special cases.  CPU only."""
import itertools

import numpy as np
import pytest

import oracle


def total_w1(q, B, r, R):
    """Sum over full windows of the W1 numerators against the reference R
    (N_ref = (2r+1)^2 = N_loc, so D / T^2 is the sorted-matching cost)."""
    d, H, W = q.shape
    T2 = (2 * r + 1) ** 2
    _, numer, nloc = oracle.score(q, B, r, R, T2)
    inner = numer[:, r:H - r, r:W - r]
    assert (nloc[r:H - r, r:W - r] == T2).all()
    return inner.sum(axis=(1, 2)) // T2


def multisets(total, B):
    for cuts in itertools.combinations(range(total + B - 1), B - 1):
        prev, h = -1, []
        for c in cuts + (total + B - 1,):
            h.append(c - prev - 1)
            prev = c
        yield np.array(h, np.uint32)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_median_reference_minimises_total_w1_exhaustively(seed):
    rng = np.random.default_rng(20 + seed)
    B, r = 3, 1
    q = rng.integers(0, B, (1, 7, 8)).astype(np.uint8)
    R = oracle.median_ref(q, B, r)
    assert R.sum() == 9
    best = min(int(total_w1(q, B, r, h[None, :])[0]) for h in multisets(9, B))
    assert int(total_w1(q, B, r, R)[0]) == best


def test_median_reference_local_moves_do_not_help():
    rng = np.random.default_rng(30)
    B, r = 8, 2
    q = np.minimum(rng.integers(0, 4, (2, 14, 15)) + rng.integers(0, 5, (2, 14, 15)), B - 1).astype(np.uint8)
    R = oracle.median_ref(q, B, r).astype(np.int64)
    base = total_w1(q, B, r, R.astype(np.uint32))
    for k in range(2):
        for b in range(B):
            if R[k, b] == 0:
                continue
            for nb in (b - 1, b + 1):
                if 0 <= nb < B:
                    R2 = R.copy()
                    R2[k, b] -= 1
                    R2[k, nb] += 1
                    assert total_w1(q, B, r, R2.astype(np.uint32))[k] >= base[k]
    # the image-global histogram at the same mass is no better
    g = oracle.ref_hist(q, B).astype(np.float64)
    for k in range(2):
        cdf = np.cumsum(g[k]) / g[k].sum()
        vals = np.searchsorted(cdf, (np.arange(25) + 0.5) / 25)
        Rg = np.bincount(vals, minlength=B).astype(np.uint32)
        assert total_w1(q[k:k + 1], B, r, Rg[None, :])[0] >= base[k]


def test_median_reference_closed_forms():
    r, T = 1, 3
    # every full window of a T-periodic image holds one period: the reference is that period
    tile = np.array([[0, 4, 2], [1, 1, 5], [3, 0, 2]], np.uint8)
    q = np.tile(tile, (4, 4))[None, :11, :10]
    R = oracle.median_ref(q, 6, r)
    np.testing.assert_array_equal(R[0], np.bincount(tile.ravel(), minlength=6))
    # constant planes
    qc = np.full((2, 6, 7), 4, np.uint8)
    R = oracle.median_ref(qc, 6, 2)
    assert (R[:, 4] == 25).all() and R.sum() == 50
    with pytest.raises(ValueError):
        oracle.median_ref(np.zeros((1, 4, 9), np.uint8), 4, 2)
