"""Pins for the oracle's value-unit option (Sec. 3.1: Algorithm 1 charges each
transported amount at the distance |Q_i - Q_j| of the quantized values, not of
the bin indices).  With uniform bins the value distance is |i - j| times the
component's bin width (hi - lo) / B, so components of different ranges get
different weights before the channel mean.

Pinned by: a 1x3 two-component map worked out by hand (tests/golden); scipy's
1-D Wasserstein distance on the quantized values themselves (a library routine
for exactly this W1); the sort-and-match brute force of the supplement on the
values; and the closed-form link to the bin-unit result (value = bin width x
bin units, per component).
"""
import json
import pathlib
from fractions import Fraction

import numpy as np
import pytest
from scipy.stats import wasserstein_distance

import oracle
from paper_2510_15602_gb300 import synth

GOLD = json.loads((pathlib.Path(__file__).parent / "golden" / "hand_examples.json").read_text())


def frac(v):
    return np.array([float(Fraction(x)) for x in v], np.float64)


def qvalues(lo, hi, B):
    return lo + (np.arange(B) + 0.5) * (hi - lo) / B


def test_value_units_hand_case():
    g = GOLD["value_units_1x3"]
    q = np.array(g["q"], np.uint8)
    B, r = g["B"], g["r"]
    R = oracle.ref_hist(q, B)
    s_v, _, _ = oracle.score(q, B, r, R, 3, lo=g["lo"], hi=g["hi"])
    np.testing.assert_allclose(s_v[0], frac(g["score_value"]), rtol=1e-14, atol=1e-15)
    s_b, _, _ = oracle.score(q, B, r, R, 3)
    np.testing.assert_allclose(s_b[0], frac(g["score_bin"]), rtol=1e-14, atol=1e-15)
    _, raw, comp = oracle.assoc(q, B, r, R, 3, sigma_s=0.0, lo=g["lo"], hi=g["hi"])
    for k in range(2):
        np.testing.assert_allclose(comp[k, 0], frac(g["assoc_comp_value"][k]), rtol=1e-14, atol=1e-15)
    np.testing.assert_allclose(raw[0], frac(g["assoc_raw_value"]), rtol=1e-14, atol=1e-15)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_value_units_against_scipy_on_the_quantized_values(seed):
    rng = np.random.default_rng(seed)
    d, H, W, B, r = 3, 7, 9, 8, 2
    q = synth.random_bins(rng, d, H, W, B)
    lo = rng.uniform(-3, 1, d)
    hi = lo + rng.uniform(0.1, 5, d)
    R = oracle.ref_hist(q, B)
    s, _, _ = oracle.score(q, B, r, R, H * W, lo=lo, hi=hi)
    for (y, x) in [(0, 0), (3, 4), (6, 8), (2, 7)]:
        ref = 0.0
        for k in range(d):
            Q = qvalues(lo[k], hi[k], B)
            win = q[k, max(0, y - r):y + r + 1, max(0, x - r):x + r + 1].ravel()
            ref += wasserstein_distance(Q[win], Q[q[k].ravel()])
        assert s[y, x] == pytest.approx(ref / d, rel=1e-12, abs=1e-14)


@pytest.mark.parametrize("seed", [3, 4])
def test_alg1_values_sort_and_match(seed):
    # equal masses: the supplement's sort-and-match on the quantized values gives
    # the same total as Algorithm 1 charged at value distances
    rng = np.random.default_rng(seed)
    B = 6
    Q = qvalues(-2.0, 1.0, B)
    a = rng.integers(0, B, 25)
    b = rng.integers(0, B, 25)
    P = np.bincount(a, minlength=B)
    Rr = np.bincount(b, minlength=B)
    Ev, steps = oracle.alg1_values(P, Rr, Q)
    match = np.abs(np.sort(Q[a]) - np.sort(Q[b])).sum() * 25  # masses scaled to 25 x 25
    assert Ev.sum() == pytest.approx(match, rel=1e-12)
    assert steps <= 2 * B - 1


def test_value_units_equal_bin_width_times_bin_units():
    rng = np.random.default_rng(11)
    d, H, W, B, r = 2, 8, 10, 16, 3
    q = synth.random_bins(rng, d, H, W, B)
    lo = np.array([-1.0, 10.0])
    hi = np.array([3.0, 10.5])
    R = oracle.ref_hist(q, B)
    w = (hi - lo) / B
    _, raw_b, comp_b = oracle.assoc(q, B, r, R, H * W, sigma_s=0.0)
    _, raw_v, comp_v = oracle.assoc(q, B, r, R, H * W, sigma_s=0.0, lo=lo, hi=hi)
    for k in range(d):
        np.testing.assert_allclose(comp_v[k], w[k] * comp_b[k], rtol=1e-12, atol=1e-15)
    s_b, numer, nloc = oracle.score(q, B, r, R, H * W)
    s_v, _, _ = oracle.score(q, B, r, R, H * W, lo=lo, hi=hi)
    ref = sum(w[k] * numer[k] for k in range(d)) / (d * nloc * float(H * W))
    np.testing.assert_allclose(s_v, ref, rtol=1e-12, atol=1e-15)
    # a constant range (hi == lo) contributes nothing in value units
    _, _, comp0 = oracle.assoc(q, B, r, R, H * W, sigma_s=0.0, lo=[0.0, 1.0], hi=[0.0, 1.0])
    assert np.all(comp0 == 0.0)
