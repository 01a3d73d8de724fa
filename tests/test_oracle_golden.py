"""Pins for the oracle against small cases worked out by hand
(`tests/golden/hand_examples.json`): Algorithm 1's per-bin transport (Sec. 3.1),
the uniform quantiser (Sec. 3.1), the window-EMD score (Sec. 3.1, Sec. 3), the
error-to-pixel association (Sec. 3.1), the median reference (Sec. 3.2), the
QFCA+ residual (Sec. 3.3) and the whole path on a 1x4 two-channel image.  Each
fixture carries its derivation; the expected values are exact fractions.
"""
import json
import pathlib
from fractions import Fraction

import numpy as np
import pytest

import oracle

GOLD = json.loads((pathlib.Path(__file__).parent / "golden" / "hand_examples.json").read_text())


def frac(v):
    return np.array([float(Fraction(x)) for x in v], np.float64)


@pytest.mark.parametrize("case", GOLD["alg1"], ids=lambda c: str(c["P"]))
def test_alg1_hand(case):
    P = np.array(case["P"], np.int64)
    R = np.array(case["R"], np.int64)
    En, _ = oracle.alg1(P, R)
    np.testing.assert_array_equal(En, case["Enum"])
    Nloc, Nref = int(P.sum()), int(R.sum())
    assert Fraction(int(En.sum()), Nloc * Nref) == Fraction(case["emd"])
    E = [Fraction(int(e), int(p) * Nref) if p else Fraction(0) for e, p in zip(En, P)]
    assert E == [Fraction(x) for x in case["E"]]


def test_quantize_hand():
    g = GOLD["quantize"]
    q, lo, hi = oracle.quantize(np.array([g["Y"]], np.float64), g["B"])
    np.testing.assert_array_equal(q[0], g["q"])
    assert lo[0] == min(g["Y"]) and hi[0] == max(g["Y"])


def test_score_hand():
    g = GOLD["score_1x3"]
    q = np.array(g["q"], np.uint8)
    R = oracle.ref_hist(q, g["B"])
    s, _, _ = oracle.score(q, g["B"], g["r"], R)
    np.testing.assert_allclose(s[0], frac(g["score"]), rtol=0, atol=1e-15)


def test_assoc_hand():
    g = GOLD["assoc_1x3"]
    q = np.array(g["q"], np.uint8)
    R = oracle.ref_hist(q, g["B"])
    s, raw, comp = oracle.assoc(q, g["B"], g["r"], R, sigma_s=0.0)
    np.testing.assert_allclose(raw[0], frac(g["raw"]), rtol=0, atol=1e-15)
    np.testing.assert_array_equal(s, raw)
    np.testing.assert_array_equal(comp[0], raw)  # one component: its map is the mean


@pytest.mark.parametrize("key", ["median_3x5", "median_3x4_even"])
def test_median_reference_hand(key):
    g = GOLD[key]
    q = np.array(g["q"], np.uint8)
    np.testing.assert_array_equal(oracle.median_ref(q, g["B"], g["r"])[0], g["ref"])


def test_residual_hand():
    g = GOLD["residual_1x4"]
    X = np.array(g["X"], np.float64)
    mean, V, ev, allev = oracle.fit(X, g["dres"])
    np.testing.assert_allclose(allev, frac(g["eigvals"]), rtol=1e-14)
    np.testing.assert_allclose(np.abs(V[:, 0]), [1.0, 0.0], atol=1e-14)
    F = oracle.residual(X, mean, V)
    np.testing.assert_allclose(F, np.array(g["F"]), atol=1e-14)


def test_pipeline_hand():
    g = GOLD["pipeline_1x4"]
    X = np.array(g["X"], np.float64)
    mean, V, ev, _ = oracle.fit(X, g["d"])
    np.testing.assert_array_equal(V[:, 0], [1.0, 0.0])  # sign rule: the largest entry is positive
    Y = oracle.project(X, mean, V)
    np.testing.assert_allclose(Y[0, 0], g["Y"], atol=1e-14)
    q, _, _ = oracle.quantize(Y, g["B"])
    np.testing.assert_array_equal(q[0, 0], g["q"])
    R = oracle.ref_hist(q, g["B"])
    np.testing.assert_array_equal(R[0], g["R"])
    s, _, _ = oracle.score(q, g["B"], g["r"], R)
    np.testing.assert_allclose(s[0], frac(g["score"]), rtol=0, atol=1e-15)
