"""Pins for the FP64 CPU oracle: checks against facts fixed by the paper and
by mathematics, never against the oracle's own formulas.

* Sec. 3.1 / supplement (Wasserstein closed form): W1 of 1-D distributions is
  the integral of |F^-1 - G^-1| over the quantile axis.  The oracle evaluates
  it as the L1 distance of the CDFs over bins; the tests evaluate it through
  the quantile integral on merged breakpoints, through scipy's
  ``wasserstein_distance``, and through the equal-mass sort-and-match form.
* Invariants: window counts sum to the window area, identical histograms give
  0, two point masses give their bin distance, a constant map scores 0.
* Sec. 3.3 PCA: covariance against numpy, eigendecomposition against LAPACK
  (numpy.linalg.eigh), a planted spectrum, and a selection basis whose
  projection has a closed form.
"""
import numpy as np
import pytest

import oracle
from paper_2510_15602_gb300 import synth
from paper_2510_15602_gb300.metrics import auroc


# ----------------------------------------------------------------- helpers (independent formulas)

def w1_quantile(a_vals, b_vals):
    """W1 between two empirical 1-D samples via the quantile integral
    int_0^1 |F^-1(u) - G^-1(u)| du, evaluated exactly on merged breakpoints."""
    a = np.sort(np.asarray(a_vals, np.float64))
    b = np.sort(np.asarray(b_vals, np.float64))
    na, nb = len(a), len(b)
    # breakpoints of the two step quantile functions
    u = np.union1d(np.arange(na + 1) / na, np.arange(nb + 1) / nb)
    total = 0.0
    for u0, u1 in zip(u[:-1], u[1:]):
        mid = 0.5 * (u0 + u1)
        ia = min(int(np.floor(mid * na)), na - 1)
        ib = min(int(np.floor(mid * nb)), nb - 1)
        total += (u1 - u0) * abs(a[ia] - b[ib])
    return total


def brute_window(qk, r, y, x):
    H, W = qk.shape
    return qk[max(0, y - r):min(H, y + r + 1), max(0, x - r):min(W, x + r + 1)].ravel()


# ----------------------------------------------------------------- score / EMD pins

def test_window_counts_sum_to_area_and_match_slicing():
    rng = np.random.default_rng(3)
    H, W, B, r = 11, 9, 7, 3
    qk = rng.integers(0, B, size=(H, W)).astype(np.uint8)
    for y in range(H):
        for x in range(W):
            L, n = oracle.window_hist(qk, B, r, y, x)
            win = brute_window(qk, r, y, x)
            assert n == win.size
            assert L.sum() == n
            np.testing.assert_array_equal(L, np.bincount(win, minlength=B))
    # corner window is clipped to (r+1)^2, interior is (2r+1)^2
    assert oracle.window_hist(qk, B, r, 0, 0)[1] == (r + 1) ** 2
    assert oracle.window_hist(qk, B, r, 5, 4)[1] == (2 * r + 1) ** 2


def test_constant_map_scores_zero():
    q = np.full((3, 10, 12), 5, np.uint8)
    R = oracle.ref_hist(q, 8)
    s, numer, _ = oracle.score(q, 8, 2, R)
    assert np.all(s == 0.0) and np.all(numer == 0)


def test_identical_histograms_give_zero():
    # q(y, x) = x mod 3 with W a multiple of 3: every window whose columns are
    # not clipped holds each value in the same proportion as the whole image.
    H, W, r, B = 7, 12, 4, 3
    q = np.tile((np.arange(W) % 3).astype(np.uint8), (H, 1))[None]
    R = oracle.ref_hist(q, B)
    s, numer, _ = oracle.score(q, B, r, R)
    # window width 9 = 3 full periods
    interior = s[:, r:W - r]
    assert np.all(interior == 0.0)
    assert np.all(numer[0][:, r:W - r] == 0)
    assert np.any(s[:, :r] > 0)  # clipped windows do differ


@pytest.mark.parametrize("a,b", [(0, 5), (5, 0), (3, 3), (0, 15), (7, 8)])
def test_point_masses_give_bin_distance(a, b):
    H, W, B, r = 6, 5, 16, 2
    q = np.full((1, H, W), a, np.uint8)
    R = np.zeros((1, B), np.uint32)
    R[0, b] = 1000  # reference: point mass at bin b with mass 1000
    s, numer, nloc = oracle.score(q, B, r, R, Nref=1000)
    np.testing.assert_array_equal(s, np.full((H, W), float(abs(a - b))))
    np.testing.assert_array_equal(numer[0], abs(a - b) * nloc.astype(np.int64) * 1000)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_brute_force_8x8_against_quantile_integral_and_scipy(seed):
    scipy_stats = pytest.importorskip("scipy.stats")
    rng = np.random.default_rng(seed)
    d, H, W, B, r = 3, 8, 8, 6, 2
    q = rng.integers(0, B, size=(d, H, W)).astype(np.uint8)
    R = oracle.ref_hist(q, B)
    s, numer, nloc = oracle.score(q, B, r, R)
    for y in range(H):
        for x in range(W):
            emds = []
            for k in range(d):
                win = brute_window(q[k], r, y, x)
                ref = q[k].ravel()
                w_q = w1_quantile(win, ref)
                w_s = scipy_stats.wasserstein_distance(win.astype(float), ref.astype(float))
                assert abs(w_q - w_s) < 1e-12
                emd_k = numer[k, y, x] / (nloc[y, x] * H * W)
                assert abs(emd_k - w_q) < 1e-12
                emds.append(w_q)
            assert abs(s[y, x] - np.mean(emds)) < 1e-12


@pytest.mark.parametrize("seed", [0, 1])
def test_score_at_against_scipy_and_point_masses(seed):
    # one pixel at a time: W1 of the clipped window against the image (scipy),
    # and point masses at bin distance |a - b|
    scipy_stats = pytest.importorskip("scipy.stats")
    rng = np.random.default_rng(10 + seed)
    d, H, W, B, r = 2, 9, 11, 7, 3
    q = rng.integers(0, B, size=(d, H, W)).astype(np.uint8)
    R = oracle.ref_hist(q, B)
    for y, x in [(0, 0), (4, 5), (8, 10), (2, 9)]:
        s, numer = oracle.score_at(q, B, r, R, H * W, y, x)
        emds = []
        for k in range(d):
            win = brute_window(q[k], r, y, x)
            w = scipy_stats.wasserstein_distance(win.astype(float), q[k].ravel().astype(float))
            assert abs(numer[k] / (win.size * H * W) - w) < 1e-12
            emds.append(w)
        assert abs(s - np.mean(emds)) < 1e-12
    qa = np.full((1, 5, 6), 2, np.uint8)
    Rb = np.zeros((1, 16), np.uint32)
    Rb[0, 11] = 77
    s, numer = oracle.score_at(qa, 16, 2, Rb, 77, 0, 5)
    assert s == 9.0 and numer[0] == 9 * (3 * 3) * 77


def test_equal_mass_sort_and_match():
    # window of 81 pixels against an external reference of mass 81:
    # W1 = (1/81) sum_i |sorted(window)_i - sorted(ref)_i|  (textbook equal-mass form)
    rng = np.random.default_rng(11)
    B, r = 10, 4
    q = rng.integers(0, B, size=(1, 9, 9)).astype(np.uint8)
    ref_vals = rng.integers(0, B, size=81)
    R = np.bincount(ref_vals, minlength=B).astype(np.uint32)[None]
    s, numer, nloc = oracle.score(q, B, r, R, Nref=81)
    win = q[0].ravel()  # centre pixel's window is the whole 9x9 map
    expect = np.abs(np.sort(win).astype(float) - np.sort(ref_vals).astype(float)).sum() / 81.0
    assert nloc[4, 4] == 81
    assert abs(s[4, 4] - expect) < 1e-13
    assert numer[0, 4, 4] == round(expect * 81 * 81)


def test_score_is_mean_over_components():
    rng = np.random.default_rng(5)
    q = rng.integers(0, 5, size=(4, 7, 6)).astype(np.uint8)
    R = oracle.ref_hist(q, 5)
    s, _, _ = oracle.score(q, 5, 1, R)
    per = [oracle.score(q[k:k + 1], 5, 1, R[k:k + 1])[0] for k in range(4)]
    np.testing.assert_allclose(s, np.mean(per, axis=0), rtol=0, atol=1e-15)


# ----------------------------------------------------------------- quantize pins

def test_quantize_edges_and_counts():
    B = 4
    lo, hi = -2.0, 6.0
    edges = lo + (hi - lo) * np.arange(B + 1) / B  # -2, 0, 2, 4, 6
    Y = np.array([[edges[0], edges[1], edges[2], edges[3], edges[4], 1.999, 2.001, 5.9999]])
    q, lo_o, hi_o = oracle.quantize(Y[:, None, :], B)
    assert lo_o[0] == lo and hi_o[0] == hi
    # an edge value belongs to the bin it opens; the maximum goes to bin B-1
    np.testing.assert_array_equal(q.ravel(), [0, 1, 2, 3, 3, 1, 2, 3])
    # counts sum to N
    R = oracle.ref_hist(q, B)
    assert R.sum() == Y.size


def test_quantize_degenerate_and_fixed_range():
    Y = np.full((2, 3, 3), 1.25)
    q, lo, hi = oracle.quantize(Y, 8)
    assert np.all(q == 0) and lo[0] == hi[0] == 1.25
    Y = np.array([[[-5.0, 0.0, 0.49, 0.5, 0.99, 7.0]]])
    q, _, _ = oracle.quantize(Y, 4, lo=np.array([0.0]), hi=np.array([1.0]))
    np.testing.assert_array_equal(q.ravel(), [0, 0, 1, 2, 3, 3])


def test_quantize_fp32_decision_matches_float_formula():
    rng = np.random.default_rng(2)
    Y = rng.standard_normal((3, 20, 20)).astype(np.float32).astype(np.float64)
    B = 32
    q32, lo, hi = oracle.quantize(Y, B, fp32_decision=True)
    y = Y.astype(np.float32)
    l32, h32 = lo.astype(np.float32)[:, None, None], hi.astype(np.float32)[:, None, None]
    t = (y - l32) / (h32 - l32)
    expect = np.clip((t * np.float32(B)).astype(np.int64), 0, B - 1)
    np.testing.assert_array_equal(q32, expect)
    q64, _, _ = oracle.quantize(Y, B)
    assert (q64 != q32).mean() < 1e-3


# ----------------------------------------------------------------- fit / project pins

def test_covariance_matches_numpy_both_layouts():
    img = synth.small_case(C=12, H=16, W=14, sigma=1.5, seed=4)
    mean, cov = oracle.covariance(img.X)
    Xm = img.X.reshape(12, -1).astype(np.float64)
    np.testing.assert_allclose(mean, Xm.mean(1), rtol=0, atol=1e-12)
    np.testing.assert_allclose(cov, np.cov(Xm, bias=True), rtol=0, atol=1e-12)
    mean2, cov2 = oracle.covariance(np.transpose(img.X, (1, 2, 0)), layout=oracle.NHWC)
    np.testing.assert_allclose(cov2, cov, rtol=0, atol=1e-13)
    np.testing.assert_allclose(mean2, mean, rtol=0, atol=1e-14)


@pytest.mark.parametrize("C,d", [(8, 3), (40, 10), (64, 16)])
def test_jacobi_matches_lapack(C, d):
    rng = np.random.default_rng(C)
    A = rng.standard_normal((C, 3 * C))
    S = A @ A.T / (3 * C)
    V, ev, allev = oracle.eigh_topd(S, d)
    w, U = np.linalg.eigh(S)
    w, U = w[::-1], U[:, ::-1]
    np.testing.assert_allclose(allev, w, rtol=1e-12, atol=1e-12 * w[0])
    gaps = np.abs(np.diff(w))
    for k in range(d):
        u = U[:, k]
        u = u * (1.0 if u[np.argmax(np.abs(u))] > 0 else -1.0)
        gap = min(gaps[k - 1] if k > 0 else np.inf, gaps[k])
        assert np.max(np.abs(V[:, k] - u)) < 1e-11 / gap
        # canonical sign: the largest-magnitude entry is positive
        assert V[np.argmax(np.abs(V[:, k])), k] > 0
    np.testing.assert_allclose(V.T @ V, np.eye(d), atol=1e-12)
    np.testing.assert_allclose(S @ V, V * ev[None, :], atol=1e-11)


def test_planted_spectrum_recovers_axes():
    # X = Q diag(sqrt(lam)) Z with white Z: the principal axes are Q's columns
    rng = np.random.default_rng(9)
    C, d = 10, 4
    Q = synth.random_orthogonal(rng, C)
    lam = np.array([9.0, 6.0, 4.0, 2.5] + [0.5] * (C - 4))
    N = 200_000
    Z = rng.standard_normal((C, N))
    X = (Q * np.sqrt(lam)[None, :]) @ Z
    X = X.reshape(C, 400, 500).astype(np.float32)
    mean, V, ev, _ = oracle.fit(X, d)
    np.testing.assert_allclose(ev, lam[:d], rtol=0.02)
    for k in range(d):
        assert abs(abs(V[:, k] @ Q[:, k]) - 1.0) < 5e-3


def test_projection_selection_basis_closed_form():
    # V = columns of the identity selecting channels (3, 0, 5): Y_k = x_sel(k) - mean
    img = synth.small_case(C=7, H=9, W=11, sigma=1.0, seed=1)
    sel = [3, 0, 5]
    V = np.zeros((7, 3))
    for k, c in enumerate(sel):
        V[c, k] = 1.0
    mean = img.X.reshape(7, -1).astype(np.float64).mean(1)
    Y = oracle.project(img.X, mean, V)
    for k, c in enumerate(sel):
        np.testing.assert_array_equal(Y[k], img.X[c].astype(np.float64) - mean[c])
    # NHWC gives the same result
    Y2 = oracle.project(np.transpose(img.X, (1, 2, 0)), mean, V, layout=oracle.NHWC)
    np.testing.assert_array_equal(Y2, Y)


def test_projection_general_basis_against_matmul():
    img = synth.small_case(C=6, H=5, W=4, sigma=1.0, seed=8)
    rng = np.random.default_rng(0)
    V = rng.standard_normal((6, 2))
    mean = rng.standard_normal(6)
    Y = oracle.project(img.X, mean, V)
    Xc = img.X.reshape(6, -1).astype(np.float64) - mean[:, None]
    np.testing.assert_allclose(Y.reshape(2, -1), V.T @ Xc, rtol=0, atol=1e-12)


def test_fit_layout_invariance_and_residual():
    img = synth.small_case(C=16, H=20, W=18, sigma=1.5, seed=6)
    m1, V1, e1, a1 = oracle.fit(img.X, 5)
    m2, V2, e2, a2 = oracle.fit(np.transpose(img.X, (1, 2, 0)), 5, layout=oracle.NHWC)
    np.testing.assert_allclose(V1, V2, atol=1e-10)
    np.testing.assert_allclose(e1, e2, rtol=1e-12)
    _, cov = oracle.covariance(img.X)
    np.testing.assert_allclose(cov @ V1, V1 * e1[None, :], atol=1e-12)
    assert np.all(np.diff(a1) <= 0)


# ----------------------------------------------------------------- pipeline sanity

def test_pipeline_detects_planted_square():
    img = synth.make_image("plain_128_c64", 0)
    out = oracle.pipeline(img.X, d=16, B=16, r=4)
    assert out["R"].sum(axis=1).tolist() == [128 * 128] * 16
    a = auroc(out["score"], img.mask)
    assert a > 0.9, a


# ----------------------------------------------------------------- AUROC metric pins

def test_auroc_against_pair_counting_and_sklearn():
    rng = np.random.default_rng(0)
    s = rng.integers(0, 6, size=200).astype(float)  # many ties
    m = (rng.random(200) < 0.3).astype(np.uint8)
    pos, neg = s[m == 1], s[m == 0]
    pairs = (pos[:, None] > neg[None, :]).sum() + 0.5 * (pos[:, None] == neg[None, :]).sum()
    assert abs(auroc(s, m) - pairs / (len(pos) * len(neg))) < 1e-12
    skm = pytest.importorskip("sklearn.metrics")
    assert abs(auroc(s, m) - skm.roc_auc_score(m, s)) < 1e-12
