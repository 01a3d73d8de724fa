"""Pins of the oracle's QFCA+ residual (arXiv 2510.15602, Sec. 3.3) against
facts of the eigendecomposition fixed independently (numpy/LAPACK): the
residual is orthogonal to the kept components, its energy is N times the sum
of the dropped eigenvalues, and the extreme component counts reduce to closed
forms.  CPU only."""
import numpy as np
import pytest

import oracle
from paper_2510_15602_gb300 import synth


@pytest.fixture(scope="module")
def case():
    img = synth.small_case(12, 20, 22, 2.0, seed=5)
    return img.X  # [C, H, W] float32


@pytest.mark.parametrize("dres", [1, 3, 7])
def test_residual_orthogonal_and_energy(case, dres):
    X = case
    C, H, W = X.shape
    mean, V, ev, allev = oracle.fit(X, dres)
    F = oracle.residual(X, mean, V)
    Fm = F.reshape(C, -1)
    # orthogonal to the kept components
    assert np.abs(V.T @ Fm).max() < 1e-10 * np.abs(Fm).max()
    # energy: sum_p |F_p|^2 = N * sum of the dropped eigenvalues of the 1/N covariance (LAPACK)
    Xc = X.reshape(C, -1).astype(np.float64)
    Xc = Xc - Xc.mean(axis=1, keepdims=True)
    lam = np.sort(np.linalg.eigvalsh(Xc @ Xc.T / Xc.shape[1]))[::-1]
    assert (Fm ** 2).sum() == pytest.approx(Xc.shape[1] * lam[dres:].sum(), rel=1e-9)
    # F = X - mean - reconstruction, checked with a matmul
    np.testing.assert_allclose(Fm, Xc - V @ (V.T @ Xc), rtol=0, atol=1e-9 * np.abs(Xc).max())


def test_residual_extremes(case):
    X = case
    C = X.shape[0]
    mean, V, _, _ = oracle.fit(X, C)
    F = oracle.residual(X, mean, V)
    assert np.abs(F).max() < 1e-9 * np.abs(X).max()  # all components kept: nothing left
    Z = np.zeros((C, 0))
    F0 = oracle.residual(X, mean, Z)
    np.testing.assert_allclose(F0, X - mean[:, None, None], rtol=0, atol=1e-12)  # none kept: centred features


def _brute_qfca_plus(X, dres, B, r):
    """QFCA+ on a tiny image from the definitions alone: the 1/N covariance and its top dres
    eigenvectors (LAPACK), the residual from the projector onto them (independent of their
    signs and of rotations inside the kept subspace), B uniform bins over each channel's own
    range, each channel's global histogram as its reference, and per pixel the W1 distance
    between the clipped window's histogram and the reference (both normalised, unit bin
    spacing) as a sum over bins of the absolute difference of the CDFs, averaged over the C
    planes."""
    C, H, W = X.shape
    Xc = X.reshape(C, -1).astype(np.float64)
    Xc = Xc - Xc.mean(axis=1, keepdims=True)
    lam, U = np.linalg.eigh(Xc @ Xc.T / Xc.shape[1])
    Vk = U[:, np.argsort(lam)[::-1][:dres]]
    F = (Xc - Vk @ (Vk.T @ Xc)).reshape(C, H, W)
    lo, hi = F.reshape(C, -1).min(axis=1), F.reshape(C, -1).max(axis=1)
    q = np.zeros((C, H, W), np.int64)
    for c in range(C):
        t = (F[c] - lo[c]) / (hi[c] - lo[c]) * B if hi[c] > lo[c] else np.zeros((H, W))
        q[c] = np.clip(np.floor(t), 0, B - 1)
    s = np.zeros((H, W))
    for c in range(C):
        ref = np.bincount(q[c].ravel(), minlength=B) / (H * W)
        for y in range(H):
            for x in range(W):
                win = q[c, max(0, y - r):y + r + 1, max(0, x - r):x + r + 1].ravel()
                loc = np.bincount(win, minlength=B) / win.size
                s[y, x] += np.abs(np.cumsum(loc) - np.cumsum(ref)).sum() / C
    return F, lo, hi, q, s


@pytest.mark.parametrize("dres,B,r", [(2, 5, 1), (4, 8, 2), (0, 6, 3)])
def test_pipeline_plus_against_definitions(dres, B, r):
    # a small image whose covariance has distinct eigenvalues around the cut (the residual is
    # then well defined), 7 x 9 pixels so windows clip at every border
    X = synth.small_case(7, 7, 9, 1.0, seed=31 + dres).X
    F_b, lo_b, hi_b, q_b, s_b = _brute_qfca_plus(X, dres, B, r)
    out = oracle.pipeline_plus(X, dres, B, r)
    np.testing.assert_allclose(out["F"], F_b, rtol=0, atol=1e-10 * np.abs(F_b).max())
    np.testing.assert_allclose(out["lo"], lo_b, rtol=0, atol=1e-10)
    np.testing.assert_allclose(out["hi"], hi_b, rtol=0, atol=1e-10)
    # the bins agree exactly: no value of these images lies within the residual's rounding of
    # an interior edge (each channel's minimum and maximum sit on the outer edges, t = 0 and
    # t = B, whose bins are not in doubt)
    t = (F_b - lo_b[:, None, None]) / (hi_b - lo_b)[:, None, None] * B
    k = np.round(t)
    assert not ((np.abs(t - k) < 1e-8) & (k > 0) & (k < B)).any()
    np.testing.assert_array_equal(out["q"], q_b)
    np.testing.assert_array_equal(out["R"], np.stack([np.bincount(qc.ravel(), minlength=B) for qc in q_b]))
    np.testing.assert_allclose(out["score"], s_b, rtol=1e-12, atol=1e-15)
