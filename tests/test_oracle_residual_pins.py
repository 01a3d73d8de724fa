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
