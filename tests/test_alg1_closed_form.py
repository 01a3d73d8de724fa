"""The closed form of Algorithm 1 (Sec. 3.1) that the association kernel evaluates,
checked in exact integers against the oracle's two-pointer walk.

On the common mass axis [0, N_loc N_ref), local bin i holds [a_i, b_i) =
[N_ref cumP_i, N_ref cumP_{i+1}) and reference bin j holds [N_loc cumR_j,
N_loc cumR_{j+1}) (cum* exclusive prefix sums).  The walk moves the mass at
position s from local bin i to the reference bin J(s) containing s, so

    Enum_i = F_i(b_i) - F_i(a_i),  F_i(t) = int_0^t |i - J(s)| ds
           = N_loc T[i][J] + |i - J| (t - N_loc cumR_J),  J = J(t),
    T[i][x] = sum_{j < x} |i - j| R_j,

and for full-size windows (N_loc the same for every window) the two terms fold
into one table, F_i(t) = U[i][J] + |i - J| t with U[i][J] = N_loc T[i][J] -
|i - J| N_loc cumR_J.  F is continuous, so J may be taken on either side of a
boundary.  This file restates the formula independently of the CUDA source.
"""
import numpy as np
import pytest

import oracle


def closed_form(P, R, Nloc, Nref, folded=False):
    B = len(P)
    cumP = np.concatenate([[0], np.cumsum(P)]).astype(object)
    cumR = np.concatenate([[0], np.cumsum(R)]).astype(object)
    T = [[sum(abs(i - j) * int(R[j]) for j in range(x)) for x in range(B + 1)] for i in range(B)]
    U = [[Nloc * T[i][x] - abs(i - x) * Nloc * cumR[x] for x in range(B + 1)] for i in range(B)]

    def J(t, right):
        # the reference bin containing position t (the right one on a boundary when right=True)
        j = 0
        while j < B - 1 and (Nloc * cumR[j + 1] < t or (right and Nloc * cumR[j + 1] == t)):
            j += 1
        return j

    def F(i, t, right):
        j = J(t, right)
        if folded:
            return U[i][j] + abs(i - j) * t
        return Nloc * T[i][j] + abs(i - j) * (t - Nloc * cumR[j])

    out = []
    for i in range(B):
        a, b = Nref * cumP[i], Nref * cumP[i + 1]
        out.append(F(i, b, False) - F(i, a, True))
    return np.array(out, dtype=np.int64)


@pytest.mark.parametrize("seed", range(6))
def test_closed_form_equals_the_walk(seed):
    rng = np.random.default_rng(seed)
    for _ in range(40):
        B = int(rng.integers(2, 24))
        # sparse and dense histograms, windows and references of different totals
        P = rng.integers(0, 6, B) * (rng.random(B) < 0.6)
        R = rng.integers(0, 9, B) * (rng.random(B) < 0.8)
        if P.sum() == 0:
            P[rng.integers(B)] = 1
        if R.sum() == 0:
            R[rng.integers(B)] = 1
        Nloc, Nref = int(P.sum()), int(R.sum())
        walk, _ = oracle.alg1(P, R, Nloc, Nref)
        np.testing.assert_array_equal(closed_form(P, R, Nloc, Nref), walk)
        np.testing.assert_array_equal(closed_form(P, R, Nloc, Nref, folded=True), walk)


def test_boundary_side_does_not_matter():
    # F is continuous: evaluating J on either side of a reference boundary gives the same value
    P, R = np.array([2, 0, 1, 3]), np.array([1, 2, 2, 1])
    Nloc, Nref = int(P.sum()), int(R.sum())
    walk, _ = oracle.alg1(P, R, Nloc, Nref)
    np.testing.assert_array_equal(closed_form(P, R, Nloc, Nref), walk)
