"""The exact-integer covariance method of the PCA fit (Sec. 3.3) checked on the
CPU, independently of the CUDA source: each channel is scaled by its power-of-two
range R_c = 2^e_c (max |x| < R_c), rounded to 27-bit fixed point and written as
four signed 7-bit digits, y = sum_i d_i 2^(-6-7i), d_i in [-64, 64]; the Gram is
formed from the digit-level sums A_L = sum_{i+j=L} sum_p d_i d_j for L = 0..3
(plus the level-4 products on the diagonal), and

    Sigma_ij = R_i R_j T_ij 2^-40 / N - mu_i mu_j,   T = sum_L A_L 2^(7(4-L)).

Claims checked: the digits are exact integers in [-64, 64] that reconstruct the
fixed-point value; partial sums over a 512-pixel window stay within 2^23 (so an
FP32 accumulator holds them exactly); and the covariance is within
2^-25 R_i R_j of the FP64 definition."""
import numpy as np
import pytest


def digits(y27):
    """Balanced base-128 digits of integers |y27| <= 2^26: y27 = d0 2^21 + d1 2^14 + d2 2^7 + d3."""
    out = []
    rest = y27.astype(np.int64)
    for w in (21, 14, 7, 0):
        d = np.floor(rest / 2.0 ** w + 0.5).astype(np.int64) if w else rest.copy()
        out.append(d)
        rest = rest - d * (1 << w)
    assert (rest == 0).all()
    return out


def gram_cov(X):
    C, N = X.shape
    amax = np.abs(X).max(axis=1)
    e = np.ceil(np.log2(np.maximum(amax, 1e-300) * (1 + 2.0 ** -23))).astype(int)  # max|x| < 2^e
    y27 = np.rint(X.astype(np.float64) * 2.0 ** (27 - e)[:, None]).astype(np.int64)
    D = digits(y27)
    for d in D:
        assert np.abs(d).max() <= 64
    # level sums over 512-pixel windows: every partial sum <= 2^23 (exact in FP32)
    for L in range(4):
        for p0 in range(0, N, 512):
            AL = sum(D[i][:, p0:p0 + 512] @ D[L - i][:, p0:p0 + 512].T for i in range(L + 1))
            assert np.abs(AL).max() <= 2 ** 23
    T = np.zeros((C, C), dtype=object)
    for L in range(4):
        AL = sum(D[i] @ D[L - i].T for i in range(L + 1))
        T = T + AL.astype(object) * (1 << (7 * (4 - L)))
    # level 4 on the diagonal: 2 d1 d3 + d2^2 (units 2^-40 exactly)
    diag4 = (2 * D[1] * D[3] + D[2] * D[2]).sum(axis=1)
    for c in range(C):
        T[c, c] += int(diag4[c])
    S = np.array([[float(T[i, j]) for j in range(C)] for i in range(C)]) * 2.0 ** -40
    Rr = 2.0 ** e
    mu = Rr * (y27.sum(axis=1) * 2.0 ** -27) / N
    Sigma = np.outer(Rr, Rr) * S / N - np.outer(mu, mu)
    return Sigma, Rr


@pytest.mark.parametrize("seed,C,N", [(0, 8, 1000), (1, 12, 777), (2, 5, 4096)])
def test_digit_gram_within_bound(seed, C, N):
    rng = np.random.default_rng(seed)
    scales = 2.0 ** rng.uniform(-6, 6, C)                 # channels of very different ranges
    X = (rng.standard_normal((C, N)) * scales[:, None] + rng.normal(0, 1, C)[:, None] * scales[:, None])
    X = X.astype(np.float32)
    Sigma, Rr = gram_cov(X)
    Xd = X.astype(np.float64)
    ref = np.cov(Xd, bias=True)
    bound = 2.0 ** -25 * np.outer(Rr, Rr)
    assert (np.abs(Sigma - ref) <= bound).all(), (np.abs(Sigma - ref) / bound).max()


@pytest.mark.parametrize("seed,C,N", [(3, 9, 1500), (4, 16, 640)])
def test_symmetric_form_of_a_diagonal_tile(seed, C, N):
    """A diagonal tile (the block against itself) keeps only the symmetric part of the
    level sums: Y_L = sum over i <= j, i + j = L of c_ij D_i D_j^T with c_ij = 1 (i < j)
    and 1/2 (i = j); then Y_L + Y_L^T equals the full level sum exactly, and every
    partial sum of Y_L over a 512-pixel window is a half-integer of magnitude <= 2^22
    (exact in an FP32 accumulator, and twice it converts exactly to an integer)."""
    rng = np.random.default_rng(seed)
    X = (rng.standard_normal((C, N)) * 2.0 ** rng.uniform(-4, 4, C)[:, None]).astype(np.float32)
    amax = np.abs(X).max(axis=1)
    e = np.ceil(np.log2(amax * (1 + 2.0 ** -23))).astype(int)
    D = digits(np.rint(X.astype(np.float64) * 2.0 ** (27 - e)[:, None]).astype(np.int64))
    for L in range(4):
        full = sum(D[i] @ D[L - i].T for i in range(L + 1))
        # 2 Y_L in integers: 2 D_i D_j^T for i < j, D_i D_i^T for i = j
        twoY = sum((1 if i == L - i else 2) * (D[i] @ D[L - i].T) for i in range(L + 1) if i <= L - i)
        assert np.array_equal(twoY + twoY.T, 2 * full)
        for p0 in range(0, N, 512):
            sl = slice(p0, p0 + 512)
            tw = sum((1 if i == L - i else 2) * (D[i][:, sl] @ D[L - i][:, sl].T) for i in range(L + 1) if i <= L - i)
            assert np.abs(tw).max() <= 2 ** 23
