"""GPU parity: the CUDA path through the C ABI against the FP64 CPU oracle.

Tolerances:
  * integer stages (window histograms, EMD numerators, reference histogram,
    bins given identical inputs): bit-exact;
  * FP32 projection: |Y_gpu - Y_oracle| <= 1e-5 * max_p |Y_oracle[k]| per
    component; a bin may differ from the oracle's only where the oracle value
    lies within 1e-5 * range of a bin edge;
  * bins from the GPU's own Y: identical to the oracle's FP32-precision
    decision on the same values (both decide in FP32);
  * score: the GPU rounds the exact sum_k D_k / (d N_loc N_ref) once to FP32,
    so it is within one FP32 rounding (2^-23 relative) of the FP64 oracle;
  * covariance: the GPU represents each element as a 27-bit fixed-point
    number of its channel's power-of-two range R_c (|x| < R_c <= 2 max|x|) and
    sums digit products exactly except the dropped products of digit levels
    >= 4 (<= 3 * 64^2 * 2^-40 R_i R_j each), so |Sigma_gpu - Sigma_oracle|_ij
    <= 2^-25 R_i R_j (representation of both factors, of the mean, and the
    dropped levels) -- tested elementwise;
  * fit: eigenvalues within 1e-8 relative and eigenvectors within
    1e-8 ||Sigma|| / gap_k + 1e-10 (first-order perturbation of the
    covariance error above), far inside the 1e-5 projection tolerance;
  * BF16 projection: <= 1% bin flips and pixel AUROC within 0.005.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2510_15602_gb300 import synth
from paper_2510_15602_gb300.metrics import auroc
from tests.gpu_helpers import bins_np, edge_distance, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def q():
    from paper_2510_15602_gb300 import qfca
    assert torch.cuda.is_available()
    return qfca


# ------------------------------------------------------------------ window histogram + EMD (integer, bit-exact)

@pytest.mark.parametrize("d,H,W,B,r,seed", [
    (3, 70, 150, 16, 4, 0),     # several tiles, ragged in both directions
    (2, 33, 129, 32, 7, 1),     # one row past a band, one column past a strip
    (1, 5, 7, 8, 4, 2),         # window larger than the image
    (2, 1, 40, 16, 3, 3),       # a single row
    (2, 40, 1, 16, 3, 4),       # a single column
    (4, 64, 96, 64, 12, 5),     # B=64, r=12
    (2, 50, 60, 255, 2, 6),     # maximum bin count
])
def test_score_bit_exact_numerators(q, d, H, W, B, r, seed):
    rng = np.random.default_rng(seed)
    qb = synth.random_bins(rng, d, H, W, B, smooth=(seed % 2 == 0))
    R = oracle.ref_hist(qb, B)
    s_o, num_o, _ = oracle.score(qb, B, r, R, H * W)
    pitch = q.bins_pitch(W)
    bins = torch.zeros(d, H, pitch, dtype=torch.uint8, device="cuda")
    bins[:, :, :W] = to_dev(qb)
    s_g, num_g = q.score(bins, W, B, r, to_dev(R.astype(np.int32)), H * W, want_numer=True)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(num_g.cpu().numpy(), num_o)
    np.testing.assert_allclose(s_g.cpu().numpy(), s_o, rtol=2.0 ** -23, atol=1e-12)


@pytest.mark.parametrize("d,H,W,B,r,seed", [
    (2, 192, 200, 255, 12, 0),   # (B-1)(2r+1)^2 N_ref >= 2^32: 64-bit CDF walk
    (1, 600, 610, 255, 63, 1),   # widest window; N_ref (2r+1)^2 >= 2^32; narrow strips
    (3, 300, 260, 64, 9, 2),     # compile-time B = 64 path with ragged bands and strips
])
def test_score_wide_and_large_windows_sampled(q, d, H, W, B, r, seed):
    # exact numerators at sampled pixels (corners, edges, interior), each
    # computed one by one by the oracle
    rng = np.random.default_rng(100 + seed)
    qb = synth.random_bins(rng, d, H, W, B, smooth=True)
    R = oracle.ref_hist(qb, B)
    bins = torch.zeros(d, H, q.bins_pitch(W), dtype=torch.uint8, device="cuda")
    bins[:, :, :W] = to_dev(qb)
    s_g, num_g = q.score(bins, W, B, r, to_dev(R.astype(np.int32)), H * W, want_numer=True)
    torch.cuda.synchronize()
    s_g, num_g = s_g.cpu().numpy(), num_g.cpu().numpy()
    pts = [(0, 0), (0, W - 1), (H - 1, 0), (H - 1, W - 1), (r, r), (H // 2, W // 2)]
    pts += [(int(y), int(x)) for y, x in zip(rng.integers(0, H, 40), rng.integers(0, W, 40))]
    for y, x in pts:
        s_o, n_o = oracle.score_at(qb, B, r, R, H * W, y, x)
        np.testing.assert_array_equal(num_g[:, y, x].astype(np.int64), n_o)
        assert abs(s_g[y, x] - s_o) <= 2.0 ** -23 * abs(s_o) + 1e-12


def test_score_bins_above_range_clamp_to_last_bin(q):
    # input bins >= B count as bin B-1 (documented for qfca_score)
    d, H, W, B, r = 2, 40, 70, 16, 3
    rng = np.random.default_rng(7)
    qb = synth.random_bins(rng, d, H, W, B, smooth=False)
    raw = qb.copy()
    hi = rng.random((d, H, W)) < 0.2
    raw[hi & (qb == B - 1)] = rng.integers(B, 256, size=int(np.sum(hi & (qb == B - 1))))
    R = oracle.ref_hist(qb, B)
    _, num_o, _ = oracle.score(qb, B, r, R, H * W)
    bins = torch.zeros(d, H, q.bins_pitch(W), dtype=torch.uint8, device="cuda")
    bins[:, :, :W] = to_dev(raw)
    _, num_g = q.score(bins, W, B, r, to_dev(R.astype(np.int32)), H * W, want_numer=True)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(num_g.cpu().numpy(), num_o)


def test_score_external_reference_point_masses(q):
    # reference = point mass at bin 9 (mass 1000), map = constant bin 2: EMD = 7 everywhere
    d, H, W, B, r = 2, 20, 30, 16, 3
    bins = torch.full((d, H, q.bins_pitch(W)), 2, dtype=torch.uint8, device="cuda")
    R = torch.zeros(d, B, dtype=torch.int32, device="cuda")
    R[:, 9] = 1000
    s = q.score(bins, W, B, r, R, 1000)
    torch.cuda.synchronize()
    assert torch.all(s == 7.0)


# ------------------------------------------------------------------ projection + quantisation (oracle basis fed in)

def _case(C, H, W, seed):
    return synth.small_case(C=C, H=H, W=W, sigma=2.0, seed=seed, n_square=2, side=8, nch=6)


@pytest.mark.parametrize("C,H,W,d,B,layout", [
    (64, 128, 128, 16, 16, 0),
    (256, 45, 77, 32, 32, 0),   # ragged pixel count
    (40, 30, 50, 8, 16, 1),     # NHWC, C not a multiple of 32
    (512, 24, 40, 32, 64, 0),
])
def test_project_quantize_against_oracle(q, C, H, W, d, B, layout):
    img = _case(C, H, W, seed=C + H)
    X = img.X if layout == 0 else np.ascontiguousarray(np.transpose(img.X, (1, 2, 0)))
    mean, V, ev, _ = oracle.fit(img.X, d)
    Y_o = oracle.project(img.X, mean, V)
    qb_o, lo_o, hi_o = oracle.quantize(Y_o, B)
    Xd = to_dev(X)
    out = q.quantize(Xd, (to_dev(mean), to_dev(V)), B, "f32", layout=layout, want_Y=True)
    torch.cuda.synchronize()
    Y_g = out["Y"].cpu().numpy().astype(np.float64)
    scale = np.abs(Y_o).reshape(d, -1).max(axis=1)
    err = np.abs(Y_g - Y_o).reshape(d, -1).max(axis=1)
    assert np.all(err <= 1e-5 * scale), (err / scale).max()
    qb_g = bins_np(out["bins"], W)
    # same-precision decision on the GPU's own Y: bit-exact
    qb_f32, lo_f, hi_f = oracle.quantize(Y_g, B, fp32_decision=True)
    np.testing.assert_array_equal(qb_g, qb_f32)
    np.testing.assert_array_equal(out["lo"].cpu().numpy(), lo_f.astype(np.float32))
    np.testing.assert_array_equal(out["hi"].cpu().numpy(), hi_f.astype(np.float32))
    # against the FP64 oracle: flips only next to a bin edge
    flip = qb_g != qb_o
    if flip.any():
        dist = edge_distance(Y_o, lo_o, hi_o, B)
        assert np.all(dist[flip] <= 1e-5), dist[flip].max()
    # reference histogram: bit-exact on the GPU's bins
    np.testing.assert_array_equal(out["hist"].cpu().numpy().astype(np.uint32), oracle.ref_hist(qb_g, B))


def test_quantize_fixed_range_clamps(q):
    img = _case(32, 20, 24, seed=3)
    mean, V, _, _ = oracle.fit(img.X, 4)
    Y_o = oracle.project(img.X, mean, V)
    lo = np.quantile(Y_o.reshape(4, -1), 0.1, axis=1).astype(np.float32)
    hi = np.quantile(Y_o.reshape(4, -1), 0.9, axis=1).astype(np.float32)
    out = q.quantize(to_dev(img.X), (to_dev(mean), to_dev(V)), 16, "f32", lo=to_dev(lo), hi=to_dev(hi),
                     want_Y=True)
    torch.cuda.synchronize()
    Y_g = out["Y"].cpu().numpy().astype(np.float64)
    exp, _, _ = oracle.quantize(Y_g, 16, lo=lo.astype(np.float64), hi=hi.astype(np.float64), fp32_decision=True)
    np.testing.assert_array_equal(bins_np(out["bins"], 24), exp)
    assert (exp == 0).any() and (exp == 15).any()


def test_quantize_histogram_of_constant_and_blocky_components(q):
    # a zero basis column makes its component constant (hi == lo: every pixel in bin 0), the others
    # come from a smooth field: whole warps share a bin, the counting groups lanes by bin
    img = _case(48, 64, 96, seed=21)
    mean, V, _, _ = oracle.fit(img.X, 6)
    V[:, 2] = 0.0
    for W in (96, 93):  # four pixels per thread, and the per-pixel route for a ragged width
        X = np.ascontiguousarray(img.X[:, :, :W])
        out = q.quantize(to_dev(X), (to_dev(mean), to_dev(V)), 32, "f32", want_Y=True)
        torch.cuda.synchronize()
        Y_g = out["Y"].cpu().numpy().astype(np.float64)
        exp, _, _ = oracle.quantize(Y_g, 32, fp32_decision=True)
        qb = bins_np(out["bins"], W)
        np.testing.assert_array_equal(qb, exp)
        hist = out["hist"].cpu().numpy().astype(np.uint32)
        np.testing.assert_array_equal(hist, oracle.ref_hist(qb, 32))
        assert hist[2, 0] == 64 * W and hist.sum() == 6 * 64 * W


@pytest.mark.parametrize("lo,hi,B", [(-2.7, 3.1, 32), (-1e-3, 5e-4, 64), (0.0, 1.0, 16), (10.0, 13.0, 255)])
def test_quantize_at_the_bin_edges(q, lo, hi, B):
    # values exactly at every bin edge and at the floats on either side of it, through a one-hot
    # basis (the projection returns the values themselves) and a fixed range: the bins must be the
    # FP32 decision taken per value on the host
    from tests.quant_edges import decision, edges
    lo, hi = np.float32(lo), np.float32(hi)
    e = edges(lo, hi, B)
    vals = np.concatenate([e, np.nextafter(e, np.float32(-np.inf)), np.nextafter(e, np.float32(np.inf)),
                           np.array([lo, hi, -np.inf, np.inf, 0.0, -0.0], dtype=np.float32)])
    vals = vals[np.isfinite(vals)]
    W = 64
    H = -(-vals.size // W)
    C = 4
    X = np.zeros((C, H, W), dtype=np.float32)
    X[0].reshape(-1)[:vals.size] = vals
    X[1] = 7.0  # weighed by zero in the basis
    mean = np.zeros(C)
    V = np.zeros((C, 1))
    V[0, 0] = 1.0
    out = q.quantize(to_dev(X), (to_dev(mean), to_dev(V)), B, "f32", lo=to_dev(np.array([lo], np.float32)),
                     hi=to_dev(np.array([hi], np.float32)), want_Y=True)
    torch.cuda.synchronize()
    Y = out["Y"].cpu().numpy().reshape(1, H, W)
    np.testing.assert_array_equal(Y[0], X[0])
    exp = np.array([decision(y, lo, hi, B) for y in X[0].reshape(-1)]).reshape(1, H, W)
    np.testing.assert_array_equal(bins_np(out["bins"], W), exp)


# ------------------------------------------------------------------ PCA fit (FP64)

@pytest.mark.parametrize("C,H,W,d,layout", [
    (64, 128, 128, 16, 0),
    (256, 40, 52, 32, 0),
    (48, 30, 33, 12, 1),
    (2, 9, 7, 2, 0),
])
def test_fit_against_oracle(q, C, H, W, d, layout):
    img = _case(C, H, W, seed=7 * C + d)
    X = img.X if layout == 0 else np.ascontiguousarray(np.transpose(img.X, (1, 2, 0)))
    mean_o, V_o, ev_o, all_o = oracle.fit(img.X, d)
    mean_g, V_g, ev_g = q.fit_pca(to_dev(X), d, layout=layout)
    torch.cuda.synchronize()
    mean_g, V_g, ev_g = mean_g.cpu().numpy(), V_g.cpu().numpy(), ev_g.cpu().numpy()
    Rc = 2.0 ** np.ceil(np.log2(np.abs(img.X).reshape(C, -1).max(axis=1) * (1 + 2 ** -23)))
    np.testing.assert_array_less(np.abs(mean_g - mean_o), 2.0 ** -27 * Rc + 1e-15)
    # |dlambda| <= ||dSigma||_2 <= C * max_ij |dSigma_ij| <= C * 2^-25 * max R^2
    ev_tol = C * 2.0 ** -25 * Rc.max() ** 2
    assert np.all(np.abs(ev_g - ev_o) <= ev_tol), (np.abs(ev_g - ev_o).max(), ev_tol)
    gaps = np.abs(np.diff(all_o))
    for k in range(d):
        gap = min(gaps[k - 1] if k > 0 else np.inf, gaps[k] if k < C - 1 else np.inf)
        err = np.max(np.abs(V_g[:, k] - V_o[:, k]))
        assert err < 1e-8 * all_o[0] / gap + 1e-10, (k, err, gap)


@pytest.mark.parametrize("C,H,W,layout", [(64, 128, 128, 0), (256, 45, 77, 0), (130, 20, 30, 1), (512, 32, 40, 0)])
def test_covariance_exact_slices_against_oracle(q, C, H, W, layout):
    img = _case(C, H, W, seed=C + W)
    X = img.X if layout == 0 else np.ascontiguousarray(np.transpose(img.X, (1, 2, 0)))
    mean_o, cov_o = oracle.covariance(img.X)
    mean_g, cov_g = q.covariance(to_dev(X), layout=layout)
    torch.cuda.synchronize()
    mean_g, cov_g = mean_g.cpu().numpy(), cov_g.cpu().numpy()
    Rc = 2.0 ** np.ceil(np.log2(np.abs(img.X).reshape(C, -1).max(axis=1) * (1 + 2 ** -23)))
    bound = 2.0 ** -25 * np.outer(Rc, Rc) + 1e-14 * np.abs(cov_o).max()
    assert np.all(np.abs(cov_g - cov_o) <= bound), np.max(np.abs(cov_g - cov_o) / bound)
    np.testing.assert_array_equal(cov_g, cov_g.T)
    np.testing.assert_array_less(np.abs(mean_g - mean_o), 2.0 ** -27 * Rc + 1e-15)


# ------------------------------------------------------------------ the whole path

@pytest.mark.parametrize("layout", [0, 1])
def test_pipeline_fp32_plain_128_c64(q, layout):
    img = synth.make_image("plain_128_c64", 0)
    d, B, r = 16, 16, 4
    ref = oracle.pipeline(img.X, d, B, r)
    X = img.X if layout == 0 else np.ascontiguousarray(np.transpose(img.X, (1, 2, 0)))
    Xd = to_dev(X)
    basis = q.fit_pca(Xd, d, layout=layout)
    out = q.quantize(Xd, basis, B, "f32", layout=layout, want_Y=True)
    s, num = q.score(out["bins"], 128, B, r, out["hist"], 128 * 128, want_numer=True)
    torch.cuda.synchronize()
    Y_g = out["Y"].cpu().numpy().astype(np.float64)
    scale = np.abs(ref["Y"]).reshape(d, -1).max(axis=1)
    assert np.all(np.abs(Y_g - ref["Y"]).reshape(d, -1).max(axis=1) <= 1e-5 * scale)
    qb_g = bins_np(out["bins"], 128)
    flip = qb_g != ref["q"]
    if flip.any():
        assert np.all(edge_distance(ref["Y"], ref["lo"], ref["hi"], B)[flip] <= 1e-5)
    # integer stages bit-exact on the GPU's bins
    R_g = oracle.ref_hist(qb_g, B)
    s_o, num_o, _ = oracle.score(qb_g, B, r, R_g, 128 * 128)
    np.testing.assert_array_equal(num.cpu().numpy(), num_o)
    np.testing.assert_allclose(s.cpu().numpy(), s_o, rtol=2.0 ** -23, atol=1e-12)
    a_g, a_o = auroc(s.cpu().numpy(), img.mask), auroc(ref["score"], img.mask)
    assert abs(a_g - a_o) < 1e-3 and a_g > 0.9


def test_pipeline_full_size_256_c256_sampled(q):
    # one full-size image of the 16 x 256^2 x C256 workload
    img = synth.make_image("batch16_256_c256", 0)
    d, B, r = 32, 32, 7
    mean_o, V_o, ev_o, _ = oracle.fit(img.X, d)
    Xd = to_dev(img.X)
    mean_g, V_g, ev_g = q.fit_pca(Xd, d)
    out = q.quantize(Xd, (mean_g, V_g), B, "f32", want_Y=True)
    s = q.score(out["bins"], 256, B, r, out["hist"], 256 * 256)
    torch.cuda.synchronize()
    np.testing.assert_allclose(ev_g.cpu().numpy(), ev_o, rtol=1e-8)
    assert np.max(np.abs(V_g.cpu().numpy() - V_o)) < 1e-5
    # projection at 4096 sampled pixels, computed one by one by the oracle
    rng = np.random.default_rng(0)
    idx = rng.choice(256 * 256, 4096, replace=False)
    Xs = img.X.reshape(256, -1)[:, idx].reshape(256, 64, 64)
    Y_o = oracle.project(Xs, mean_o, V_o).reshape(d, -1)
    Y_g = out["Y"].reshape(d, -1)[:, torch.from_numpy(idx).cuda()].cpu().numpy()
    scale = np.abs(Y_o).max(axis=1)
    assert np.all(np.abs(Y_g - Y_o).max(axis=1) <= 1e-5 * scale)
    # integer stages: the oracle's window EMD on the GPU's bins, full image
    qb = bins_np(out["bins"], 256)
    R = oracle.ref_hist(qb, B)
    np.testing.assert_array_equal(out["hist"].cpu().numpy().astype(np.uint32), R)
    s_o, _, _ = oracle.score(qb, B, r, R, 256 * 256)
    np.testing.assert_allclose(s.cpu().numpy(), s_o, rtol=2.0 ** -23, atol=1e-12)


# ------------------------------------------------------------------ argument validation through the ABI

def test_invalid_arguments_rejected(q):
    X = torch.zeros(8, 4, 4, device="cuda")
    with pytest.raises(q.QfcaError) as e:
        q.fit_pca(X, 9)  # d > C
    assert e.value.status == q.ERR_INVALID_ARG
    bins = torch.zeros(2, 4, 16, dtype=torch.uint8, device="cuda")
    R = torch.zeros(2, 8, dtype=torch.int32, device="cuda")
    with pytest.raises(q.QfcaError):
        q.score(bins, 4, 8, 0, R, 16)  # r = 0
    with pytest.raises(q.QfcaError):
        q.score(bins, 4, 1, 1, R, 16)  # B = 1


# ------------------------------------------------------------------ BF16 projection on tcgen05

def bf16_round(a):
    """Round to the nearest BF16 (ties to even), returned as float32."""
    u = np.ascontiguousarray(a, np.float32).view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32)


@pytest.mark.parametrize("C,H,W,d,layout", [
    (256, 45, 77, 32, 0),   # ragged pixel count (last tile partial)
    (64, 128, 128, 16, 0),
    (512, 24, 40, 64, 0),   # 8 K-chunks, N = 64
    (40, 30, 50, 8, 1),     # NHWC, C padded to 64
    (200, 16, 17, 32, 1),
])
def test_project_bf16_matches_rounded_operands(q, C, H, W, d, layout):
    # the tensor-core result equals the FP64 sum of the same BF16-rounded
    # operands up to FP32 accumulation: checks operand layouts, swizzle,
    # descriptors and the TMEM read-back element by element
    img = _case(C, H, W, seed=C * 3 + W)
    X = img.X if layout == 0 else np.ascontiguousarray(np.transpose(img.X, (1, 2, 0)))
    mean, V, _, _ = oracle.fit(img.X, d)
    out = q.quantize(to_dev(X), (to_dev(mean), to_dev(V)), 16, "bf16", layout=layout, want_Y=True)
    torch.cuda.synchronize()
    Xc = bf16_round(img.X.reshape(C, -1) - mean.astype(np.float32)[:, None]).astype(np.float64)
    Vb = bf16_round(V.astype(np.float32)).astype(np.float64)
    Y_ref = (Vb.T @ Xc).reshape(d, H, W)
    bound = (np.abs(Vb).T @ np.abs(Xc)).reshape(d, H, W) * 1e-6 + 1e-30
    Y_g = out["Y"].cpu().numpy().astype(np.float64)
    assert np.all(np.abs(Y_g - Y_ref) <= bound), np.max(np.abs(Y_g - Y_ref) / bound)
    # bins still decided in FP32 on the kernel's own Y
    qb, _, _ = oracle.quantize(Y_g, 16, fp32_decision=True)
    np.testing.assert_array_equal(bins_np(out["bins"], W), qb)


def test_bf16_flips_and_auroc_plain_128_c64(q):
    img = synth.make_image("plain_128_c64", 0)
    d, B, r = 16, 16, 4
    ref = oracle.pipeline(img.X, d, B, r)
    Xd = to_dev(img.X)
    basis = q.fit_pca(Xd, d)
    out = q.quantize(Xd, basis, B, "bf16", want_Y=True)
    s = q.score(out["bins"], 128, B, r, out["hist"], 128 * 128)
    torch.cuda.synchronize()
    flips = float((bins_np(out["bins"], 128) != ref["q"]).mean())
    assert flips <= 0.01, flips
    a_g, a_o = auroc(s.cpu().numpy(), img.mask), auroc(ref["score"], img.mask)
    assert abs(a_g - a_o) <= 0.005, (a_g, a_o)


def test_bf16_flips_and_auroc_full_size_image(q):
    img = synth.make_image("batch16_256_c256", 1)
    d, B, r = 32, 32, 7
    mean_o, V_o, _, _ = oracle.fit(img.X, d)
    Y_o = oracle.project(img.X, mean_o, V_o)
    qb_o, _, _ = oracle.quantize(Y_o, B)
    R_o = oracle.ref_hist(qb_o, B)
    s_o, _, _ = oracle.score(qb_o, B, r, R_o, 256 * 256)
    Xd = to_dev(img.X)
    basis = q.fit_pca(Xd, d)
    out = q.quantize(Xd, basis, B, "bf16")
    s = q.score(out["bins"], 256, B, r, out["hist"], 256 * 256)
    torch.cuda.synchronize()
    flips = float((bins_np(out["bins"], 256) != qb_o).mean())
    assert flips <= 0.01, flips
    a_g, a_o = auroc(s.cpu().numpy(), img.mask), auroc(s_o, img.mask)
    assert abs(a_g - a_o) <= 0.005, (a_g, a_o)


def test_device_status_clean_after_bf16(q):
    ctx = q.default_context()
    img = _case(64, 32, 32, seed=2)
    mean, V, _, _ = oracle.fit(img.X, 16)
    q.quantize(to_dev(img.X), (to_dev(mean), to_dev(V)), 16, "bf16", ctx=ctx)
    assert ctx.device_status() == 0


# ------------------------------------------------------------------ batched entry point

@pytest.mark.parametrize("precision", ["f32", "bf16"])
def test_batch_run_equals_single_image_calls(q, precision):
    # every stage of qfca_batch_run shares one grid across the batch; the
    # results must equal per-image calls bit for bit (integer stages are exact
    # and order-independent, the floating stages use the same per-image order)
    C, H, W, d, B, r, n = 64, 48, 40, 16, 16, 4, 3
    imgs = [synth.small_case(C=C, H=H, W=W, sigma=2.0, seed=50 + i, n_square=1, side=8, nch=6) for i in range(n)]
    Xb = to_dev(np.stack([im.X for im in imgs]))
    sb, ex = q.batch_run(Xb, d, B, r, precision, extras=True)
    torch.cuda.synchronize()
    for i in range(n):
        basis = q.fit_pca(Xb[i], d)
        out = q.quantize(Xb[i], basis, B, precision)
        s1 = q.score(out["bins"], W, B, r, out["hist"], H * W)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(ex["eigvals"][i].cpu().numpy(), basis[2].cpu().numpy())
        np.testing.assert_array_equal(ex["V"][i].cpu().numpy(), basis[1].cpu().numpy())
        np.testing.assert_array_equal(ex["bins"][i][:, :, :W].cpu().numpy(), out["bins"][:, :, :W].cpu().numpy())
        np.testing.assert_array_equal(sb[i].cpu().numpy(), s1.cpu().numpy())


def test_batch_run_full_size_against_oracle_integer_stages(q):
    # two images of the 256^2 x C256 workload through the batch path; integer
    # stages of each image checked bit-exactly against the oracle on the GPU bins
    imgs = [synth.make_image("batch16_256_c256", i) for i in range(2)]
    Xb = to_dev(np.stack([im.X for im in imgs]))
    sb, ex = q.batch_run(Xb, 32, 32, 7, "bf16", extras=True)
    torch.cuda.synchronize()
    for i in range(2):
        qb = ex["bins"][i][:, :, :256].cpu().numpy()
        R = oracle.ref_hist(qb, 32)
        np.testing.assert_array_equal(ex["ref_hist"][i].cpu().numpy().astype(np.uint32), R)
        s_o, _, _ = oracle.score(qb, 32, 7, R, 256 * 256)
        np.testing.assert_allclose(sb[i].cpu().numpy(), s_o, rtol=2.0 ** -23, atol=1e-12)


# ------------------------------------------------------------------ uneven batch (one launch per stage over an image table)

def _uneven_images(C, sizes, seed0):
    return [synth.small_case(C=C, H=h, W=w, sigma=2.0, seed=seed0 + i, n_square=1, side=8, nch=6)
            for i, (h, w) in enumerate(sizes)]


@pytest.mark.parametrize("precision", ["bf16", "f32"])
def test_score_batch_uneven_equals_single_image_calls(q, precision):
    # sizes and radii differ per image; the table-driven launches must give
    # each image exactly what the single-image entry points give it
    C, d, B = 64, 16, 64
    sizes = [(96, 104), (64, 72), (120, 88), (48, 160)]
    rs = [5, 7, 9, 12]
    imgs = _uneven_images(C, sizes, 70)
    Xs = [to_dev(im.X) for im in imgs]
    ctx = q.Context()
    sb = q.score_batch(Xs, rs, d, B, precision, ctx=ctx)
    torch.cuda.synchronize()
    for i, (X, (H, W), r) in enumerate(zip(Xs, sizes, rs)):
        basis = q.fit_pca(X, d, ctx=ctx)
        out = q.quantize(X, basis, B, precision, ctx=ctx)
        s1 = q.score(out["bins"], W, B, r, out["hist"], H * W, ctx=ctx)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(sb[i].cpu().numpy(), s1.cpu().numpy())
    assert ctx.device_status() == 0


def test_score_batch_uneven_c512_equals_single_image_calls(q):
    # C = 512 (the float-float cluster solver, the TMA projection's image cursor over a table of
    # mixed sizes, B = 64, mixed radii): the batch equals the single-image calls bit for bit
    C, d, B = 512, 32, 64
    sizes = [(40, 48), (32, 56), (48, 40)]
    rs = [5, 12, 9]
    imgs = _uneven_images(C, sizes, 130)
    Xs = [to_dev(im.X) for im in imgs]
    ctx = q.Context()
    sb = q.score_batch(Xs, rs, d, B, "bf16", ctx=ctx)
    torch.cuda.synchronize()
    for i, (X, (H, W), r) in enumerate(zip(Xs, sizes, rs)):
        basis = q.fit_pca(X, d, ctx=ctx)
        out = q.quantize(X, basis, B, "bf16", ctx=ctx)
        s1 = q.score(out["bins"], W, B, r, out["hist"], H * W, ctx=ctx)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(sb[i].cpu().numpy(), s1.cpu().numpy())
    assert ctx.device_status() == 0


def test_score_batch_uneven_integer_stages_against_oracle(q):
    # one image of the batch checked end to end: eigenvalues against the
    # oracle's fit, and the oracle's window EMD on the GPU's own bins
    C, d, B = 64, 16, 64
    sizes = [(72, 80), (104, 96)]
    rs = [7, 5]
    imgs = _uneven_images(C, sizes, 90)
    Xs = [to_dev(im.X) for im in imgs]
    sb = q.score_batch(Xs, rs, d, B, "f32")
    torch.cuda.synchronize()
    for i, (X, (H, W), r) in enumerate(zip(Xs, sizes, rs)):
        basis = q.fit_pca(X, d)
        out = q.quantize(X, basis, B, "f32")
        torch.cuda.synchronize()
        qb = bins_np(out["bins"], W)
        R = oracle.ref_hist(qb, B)
        s_o, _, _ = oracle.score(qb, B, r, R, H * W)
        np.testing.assert_allclose(sb[i].cpu().numpy(), s_o, rtol=2.0 ** -23, atol=1e-12)


def test_score_batch_autotune_keeps_results(q):
    C, d, B = 64, 16, 32
    sizes = [(80, 96), (96, 64), (64, 64)]
    rs = [7, 5, 9]
    imgs = _uneven_images(C, sizes, 110)
    Xs = [to_dev(im.X) for im in imgs]
    ctx = q.Context()
    s_model = [s.clone() for s in q.score_batch(Xs, rs, d, B, "bf16", ctx=ctx)]
    model_tiling = ctx.last_tiling()
    ctx.set_autotune(True)
    s_tuned = q.score_batch(Xs, rs, d, B, "bf16", ctx=ctx)
    tuned = ctx.last_tiling()
    s_again = q.score_batch(Xs, rs, d, B, "bf16", ctx=ctx)
    torch.cuda.synchronize()
    assert tuned[0] in (64, 128) and 1 <= tuned[1] <= 64 and 1 <= tuned[2] <= d
    assert ctx.last_tiling() == tuned  # cached for the same shapes
    assert model_tiling[0] in (64, 128)
    for a, b, c in zip(s_model, s_tuned, s_again):
        np.testing.assert_array_equal(a.cpu().numpy(), b.cpu().numpy())
        np.testing.assert_array_equal(a.cpu().numpy(), c.cpu().numpy())


def test_score_batch_rejects_bad_arguments(q):
    X = to_dev(synth.small_case(C=16, H=16, W=16, sigma=1.0, seed=1, n_square=0, side=4, nch=2).X)
    with pytest.raises(q.QfcaError):
        q.score_batch([X], [0], 4, 16)          # r < 1
    with pytest.raises(q.QfcaError):
        q.score_batch([X], [64], 4, 16)         # 2r+1 > 127
    with pytest.raises(q.QfcaError):
        q.score_batch([X], [3], 4, 1)           # B < 2
    with pytest.raises(ValueError):
        q.score_batch([X], [3, 4], 4, 16)       # one radius per image


# ------------------------------------------------------------------ FP8 (e4m3) projection

def _e4m3(a):
    return torch.from_numpy(np.ascontiguousarray(a, np.float32)).to(torch.float8_e4m3fn).to(torch.float32).numpy()


def _fp8_operands(X, mean, V):
    """The documented FP8 operands, from the same inputs: per-channel and
    per-component power-of-two scales, e4m3 A and the e4m3 hi + lo basis."""
    C = X.shape[0]
    amax = np.abs(X.reshape(C, -1)).max(axis=1).astype(np.float32).astype(np.float64)
    bound = amax + np.abs(mean)
    s = np.where(bound > 0, np.exp2(np.floor(np.log2(448.0 / np.where(bound > 0, bound, 1.0)))), 1.0)
    m = (np.abs(V) / s[:, None]).max(axis=0)
    t = np.where(m > 0, np.exp2(np.floor(np.log2(448.0 / np.where(m > 0, m, 1.0)))), 1.0)
    b = (V / s[:, None] * t[None, :]).astype(np.float32)
    hi = _e4m3(b)
    lo = _e4m3(b - hi)
    xc = (X.reshape(C, -1).astype(np.float32) - mean.astype(np.float32)[:, None]) * s.astype(np.float32)[:, None]
    A = _e4m3(xc.astype(np.float32))
    return A.astype(np.float64), (hi.astype(np.float64) + lo.astype(np.float64)) / t[None, :]


@pytest.mark.parametrize("C,H,W,d", [(64, 40, 48, 16), (256, 32, 64, 32), (200, 24, 40, 64), (512, 16, 32, 32)])
def test_project_fp8_matches_rounded_operands(q, C, H, W, d):
    # tcgen05 kind::f8f6f4 result equals the FP64 sum of the same e4m3 operands
    # up to FP32 accumulation: checks scales, packing, 128-channel chunk
    # assembly, descriptors and the epilogue's component scale element by element
    img = _case(C, H, W, seed=C * 5 + W)
    mean, V, _, _ = oracle.fit(img.X, d)
    out = q.quantize(to_dev(img.X), (to_dev(mean), to_dev(V)), 16, "fp8", want_Y=True)
    torch.cuda.synchronize()
    A, Bm = _fp8_operands(img.X, mean, V)
    Y_ref = (Bm.T @ A).reshape(d, H, W)
    bound = (np.abs(Bm).T @ np.abs(A)).reshape(d, H, W) * 1e-6 + 1e-30
    Y_g = out["Y"].cpu().numpy().astype(np.float64)
    assert np.all(np.abs(Y_g - Y_ref) <= bound), np.max(np.abs(Y_g - Y_ref) / bound)
    qb, _, _ = oracle.quantize(Y_g, 16, fp32_decision=True)
    np.testing.assert_array_equal(bins_np(out["bins"], W), qb)


def test_fp8_precision_sweep_plain_128_c64(q):
    # precision sweep on the single-image workload: FP32 / BF16 / FP8 projection
    # against the FP64 oracle (bin flips, score error, AUROC)
    img = synth.make_image("plain_128_c64", 0)
    d, B, r = 16, 16, 4
    ref = oracle.pipeline(img.X, d, B, r)
    Xd = to_dev(img.X)
    basis = q.fit_pca(Xd, d)
    res = {}
    for prec in ("f32", "bf16", "fp8"):
        out = q.quantize(Xd, basis, B, prec)
        s = q.score(out["bins"], 128, B, r, out["hist"], 128 * 128)
        torch.cuda.synchronize()
        sg = s.cpu().numpy()
        res[prec] = dict(flips=float((bins_np(out["bins"], 128) != ref["q"]).mean()),
                         max_err=float(np.abs(sg - ref["score"]).max()),
                         auroc=auroc(sg, img.mask))
    a_o = auroc(ref["score"], img.mask)
    print("precision sweep", res, "oracle auroc", a_o)
    assert res["f32"]["flips"] <= res["bf16"]["flips"] <= res["fp8"]["flips"]
    # measured on GB300: flips 0 / 0.45% / 5.2%, AUROC within 0.002 of the oracle for all three
    assert res["f32"]["flips"] <= 1e-3 and res["bf16"]["flips"] <= 0.01 and res["fp8"]["flips"] <= 0.08
    assert abs(res["fp8"]["auroc"] - a_o) <= 0.01 and abs(res["bf16"]["auroc"] - a_o) <= 0.005
