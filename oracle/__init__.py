"""FP64 CPU oracle for the QFCA hot path -- TEST INFRASTRUCTURE ONLY.

Only the test suite, ``__graft_entry__.smoke()`` and the benchmark's CPU
baseline leg may import this package.  The product path (the CUDA library and
its binding) never imports, links or calls it, and it imports nothing from the
product package.

The arithmetic lives in ``qfca_oracle.c`` (plain C, FP64, following the
paper's definitions step by step); this module compiles it with gcc when
needed and wraps it with ctypes.  Every function cites the passage of
arXiv 2510.15602 it follows.

Parity status: ``fit`` (Sec. 3.3), ``project`` (Sec. 3.3), ``quantize``
(Sec. 3.1), ``ref_hist`` and ``score`` (Sec. 3.1, supplement's Wasserstein
closed form), ``alg1`` (Algorithm 1; the supplement's correctness proof) and
``assoc`` (Sec. 3.1's error-to-pixel association, the final blur) and
``median_ref`` (Sec. 3.2's median reference) and ``residual`` (Sec. 3.3's
QFCA+ features) are each
pinned by tests against closed forms, library routines, brute force and
hand-worked cases (tests/test_oracle_pins.py, tests/test_oracle_golden.py and
the assoc, median and residual pin files); tests/test_oracle_mutants.py checks
that planted mistakes fail those pins.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "qfca_oracle.c")
_LIB_PATH = os.path.join(_HERE, "_build", "liboracle.so")
_lib = None
_lock = threading.Lock()

NCHW = 0
NHWC = 1


def build(force: bool = False) -> str:
    """Compile the oracle's C source into ``oracle/_build/liboracle.so``."""
    os.makedirs(os.path.dirname(_LIB_PATH), exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-ffp-contract=off", "-std=c99",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB_PATH)
            P = ctypes.c_void_p
            I = ctypes.c_int
            L = ctypes.c_long
            lib.orc_covariance.argtypes = [P, I, I, I, I, P, P]
            lib.orc_covariance.restype = None
            lib.orc_eigh_topd.argtypes = [P, I, I, P, P, P]
            lib.orc_eigh_topd.restype = I
            lib.orc_fit.argtypes = [P, I, I, I, I, I, P, P, P, P, P]
            lib.orc_fit.restype = I
            lib.orc_project.argtypes = [P, I, I, I, I, P, P, I, P]
            lib.orc_project.restype = None
            lib.orc_quantize.argtypes = [P, I, L, I, I, P, P, I, P, P, P]
            lib.orc_quantize.restype = None
            lib.orc_ref_hist.argtypes = [P, I, L, I, P]
            lib.orc_ref_hist.restype = None
            lib.orc_window_hist.argtypes = [P, I, I, I, I, I, I, P]
            lib.orc_window_hist.restype = L
            lib.orc_score.argtypes = [P, I, I, I, I, I, P, ctypes.c_uint64, P, P, P, P, P]
            lib.orc_score.restype = I
            lib.orc_score_at.argtypes = [P, I, I, I, I, I, P, ctypes.c_uint64, I, I, P]
            lib.orc_score_at.restype = ctypes.c_double
            lib.orc_alg1.argtypes = [P, P, I, ctypes.c_int64, ctypes.c_int64, P]
            lib.orc_alg1_values.argtypes = [P, P, I, ctypes.c_int64, ctypes.c_int64, P, P]
            lib.orc_alg1_values.restype = I
            lib.orc_alg1.restype = I
            lib.orc_assoc.argtypes = [P, I, I, I, I, I, P, ctypes.c_uint64, ctypes.c_double, P, P, P, P, P]
            lib.orc_assoc.restype = I
            lib.orc_blur.argtypes = [P, I, I, ctypes.c_double, P]
            lib.orc_blur.restype = I
            lib.orc_median_ref.argtypes = [P, I, I, I, I, I, P]
            lib.orc_median_ref.restype = I
            lib.orc_residual.argtypes = [P, I, I, I, I, P, P, I, P]
            lib.orc_residual.restype = None
            _lib = lib
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _fmap(X: np.ndarray, layout: int):
    X = np.ascontiguousarray(X, dtype=np.float32)
    if layout == NCHW:
        C, H, W = X.shape
    else:
        H, W, C = X.shape
    return X, C, H, W


def covariance(X: np.ndarray, layout: int = NCHW):
    """Mean and 1/N covariance of the channels (Sec. 3.3, single-image PCA)."""
    X, C, H, W = _fmap(X, layout)
    mean = np.zeros(C, np.float64)
    cov = np.zeros((C, C), np.float64)
    _load().orc_covariance(_p(X), layout, H, W, C, _p(mean), _p(cov))
    return mean, cov


def eigh_topd(S: np.ndarray, d: int):
    """Cyclic-Jacobi eigendecomposition, top-d descending, sign-normalised."""
    S = np.ascontiguousarray(S, dtype=np.float64)
    C = S.shape[0]
    V = np.zeros((C, d), np.float64)
    ev = np.zeros(d, np.float64)
    allev = np.zeros(C, np.float64)
    rc = _load().orc_eigh_topd(_p(S), C, d, _p(V), _p(ev), _p(allev))
    if rc < 0:
        raise MemoryError("oracle eigh_topd")
    return V, ev, allev


def fit(X: np.ndarray, d: int, layout: int = NCHW):
    """PCA fit on one image (Sec. 3.3): returns mean[C], V[C,d], eigvals[d], all eigvals[C]."""
    X, C, H, W = _fmap(X, layout)
    mean = np.zeros(C, np.float64)
    V = np.zeros((C, d), np.float64)
    ev = np.zeros(d, np.float64)
    allev = np.zeros(C, np.float64)
    rc = _load().orc_fit(_p(X), layout, H, W, C, d, _p(mean), _p(V), _p(ev), _p(allev), None)
    if rc < 0:
        raise MemoryError("oracle fit")
    return mean, V, ev, allev


def project(X: np.ndarray, mean: np.ndarray, V: np.ndarray, layout: int = NCHW) -> np.ndarray:
    """Principal components Y[k, y, x] = sum_c (x_c - mean_c) V[c, k] in FP64 (Sec. 3.3)."""
    X, C, H, W = _fmap(X, layout)
    mean = np.ascontiguousarray(mean, np.float64)
    V = np.ascontiguousarray(V, np.float64)
    d = V.shape[1]
    Y = np.zeros((d, H, W), np.float64)
    _load().orc_project(_p(X), layout, H, W, C, _p(mean), _p(V), d, _p(Y))
    return Y


def quantize(Y: np.ndarray, B: int, lo=None, hi=None, fp32_decision: bool = False):
    """Uniform quantisation into B bins (Sec. 3.1).

    With ``lo``/``hi`` None the range is each component's image-wide min/max,
    otherwise the given fixed range (values clamped).  Returns (q uint8
    [d,H,W], lo[d], hi[d]).
    """
    Y = np.ascontiguousarray(Y, np.float64)
    d = Y.shape[0]
    N = int(np.prod(Y.shape[1:]))
    q = np.zeros(Y.shape, np.uint8)
    lo_out = np.zeros(d, np.float64)
    hi_out = np.zeros(d, np.float64)
    mode = 0 if lo is None else 1
    lo_in = np.ascontiguousarray(lo if lo is not None else np.zeros(d), np.float64)
    hi_in = np.ascontiguousarray(hi if hi is not None else np.zeros(d), np.float64)
    _load().orc_quantize(_p(Y), d, N, B, mode, _p(lo_in), _p(hi_in), int(bool(fp32_decision)),
                         _p(lo_out), _p(hi_out), _p(q))
    return q, lo_out, hi_out


def ref_hist(q: np.ndarray, B: int) -> np.ndarray:
    """Reference histogram R[k, b] = #pixels of component k in bin b."""
    q = np.ascontiguousarray(q, np.uint8)
    d = q.shape[0]
    N = int(np.prod(q.shape[1:]))
    R = np.zeros((d, B), np.uint32)
    _load().orc_ref_hist(_p(q), d, N, B, _p(R))
    return R


def window_hist(qk: np.ndarray, B: int, r: int, y: int, x: int):
    """Histogram of one component plane over the clipped window of (y, x) (Sec. 3.1).

    Returns (L int64 [B], N_loc).
    """
    qk = np.ascontiguousarray(qk, np.uint8)
    H, W = qk.shape
    L = np.zeros(B, np.int64)
    n = _load().orc_window_hist(_p(qk), H, W, B, r, y, x, _p(L))
    return L, int(n)


def _ranges(lo, hi, d):
    if lo is None:
        return None, None
    lo = np.ascontiguousarray(np.asarray(lo, np.float64).reshape(d))
    hi = np.ascontiguousarray(np.asarray(hi, np.float64).reshape(d))
    return lo, hi


def score(q: np.ndarray, B: int, r: int, R: np.ndarray, Nref: int | None = None, lo=None, hi=None):
    """Window histograms + 1-D EMD to R + mean over components (Sec. 3.1, Sec. 3).

    Bin units by default; with each component's quantisation range lo/hi [d]
    the EMD is in value units (distances of the quantized values, the cost of
    Algorithm 1 as Sec. 3.1 states it).
    Returns (score float64 [H,W], numer int64 [d,H,W] (bin units), nloc int32 [H,W]).
    """
    q = np.ascontiguousarray(q, np.uint8)
    d, H, W = q.shape
    R = np.ascontiguousarray(R, np.uint32)
    if Nref is None:
        Nref = int(R[0].sum())
    s = np.zeros((H, W), np.float64)
    numer = np.zeros((d, H, W), np.int64)
    nloc = np.zeros((H, W), np.int32)
    lo, hi = _ranges(lo, hi, d)
    rc = _load().orc_score(_p(q), d, H, W, B, r, _p(R), int(Nref), _p(s), _p(numer), _p(nloc),
                           None if lo is None else _p(lo), None if hi is None else _p(hi))
    if rc < 0:
        raise MemoryError("oracle score")
    return s, numer, nloc


def score_at(q: np.ndarray, B: int, r: int, R: np.ndarray, Nref: int, y: int, x: int):
    """One pixel of `score`: (score float64, numer int64 [d]) at (y, x)."""
    q = np.ascontiguousarray(q, np.uint8)
    d, H, W = q.shape
    R = np.ascontiguousarray(R, np.uint32)
    numer = np.zeros(d, np.int64)
    s = _load().orc_score_at(_p(q), d, H, W, B, r, _p(R), int(Nref), int(y), int(x), _p(numer))
    if s < 0:
        raise MemoryError("oracle score_at")
    return s, numer


def alg1(P: np.ndarray, R: np.ndarray, Nloc: int | None = None, Nref: int | None = None):
    """Algorithm 1 (Sec. 3.1) on one window histogram P against the reference R.

    Masses are made equal by scaling (P * N_ref, R * N_loc).  Returns
    (Enum int64 [B], steps): Enum[i] is the mass-weighted transport distance
    charged to bin i (bin units); E_i = Enum[i] / (P[i] * N_ref).
    """
    P = np.ascontiguousarray(P, np.int64)
    R = np.ascontiguousarray(R, np.int64)
    B = P.shape[0]
    Nloc = int(P.sum()) if Nloc is None else int(Nloc)
    Nref = int(R.sum()) if Nref is None else int(Nref)
    En = np.zeros(B, np.int64)
    steps = _load().orc_alg1(_p(P), _p(R), B, Nloc, Nref, _p(En))
    if steps < 0:
        raise MemoryError("oracle alg1")
    return En, int(steps)


def alg1_values(P: np.ndarray, R: np.ndarray, Qv: np.ndarray, Nloc: int | None = None, Nref: int | None = None):
    """Algorithm 1 with the cost in value units: transported amounts charged at
    |Q_i - Q_j| (Qv [B] the quantized values).  Returns (Ev float64 [B], steps)."""
    P = np.ascontiguousarray(P, np.int64)
    R = np.ascontiguousarray(R, np.int64)
    Qv = np.ascontiguousarray(Qv, np.float64)
    B = P.shape[0]
    Nloc = int(P.sum()) if Nloc is None else int(Nloc)
    Nref = int(R.sum()) if Nref is None else int(Nref)
    Ev = np.zeros(B, np.float64)
    steps = _load().orc_alg1_values(_p(P), _p(R), B, Nloc, Nref, _p(Qv), _p(Ev))
    if steps < 0:
        raise MemoryError("oracle alg1_values")
    return Ev, int(steps)


def residual(X: np.ndarray, mean: np.ndarray, V: np.ndarray, layout: int = NCHW) -> np.ndarray:
    """QFCA+ features (Sec. 3.3): X minus its PCA reconstruction from the columns
    of V, F[c, y, x] = (x_c - mean_c) - sum_k V[c, k] y_k, in FP64."""
    X, C, H, W = _fmap(X, layout)
    mean = np.ascontiguousarray(mean, np.float64)
    V = np.ascontiguousarray(V, np.float64)
    dres = V.shape[1]
    F = np.zeros((C, H, W), np.float64)
    _load().orc_residual(_p(X), layout, H, W, C, _p(mean), _p(V), dres, _p(F))
    return F


def pipeline_plus(X: np.ndarray, dres: int, B: int, r: int, layout: int = NCHW):
    """QFCA+ on one image: fit dres components, residual features over all C
    channels, per-channel quantisation, global histograms, window EMD."""
    mean, V, ev, allev = fit(X, dres, layout)
    F = residual(X, mean, V, layout)
    q, lo, hi = quantize(F, B)
    R = ref_hist(q, B)
    H, W = q.shape[1:]
    s, numer, nloc = score(q, B, r, R, H * W)
    return dict(mean=mean, V=V, all_eigvals=allev, F=F, q=q, lo=lo, hi=hi, R=R, score=s, numer=numer)


def median_ref(q: np.ndarray, B: int, r: int) -> np.ndarray:
    """The median reference (Sec. 3.2): per component, the lower median over all
    full windows of each rank's value, as a histogram R [d, B] with N_ref = (2r+1)^2."""
    q = np.ascontiguousarray(q, np.uint8)
    d, H, W = q.shape
    R = np.zeros((d, B), np.uint32)
    rc = _load().orc_median_ref(_p(q), d, H, W, B, r, _p(R))
    if rc == -2:
        raise ValueError("no full window: H and W must exceed 2r")
    if rc < 0:
        raise MemoryError("oracle median_ref")
    return R


def blur(a: np.ndarray, sigma: float) -> np.ndarray:
    """Gaussian smoothing of a map (the final low-pass step with sigma_s): separable,
    taps |t| <= ceil(4 sigma), weights renormalised over the taps inside the image."""
    a = np.ascontiguousarray(a, np.float64)
    H, W = a.shape
    out = np.zeros_like(a)
    if _load().orc_blur(_p(a), H, W, float(sigma), _p(out)) < 0:
        raise MemoryError("oracle blur")
    return out


def assoc(q: np.ndarray, B: int, r: int, R: np.ndarray, Nref: int | None = None, sigma_s: float = 1.0,
          lo=None, hi=None):
    """The paper's scoring: Algorithm 1 per window and component, error-to-pixel
    association (each pixel averages its own bin's error over the windows that
    contain it, sigma_p = infinity), mean over components, Gaussian blur sigma_s
    (Sec. 3.1 and its association paragraph; smoothing as in the sigma_s study).
    Bin units by default; value units with each component's range lo/hi [d].

    Returns (score float64 [H,W], raw float64 [H,W] before the blur,
    comp float64 [d,H,W] per-component associated errors).
    """
    q = np.ascontiguousarray(q, np.uint8)
    d, H, W = q.shape
    R = np.ascontiguousarray(R, np.uint32)
    if Nref is None:
        Nref = int(R[0].sum())
    s = np.zeros((H, W), np.float64)
    raw = np.zeros((H, W), np.float64)
    comp = np.zeros((d, H, W), np.float64)
    lo, hi = _ranges(lo, hi, d)
    rc = _load().orc_assoc(_p(q), d, H, W, B, r, _p(R), int(Nref), float(sigma_s), _p(raw), _p(s), _p(comp),
                           None if lo is None else _p(lo), None if hi is None else _p(hi))
    if rc < 0:
        raise MemoryError("oracle assoc")
    return s, raw, comp


def pipeline(X: np.ndarray, d: int, B: int, r: int, layout: int = NCHW):
    """The whole path on one image: fit, project, quantize, ref hist, score."""
    mean, V, ev, allev = fit(X, d, layout)
    Y = project(X, mean, V, layout)
    q, lo, hi = quantize(Y, B)
    R = ref_hist(q, B)
    H, W = q.shape[1:]
    s, numer, nloc = score(q, B, r, R, H * W)
    return dict(mean=mean, V=V, eigvals=ev, all_eigvals=allev, Y=Y, q=q, lo=lo, hi=hi, R=R,
                score=s, numer=numer, nloc=nloc)
