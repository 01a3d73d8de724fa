"""Thin Python binding over libqfca.so (the C ABI of include/qfca.h).

Argument marshalling only: tensors become device pointers, the current torch
CUDA stream becomes the ``stream`` argument, and every step of the path runs
in the library's CUDA kernels.  PyTorch provides device memory and streams.

Importing this module loads ``libqfca.so`` and raises ImportError when the
library has not been built -- there is no fallback path.
"""
from __future__ import annotations

import ctypes
import os
import re
import threading

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libqfca.so")
HEADER = os.path.join(os.path.dirname(_HERE), "include", "qfca.h")

if not os.path.exists(LIB_PATH):
    raise ImportError(f"{LIB_PATH} is missing: build it with paper_2510_15602_gb300/build.py "
                      "(or __graft_entry__.build()); the QFCA path has no CPU fallback")

_lib = ctypes.CDLL(LIB_PATH)

# status codes and enums (include/qfca.h)
OK, PENDING = 0, 1
ERR_INVALID_ARG, ERR_UNSUPPORTED, ERR_OOM, ERR_CUDA, ERR_TIMEOUT, ERR_BUSY = -1, -2, -3, -4, -5, -6
NCHW, NHWC = 0, 1
F32, BF16, FP8_E4M3 = 0, 1, 2
RANGE_IMAGE, RANGE_FIXED = 0, 1
_PREC = {"f32": F32, "fp32": F32, "bf16": BF16, "fp8": FP8_E4M3, F32: F32, BF16: BF16, FP8_E4M3: FP8_E4M3}


class Fmap(ctypes.Structure):
    _fields_ = [("H", ctypes.c_int), ("W", ctypes.c_int), ("C", ctypes.c_int), ("layout", ctypes.c_int)]


class Basis(ctypes.Structure):
    _fields_ = [("mean", ctypes.c_void_p), ("V", ctypes.c_void_p), ("eigvals", ctypes.c_void_p)]


_P = ctypes.c_void_p
_I = ctypes.c_int
_lib.qfca_create.argtypes = [_I, ctypes.c_size_t, ctypes.POINTER(_P)]
_lib.qfca_create.restype = _I
_lib.qfca_destroy.argtypes = [_P]
_lib.qfca_destroy.restype = _I
_lib.qfca_status_string.argtypes = [_I]
_lib.qfca_status_string.restype = ctypes.c_char_p
_lib.qfca_last_error.argtypes = [_P]
_lib.qfca_last_error.restype = ctypes.c_char_p
_lib.qfca_version.argtypes = []
_lib.qfca_version.restype = ctypes.c_char_p
_lib.qfca_fit_pca.argtypes = [_P, _P, Fmap, _I, ctypes.POINTER(Basis), _P]
_lib.qfca_fit_pca.restype = _I
_lib.qfca_covariance.argtypes = [_P, _P, Fmap, _P, _P, _P]
_lib.qfca_covariance.restype = _I
_lib.qfca_quantize.argtypes = [_P, _P, Fmap, ctypes.POINTER(Basis), _I, _I, _I, _I, _P, _P, _P, _I, _P, _P, _P,
                               _P, _P]
_lib.qfca_quantize.restype = _I
_lib.qfca_score.argtypes = [_P, _P, _I, _I, _I, _I, _I, _I, _P, ctypes.c_uint32, _P, _P, _P, _P, _P]
_lib.qfca_score.restype = _I
_lib.qfca_device_status.argtypes = [_P, ctypes.POINTER(ctypes.c_int)]
_lib.qfca_device_status.restype = _I
_lib.qfca_launch_count.argtypes = [_P, ctypes.POINTER(ctypes.c_uint64)]
_lib.qfca_launch_count.restype = _I
_lib.qfca_trace_start.argtypes = [_P, ctypes.c_char_p]
_lib.qfca_trace_start.restype = _I
_lib.qfca_trace_stop.argtypes = [_P]
_lib.qfca_trace_stop.restype = _I
_lib.qfca_trace_get.argtypes = [_P, _I, ctypes.c_char_p, ctypes.POINTER(ctypes.c_double),
                                ctypes.POINTER(ctypes.c_uint64)]
_lib.qfca_trace_get.restype = _I


class BatchOutputs(ctypes.Structure):
    _fields_ = [("mean", ctypes.c_void_p), ("V", ctypes.c_void_p), ("eigvals", ctypes.c_void_p),
                ("bins", ctypes.c_void_p), ("pitch", ctypes.c_int), ("ref_hist", ctypes.c_void_p),
                ("lo", ctypes.c_void_p), ("hi", ctypes.c_void_p)]


_lib.qfca_batch_run.argtypes = [_P, _P, _I, Fmap, _I, _I, _I, _I, _P, ctypes.POINTER(BatchOutputs), _P]
_lib.qfca_batch_run.restype = _I
_lib.qfca_batch_run_host.argtypes = [_P, _P, _I, Fmap, _I, _I, _I, _I, _P, _P]
_lib.qfca_batch_run_host.restype = _I
_lib.qfca_metrics.argtypes = [_P, _P, _P, _I, _I, _I, _I, ctypes.c_double, _P, _P]
_lib.qfca_metrics.restype = _I
_lib.qfca_batch_run_basis.argtypes = [_P, _P, _I, Fmap, _P, _P, _I, _I, _I, _I, _P, ctypes.POINTER(BatchOutputs), _P]
_lib.qfca_batch_run_basis.restype = _I
_lib.qfca_last_projection_tiling.argtypes = [_P, ctypes.POINTER(_I), ctypes.POINTER(_I)]
_lib.qfca_last_projection_tiling.restype = _I
_lib.qfca_set_tiling.argtypes = [_P, _I, _I, _I]
_lib.qfca_set_tiling.restype = _I
_lib.qfca_set_eig_tolerance.argtypes = [_P, ctypes.c_double]
_lib.qfca_set_eig_tolerance.restype = _I
_lib.qfca_eig_redo_count.argtypes = [_P, ctypes.POINTER(ctypes.c_uint64)]
_lib.qfca_eig_redo_count.restype = _I
_lib.qfca_batch_run_plus.argtypes = [_P, _P, _I, Fmap, _I, _I, _I, _P, ctypes.POINTER(BatchOutputs), _P]
_lib.qfca_batch_run_plus.restype = _I


class Image(ctypes.Structure):
    _fields_ = [("X", ctypes.c_void_p), ("H", ctypes.c_int), ("W", ctypes.c_int), ("r", ctypes.c_int),
                ("score", ctypes.c_void_p)]


_lib.qfca_score_batch.argtypes = [_P, ctypes.POINTER(Image), _I, _I, _I, _I, _I, _I, _P]
_lib.qfca_score_batch.restype = _I
_lib.qfca_score_assoc.argtypes = [_P, _P, _I, _I, _I, _I, _I, _I, _P, ctypes.c_uint32, ctypes.c_float, _P, _P, _P,
                                  _P, _P, _P]
_lib.qfca_score_assoc.restype = _I


class AssocImage(ctypes.Structure):
    _fields_ = [("bins", ctypes.c_void_p), ("H", ctypes.c_int), ("W", ctypes.c_int), ("pitch", ctypes.c_int),
                ("r", ctypes.c_int), ("ref_hist", ctypes.c_void_p), ("ref_total", ctypes.c_uint32),
                ("score", ctypes.c_void_p), ("raw", ctypes.c_void_p), ("lo", ctypes.c_void_p),
                ("hi", ctypes.c_void_p)]


_lib.qfca_score_assoc_batch.argtypes = [_P, ctypes.POINTER(AssocImage), _I, _I, _I, ctypes.c_float, _P]
_lib.qfca_score_assoc_batch.restype = _I
_lib.qfca_quantize_residual.argtypes = [_P, _P, Fmap, ctypes.POINTER(Basis), _I, _I, _P, _I, _P, _P, _P, _P, _P]
_lib.qfca_quantize_residual.restype = _I
_lib.qfca_median_reference.argtypes = [_P, _P, _I, _I, _I, _I, _I, _I, _P, _P]
_lib.qfca_median_reference.restype = _I


class MedianImage(ctypes.Structure):
    _fields_ = [("bins", ctypes.c_void_p), ("H", ctypes.c_int), ("W", ctypes.c_int), ("pitch", ctypes.c_int),
                ("r", ctypes.c_int), ("ref_out", ctypes.c_void_p)]


_lib.qfca_median_reference_batch.argtypes = [_P, ctypes.POINTER(MedianImage), _I, _I, _I, _P]
_lib.qfca_median_reference_batch.restype = _I
_lib.qfca_set_autotune.argtypes = [_P, _I]
_lib.qfca_set_autotune.restype = _I
_lib.qfca_last_tiling.argtypes = [_P, ctypes.POINTER(_I), ctypes.POINTER(_I), ctypes.POINTER(_I)]
_lib.qfca_last_tiling.restype = _I
_lib.qfca_set_cdf_walk.argtypes = [_P, _I]
_lib.qfca_set_cdf_walk.restype = _I
_lib.qfca_last_cdf_walk.argtypes = [_P, ctypes.POINTER(_I)]
_lib.qfca_last_cdf_walk.restype = _I
_lib.qfca_set_band_run.argtypes = [_P, _I]
_lib.qfca_set_band_run.restype = _I
_lib.qfca_last_band_run.argtypes = [_P, ctypes.POINTER(_I)]
_lib.qfca_last_band_run.restype = _I


class ServeConfig(ctypes.Structure):
    _fields_ = [("C", ctypes.c_int), ("d", ctypes.c_int), ("B", ctypes.c_int), ("precision", ctypes.c_int),
                ("max_batch", ctypes.c_int), ("streams", ctypes.c_int), ("max_queue", ctypes.c_int),
                ("arena_bytes", ctypes.c_size_t)]


class Request(ctypes.Structure):
    _fields_ = [("class_id", ctypes.c_int), ("X", ctypes.c_void_p), ("H", ctypes.c_int), ("W", ctypes.c_int),
                ("r", ctypes.c_int), ("score", ctypes.c_void_p), ("flags", ctypes.c_int)]


class Result(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("batch_size", ctypes.c_int), ("t_submit_us", ctypes.c_double),
                ("t_start_us", ctypes.c_double), ("t_done_us", ctypes.c_double), ("stream", ctypes.c_int),
                ("reserved", ctypes.c_int), ("batch_seq", ctypes.c_uint64)]


REQ_HOST_INPUT, REQ_HOST_OUTPUT = 1, 2
_lib.qfca_serve_start.argtypes = [_P, ctypes.POINTER(ServeConfig)]
_lib.qfca_serve_start.restype = _I
_lib.qfca_register_class.argtypes = [_P, _I, _P, _P, _P, _P, _P, ctypes.c_uint32]
_lib.qfca_register_class.restype = _I
_lib.qfca_submit.argtypes = [_P, ctypes.POINTER(Request), ctypes.POINTER(ctypes.c_uint64)]
_lib.qfca_submit.restype = _I
_lib.qfca_poll.argtypes = [_P, ctypes.c_uint64, _I, ctypes.POINTER(Result)]
_lib.qfca_poll.restype = _I
_lib.qfca_serve_stop.argtypes = [_P]
_lib.qfca_serve_stop.restype = _I


class QfcaError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{_lib.qfca_status_string(status).decode()}: {msg}")
        self.status = status


def header_functions() -> list[str]:
    """Names of the functions declared in include/qfca.h."""
    with open(HEADER) as f:
        txt = f.read()
    return sorted(set(re.findall(r"\b(qfca_[a-z0-9_]+)\s*\(", txt)))


def version() -> str:
    return _lib.qfca_version().decode()


class Context:
    """A libqfca context (owns the device workspace)."""

    def __init__(self, device: int | None = None, workspace_bytes: int = 0):
        if device is None:
            device = torch.cuda.current_device()
        self.device = device
        h = _P()
        s = _lib.qfca_create(device, workspace_bytes, ctypes.byref(h))
        if s != OK:
            raise QfcaError(s, "qfca_create failed")
        self.handle = h

    def check(self, s: int):
        if s != OK:
            raise QfcaError(s, _lib.qfca_last_error(self.handle).decode())

    def device_status(self) -> int:
        """Synchronise and read-and-clear the device status word (0 = no kernel timed out)."""
        v = ctypes.c_int()
        s = _lib.qfca_device_status(self.handle, ctypes.byref(v))
        if s not in (OK, ERR_TIMEOUT):
            self.check(s)
        return int(v.value)

    def set_autotune(self, on: bool):
        """Measure the window stage's tilings once per shape set (True) or use the cost model (False)."""
        self.check(_lib.qfca_set_autotune(self.handle, 1 if on else 0))

    def set_tiling(self, strip_width: int = 0, band_height: int = 0, component_groups: int = 0):
        """Force the window stage's tiling for later calls (strip_width 0: cost model / autotuner)."""
        self.check(_lib.qfca_set_tiling(self.handle, int(strip_width), int(band_height), int(component_groups)))

    def set_cdf_walk(self, walk: int = -1):
        """CDF walk of the window stage: -1 the autotuner's choice (per thread without
        autotuning), 0 per thread, 1 warp-shuffle segmented (B = 32, 32-bit numerators)."""
        self.check(_lib.qfca_set_cdf_walk(self.handle, int(walk)))

    def set_band_run(self, bands: int = 1):
        """Bands per CTA of a tiling forced by set_tiling (1 default, 0 every band of a strip)."""
        self.check(_lib.qfca_set_band_run(self.handle, int(bands)))

    def last_band_run(self) -> int:
        """Bands per CTA of the most recent window-stage launch."""
        v = ctypes.c_int()
        self.check(_lib.qfca_last_band_run(self.handle, ctypes.byref(v)))
        return int(v.value)

    def last_cdf_walk(self) -> int:
        """The CDF walk (0 per thread, 1 warp-shuffle) of the most recent window-stage launch."""
        v = ctypes.c_int()
        self.check(_lib.qfca_last_cdf_walk(self.handle, ctypes.byref(v)))
        return int(v.value)

    def last_projection_tiling(self) -> tuple[int, int]:
        """(FP32 boxes in flight, operand chunks) of the most recent TMA-fed projection."""
        a, b = ctypes.c_int(), ctypes.c_int()
        self.check(_lib.qfca_last_projection_tiling(self.handle, ctypes.byref(a), ctypes.byref(b)))
        return int(a.value), int(b.value)

    def last_tiling(self) -> tuple[int, int, int]:
        """(strip width, band height, component groups) of the most recent window-stage launch."""
        a, b, c = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        self.check(_lib.qfca_last_tiling(self.handle, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)))
        return int(a.value), int(b.value), int(c.value)

    def set_eig_tolerance(self, tol: float):
        """Residual bound of the fit's FP32 + Newton eigensolver (relative to the largest
        eigenvalue); 0 sends every matrix to the float-float solver."""
        self.check(_lib.qfca_set_eig_tolerance(self.handle, float(tol)))

    def eig_redo_count(self) -> int:
        """Synchronise; read and clear how many matrices the float-float solver redid."""
        n = ctypes.c_uint64()
        self.check(_lib.qfca_eig_redo_count(self.handle, ctypes.byref(n)))
        return int(n.value)

    def launch_count(self) -> int:
        n = ctypes.c_uint64()
        self.check(_lib.qfca_launch_count(self.handle, ctypes.byref(n)))
        return int(n.value)

    def trace_start(self, kernel_filter: str = ""):
        self.check(_lib.qfca_trace_start(self.handle, kernel_filter.encode()))

    def trace_stop(self):
        self.check(_lib.qfca_trace_stop(self.handle))

    def trace(self) -> dict:
        """{kernel name: (total device ms, launches)} of the current trace."""
        out = {}
        i = 0
        buf = ctypes.create_string_buffer(64)
        ms = ctypes.c_double()
        n = ctypes.c_uint64()
        while _lib.qfca_trace_get(self.handle, i, buf, ctypes.byref(ms), ctypes.byref(n)) == OK:
            out[buf.value.decode()] = (ms.value, int(n.value))
            i += 1
        return out

    def close(self):
        if getattr(self, "handle", None):
            _lib.qfca_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


_ctx_lock = threading.Lock()
_default_ctx: dict[int, Context] = {}


def default_context(device: int | None = None) -> Context:
    if device is None:
        device = torch.cuda.current_device()
    with _ctx_lock:
        if device not in _default_ctx:
            _default_ctx[device] = Context(device)
        return _default_ctx[device]


def _stream_ptr(stream=None) -> int:
    st = stream if stream is not None else torch.cuda.current_stream()
    return st.cuda_stream


def _ptr(t: torch.Tensor | None):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _check_dev(t: torch.Tensor, name: str, dtype: torch.dtype):
    if not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise ValueError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")


def fmap_of(X: torch.Tensor, layout: int = NCHW) -> Fmap:
    if X.dim() != 3:
        raise ValueError("feature map must be 3-D: (C, H, W) for NCHW or (H, W, C) for NHWC")
    if layout == NCHW:
        C, H, W = X.shape
    else:
        H, W, C = X.shape
    return Fmap(int(H), int(W), int(C), int(layout))


def bins_pitch(W: int) -> int:
    return (W + 15) // 16 * 16


def fit_pca(X: torch.Tensor, d: int, layout: int = NCHW, ctx: Context | None = None, stream=None, out=None):
    """qfca_fit_pca: returns (mean[C], V[C, d], eigvals[d]) FP64 device tensors."""
    _check_dev(X, "X", torch.float32)
    fm = fmap_of(X, layout)
    ctx = ctx or default_context(X.device.index)
    if out is None:
        mean = torch.empty(fm.C, dtype=torch.float64, device=X.device)
        V = torch.empty(fm.C, d, dtype=torch.float64, device=X.device)
        ev = torch.empty(d, dtype=torch.float64, device=X.device)
    else:
        mean, V, ev = out
    b = Basis(mean.data_ptr(), V.data_ptr(), ev.data_ptr())
    ctx.check(_lib.qfca_fit_pca(ctx.handle, _ptr(X), fm, d, ctypes.byref(b), _P(_stream_ptr(stream))))
    return mean, V, ev


def covariance(X: torch.Tensor, layout: int = NCHW, ctx: Context | None = None, stream=None):
    """qfca_covariance: returns (mean[C], Sigma[C, C]) FP64 device tensors."""
    _check_dev(X, "X", torch.float32)
    fm = fmap_of(X, layout)
    ctx = ctx or default_context(X.device.index)
    mean = torch.empty(fm.C, dtype=torch.float64, device=X.device)
    cov = torch.empty(fm.C, fm.C, dtype=torch.float64, device=X.device)
    ctx.check(_lib.qfca_covariance(ctx.handle, _ptr(X), fm, _ptr(mean), _ptr(cov), _P(_stream_ptr(stream))))
    return mean, cov


def quantize(X: torch.Tensor, basis, B: int, precision="f32", layout: int = NCHW, lo=None, hi=None,
             want_Y: bool = False, want_hist: bool = True, ctx: Context | None = None, stream=None, out=None):
    """qfca_quantize: projection + quantisation (+ reference histogram).

    ``basis`` = (mean, V[, eigvals]).  ``lo``/``hi`` (f32 [d] device) select the
    fixed-range mode.  Returns a dict with bins (u8 [d, H, pitch]), lo, hi,
    hist (u32 [d, B]) and optionally Y (f32 [d, H, W]).
    """
    _check_dev(X, "X", torch.float32)
    mean, V = basis[0], basis[1]
    _check_dev(mean, "mean", torch.float64)
    _check_dev(V, "V", torch.float64)
    fm = fmap_of(X, layout)
    ctx = ctx or default_context(X.device.index)
    d = V.shape[1]
    pitch = bins_pitch(fm.W)
    dev = X.device
    if out is None:
        bins = torch.empty(d, fm.H, pitch, dtype=torch.uint8, device=dev)
        lo_o = torch.empty(d, dtype=torch.float32, device=dev)
        hi_o = torch.empty(d, dtype=torch.float32, device=dev)
        hist = torch.empty(d, B, dtype=torch.int32, device=dev) if want_hist else None
        Y = torch.empty(d, fm.H, fm.W, dtype=torch.float32, device=dev) if want_Y else None
    else:
        bins, lo_o, hi_o, hist, Y = out
    rmode = RANGE_IMAGE if lo is None else RANGE_FIXED
    b = Basis(mean.data_ptr(), V.data_ptr(), None)
    ctx.check(_lib.qfca_quantize(ctx.handle, _ptr(X), fm, ctypes.byref(b), d, B, _PREC[precision], rmode,
                                 _ptr(lo), _ptr(hi), _ptr(bins), pitch, _ptr(lo_o), _ptr(hi_o), _ptr(hist),
                                 _ptr(Y), _P(_stream_ptr(stream))))
    return dict(bins=bins, lo=lo_o, hi=hi_o, hist=hist, Y=Y, pitch=pitch)


def quantize_residual(X: torch.Tensor, basis, B: int, layout: int = NCHW, want_F: bool = False,
                      ctx: Context | None = None, stream=None):
    """qfca_quantize_residual: QFCA+ features (X minus its PCA reconstruction from the
    basis' dres components) quantised per channel.  Returns a dict with bins (u8
    [C, H, pitch]), lo, hi (f32 [C]), hist (u32 [C, B]) and optionally F (f32 [C, H, W])."""
    _check_dev(X, "X", torch.float32)
    mean, V = basis[0], basis[1]
    _check_dev(mean, "mean", torch.float64)
    _check_dev(V, "V", torch.float64)
    fm = fmap_of(X, layout)
    ctx = ctx or default_context(X.device.index)
    dres = V.shape[1]
    pitch = bins_pitch(fm.W)
    dev = X.device
    C = fm.C
    bins = torch.empty(C, fm.H, pitch, dtype=torch.uint8, device=dev)
    lo_o = torch.empty(C, dtype=torch.float32, device=dev)
    hi_o = torch.empty(C, dtype=torch.float32, device=dev)
    hist = torch.empty(C, B, dtype=torch.int32, device=dev)
    F = torch.empty(C, fm.H, fm.W, dtype=torch.float32, device=dev) if want_F else None
    b = Basis(mean.data_ptr(), V.data_ptr() if V.numel() else None, None)
    ctx.check(_lib.qfca_quantize_residual(ctx.handle, _ptr(X), fm, ctypes.byref(b), dres, B, _ptr(bins), pitch,
                                          _ptr(lo_o), _ptr(hi_o), _ptr(hist), _ptr(F), _P(_stream_ptr(stream))))
    return dict(bins=bins, lo=lo_o, hi=hi_o, hist=hist, F=F, pitch=pitch)


def _ranges(lo, hi, d):
    if (lo is None) != (hi is None):
        raise ValueError("value units need both lo and hi")
    if lo is not None:
        for t, nm in ((lo, "lo"), (hi, "hi")):
            _check_dev(t, nm, torch.float32)
            if t.numel() != d:
                raise ValueError(f"{nm} must hold one range end per component ({d})")
    return _ptr(lo), _ptr(hi)


def score(bins: torch.Tensor, W: int, B: int, r: int, ref_hist: torch.Tensor, ref_total: int,
          want_numer: bool = False, ctx: Context | None = None, stream=None, out=None, lo=None, hi=None):
    """qfca_score: window histograms + 1-D EMD + component mean -> f32 [H, W] score map.
    Bin units, or value units given each component's quantisation range lo/hi (f32 [d])."""
    _check_dev(bins, "bins", torch.uint8)
    if ref_hist.dtype not in (torch.int32, torch.uint32) or not ref_hist.is_cuda:
        raise ValueError("ref_hist must be a CUDA int32/uint32 tensor")
    d, H, pitch = bins.shape
    ctx = ctx or default_context(bins.device.index)
    if out is None:
        s = torch.empty(H, W, dtype=torch.float32, device=bins.device)
    else:
        s = out
    numer = torch.empty(d, H, W, dtype=torch.int64, device=bins.device) if want_numer else None
    plo, phi = _ranges(lo, hi, d)
    ctx.check(_lib.qfca_score(ctx.handle, _ptr(bins), H, W, pitch, d, B, r, _ptr(ref_hist), int(ref_total),
                              _ptr(s), _ptr(numer), plo, phi, _P(_stream_ptr(stream))))
    return (s, numer) if want_numer else s


def score_assoc(bins: torch.Tensor, W: int, B: int, r: int, ref_hist: torch.Tensor, ref_total: int,
                sigma_s: float = 1.0, want_raw: bool = False, want_comp: bool = False, ctx: Context | None = None,
                stream=None, out=None, lo=None, hi=None):
    """qfca_score_assoc: the paper's scoring (Algorithm 1, error-to-pixel association,
    component mean, Gaussian smoothing) -> f32 [H, W] score map; with want_raw /
    want_comp also the map before smoothing [H, W] and the per-component maps [d, H, W]."""
    _check_dev(bins, "bins", torch.uint8)
    if ref_hist.dtype not in (torch.int32, torch.uint32) or not ref_hist.is_cuda:
        raise ValueError("ref_hist must be a CUDA int32/uint32 tensor")
    d, H, pitch = bins.shape
    ctx = ctx or default_context(bins.device.index)
    s = torch.empty(H, W, dtype=torch.float32, device=bins.device) if out is None else out
    raw = torch.empty(H, W, dtype=torch.float32, device=bins.device) if want_raw else None
    comp = torch.empty(d, H, W, dtype=torch.float32, device=bins.device) if want_comp else None
    plo, phi = _ranges(lo, hi, d)
    ctx.check(_lib.qfca_score_assoc(ctx.handle, _ptr(bins), H, W, pitch, d, B, r, _ptr(ref_hist), int(ref_total),
                                    float(sigma_s), _ptr(s), _ptr(raw), _ptr(comp), plo, phi,
                                    _P(_stream_ptr(stream))))
    if not (want_raw or want_comp):
        return s
    return (s,) + ((raw,) if want_raw else ()) + ((comp,) if want_comp else ())


def score_assoc_batch(bins_list, Ws, rs, B: int, refs, ref_totals, sigma_s: float = 1.0,
                      ctx: Context | None = None, stream=None, scores=None, los=None, his=None):
    """qfca_score_assoc_batch: qfca_score_assoc for several images (bins [d, H_i, pitch_i])
    in one launch per stage.  Returns the list of score maps [H_i, W_i]."""
    n = len(bins_list)
    if not (n == len(Ws) == len(rs) == len(refs) == len(ref_totals)) or n == 0:
        raise ValueError("one width, radius, reference and total per image")
    ctx = ctx or default_context(bins_list[0].device.index)
    d = int(bins_list[0].shape[0])
    if scores is None:
        scores = [torch.empty(int(b.shape[1]), int(w), dtype=torch.float32, device=b.device)
                  for b, w in zip(bins_list, Ws)]
    arr = (AssocImage * n)()
    for i, (b, w, r, R, nt, sc) in enumerate(zip(bins_list, Ws, rs, refs, ref_totals, scores)):
        _check_dev(b, f"bins_list[{i}]", torch.uint8)
        if int(b.shape[0]) != d:
            raise ValueError("every image needs the same number of components")
        plo, phi = _ranges(None if los is None else los[i], None if his is None else his[i], d)
        arr[i] = AssocImage(_ptr(b), int(b.shape[1]), int(w), int(b.shape[2]), int(r), _ptr(R), int(nt), _ptr(sc), None,
                            plo, phi)
    ctx.check(_lib.qfca_score_assoc_batch(ctx.handle, arr, n, d, B, float(sigma_s), _P(_stream_ptr(stream))))
    return scores


def median_reference(bins: torch.Tensor, W: int, B: int, r: int, ctx: Context | None = None, stream=None, out=None):
    """qfca_median_reference: the per-rank median reference of bins [d, H, pitch] as a
    histogram int32 [d, B] (each row sums to (2r+1)^2)."""
    _check_dev(bins, "bins", torch.uint8)
    d, H, pitch = bins.shape
    ctx = ctx or default_context(bins.device.index)
    R = torch.empty(d, B, dtype=torch.int32, device=bins.device) if out is None else out
    ctx.check(_lib.qfca_median_reference(ctx.handle, _ptr(bins), H, W, pitch, d, B, r, _ptr(R),
                                         _P(_stream_ptr(stream))))
    return R


def median_reference_batch(bins_list, Ws, rs, B: int, ctx: Context | None = None, stream=None, outs=None):
    """qfca_median_reference_batch over several images; returns the list of int32 [d, B]."""
    n = len(bins_list)
    if not (n == len(Ws) == len(rs)) or n == 0:
        raise ValueError("one width and radius per image")
    ctx = ctx or default_context(bins_list[0].device.index)
    d = int(bins_list[0].shape[0])
    if outs is None:
        outs = [torch.empty(d, B, dtype=torch.int32, device=b.device) for b in bins_list]
    arr = (MedianImage * n)()
    for i, (b, w, r, o) in enumerate(zip(bins_list, Ws, rs, outs)):
        _check_dev(b, f"bins_list[{i}]", torch.uint8)
        arr[i] = MedianImage(_ptr(b), int(b.shape[1]), int(w), int(b.shape[2]), int(r), _ptr(o))
    ctx.check(_lib.qfca_median_reference_batch(ctx.handle, arr, n, d, B, _P(_stream_ptr(stream))))
    return outs


def batch_run(X: torch.Tensor, d: int, B: int, r: int, precision="bf16", ctx: Context | None = None, stream=None,
              scores: torch.Tensor | None = None, extras: bool = False):
    """qfca_batch_run: the whole path for a batch X [nimg, C, H, W] (NCHW maps).

    Returns scores [nimg, H, W] (f32), or (scores, dict of per-image mean, V,
    eigvals, bins, ref_hist, lo, hi) when ``extras`` is set.
    """
    _check_dev(X, "X", torch.float32)
    if X.dim() != 4:
        raise ValueError("X must be [nimg, C, H, W]")
    nimg, C, H, W = (int(v) for v in X.shape)
    ctx = ctx or default_context(X.device.index)
    dev = X.device
    if scores is None:
        scores = torch.empty(nimg, H, W, dtype=torch.float32, device=dev)
    ext = None
    ex = None
    if extras:
        pitch = bins_pitch(W)
        ex = dict(mean=torch.empty(nimg, C, dtype=torch.float64, device=dev),
                  V=torch.empty(nimg, C, d, dtype=torch.float64, device=dev),
                  eigvals=torch.empty(nimg, d, dtype=torch.float64, device=dev),
                  bins=torch.empty(nimg, d, H, pitch, dtype=torch.uint8, device=dev),
                  ref_hist=torch.empty(nimg, d, B, dtype=torch.int32, device=dev),
                  lo=torch.empty(nimg, d, dtype=torch.float32, device=dev),
                  hi=torch.empty(nimg, d, dtype=torch.float32, device=dev))
        ext = BatchOutputs(ex["mean"].data_ptr(), ex["V"].data_ptr(), ex["eigvals"].data_ptr(),
                           ex["bins"].data_ptr(), pitch, ex["ref_hist"].data_ptr(), ex["lo"].data_ptr(),
                           ex["hi"].data_ptr())
    fm = Fmap(H, W, C, NCHW)
    ctx.check(_lib.qfca_batch_run(ctx.handle, _ptr(X), nimg, fm, d, B, r, _PREC[precision], _ptr(scores),
                                  ctypes.byref(ext) if ext is not None else None, _P(_stream_ptr(stream))))
    return (scores, ex) if extras else scores


def batch_run_host(X: torch.Tensor, d: int, B: int, r: int, precision="bf16", ctx: Context | None = None,
                   stream=None, scores: torch.Tensor | None = None, device: int = 0):
    """qfca_batch_run_host: the whole path for a batch X [nimg, C, H, W] (NCHW maps) held in
    host memory (pinned for asynchronous copies); the score maps come back into the host tensor
    ``scores`` [nimg, H, W] (f32, allocated pinned when not given).  Enqueued on ``stream``: the
    host tensors must stay alive until the stream has passed the call."""
    if X.is_cuda or X.dtype != torch.float32 or not X.is_contiguous() or X.dim() != 4:
        raise ValueError("X must be a contiguous host float32 tensor [nimg, C, H, W]")
    nimg, C, H, W = (int(v) for v in X.shape)
    ctx = ctx or default_context(device)
    if scores is None:
        scores = torch.empty(nimg, H, W, dtype=torch.float32).pin_memory()
    if scores.is_cuda or scores.dtype != torch.float32 or not scores.is_contiguous() or tuple(scores.shape) != (nimg, H, W):
        raise ValueError("scores must be a contiguous host float32 tensor [nimg, H, W]")
    ctx.check(_lib.qfca_batch_run_host(ctx.handle, _P(X.data_ptr()), nimg, Fmap(H, W, C, NCHW), d, B, r,
                                       _PREC[precision], _P(scores.data_ptr()), _P(_stream_ptr(stream))))
    return scores


def metrics(scores: torch.Tensor, masks: torch.Tensor, border: int = 0, fpr_limit: float = 0.3,
            ctx: Context | None = None, stream=None) -> dict:
    """qfca_metrics on device maps scores [nimg, H, W] (f32) and masks [nimg, H, W] (u8 or bool):
    pixel AUROC, F1 max, AUPRO up to ``fpr_limit`` and image AUROC after a ``border`` discard.
    Synchronises the stream to return the four values."""
    _check_dev(scores, "scores", torch.float32)
    if scores.dim() == 2:
        scores, masks = scores[None], masks[None]
    if masks.dtype == torch.bool:
        masks = masks.to(torch.uint8)
    _check_dev(masks, "masks", torch.uint8)
    if tuple(masks.shape) != tuple(scores.shape):
        raise ValueError("scores and masks must have the same shape [nimg, H, W]")
    nimg, H, W = (int(v) for v in scores.shape)
    ctx = ctx or default_context(scores.device.index)
    out = torch.empty(4, dtype=torch.float64, device=scores.device)
    ctx.check(_lib.qfca_metrics(ctx.handle, _ptr(scores), _ptr(masks), nimg, H, W, int(border), float(fpr_limit),
                                _ptr(out), _P(_stream_ptr(stream))))
    v = out.cpu().tolist()
    return {"pixel_auroc": v[0], "f1_max": v[1], "aupro": v[2], "image_auroc": v[3]}


def batch_run_basis(X: torch.Tensor, mean: torch.Tensor, V: torch.Tensor, B: int, r: int, precision="bf16",
                    ctx: Context | None = None, stream=None, scores: torch.Tensor | None = None):
    """qfca_batch_run_basis: the path after the fit for a batch X [nimg, C, H, W]
    (NCHW maps) with given bases mean [nimg, C] and V [nimg, C, d] (FP64).
    Returns scores [nimg, H, W] (f32)."""
    _check_dev(X, "X", torch.float32)
    _check_dev(mean, "mean", torch.float64)
    _check_dev(V, "V", torch.float64)
    if X.dim() != 4 or V.dim() != 3:
        raise ValueError("X must be [nimg, C, H, W] and V [nimg, C, d]")
    nimg, C, H, W = (int(v) for v in X.shape)
    d = int(V.shape[2])
    if tuple(mean.shape) != (nimg, C) or tuple(V.shape[:2]) != (nimg, C):
        raise ValueError("mean must be [nimg, C] and V [nimg, C, d]")
    ctx = ctx or default_context(X.device.index)
    if scores is None:
        scores = torch.empty(nimg, H, W, dtype=torch.float32, device=X.device)
    fm = Fmap(H, W, C, NCHW)
    ctx.check(_lib.qfca_batch_run_basis(ctx.handle, _ptr(X), nimg, fm, _ptr(mean), _ptr(V), d, B, r,
                                        _PREC[precision], _ptr(scores), None, _P(_stream_ptr(stream))))
    return scores


def batch_run_plus(X: torch.Tensor, dres: int, B: int, r: int, ctx: Context | None = None, stream=None,
                   scores: torch.Tensor | None = None, extras: bool = False):
    """qfca_batch_run_plus: QFCA+ for a batch X [nimg, C, H, W] (NCHW maps): fit of dres
    components, residual features of all C channels, per-channel quantisation, EMD over
    the C planes.  Returns scores [nimg, H, W], or (scores, dict of mean, V, eigvals,
    bins [nimg, C, H, pitch], ref_hist [nimg, C, B], lo, hi) when ``extras`` is set."""
    _check_dev(X, "X", torch.float32)
    if X.dim() != 4:
        raise ValueError("X must be [nimg, C, H, W]")
    nimg, C, H, W = (int(v) for v in X.shape)
    ctx = ctx or default_context(X.device.index)
    dev = X.device
    if scores is None:
        scores = torch.empty(nimg, H, W, dtype=torch.float32, device=dev)
    ext = None
    ex = None
    if extras:
        pitch = bins_pitch(W)
        ex = dict(mean=torch.empty(nimg, C, dtype=torch.float64, device=dev),
                  V=torch.empty(nimg, C, dres, dtype=torch.float64, device=dev),
                  eigvals=torch.empty(nimg, dres, dtype=torch.float64, device=dev),
                  bins=torch.empty(nimg, C, H, pitch, dtype=torch.uint8, device=dev),
                  ref_hist=torch.empty(nimg, C, B, dtype=torch.int32, device=dev),
                  lo=torch.empty(nimg, C, dtype=torch.float32, device=dev),
                  hi=torch.empty(nimg, C, dtype=torch.float32, device=dev))
        ext = BatchOutputs(_ptr(ex["mean"]), _ptr(ex["V"]), _ptr(ex["eigvals"]), _ptr(ex["bins"]), pitch,
                           _ptr(ex["ref_hist"]), _ptr(ex["lo"]), _ptr(ex["hi"]))
    fm = Fmap(H, W, C, NCHW)
    ctx.check(_lib.qfca_batch_run_plus(ctx.handle, _ptr(X), nimg, fm, dres, B, r, _ptr(scores),
                                       ctypes.byref(ext) if ext is not None else None, _P(_stream_ptr(stream))))
    return (scores, ex) if extras else scores


def score_batch(Xs, rs, d: int, B: int, precision="bf16", layout: int = NCHW, ctx: Context | None = None,
                stream=None, scores=None):
    """qfca_score_batch: the whole path for images of different sizes and radii.

    Xs: list of device FP32 maps [C, H_i, W_i] (NCHW) or [H_i, W_i, C] (NHWC);
    rs: one window radius per image.  Returns the list of score maps [H_i, W_i].
    """
    if len(Xs) != len(rs) or not Xs:
        raise ValueError("one radius per image, at least one image")
    fms = [fmap_of(X, layout) for X in Xs]
    C = fms[0].C
    if any(fm.C != C for fm in fms):
        raise ValueError("every image needs the same channel count")
    ctx = ctx or default_context(Xs[0].device.index)
    if scores is None:
        scores = [torch.empty(fm.H, fm.W, dtype=torch.float32, device=X.device) for fm, X in zip(fms, Xs)]
    arr = (Image * len(Xs))()
    for i, (X, fm, r, sc) in enumerate(zip(Xs, fms, rs, scores)):
        _check_dev(X, f"Xs[{i}]", torch.float32)
        arr[i] = Image(_ptr(X), fm.H, fm.W, int(r), _ptr(sc))
    ctx.check(_lib.qfca_score_batch(ctx.handle, arr, len(Xs), C, layout, d, B, _PREC[precision],
                                    _P(_stream_ptr(stream))))
    return scores


class Server:
    """A serving session on a context (qfca_serve_start ... qfca_serve_stop).

    Classes carry resident bases, fixed ranges and reference histograms;
    requests are single NCHW feature maps [C, H, W] scored against their
    class.  submit() queues a request and returns its ticket (None when the
    queue is full); poll() returns a Result once it has finished.
    """

    def __init__(self, C: int, d: int, B: int, precision="bf16", max_batch: int = 16, streams: int = 2,
                 max_queue: int = 4096, arena_bytes: int = 4 << 30, ctx: Context | None = None):
        self.ctx = ctx or Context()
        self.C, self.d, self.B = C, d, B
        cfg = ServeConfig(C, d, B, _PREC[precision], max_batch, streams, max_queue, arena_bytes)
        self.ctx.check(_lib.qfca_serve_start(self.ctx.handle, ctypes.byref(cfg)))
        self._keep = {}  # ticket -> tensors the GPU reads or writes until the request is polled

    def register_class(self, class_id: int, mean, V, lo, hi, ref_hist, ref_total: int):
        _check_dev(mean, "mean", torch.float64)
        _check_dev(V, "V", torch.float64)
        self.ctx.check(_lib.qfca_register_class(self.ctx.handle, int(class_id), _ptr(mean), _ptr(V), _ptr(lo),
                                                _ptr(hi), _ptr(ref_hist), int(ref_total)))

    def submit(self, class_id: int, X: torch.Tensor, r: int, score: torch.Tensor | None = None):
        C, H, W = (int(v) for v in X.shape)
        if C != self.C:
            raise ValueError(f"X has {C} channels, the session {self.C}")
        host_in = not X.is_cuda
        if score is None:
            score = torch.empty(H, W, dtype=torch.float32, device="cpu" if host_in else X.device,
                                pin_memory=host_in)
        flags = (REQ_HOST_INPUT if host_in else 0) | (REQ_HOST_OUTPUT if not score.is_cuda else 0)
        req = Request(int(class_id), X.data_ptr(), H, W, int(r), score.data_ptr(), flags)
        t = ctypes.c_uint64()
        s = _lib.qfca_submit(self.ctx.handle, ctypes.byref(req), ctypes.byref(t))
        if s == ERR_BUSY:
            return None
        if s != OK:
            raise QfcaError(s, "qfca_submit")
        self._keep[int(t.value)] = (X, score)
        return int(t.value)

    def poll(self, ticket: int, timeout_us: int = 0):
        """(Result, score tensor) when the request is done, else None."""
        res = Result()
        s = _lib.qfca_poll(self.ctx.handle, ctypes.c_uint64(ticket), int(timeout_us), ctypes.byref(res))
        if s == PENDING:
            return None
        if s != OK:
            raise QfcaError(s, "qfca_poll")
        _, score = self._keep.pop(ticket)
        return res, score

    def stop(self):
        if self.ctx is not None and getattr(self.ctx, "handle", None):
            self.ctx.check(_lib.qfca_serve_stop(self.ctx.handle))
        self._keep.clear()


def run_image(X: torch.Tensor, d: int, B: int, r: int, precision="f32", layout: int = NCHW,
              ctx: Context | None = None, stream=None):
    """The whole path on one image: fit, project + quantize, window EMD score."""
    basis = fit_pca(X, d, layout, ctx=ctx, stream=stream)
    q = quantize(X, basis, B, precision, layout, ctx=ctx, stream=stream)
    fm = fmap_of(X, layout)
    s = score(q["bins"], fm.W, B, r, q["hist"], fm.H * fm.W, ctx=ctx, stream=stream)
    return s, basis, q
