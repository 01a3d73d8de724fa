"""Seeded synthetic feature maps with anomaly masks.

These inputs stand in for the paper's texture datasets (MVTec AD textures,
DTD-Synthetic, WFT; Sec. 4.1), which are not available here.  They mimic the
shape of the paper's WideResNet-50 feature maps (stride-8 features with
hundreds of channels, Sec. 3.3) with a stationary, spatially smoothed Gaussian
random field, and plant anomalies whose statistics differ from the rest of the
field.  Nothing in this module computes any part of the anomaly-scoring
method: it only draws inputs.  Both the GPU library's tests and the CPU oracle
consume these arrays.

Recipe
------
* Field: per channel, i.i.d. N(0, 1) on an (H + 2p) x (W + 2p) grid with
  p = ceil(4 sigma), separable Gaussian blur (std sigma px, truncated at
  4 sigma, kernel normalised to sum 1), valid crop to H x W, then division by
  the analytic std of the blurred field (sum of squared 1-D taps, squared for
  2-D) so every channel has unit variance.
* Anomalies (mask value 1 where planted):
    - ``square``: a 12 x 12 square fully inside the image, +1.5 on 8 distinct
      random channels;
    - ``scratch``: a segment of length U(0.3, 0.8) * W through a random point at a
      random angle, width 1-3 px, +1.5 on 8 random channels;
    - ``blob``: an ellipse with semi-axes U(6, 20) px at a random angle, features
      multiplied by sqrt(2) (variance x2);
    - ``rotcov``: a square of side 16-32 px whose channel vectors are rotated
      by a seeded random orthogonal C x C matrix.
* Seeds: numpy PCG64 ``default_rng(1000 * config + image_index)``
  (+ 100000 * class for the serving workload's class fields).

All arrays are float32 ``(C, H, W)`` (NCHW without the batch axis) and masks
uint8 ``(H, W)``.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field as dc_field

import numpy as np

try:  # scipy is present on both the build host and the GPU host
    from scipy.ndimage import convolve1d as _convolve1d
except Exception:  # pragma: no cover - fallback keeps the generator usable
    _convolve1d = None


def _blur1d(z: np.ndarray, g: np.ndarray, axis: int) -> np.ndarray:
    if _convolve1d is not None:
        return _convolve1d(z, g, axis=axis, mode="constant")
    # plain numpy fallback: explicit shifted sums
    out = np.zeros_like(z)
    p = (len(g) - 1) // 2
    n = z.shape[axis]
    for i, gi in enumerate(g):
        s = i - p
        src = [slice(None)] * z.ndim
        dst = [slice(None)] * z.ndim
        if s >= 0:
            src[axis] = slice(s, n)
            dst[axis] = slice(0, n - s)
        else:
            src[axis] = slice(0, n + s)
            dst[axis] = slice(-s, n)
        out[tuple(dst)] += gi * z[tuple(src)]
    return out


def gaussian_field(rng: np.random.Generator, C: int, H: int, W: int, sigma: float) -> np.ndarray:
    """Unit-variance stationary Gaussian random field, float32 (C, H, W)."""
    p = int(math.ceil(4.0 * sigma))
    z = rng.standard_normal((C, H + 2 * p, W + 2 * p), dtype=np.float32)
    x = np.arange(-p, p + 1, dtype=np.float64)
    g = np.exp(-0.5 * (x / sigma) ** 2)
    g /= g.sum()
    g32 = g.astype(np.float32)
    z = _blur1d(z, g32, axis=1)
    z = _blur1d(z, g32, axis=2)
    z = z[:, p:p + H, p:p + W]
    std = float(np.sum(g ** 2))  # std of the 2-D blurred white field = (sum g^2)
    return np.ascontiguousarray(z / np.float32(std), dtype=np.float32)


def random_orthogonal(rng: np.random.Generator, n: int) -> np.ndarray:
    """Haar-distributed orthogonal matrix (QR of a Gaussian, sign-fixed)."""
    a = rng.standard_normal((n, n))
    q, r = np.linalg.qr(a)
    q *= np.sign(np.diag(r))[None, :]
    return q


# --------------------------------------------------------------------------- anomalies

def _plant_square(rng, X, mask, side=12, shift=1.5, nch=8):
    C, H, W = X.shape
    y0 = int(rng.integers(0, H - side + 1))
    x0 = int(rng.integers(0, W - side + 1))
    ch = rng.choice(C, size=min(nch, C), replace=False)
    X[np.ix_(ch, np.arange(y0, y0 + side), np.arange(x0, x0 + side))] += np.float32(shift)
    mask[y0:y0 + side, x0:x0 + side] = 1


def _plant_scratch(rng, X, mask, shift=1.5, nch=8):
    C, H, W = X.shape
    length = rng.uniform(0.3, 0.8) * W
    cy, cx = rng.uniform(0, H), rng.uniform(0, W)
    ang = rng.uniform(0, math.pi)
    width = int(rng.integers(1, 4))
    dy, dx = math.sin(ang), math.cos(ang)
    yy, xx = np.mgrid[0:H, 0:W].astype(np.float64)
    # distance from pixel centres to the segment
    t = np.clip((yy - cy) * dy + (xx - cx) * dx, -length / 2, length / 2)
    dist = np.hypot(yy - (cy + t * dy), xx - (cx + t * dx))
    m = dist <= width / 2.0
    if not m.any():
        iy, ix = min(int(cy), H - 1), min(int(cx), W - 1)
        m[iy, ix] = True
    ch = rng.choice(C, size=min(nch, C), replace=False)
    for c in ch:
        X[c][m] += np.float32(shift)
    mask[m] = 1


def _plant_blob(rng, X, mask):
    C, H, W = X.shape
    a, b = rng.uniform(6, 20), rng.uniform(6, 20)
    cy, cx = rng.uniform(0, H), rng.uniform(0, W)
    ang = rng.uniform(0, math.pi)
    yy, xx = np.mgrid[0:H, 0:W].astype(np.float64)
    u = (xx - cx) * math.cos(ang) + (yy - cy) * math.sin(ang)
    v = -(xx - cx) * math.sin(ang) + (yy - cy) * math.cos(ang)
    m = (u / a) ** 2 + (v / b) ** 2 <= 1.0
    if not m.any():
        m[min(int(cy), H - 1), min(int(cx), W - 1)] = True
    X[:, m] *= np.float32(math.sqrt(2.0))
    mask[m] = 1


def _plant_rotcov(rng, X, mask):
    C, H, W = X.shape
    side = int(rng.integers(16, 33))
    side = min(side, H, W)
    y0 = int(rng.integers(0, H - side + 1))
    x0 = int(rng.integers(0, W - side + 1))
    Q = random_orthogonal(rng, C).astype(np.float32)
    patch = X[:, y0:y0 + side, x0:x0 + side].reshape(C, -1)
    X[:, y0:y0 + side, x0:x0 + side] = (Q @ patch).reshape(C, side, side)
    mask[y0:y0 + side, x0:x0 + side] = 1


_PLANTERS = {
    "square": _plant_square,
    "scratch": _plant_scratch,
    "blob": _plant_blob,
    "rotcov": _plant_rotcov,
}


# --------------------------------------------------------------------------- workloads

@dataclass
class Workload:
    """Parameters of one synthetic workload (a named configuration)."""

    name: str
    config_id: int
    n_images: int
    C: int
    sigma: float
    d: int
    B: int
    sizes: tuple = ()            # allowed square sides
    radii: tuple = ()            # allowed window radii
    kinds: tuple = ("square",)   # anomaly kinds drawn uniformly
    n_anom: tuple = (1, 1)       # inclusive range of anomalies per image
    precision: str = "f32"
    extra: dict = dc_field(default_factory=dict)


WORKLOADS = {
    # one 128x128xC64 image, one 12x12 mean-shift square, d=16, B=16, 9x9 window
    "plain_128_c64": Workload("plain_128_c64", 1, 1, 64, 2.0, 16, 16, sizes=(128,), radii=(4,),
                              kinds=("square",), n_anom=(1, 1)),
    # 16 images of 256x256xC256, 1-3 anomalies of three kinds, d=32, B=32, 15x15 window
    "batch16_256_c256": Workload("batch16_256_c256", 2, 16, 256, 3.0, 32, 32, sizes=(256,), radii=(7,),
                                 kinds=("scratch", "blob", "rotcov"), n_anom=(1, 3)),
    # 64 uneven images 96..320 (multiples of 8) x C512, d=32, B=64, radii {5,7,9,12}
    "uneven64_c512": Workload("uneven64_c512", 4, 64, 512, 3.0, 32, 64,
                              sizes=tuple(range(96, 321, 8)), radii=(5, 7, 9, 12),
                              kinds=("square", "scratch", "blob", "rotcov"), n_anom=(1, 3),
                              precision="bf16"),
    # serving stream: sizes {128,224,320,448} x C256, d=32, B=32, 15x15 window
    "serve_c256": Workload("serve_c256", 5, 0, 256, 3.0, 32, 32, sizes=(128, 224, 320, 448), radii=(7,),
                           kinds=("square", "scratch", "blob", "rotcov"), n_anom=(1, 3),
                           precision="bf16", extra={"n_classes": 32}),
}


@dataclass
class Image:
    X: np.ndarray          # float32 (C, H, W)
    mask: np.ndarray       # uint8 (H, W)
    r: int
    seed: int
    kinds: list


def make_image(wl: Workload | str, index: int, *, side: int | None = None, r: int | None = None,
               C: int | None = None, class_id: int | None = None, class_mix: np.ndarray | None = None) -> Image:
    """Draw image ``index`` of workload ``wl`` (seeded, reproducible).

    ``side``, ``r`` and ``C`` override the workload's draws (used to make
    small cases of the same recipe).  ``class_mix`` (C x C) mixes the channels
    of the unit field, giving a class-specific channel covariance.
    """
    if isinstance(wl, str):
        wl = WORKLOADS[wl]
    seed = 1000 * wl.config_id + index + (100000 * class_id if class_id is not None else 0)
    rng = np.random.default_rng(seed)
    S = side if side is not None else int(rng.choice(np.asarray(wl.sizes)))
    rad = r if r is not None else int(rng.choice(np.asarray(wl.radii)))
    Cc = C if C is not None else wl.C
    X = gaussian_field(rng, Cc, S, S, wl.sigma)
    if class_mix is not None:
        X = np.ascontiguousarray((class_mix.astype(np.float32) @ X.reshape(Cc, -1)).reshape(Cc, S, S))
    mask = np.zeros((S, S), dtype=np.uint8)
    lo, hi = wl.n_anom
    n = int(rng.integers(lo, hi + 1))
    kinds = []
    for _ in range(n):
        kind = str(rng.choice(np.asarray(wl.kinds)))
        kinds.append(kind)
        _PLANTERS[kind](rng, X, mask)
    return Image(X=X, mask=mask, r=rad, seed=seed, kinds=kinds)


def kind_masks(wl: Workload | str, index: int, *, side: int | None = None, r: int | None = None,
               C: int | None = None) -> dict:
    """The anomaly masks of image ``index`` of ``wl``, one per anomaly kind planted
    ({kind: uint8 (H, W)}; their union is ``make_image(...).mask``).

    Replays the image's random draws in the order ``make_image`` takes them (size,
    radius, the field's normals, then each anomaly) on an all-zero field: the
    planters' draws do not depend on the feature values, so the masks are those of
    the generated image, without the cost of blurring the field."""
    if isinstance(wl, str):
        wl = WORKLOADS[wl]
    rng = np.random.default_rng(1000 * wl.config_id + index)
    S = side if side is not None else int(rng.choice(np.asarray(wl.sizes)))
    if r is None:
        rng.choice(np.asarray(wl.radii))
    Cc = C if C is not None else wl.C
    p = int(math.ceil(4.0 * wl.sigma))
    rng.standard_normal((Cc, S + 2 * p, S + 2 * p), dtype=np.float32)  # the field's draws
    X = np.zeros((Cc, S, S), np.float32)
    out = {}
    lo, hi = wl.n_anom
    for _ in range(int(rng.integers(lo, hi + 1))):
        kind = str(rng.choice(np.asarray(wl.kinds)))
        m = np.zeros((S, S), np.uint8)
        _PLANTERS[kind](rng, X, m)
        out[kind] = np.maximum(out.get(kind, np.zeros_like(m)), m)
    return out


def class_mixing(class_id: int, C: int, decay: float = 0.9) -> np.ndarray:
    """Channel-mixing matrix Q diag(sqrt(lambda)) of a texture class.

    lambda_k is proportional to decay**k, normalised to mean 1, and Q is a seeded
    random orthogonal matrix, so the class covariance is Q diag(lambda) Q^T.
    """
    rng = np.random.default_rng(5000 + 100000 * class_id)
    Q = random_orthogonal(rng, C)
    lam = decay ** np.arange(C)
    lam = lam / lam.mean()
    return (Q * np.sqrt(lam)[None, :]).astype(np.float32)


def small_case(C: int, H: int, W: int, sigma: float, seed: int, n_square: int = 1, side: int = 6,
               nch: int = 4) -> Image:
    """A small seeded field with mean-shift squares, for parity tests."""
    rng = np.random.default_rng(seed)
    X = gaussian_field(rng, C, H, W, sigma)
    mask = np.zeros((H, W), dtype=np.uint8)
    for _ in range(n_square):
        s = min(side, H, W)
        _plant_square(rng, X, mask, side=s, nch=min(nch, C))
    return Image(X=X, mask=mask, r=0, seed=seed, kinds=["square"] * n_square)


def random_bins(rng: np.random.Generator, d: int, H: int, W: int, B: int, smooth: bool = True) -> np.ndarray:
    """Random bin planes uint8 (d, H, W) in [0, B) for integer-stage tests."""
    if not smooth:
        return rng.integers(0, B, size=(d, H, W), dtype=np.int64).astype(np.uint8)
    f = gaussian_field(rng, d, H, W, 1.5).astype(np.float64)
    u = 0.5 * (1.0 + np.tanh(f / 1.2))
    return np.minimum((u * B).astype(np.int64), B - 1).astype(np.uint8)
