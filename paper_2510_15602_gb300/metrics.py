"""Evaluation metrics on the host (not part of the GPU path).

Pixel-level AUROC (Sec. 4.2): the probability that a randomly drawn anomalous
pixel scores higher than a randomly drawn normal one, ties counting one half --
the Mann-Whitney U statistic with average ranks for ties, divided by the
number of (positive, negative) pairs.  Borders can be discarded first, as the
paper's evaluation does.
"""
from __future__ import annotations

import numpy as np


def _average_ranks(v: np.ndarray) -> np.ndarray:
    order = np.argsort(v, kind="mergesort")
    sv = v[order]
    n = len(v)
    ranks = np.empty(n, np.float64)
    # boundaries of runs of equal values
    starts = np.flatnonzero(np.r_[True, sv[1:] != sv[:-1]])
    ends = np.r_[starts[1:], n]
    avg = 0.5 * (starts + ends - 1) + 1.0  # 1-based average rank of each run
    ranks[order] = np.repeat(avg, ends - starts)
    return ranks


def auroc(score: np.ndarray, mask: np.ndarray, border: int = 0) -> float:
    """Pixel AUROC of ``score`` against the binary ``mask`` (same shape).

    ``border`` pixels are discarded on each side before ranking.  Returns NaN
    when either class is empty.
    """
    s = np.asarray(score, np.float64)
    m = np.asarray(mask) != 0
    if border > 0:
        s = s[..., border:-border, border:-border]
        m = m[..., border:-border, border:-border]
    s = s.ravel()
    m = m.ravel()
    n_pos = int(m.sum())
    n_neg = int(m.size - n_pos)
    if n_pos == 0 or n_neg == 0:
        return float("nan")
    ranks = _average_ranks(s)
    u = ranks[m].sum() - n_pos * (n_pos + 1) / 2.0
    return float(u / (n_pos * n_neg))


# ---------------------------------------------------------------- the rest of the paper's metric suite (Sec. 4.2)
#
# F1 at the optimal threshold, the per-region overlap curve integrated to a
# false-positive rate of 30% (AUPRO), and the image-level AUROC of the maximum
# pixel score.  Each takes the border discard of the paper's evaluation.
# Thresholds: every distinct score value (a pixel is predicted anomalous when
# its score is >= the threshold), so the curves are exact rather than sampled.


def _crop(a: np.ndarray, border: int) -> np.ndarray:
    return a[..., border:-border, border:-border] if border > 0 else a


def _run_ends(sorted_desc: np.ndarray) -> np.ndarray:
    """Indices of the last element of each run of equal values in a descending array."""
    n = len(sorted_desc)
    return np.flatnonzero(np.r_[sorted_desc[1:] != sorted_desc[:-1], True]) if n else np.zeros(0, np.int64)


def f1_max(score, mask, border: int = 0) -> float:
    """Maximum pixel F1 = 2 P R / (P + R) over all thresholds (score >= t is
    predicted anomalous).  ``score`` and ``mask`` may be single maps or stacks of
    maps (pooled over all pixels).  NaN without anomalous pixels."""
    s = _crop(np.asarray(score, np.float64), border).ravel()
    m = _crop(np.asarray(mask) != 0, border).ravel()
    n_pos = int(m.sum())
    if n_pos == 0:
        return float("nan")
    order = np.argsort(-s, kind="mergesort")
    tp = np.cumsum(m[order])
    k = _run_ends(s[order])
    tp, npred = tp[k].astype(np.float64), (k + 1).astype(np.float64)
    f1 = 2.0 * tp / (npred + n_pos)
    return float(f1.max())


def _label8(mask2d: np.ndarray):
    from scipy import ndimage
    return ndimage.label(mask2d, structure=np.ones((3, 3), dtype=int))


def pro_curve(scores, masks, border: int = 0):
    """The per-region overlap curve over all thresholds: for each threshold, the
    false-positive rate over all normal pixels and the mean, over every
    connected anomalous region (8-connectivity) of every image, of the fraction
    of the region's pixels at or above the threshold.  Returns (fpr, pro) with a
    leading (0, 0) point, in threshold-descending order."""
    maps = [np.asarray(s, np.float64) for s in scores]
    ms = [np.asarray(m) != 0 for m in masks]
    vals, w_fpr, w_pro = [], [], []
    n_neg = sum(int((~_crop(m, border)).sum()) for m in ms)
    regions = []
    for s, m in zip(maps, ms):
        s, m = _crop(s, border), _crop(m, border)
        lab, nreg = _label8(m)
        regions.append((s, m, lab, nreg))
    n_reg = sum(r[3] for r in regions)
    if n_neg == 0 or n_reg == 0:
        return np.zeros(1), np.zeros(1)
    for s, m, lab, nreg in regions:
        sizes = np.bincount(lab.ravel(), minlength=nreg + 1).astype(np.float64)
        vals.append(s.ravel())
        w_fpr.append((~m).ravel() / n_neg)
        wl = np.where(lab.ravel() > 0, 1.0 / (n_reg * sizes[lab.ravel()]), 0.0)
        w_pro.append(wl)
    v = np.concatenate(vals)
    order = np.argsort(-v, kind="mergesort")
    fpr = np.cumsum(np.concatenate(w_fpr)[order])
    pro = np.cumsum(np.concatenate(w_pro)[order])
    k = _run_ends(v[order])
    return np.r_[0.0, fpr[k]], np.r_[0.0, pro[k]]


def aupro(scores, masks, fpr_limit: float = 0.3, border: int = 0) -> float:
    """Area under the per-region overlap curve up to ``fpr_limit``, divided by
    ``fpr_limit`` (the PRO score at 30% FPR).  Trapezoids between thresholds,
    linear interpolation at the limit."""
    fpr, pro = pro_curve(scores, masks, border)
    if len(fpr) < 2:
        return float("nan")
    fpr = np.minimum(fpr, 1.0)
    keep = fpr <= fpr_limit
    x, y = list(fpr[keep]), list(pro[keep])
    j = int(keep.sum())
    if j < len(fpr) and x[-1] < fpr_limit:
        f0, f1, p0, p1 = fpr[j - 1], fpr[j], pro[j - 1], pro[j]
        x.append(fpr_limit)
        y.append(p0 + (p1 - p0) * (fpr_limit - f0) / (f1 - f0))
    x, y = np.asarray(x), np.asarray(y)
    return float(np.sum(0.5 * (y[1:] + y[:-1]) * np.diff(x)) / fpr_limit)


def image_auroc(scores, masks, border: int = 0) -> float:
    """Image-level AUROC: each image scores the maximum of its (border-cropped)
    map; an image is anomalous when its mask has any anomalous pixel.  NaN when
    all images fall in one class."""
    s = np.array([_crop(np.asarray(x, np.float64), border).max() for x in scores])
    y = np.array([bool((np.asarray(m) != 0).any()) for m in masks], np.uint8)
    return auroc(s[None, :], y[None, :])
