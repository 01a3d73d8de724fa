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
