"""Shared helpers for the GPU parity tests (no method arithmetic here)."""
import numpy as np
import torch


def to_dev(a, dtype=None):
    t = torch.from_numpy(np.ascontiguousarray(a))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda()


def bins_np(bins_dev, W):
    """Device bins [d, H, pitch] -> numpy [d, H, W]."""
    return bins_dev[:, :, :W].cpu().numpy()


def edge_distance(Y, lo, hi, B):
    """Distance (in units of the range) from each value to the nearest interior bin edge."""
    rng = (hi - lo)[:, None, None]
    t = (Y - lo[:, None, None]) / np.where(rng > 0, rng, 1.0) * B
    return np.abs(t - np.round(t)) / B
