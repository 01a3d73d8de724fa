"""The counting form of the median reference (Sec. 3.2) that the median kernel
evaluates, checked against the oracle's sort-based definition.

The m-th smallest value of a window is <= b exactly when the window's cumulative
count up to bin b reaches m, so with G[b][m] = #{full windows w : cumP_b(w) >= m}
the lower median of the windows' m-th values is min{b : G[b][m] >= ceil(Np / 2)}
for Np full windows.  Restated here with numpy, independently of the CUDA source."""
import numpy as np
import pytest

import oracle
from paper_2510_15602_gb300 import synth


def counting_form(q, B, r):
    d, H, W = q.shape
    T2 = (2 * r + 1) ** 2
    R = np.zeros((d, B), np.int64)
    for k in range(d):
        cums = []
        for y in range(r, H - r):
            for x in range(r, W - r):
                win = q[k, y - r:y + r + 1, x - r:x + r + 1].ravel()
                cums.append(np.cumsum(np.bincount(np.minimum(win, B - 1), minlength=B)))
        cums = np.array(cums)                  # [Np][B]
        Np = len(cums)
        half = (Np + 1) // 2
        for m in range(1, T2 + 1):
            G = (cums >= m).sum(axis=0)        # G[b][m] for every b
            R[k, int(np.argmax(G >= half))] += 1
    return R


@pytest.mark.parametrize("d,H,W,B,r,seed", [(2, 9, 11, 6, 2, 0), (1, 8, 8, 4, 1, 1), (2, 12, 7, 16, 2, 2),
                                            (1, 5, 6, 3, 2, 3)])
def test_counting_form_equals_sorted_medians(d, H, W, B, r, seed):
    rng = np.random.default_rng(700 + seed)
    q = synth.random_bins(rng, d, H, W, B, smooth=seed % 2 == 0)
    np.testing.assert_array_equal(counting_form(q, B, r), oracle.median_ref(q, B, r))
