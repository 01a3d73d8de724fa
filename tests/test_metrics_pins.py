"""Pins of the evaluation metrics (Sec. 4.2) against brute force, sklearn and
closed forms.  CPU only."""
import numpy as np
import pytest

from paper_2510_15602_gb300.metrics import aupro, auroc, f1_max, image_auroc, pro_curve

ndimage = pytest.importorskip("scipy.ndimage")


def test_f1_max_brute_force_and_sklearn():
    rng = np.random.default_rng(1)
    s = rng.integers(0, 20, size=(2, 9, 11)).astype(float)  # ties
    m = (rng.random((2, 9, 11)) < 0.25).astype(np.uint8)
    best = 0.0
    for t in np.unique(s):
        pred = s >= t
        tp = (pred & (m == 1)).sum()
        p, r = tp / pred.sum(), tp / m.sum()
        if tp:
            best = max(best, 2 * p * r / (p + r))
    assert f1_max(s, m) == pytest.approx(best, abs=1e-12)
    skm = pytest.importorskip("sklearn.metrics")
    pr, rc, _ = skm.precision_recall_curve(m.ravel(), s.ravel())
    f = np.where(pr + rc > 0, 2 * pr * rc / np.maximum(pr + rc, 1e-300), 0)
    assert f1_max(s, m) == pytest.approx(f.max(), abs=1e-12)


def pro_brute(scores, masks, limit):
    """Threshold loop over every distinct score, scipy labelling, trapezoids."""
    allv = np.unique(np.concatenate([np.ravel(s) for s in scores]))[::-1]
    n_neg = sum(int((m == 0).sum()) for m in masks)
    regs = []
    for s, m in zip(scores, masks):
        lab, n = ndimage.label(m, structure=np.ones((3, 3), int))
        regs += [(s, lab == i) for i in range(1, n + 1)]
    pts = [(0.0, 0.0)]
    for t in allv:
        fp = sum(int(((s >= t) & (m == 0)).sum()) for s, m in zip(scores, masks))
        pro = np.mean([((s >= t) & reg).sum() / reg.sum() for s, reg in regs])
        pts.append((fp / n_neg, pro))
    area, prev = 0.0, pts[0]
    for f, p in pts[1:]:
        if f > limit:
            p_lim = prev[1] + (p - prev[1]) * (limit - prev[0]) / (f - prev[0])
            area += 0.5 * (prev[1] + p_lim) * (limit - prev[0])
            return area / limit
        area += 0.5 * (prev[1] + p) * (f - prev[0])
        prev = (f, p)
    return area / limit


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_aupro_brute_force(seed):
    rng = np.random.default_rng(10 + seed)
    scores, masks = [], []
    for _ in range(2):
        m = np.zeros((12, 14), np.uint8)
        m[2:5, 3:7] = 1
        m[8:11, 9:10] = 1
        m[7, 0] = 1  # a one-pixel region
        s = rng.integers(0, 12, size=m.shape).astype(float) + 3 * m
        scores.append(s)
        masks.append(m)
    for lim in (0.3, 0.05, 1.0):
        assert aupro(scores, masks, lim) == pytest.approx(pro_brute(scores, masks, lim), abs=1e-12)


def test_aupro_closed_forms():
    m = np.zeros((10, 10), np.uint8)
    m[3:6, 3:6] = 1
    s_good = m.astype(float) + 0.01 * np.arange(100).reshape(10, 10) / 100
    assert aupro([s_good], [m]) == pytest.approx(1.0, abs=1e-12)  # every region found before any false positive
    assert aupro([-s_good], [m]) == pytest.approx(0.0, abs=1e-12)  # no region pixel before every normal one
    fpr, pro = pro_curve([s_good], [m])
    assert fpr[0] == 0.0 and pro[-1] == pytest.approx(1.0) and fpr[-1] == pytest.approx(1.0)


def test_border_discard_and_image_auroc():
    rng = np.random.default_rng(5)
    s = rng.random((3, 16, 16))
    m = np.zeros((3, 16, 16), np.uint8)
    m[:, 6:9, 6:9] = 1
    s[:, 0, :] = 10.0  # a hot border row, discarded with border=2
    assert auroc(s, m, border=2) == pytest.approx(auroc(s[:, 2:-2, 2:-2], m[:, 2:-2, 2:-2]))
    assert f1_max(s, m, border=2) == pytest.approx(f1_max(s[:, 2:-2, 2:-2], m[:, 2:-2, 2:-2]))
    maps = [rng.random((8, 8)) for _ in range(6)]
    lab = [np.zeros((8, 8), np.uint8) for _ in range(6)]
    for i in (1, 4):
        lab[i][2, 2] = 1
        maps[i] = maps[i] + 0.5 * (i == 1)
    skm = pytest.importorskip("sklearn.metrics")
    y = [int(l.any()) for l in lab]
    assert image_auroc(maps, lab) == pytest.approx(skm.roc_auc_score(y, [x.max() for x in maps]), abs=1e-12)


def test_degenerate_inputs():
    from paper_2510_15602_gb300 import metrics as M
    rng = np.random.default_rng(9)
    s = rng.random((12, 12))
    none = np.zeros((12, 12), np.uint8)
    allm = np.ones((12, 12), np.uint8)
    # one class only: the rank statistics are undefined
    assert np.isnan(M.auroc(s, none)) and np.isnan(M.auroc(s, allm))
    assert np.isnan(M.f1_max(s, none))
    assert np.isnan(M.aupro([s], [none]))
    assert np.isnan(M.image_auroc([s, s], [allm, allm]))
    # every pixel anomalous: predicting all of them gives precision = recall = 1
    assert M.f1_max(s, allm) == 1.0
    # a constant map cannot separate anything: AUROC one half, PRO reaches the region only at FPR 1
    m = none.copy()
    m[3:6, 3:6] = 1
    c = np.full((12, 12), 0.25)
    assert M.auroc(c, m) == 0.5
    fpr, pro = M.pro_curve([c], [m])
    np.testing.assert_allclose(fpr, [0.0, 1.0], atol=1e-12)  # sums of 1/n weights
    np.testing.assert_allclose(pro, [0.0, 1.0], atol=1e-12)
    assert M.aupro([c], [m]) == pytest.approx(0.5 * 0.3 * 0.3 / 0.3)  # the diagonal: area 0.045 over 0.3
    # a border that swallows the image leaves no pixels
    assert np.isnan(M.auroc(s, m, border=6))
