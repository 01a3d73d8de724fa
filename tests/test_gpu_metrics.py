"""The GPU metric suite (qfca_metrics: pixel AUROC, F1 at the optimal
threshold, AUPRO at an FPR limit and image-level AUROC, Sec. 4.2, after a
border discard) against the host implementation in metrics.py, which is
pinned against sklearn and brute force on the CPU.  The pixel and image AUROC
are exact integer statistics on both sides; F1 and AUPRO are FP64 sums taken
in different orders, so they agree to a few ulps of their size."""
import numpy as np
import pytest
import torch

from paper_2510_15602_gb300 import metrics as hm
from paper_2510_15602_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def q():
    from paper_2510_15602_gb300 import qfca
    assert torch.cuda.is_available()
    return qfca


def _host(scores, masks, border, limit=0.3):
    return {"pixel_auroc": hm.auroc(scores, masks, border), "f1_max": hm.f1_max(scores, masks, border),
            "aupro": hm.aupro(list(scores), list(masks), limit, border), "image_auroc": hm.image_auroc(list(scores), list(masks), border)}


def _compare(g, h):
    for k in ("pixel_auroc", "image_auroc"):
        if np.isnan(h[k]):
            assert np.isnan(g[k]), (k, g[k])
        else:
            assert abs(g[k] - h[k]) <= 1e-13, (k, g[k], h[k])
    for k in ("f1_max", "aupro"):
        if np.isnan(h[k]):
            assert np.isnan(g[k]), (k, g[k])
        else:
            assert abs(g[k] - h[k]) <= 1e-10 * max(1.0, abs(h[k])), (k, g[k], h[k])


def _random_case(rng, n, H, W, levels):
    sc = rng.random((n, H, W)).astype(np.float32)
    if levels:
        sc = (np.floor(sc * levels) / levels).astype(np.float32)  # many ties
    mk = np.zeros((n, H, W), np.uint8)
    for i in range(n):
        for _ in range(int(rng.integers(0, 5))):
            y, x = int(rng.integers(0, H - 4)), int(rng.integers(0, W - 4))
            mk[i, y:y + int(rng.integers(1, 5)), x:x + int(rng.integers(1, 5))] = 1
            sc[i, y:y + 3, x:x + 3] += np.float32(0.3)
        if rng.random() < 0.3:
            mk[i, int(rng.integers(0, H)), int(rng.integers(0, W))] = 1  # one-pixel region
    return sc, mk


@pytest.mark.parametrize("seed", range(6))
def test_metrics_random_maps_with_ties_regions_and_borders(q, seed):
    rng = np.random.default_rng(seed)
    for levels in (0, 5, 40):
        n, H, W = int(rng.integers(2, 6)), int(rng.integers(12, 70)), int(rng.integers(12, 70))
        sc, mk = _random_case(rng, n, H, W, levels)
        for border in (0, 3):
            g = q.metrics(torch.from_numpy(sc).cuda(), torch.from_numpy(mk).cuda(), border=border)
            _compare(g, _host(sc, mk, border))


def test_metrics_on_score_maps_of_the_path(q):
    # maps from the whole path on seeded anomaly images, border r as the paper's evaluation
    imgs = [synth.small_case(C=48, H=64, W=72, sigma=2.0, seed=300 + i, n_square=1, side=8, nch=6) for i in range(4)]
    X = torch.stack([torch.from_numpy(im.X).cuda() for im in imgs])
    s = q.batch_run(X, 8, 16, 4, "f32")
    masks = np.stack([im.mask for im in imgs]).astype(np.uint8)
    masks[3] = 0  # one normal image, so the image-level AUROC is defined
    torch.cuda.synchronize()
    sc = s.cpu().numpy()
    g = q.metrics(s, torch.from_numpy(masks).cuda(), border=4)
    _compare(g, _host(sc, masks, 4))


def test_metrics_eight_connected_regions(q):
    # two diagonal neighbours are one region (8-connectivity): AUPRO weighs them as one
    sc = np.zeros((1, 10, 10), np.float32)
    mk = np.zeros((1, 10, 10), np.uint8)
    mk[0, 2, 2] = mk[0, 3, 3] = 1          # one region of two pixels
    mk[0, 7, 1] = 1                        # one region of one pixel
    sc[0, 2, 2], sc[0, 3, 3], sc[0, 7, 1] = 0.9, 0.1, 0.5
    sc[0, 5, 5] = 0.7                      # a normal pixel above two anomalous ones
    g = q.metrics(torch.from_numpy(sc).cuda(), torch.from_numpy(mk).cuda(), fpr_limit=1.0)
    _compare(g, _host(sc, mk, 0, 1.0))


def test_metrics_degenerate_inputs(q):
    sc = np.random.default_rng(0).random((2, 16, 16)).astype(np.float32)
    none = np.zeros((2, 16, 16), np.uint8)
    g = q.metrics(torch.from_numpy(sc).cuda(), torch.from_numpy(none).cuda())
    assert all(np.isnan(g[k]) for k in g)
    allpos = np.ones((2, 16, 16), np.uint8)
    g = q.metrics(torch.from_numpy(sc).cuda(), torch.from_numpy(allpos).cuda())
    assert np.isnan(g["pixel_auroc"]) and np.isnan(g["aupro"]) and np.isnan(g["image_auroc"])
    assert g["f1_max"] == 1.0
    const = np.full((2, 16, 16), 0.25, np.float32)
    mk = none.copy()
    mk[0, 4:8, 4:8] = 1
    g = q.metrics(torch.from_numpy(const).cuda(), torch.from_numpy(mk).cuda())
    assert g["pixel_auroc"] == 0.5 and g["image_auroc"] == 0.5
    _compare(g, _host(const, mk, 0))
    with pytest.raises(q.QfcaError):
        q.metrics(torch.from_numpy(sc).cuda(), torch.from_numpy(mk).cuda(), border=8)


def test_metrics_full_batch_size(q):
    # the bench's 16 maps of 256 x 256 with a border of 7: 937 k kept pixels (a 2^20-word sort)
    rng = np.random.default_rng(9)
    sc = rng.random((16, 256, 256)).astype(np.float32)
    sc = (np.floor(sc * 3000) / 3000).astype(np.float32)
    mk = np.zeros((16, 256, 256), np.uint8)
    for i in range(16):
        for _ in range(3):
            y, x = int(rng.integers(10, 200)), int(rng.integers(10, 200))
            mk[i, y:y + 30, x:x + 20] = 1
            sc[i, y:y + 30, x:x + 20] += np.float32(0.2)
    mk[15] = 0
    ctx = q.Context()
    g = q.metrics(torch.from_numpy(sc).cuda(), torch.from_numpy(mk).cuda(), border=7, ctx=ctx)
    _compare(g, _host(sc, mk, 7))
    assert ctx.device_status() == 0  # no union-find loop reached its limit


def test_metrics_signed_zero_scores_are_one_threshold(q):
    # -0 and +0 are one score value: a run of ties across both signs, on anomalous and normal pixels
    rng = np.random.default_rng(21)
    sc = (np.floor(rng.random((3, 24, 20)) * 4) / 4).astype(np.float32)  # 0, 0.25, 0.5, 0.75
    sc[(sc == 0) & (rng.random(sc.shape) < 0.5)] = np.float32(-0.0)    # about half the zeros become -0
    assert np.signbit(sc[sc == 0]).any() and (~np.signbit(sc[sc == 0])).any()
    mk = np.zeros(sc.shape, np.uint8)
    mk[0, 4:12, 3:9] = 1
    mk[1, 10:20, 10:18] = 1
    g = q.metrics(torch.from_numpy(sc).cuda(), torch.from_numpy(mk).cuda(), border=2)
    _compare(g, _host(sc, mk, 2))
    # the same maps with every zero positive give the same metrics bit for bit
    g0 = q.metrics(torch.from_numpy(np.where(sc == 0, np.float32(0.0), sc)).cuda(), torch.from_numpy(mk).cuda(), border=2)
    assert g == g0
