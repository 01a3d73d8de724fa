"""The two CDF walks of the window stage (the per-pixel sum over bins of
|cumP_b N_ref - cumR_b N_loc|, the W1 closed form applied to the window and
reference histograms of Sec. 3.1) give the same exact numerators: the
per-thread sequential walk and the warp-shuffle segmented walk (two lanes per
pixel, CDF offset and partial sums exchanged by shuffles).  Every tiling and
both walks must agree bit for bit with the numerator path, which agrees with
the oracle within one FP32 rounding.  The shuffle walk exists for B = 32 with
32-bit numerators; elsewhere the per-thread walk runs and the context reports
it."""
import numpy as np
import pytest
import torch

import oracle
from paper_2510_15602_gb300 import synth
from tests.gpu_helpers import to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def q():
    from paper_2510_15602_gb300 import qfca
    assert torch.cuda.is_available()
    return qfca


TILINGS = [(128, 32, 1), (64, 8, 1), (128, 16, 4), (64, 64, 2), (128, 8, 64)]


def _case(q, d, H, W, B, r, seed):
    rng = np.random.default_rng(seed)
    qb = synth.random_bins(rng, d, H, W, B)
    R = oracle.ref_hist(qb, B)
    bins = torch.zeros(d, H, q.bins_pitch(W), dtype=torch.uint8, device="cuda")
    bins[:, :, :W] = to_dev(qb)
    return qb, R, bins, to_dev(R.astype(np.int32))


# ragged widths (lanes past the image), one-row and one-column-band images, windows
# wider than the image, the 15 x 15 window's radius and larger ones
@pytest.mark.parametrize("d,H,W,B,r,seed", [(5, 70, 150, 32, 7, 0), (32, 64, 64, 32, 7, 1), (3, 1, 45, 32, 3, 2),
                                            (2, 40, 7, 32, 12, 3), (4, 97, 131, 32, 1, 4), (2, 60, 200, 32, 20, 5)])
def test_both_walks_give_the_same_map(q, d, H, W, B, r, seed):
    qb, R, bins, Rd = _case(q, d, H, W, B, r, seed)
    s_o, _, _ = oracle.score(qb, B, r, R, H * W)
    ctx = q.Context()
    ref, numer = q.score(bins, W, B, r, Rd, H * W, want_numer=True, ctx=ctx)
    torch.cuda.synchronize()
    ref, numer = ref.cpu().numpy(), numer.cpu().numpy()
    np.testing.assert_allclose(ref, s_o, rtol=2.0 ** -23, atol=1e-12)
    seen = set()
    for walk in (0, 1):
        ctx.set_cdf_walk(walk)
        # the numerator path with this walk
        _, nw = q.score(bins, W, B, r, Rd, H * W, want_numer=True, ctx=ctx)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(nw.cpu().numpy(), numer)
        for tl in TILINGS:
            for run in (1, 0):  # one band per CTA, or every band of a strip (windows carried over)
                ctx.set_tiling(*tl)
                ctx.set_band_run(run)
                try:
                    s = q.score(bins, W, B, r, Rd, H * W, ctx=ctx)
                except q.QfcaError:
                    continue  # this tiling does not fit shared memory for (B, r)
                torch.cuda.synchronize()
                assert ctx.last_tiling() == tl
                seen.add(ctx.last_cdf_walk())
                np.testing.assert_array_equal(s.cpu().numpy(), ref)
        ctx.set_tiling(0)
        ctx.set_band_run(1)
    assert seen == {0, 1}
    ctx.set_cdf_walk(-1)
    assert ctx.device_status() == 0


def test_shuffle_walk_falls_back_where_it_does_not_exist(q):
    ctx = q.Context()
    ctx.set_cdf_walk(1)
    # B = 64: per-thread walk
    qb, R, bins, Rd = _case(q, 3, 50, 70, 64, 5, 10)
    s = q.score(bins, 70, 64, 5, Rd, 50 * 70, ctx=ctx)
    torch.cuda.synchronize()
    assert ctx.last_cdf_walk() == 0
    s_o, _, _ = oracle.score(qb, 64, 5, R, 50 * 70)
    np.testing.assert_allclose(s.cpu().numpy(), s_o, rtol=2.0 ** -23, atol=1e-12)
    # B = 32 with a numerator past 32 bits ((B-1)(2r+1)^2 N_ref >= 2^32): the 64-bit walk, per thread
    H = W = 300
    qb, R, bins, Rd = _case(q, 1, H, W, 32, 20, 11)
    s = q.score(bins, W, 32, 20, Rd, H * W, ctx=ctx)
    torch.cuda.synchronize()
    assert ctx.last_cdf_walk() == 0
    s_o, _, _ = oracle.score(qb, 32, 20, R, H * W)
    np.testing.assert_allclose(s.cpu().numpy(), s_o, rtol=2.0 ** -23, atol=1e-12)
    with pytest.raises(q.QfcaError):
        ctx.set_cdf_walk(2)
    assert ctx.device_status() == 0


def test_autotuner_chooses_a_walk_and_keeps_results(q):
    # the batch entry points measure both walks (B = 32) with every tiling and keep the fastest
    C, d, B = 64, 16, 32
    sizes, rs = [(80, 96), (96, 64), (64, 136)], [7, 5, 9]
    Xs = [to_dev(synth.small_case(C=C, H=h, W=w, sigma=2.0, seed=120 + i, n_square=1, side=8, nch=6).X)
          for i, (h, w) in enumerate(sizes)]
    ctx = q.Context()
    ctx.set_cdf_walk(0)
    s0 = [s.clone() for s in q.score_batch(Xs, rs, d, B, "bf16", ctx=ctx)]
    ctx.set_cdf_walk(1)
    s1 = [s.clone() for s in q.score_batch(Xs, rs, d, B, "bf16", ctx=ctx)]
    torch.cuda.synchronize()
    assert ctx.last_cdf_walk() == 1
    ctx.set_cdf_walk(-1)
    ctx.set_autotune(True)
    st = q.score_batch(Xs, rs, d, B, "bf16", ctx=ctx)
    torch.cuda.synchronize()
    assert ctx.last_cdf_walk() in (0, 1)
    for a, b, c in zip(s0, s1, st):
        np.testing.assert_array_equal(a.cpu().numpy(), b.cpu().numpy())
        np.testing.assert_array_equal(a.cpu().numpy(), c.cpu().numpy())
    assert ctx.device_status() == 0
