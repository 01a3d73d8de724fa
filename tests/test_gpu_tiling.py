"""The window stage's tilings give identical maps (Sec. 3.1 window EMD and the
channel mean): with one component group per CTA the kernel sums all d exact
numerators per pixel in shared memory and writes the score itself (the fused
form); with several groups the per-component numerators go through the
finalisation launch.  Both divide the same exact integer sum once in FP64, so
every tiling must agree bit for bit with the numerator path, and within one
FP32 rounding with the oracle.  Tilings are forced through qfca_set_tiling;
a CTA may also take a run of consecutive bands (qfca_set_band_run), sliding
its windows on from one band into the next, which must not change a bit
either."""
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


TILINGS = [(128, 32, 1), (128, 16, 1), (64, 8, 1), (64, 64, 1), (128, 32, 2), (64, 16, 4), (128, 8, 64)]


@pytest.mark.parametrize("d,H,W,B,r,seed", [(5, 70, 150, 32, 7, 0), (3, 33, 129, 64, 12, 1), (1, 1, 40, 16, 3, 2),
                                            (32, 64, 64, 32, 7, 3), (4, 90, 37, 255, 4, 4)])
def test_every_tiling_gives_the_same_map(q, d, H, W, B, r, seed):
    rng = np.random.default_rng(seed)
    qb = synth.random_bins(rng, d, H, W, B)
    R = oracle.ref_hist(qb, B)
    s_o, _, _ = oracle.score(qb, B, r, R, H * W)
    bins = torch.zeros(d, H, q.bins_pitch(W), dtype=torch.uint8, device="cuda")
    bins[:, :, :W] = to_dev(qb)
    Rd = to_dev(R.astype(np.int32))
    ctx = q.Context()
    ref, _ = q.score(bins, W, B, r, Rd, H * W, want_numer=True, ctx=ctx)  # the numerator path, never fused
    torch.cuda.synchronize()
    ref = ref.cpu().numpy()
    np.testing.assert_allclose(ref, s_o, rtol=2.0 ** -23, atol=1e-12)
    fused_seen = False
    runs_seen = set()
    for tl in TILINGS:
        for run in (1, 2, 3, 0):
            ctx.set_tiling(*tl)
            ctx.set_band_run(run)
            try:
                s = q.score(bins, W, B, r, Rd, H * W, ctx=ctx)
            except q.QfcaError:
                continue  # this tiling does not fit shared memory for (B, r)
            torch.cuda.synchronize()
            used = ctx.last_tiling()
            assert used == tl
            nby = (H + tl[1] - 1) // tl[1]
            kg = -(-d // tl[2])
            fused = -(-d // kg) == 1
            # a fused tiling (one group) takes one band; 0 asks for every band of the strip
            want = 1 if fused else min(run if run > 0 else nby, nby)
            assert ctx.last_band_run() == want
            runs_seen.add(want)
            fused_seen = fused_seen or fused
            np.testing.assert_array_equal(s.cpu().numpy(), ref)
    ctx.set_tiling(0)
    ctx.set_band_run(1)
    assert fused_seen
    if d > 1 and H > 16:
        assert max(runs_seen) > 1
    assert ctx.device_status() == 0
