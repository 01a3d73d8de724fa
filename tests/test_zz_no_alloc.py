"""qfca_score_noalloc: the window-EMD score for callers that cannot allocate
device memory (no context, scratch in a fixed device array of the library).

Checked through the C ABI against qfca_score on two calls in a row -- the
second on a smaller image, so scratch left over from the first call would show
-- and for the rejection of images larger than its fixed scratch.  Kept in a
file of its own that pytest collects last.
"""
import ctypes

import numpy as np
import pytest
import torch

from paper_2510_15602_gb300 import synth

pytestmark = pytest.mark.gpu

OK, ERR_UNSUPPORTED = 0, -2


def _lib():
    from paper_2510_15602_gb300 import qfca
    f = qfca._lib.qfca_score_noalloc
    P, I = ctypes.c_void_p, ctypes.c_int
    f.argtypes = [P, I, I, I, I, I, I, P, ctypes.c_uint32, P, P]
    f.restype = I
    return qfca, f


def _case(rng, d, H, W, B):
    qb = synth.random_bins(rng, d, H, W, B)
    pitch = (W + 15) // 16 * 16
    bins = torch.zeros(d, H, pitch, dtype=torch.uint8, device="cuda")
    bins[:, :, :W] = torch.from_numpy(qb).cuda()
    R = np.stack([np.bincount(qb[k].ravel(), minlength=B) for k in range(d)]).astype(np.int32)
    return bins, torch.from_numpy(R).cuda(), pitch


def test_noalloc_score_matches_score_on_two_calls():
    q, f = _lib()
    rng = np.random.default_rng(2024)
    stream = torch.cuda.current_stream()
    for d, H, W, B, r in [(8, 150, 200, 32, 7), (3, 70, 90, 16, 4)]:
        bins, R, pitch = _case(rng, d, H, W, B)
        ref = q.score(bins, W, B, r, R, H * W)
        out = torch.full((H, W), float("nan"), dtype=torch.float32, device="cuda")
        st = f(bins.data_ptr(), H, W, pitch, d, B, r, R.data_ptr(), H * W, out.data_ptr(), stream.cuda_stream)
        assert st == OK
        torch.cuda.synchronize()
        np.testing.assert_allclose(out.cpu().numpy(), ref.cpu().numpy(), rtol=2.0 ** -23, atol=1e-12)


def test_noalloc_rejects_images_beyond_its_scratch():
    q, f = _lib()
    bins = torch.zeros(1, 1, 16, dtype=torch.uint8, device="cuda")
    R = torch.zeros(1, 16, dtype=torch.int32, device="cuda")
    out = torch.zeros(1, dtype=torch.float32, device="cuda")
    st = f(bins.data_ptr(), 1024, 1024, 1024, 1, 16, 3, R.data_ptr(), 1 << 20, out.data_ptr(),
           torch.cuda.current_stream().cuda_stream)
    assert st == ERR_UNSUPPORTED
