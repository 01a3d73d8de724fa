"""qfca_score_noalloc: the window-EMD score for callers that cannot allocate
device memory -- code whose host application or memory manager owns every
device allocation, processes with a hard device-memory budget, loops that
cannot take cudaMalloc's implicit synchronisation.  It takes no context and
keeps its scratch in a fixed device array of the library.

Checked through the C ABI against qfca_score: bit for bit (both sum the same
exact integer numerators and divide once in FP64) on two calls in a row -- the
second on a smaller image, so scratch left over from the first call would show
-- and on two calls enqueued back to back on one stream with no host
synchronisation between them; images larger than the fixed scratch are
rejected; a bounded wait made to run out is reported by
qfca_score_noalloc_status and cleared by it.  Kept in a file of its own that
pytest collects last.
"""
import ctypes

import numpy as np
import pytest
import torch

from paper_2510_15602_gb300 import synth

pytestmark = pytest.mark.gpu

OK, ERR_UNSUPPORTED, ERR_TIMEOUT = 0, -2, -5


def _lib():
    from paper_2510_15602_gb300 import qfca
    lib = qfca._lib
    P, I = ctypes.c_void_p, ctypes.c_int
    f = lib.qfca_score_noalloc
    f.argtypes = [P, I, I, I, I, I, I, P, ctypes.c_uint32, P, P]
    f.restype = I
    lib.qfca_score_noalloc_status.argtypes = [ctypes.POINTER(I), P]
    lib.qfca_score_noalloc_status.restype = I
    lib.qfca_score_noalloc_test_wait_limit.argtypes = [I]
    lib.qfca_score_noalloc_test_wait_limit.restype = I
    return qfca, lib


def _case(rng, d, H, W, B):
    qb = synth.random_bins(rng, d, H, W, B)
    pitch = (W + 15) // 16 * 16
    bins = torch.zeros(d, H, pitch, dtype=torch.uint8, device="cuda")
    bins[:, :, :W] = torch.from_numpy(qb).cuda()
    R = np.stack([np.bincount(qb[k].ravel(), minlength=B) for k in range(d)]).astype(np.int32)
    return bins, torch.from_numpy(R).cuda(), pitch


def _status(lib, stream):
    w = ctypes.c_int(-1)
    st = lib.qfca_score_noalloc_status(ctypes.byref(w), stream.cuda_stream)
    return st, w.value


def test_noalloc_score_equals_score_on_two_calls():
    q, lib = _lib()
    rng = np.random.default_rng(2024)
    stream = torch.cuda.current_stream()
    for d, H, W, B, r in [(8, 150, 200, 32, 7), (3, 70, 90, 16, 4)]:
        bins, R, pitch = _case(rng, d, H, W, B)
        ref = q.score(bins, W, B, r, R, H * W)
        out = torch.full((H, W), float("nan"), dtype=torch.float32, device="cuda")
        st = lib.qfca_score_noalloc(bins.data_ptr(), H, W, pitch, d, B, r, R.data_ptr(), H * W, out.data_ptr(),
                                    stream.cuda_stream)
        assert st == OK
        torch.cuda.synchronize()
        np.testing.assert_array_equal(out.cpu().numpy(), ref.cpu().numpy())
    assert _status(lib, stream) == (OK, 0)


def test_noalloc_back_to_back_on_one_stream():
    # two calls enqueued one after the other with no host synchronisation: the
    # second call's clearing of the shared scratch is ordered after the first
    # call's finalisation by the stream alone
    q, lib = _lib()
    rng = np.random.default_rng(77)
    stream = torch.cuda.current_stream()
    cases = [(5, 120, 130, 32, 6), (4, 96, 64, 64, 3)]
    made = [_case(rng, d, H, W, B) for d, H, W, B, _ in cases]
    refs = [q.score(bins, W, B, r, R, H * W) for (d, H, W, B, r), (bins, R, _) in zip(cases, made)]
    torch.cuda.synchronize()
    outs = []
    for (d, H, W, B, r), (bins, R, pitch) in zip(cases, made):
        out = torch.full((H, W), float("nan"), dtype=torch.float32, device="cuda")
        assert lib.qfca_score_noalloc(bins.data_ptr(), H, W, pitch, d, B, r, R.data_ptr(), H * W, out.data_ptr(),
                                      stream.cuda_stream) == OK
        outs.append(out)
    torch.cuda.synchronize()
    for out, ref in zip(outs, refs):
        np.testing.assert_array_equal(out.cpu().numpy(), ref.cpu().numpy())


def test_noalloc_rejects_images_beyond_its_scratch():
    q, lib = _lib()
    bins = torch.zeros(1, 1, 16, dtype=torch.uint8, device="cuda")
    R = torch.zeros(1, 16, dtype=torch.int32, device="cuda")
    out = torch.zeros(1, dtype=torch.float32, device="cuda")
    st = lib.qfca_score_noalloc(bins.data_ptr(), 1024, 1024, 1024, 1, 16, 3, R.data_ptr(), 1 << 20, out.data_ptr(),
                                torch.cuda.current_stream().cuda_stream)
    assert st == ERR_UNSUPPORTED


def test_noalloc_reports_a_wait_that_ran_out():
    # each CTA's first tile wait gives up without probing: the kernel waits for
    # its copies in flight, sets the status word and returns; the status call
    # reports it once and clears it, and the normal limit gives the right map again
    q, lib = _lib()
    rng = np.random.default_rng(9)
    stream = torch.cuda.current_stream()
    d, H, W, B, r = 4, 64, 80, 32, 5
    bins, R, pitch = _case(rng, d, H, W, B)
    ref = q.score(bins, W, B, r, R, H * W)
    torch.cuda.synchronize()
    assert _status(lib, stream) == (OK, 0)
    out = torch.full((H, W), float("nan"), dtype=torch.float32, device="cuda")
    try:
        assert lib.qfca_score_noalloc_test_wait_limit(1) == OK
        assert lib.qfca_score_noalloc(bins.data_ptr(), H, W, pitch, d, B, r, R.data_ptr(), H * W, out.data_ptr(),
                                      stream.cuda_stream) == OK
    finally:
        lib.qfca_score_noalloc_test_wait_limit(0)
    st, word = _status(lib, stream)
    assert st == ERR_TIMEOUT and word != 0
    assert _status(lib, stream) == (OK, 0)
    assert lib.qfca_score_noalloc(bins.data_ptr(), H, W, pitch, d, B, r, R.data_ptr(), H * W, out.data_ptr(),
                                  stream.cuda_stream) == OK
    assert _status(lib, stream) == (OK, 0)
    np.testing.assert_array_equal(out.cpu().numpy(), ref.cpu().numpy())
