"""qfca_batch_run_host: the batch path with the feature maps and score maps in
host memory (the copies on the call's stream) gives the device-resident
qfca_batch_run's maps bit for bit -- with pinned and with pageable buffers,
and replayed from a captured CUDA graph with new host data."""
import ctypes

import numpy as np
import pytest
import torch

from paper_2510_15602_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def q():
    from paper_2510_15602_gb300 import qfca
    assert torch.cuda.is_available()
    return qfca


def _batch(n, C, H, W, seed):
    return np.stack([synth.small_case(C=C, H=H, W=W, sigma=2.0, seed=seed + i, n_square=1, side=8, nch=6).X
                     for i in range(n)])


def test_host_batch_equals_device_batch(q):
    n, C, H, W, d, B, r = 3, 64, 72, 80, 16, 32, 5
    Xh = torch.from_numpy(_batch(n, C, H, W, 40))
    ref = q.batch_run(Xh.cuda(), d, B, r, "bf16").cpu()
    for pinned in (True, False):
        Xs = Xh.pin_memory() if pinned else Xh.clone()
        out = torch.empty(n, H, W, dtype=torch.float32)
        out = out.pin_memory() if pinned else out
        ctx = q.Context()
        s = q.batch_run_host(Xs, d, B, r, "bf16", ctx=ctx, scores=out)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(s.numpy(), ref.numpy())
        assert ctx.device_status() == 0


def test_host_batch_in_a_captured_graph(q):
    n, C, H, W, d, B, r = 2, 48, 64, 64, 8, 16, 4
    X1 = torch.from_numpy(_batch(n, C, H, W, 50)).pin_memory()
    X2 = torch.from_numpy(_batch(n, C, H, W, 60))
    out = torch.empty(n, H, W, dtype=torch.float32).pin_memory()
    ctx = q.Context()
    st = torch.cuda.Stream()
    q.batch_run_host(X1, d, B, r, "f32", ctx=ctx, stream=st, scores=out)  # grows the buffers outside capture
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=st):
        q.batch_run_host(X1, d, B, r, "f32", ctx=ctx, stream=st, scores=out)
    X1.copy_(X2)  # new host data, read by the graph's copy at replay
    g.replay()
    torch.cuda.synchronize()
    ref = q.batch_run(X2.cuda(), d, B, r, "f32").cpu()
    np.testing.assert_array_equal(out.numpy(), ref.numpy())
    assert ctx.device_status() == 0


def test_host_batch_rejects_bad_arguments(q):
    ctx = q.Context()
    fm = q.Fmap(16, 16, 8, q.NCHW)
    out = torch.empty(1, 16, 16, dtype=torch.float32)
    st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    s = q._lib.qfca_batch_run_host(ctx.handle, None, 1, fm, 4, 16, 3, q._PREC["f32"], ctypes.c_void_p(out.data_ptr()), st)
    assert s == q.ERR_INVALID_ARG
    X = torch.zeros(1, 8, 16, 16)
    s = q._lib.qfca_batch_run_host(ctx.handle, ctypes.c_void_p(X.data_ptr()), 0, fm, 4, 16, 3, q._PREC["f32"],
                                   ctypes.c_void_p(out.data_ptr()), st)
    assert s == q.ERR_INVALID_ARG
    with pytest.raises(ValueError):
        q.batch_run_host(X.cuda(), 4, 16, 3, "f32", ctx=ctx)
