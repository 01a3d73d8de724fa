"""Serving session (qfca_serve_start / register_class / submit / poll): every
result equals the same image scored alone through the single-image entry
points with the class's basis, fixed range and reference; admission limits;
host-memory requests; latency stamps."""
import numpy as np
import pytest
import torch

from paper_2510_15602_gb300 import synth
from tests.gpu_helpers import to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def q():
    from paper_2510_15602_gb300 import qfca
    assert torch.cuda.is_available()
    return qfca


def _class_from_training_image(q, ctx, C, H, W, d, B, seed, precision):
    """A class as the paper's per-texture setting fits it: PCA of a training
    image, its component ranges and its global histogram as the reference."""
    X = to_dev(synth.small_case(C=C, H=H, W=W, sigma=2.0, seed=seed, n_square=0, side=4, nch=2).X)
    mean, V, _ = q.fit_pca(X, d, ctx=ctx)
    out = q.quantize(X, (mean, V), B, precision, ctx=ctx)
    torch.cuda.synchronize()
    return dict(mean=mean, V=V, lo=out["lo"].clone(), hi=out["hi"].clone(), hist=out["hist"].clone(), total=H * W)


def _alone(q, ctx, X, cls, d, B, r, precision):
    H, W = int(X.shape[1]), int(X.shape[2])
    out = q.quantize(X, (cls["mean"], cls["V"]), B, precision, lo=cls["lo"], hi=cls["hi"], want_hist=False, ctx=ctx)
    return q.score(out["bins"], W, B, r, cls["hist"], cls["total"], ctx=ctx)


@pytest.mark.parametrize("precision", ["bf16", "f32"])
def test_serving_results_equal_alone_and_in_the_mix(q, precision):
    C, d, B = 64, 16, 32
    ctx = q.Context()
    classes = [_class_from_training_image(q, ctx, C, 64, 64, d, B, 200 + k, precision) for k in range(3)]
    srv = q.Server(C, d, B, precision, max_batch=4, streams=2, arena_bytes=256 << 20)
    try:
        for k, c in enumerate(classes):
            srv.register_class(k, c["mean"], c["V"], c["lo"], c["hi"], c["hist"], c["total"])
        rng = np.random.default_rng(5)
        sizes = [(64, 64), (96, 80), (48, 112), (72, 72)]
        reqs = []
        for i in range(14):
            H, W = sizes[i % len(sizes)]
            X = to_dev(synth.small_case(C=C, H=H, W=W, sigma=2.0, seed=300 + i, n_square=1, side=8, nch=6).X)
            reqs.append((int(rng.integers(0, 3)), X, int(rng.choice([3, 5, 7]))))
        tickets = []
        for k, X, r in reqs:
            t = srv.submit(k, X, r)
            assert t is not None
            tickets.append(t)
        got = []
        for t in tickets:
            res = None
            for _ in range(2000):
                res = srv.poll(t, timeout_us=10000)
                if res is not None:
                    break
            assert res is not None, "request did not finish"
            got.append(res)
        sizes_seen = set()
        batches = {}
        for (k, X, r), (res, sc) in zip(reqs, got):
            assert res.status == 0
            assert res.t_submit_us <= res.t_start_us <= res.t_done_us
            assert 1 <= res.batch_size <= 4
            assert 0 <= res.stream < 2 and res.batch_seq >= 1
            sizes_seen.add(res.batch_size)
            batches[res.batch_seq] = (res.stream, res.t_start_us, res.t_done_us, res.batch_size)
            ref = _alone(q, ctx, X, classes[k], d, B, r, precision)
            torch.cuda.synchronize()
            np.testing.assert_array_equal(sc.cpu().numpy(), ref.cpu().numpy())
        # the mix: some request shared its batch with others ...
        assert max(sizes_seen) > 1, sizes_seen
        # ... and two batches were in flight on the device at once (on different
        # streams, the later one launched before the earlier one completed)
        seqs = sorted(batches)
        overlap = any(batches[a][0] != batches[b][0] and batches[b][1] < batches[a][2]
                      for i, a in enumerate(seqs) for b in seqs[i + 1:])
        assert overlap, batches
    finally:
        srv.stop()
    assert ctx.device_status() == 0


def test_serving_host_memory_requests(q):
    C, d, B = 32, 8, 16
    ctx = q.Context()
    cls = _class_from_training_image(q, ctx, C, 48, 48, d, B, 400, "bf16")
    srv = q.Server(C, d, B, "bf16", max_batch=2, streams=1, arena_bytes=64 << 20)
    try:
        srv.register_class(7, cls["mean"], cls["V"], cls["lo"], cls["hi"], cls["hist"], cls["total"])
        Xh = torch.from_numpy(synth.small_case(C=C, H=40, W=56, sigma=2.0, seed=401, n_square=1, side=6, nch=4).X)
        Xh = Xh.pin_memory()
        t = srv.submit(7, Xh, 4)
        res = None
        for _ in range(1000):
            res = srv.poll(t, timeout_us=10000)
            if res is not None:
                break
        assert res is not None and res[0].status == 0
        assert not res[1].is_cuda
        ref = _alone(q, ctx, Xh.cuda(), cls, d, B, 4, "bf16")
        torch.cuda.synchronize()
        np.testing.assert_array_equal(res[1].numpy(), ref.cpu().numpy())
    finally:
        srv.stop()


def test_serving_admission_limits(q):
    C, d, B = 32, 8, 16
    ctx = q.Context()
    cls = _class_from_training_image(q, ctx, C, 32, 32, d, B, 500, "bf16")
    srv = q.Server(C, d, B, "bf16", max_batch=1, streams=1, max_queue=1, arena_bytes=2 << 20)
    try:
        srv.register_class(0, cls["mean"], cls["V"], cls["lo"], cls["hi"], cls["hist"], cls["total"])
        # a request that can never fit the arena is refused outright
        big = to_dev(np.zeros((C, 512, 512), np.float32))
        with pytest.raises(q.QfcaError):
            srv.submit(0, big, 3)
        # an unknown class is an invalid request
        small = to_dev(synth.small_case(C=C, H=64, W=64, sigma=2.0, seed=501, n_square=0, side=4, nch=2).X)
        with pytest.raises(q.QfcaError):
            srv.submit(99, small, 3)
        # with a one-slot queue, a burst of submissions meets QFCA_ERR_BUSY
        busy, tickets = 0, []
        for i in range(200):
            t = srv.submit(0, small, 3)
            if t is None:
                busy += 1
            else:
                tickets.append(t)
        assert busy > 0 and tickets
        for t in tickets:
            res = None
            for _ in range(2000):
                res = srv.poll(t, timeout_us=10000)
                if res is not None:
                    break
            assert res is not None and res[0].status == 0 and res[0].batch_size == 1
    finally:
        srv.stop()
