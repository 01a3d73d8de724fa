"""The serving session at the served workload's full size, in the settings the
benchmark runs it with: C = 256, d = 32, B = 32, r = 7, BF16, image sizes 128,
224, 320 and 448 pixels square, classes fitted on 448 x 448 training images with
their own channel covariance, batches of up to 16 requests on three streams.
A burst of requests of every size and both classes is submitted at once, so the
batches mix sizes and classes; every result must equal the same image scored
alone through the single-image entry points (the class's basis, fixed range and
reference) bit for bit, and the run must show batching and overlap."""
import numpy as np
import pytest
import torch

from paper_2510_15602_gb300 import synth

pytestmark = pytest.mark.gpu

C, D, B, R = 256, 32, 32, 7
SIZES = (128, 224, 320, 448)
TRAIN_SIDE = 448


@pytest.fixture(scope="module")
def q():
    from paper_2510_15602_gb300 import qfca
    assert torch.cuda.is_available()
    return qfca


def test_serving_full_size_mix_equals_alone(q):
    ctx = q.Context()
    classes, mixes = [], []
    for k in range(2):
        Q = synth.class_mixing(k, C)
        Xt = torch.from_numpy(synth.make_image("serve_c256", 50000 + k, side=TRAIN_SIDE, class_id=k,
                                               class_mix=Q).X).cuda()
        mean, V, _ = q.fit_pca(Xt, D, ctx=ctx)
        out = q.quantize(Xt, (mean, V), B, "bf16", ctx=ctx)
        torch.cuda.synchronize()
        classes.append(dict(mean=mean, V=V, lo=out["lo"].clone(), hi=out["hi"].clone(),
                            hist=out["hist"].clone(), total=TRAIN_SIDE * TRAIN_SIDE))
        mixes.append(torch.from_numpy(Q).cuda())
    # one unit field per size, mixed on the device by each class's channel mixing
    pool = []
    for j, S in enumerate(SIZES):
        f = torch.from_numpy(synth.make_image("serve_c256", 100 * S + j, side=S).X).cuda()
        for k in range(2):
            pool.append((k, (mixes[k] @ f.reshape(C, -1)).reshape(C, S, S).contiguous()))
    torch.cuda.synchronize()
    srv = q.Server(C, D, B, "bf16", max_batch=16, streams=3, max_queue=1 << 15, arena_bytes=8 << 30)
    try:
        for k, c in enumerate(classes):
            srv.register_class(k, c["mean"], c["V"], c["lo"], c["hi"], c["hist"], c["total"])
        rng = np.random.default_rng(11)
        reqs = [pool[int(rng.integers(0, len(pool)))] for _ in range(24)]
        tickets = []
        for k, X in reqs:
            t = srv.submit(k, X, R)
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
        sizes_seen, batches = set(), {}
        for (k, X), (res, sc) in zip(reqs, got):
            assert res.status == 0
            assert res.t_submit_us <= res.t_start_us <= res.t_done_us
            assert 1 <= res.batch_size <= 16 and 0 <= res.stream < 3
            sizes_seen.add(res.batch_size)
            batches[res.batch_seq] = (res.stream, res.t_start_us, res.t_done_us)
            c = classes[k]
            S = int(X.shape[1])
            out = q.quantize(X, (c["mean"], c["V"]), B, "bf16", lo=c["lo"], hi=c["hi"], want_hist=False, ctx=ctx)
            ref = q.score(out["bins"], S, B, R, c["hist"], c["total"], ctx=ctx)
            torch.cuda.synchronize()
            np.testing.assert_array_equal(sc.cpu().numpy(), ref.cpu().numpy())
        assert max(sizes_seen) > 1, sizes_seen
        seqs = sorted(batches)
        overlap = any(batches[a][0] != batches[b][0] and batches[b][1] < batches[a][2]
                      for i, a in enumerate(seqs) for b in seqs[i + 1:])
        assert overlap, batches
    finally:
        srv.stop()
    assert ctx.device_status() == 0
