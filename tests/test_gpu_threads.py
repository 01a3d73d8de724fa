"""Launches from several host threads at once, each thread with its own
context and stream, in a fresh process so that the threads race for every
launcher's first (once-per-device) kernel-attribute setup: the whole batch path,
the PCA fit, the QFCA+ residual quantisation, the paper's association scoring
and the median reference.  Every thread's results must equal, bit for bit, the
same calls made afterwards one after another on one stream."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SCRIPT = r"""
import threading
import numpy as np
import torch
from paper_2510_15602_gb300 import qfca, synth

C, H, W, d, B, r, dres, T = 64, 48, 40, 8, 16, 3, 4, 4
Xs = []
for t in range(T):
    imgs = [synth.small_case(C=C, H=H, W=W, sigma=2.0, seed=900 + 2 * t + j, n_square=1, side=6, nch=4).X
            for j in range(2)]
    Xs.append(torch.from_numpy(np.stack(imgs)).cuda())
torch.cuda.synchronize()


def run(X, ctx, st):
    s, ex = qfca.batch_run(X, d, B, r, "bf16", ctx=ctx, stream=st, extras=True)
    mean, V, _ = qfca.fit_pca(X[0], dres, ctx=ctx, stream=st)
    res = qfca.quantize_residual(X[0], (mean, V), B, ctx=ctx, stream=st)
    bins, hist = ex["bins"][0], ex["ref_hist"][0]
    a = qfca.score_assoc(bins, W, B, r, hist, H * W, sigma_s=1.0, ctx=ctx, stream=st)
    m = qfca.median_reference(bins, W, B, r, ctx=ctx, stream=st)
    st.synchronize()
    return [s, V, res["bins"][:, :, :W], res["hist"], a, m]  # bins without the row padding


barrier = threading.Barrier(T)
got = [None] * T
err = []


def worker(t):
    try:
        ctx = qfca.Context()
        st = torch.cuda.Stream()
        barrier.wait()
        with torch.cuda.stream(st):
            got[t] = [x.clone() for x in run(Xs[t], ctx, st)]
    except Exception as e:  # reported by the main thread
        err.append(repr(e))


ths = [threading.Thread(target=worker, args=(t,)) for t in range(T)]
for th in ths:
    th.start()
for th in ths:
    th.join()
assert not err, err
ctx = qfca.Context()
st = torch.cuda.Stream()
for t in range(T):
    with torch.cuda.stream(st):
        want = run(Xs[t], ctx, st)
    for g, w in zip(got[t], want):
        assert torch.equal(g, w), t
print("threads ok")
"""


def test_concurrent_first_launches_from_threads():
    env = dict(os.environ)
    env["PYTHONPATH"] = ROOT + os.pathsep + env.get("PYTHONPATH", "")
    p = subprocess.run([sys.executable, "-c", SCRIPT], cwd=ROOT, env=env, capture_output=True, text=True,
                       timeout=600)
    assert p.returncode == 0, p.stdout[-2000:] + p.stderr[-4000:]
    assert "threads ok" in p.stdout
