"""The edge form of the FP32 bin decision gives the decision itself: at every
edge, at the floats next to it, and on random values (IEEE float32 arithmetic
on the host; the GPU quantiser uses the same form)."""
import numpy as np

from tests.quant_edges import decision, edges, f32


def _count(y, e):
    return int(np.sum(e <= f32(y)))


def test_edges_reproduce_the_decision():
    rng = np.random.default_rng(5)
    for lo, hi, B in [(-2.7, 3.1, 32), (0.0, 1.0, 16), (-1e-3, 5e-4, 64), (-41.5, -40.25, 7), (1e6, 1e6 + 3.0, 255)]:
        lo, hi = f32(lo), f32(hi)
        e = edges(lo, hi, B)
        assert np.all(np.diff(e) >= 0)
        probes = list(e) + [np.nextafter(v, f32(-np.inf)) for v in e] + [np.nextafter(v, f32(np.inf)) for v in e]
        span = float(hi - lo)
        probes += list(rng.uniform(float(lo) - 0.2 * span, float(hi) + 0.2 * span, 400).astype(np.float32))
        probes += [lo, hi, f32(0.0), f32(-0.0), f32(np.inf), f32(-np.inf)]
        for y in probes:
            assert _count(y, e) == decision(y, lo, hi, B), (lo, hi, B, y)
        # the edges are the first floats of their bins
        for j, v in enumerate(e, start=1):
            assert decision(v, lo, hi, B) >= j > decision(np.nextafter(v, f32(-np.inf)), lo, hi, B)


def test_degenerate_range_is_bin_zero():
    assert decision(f32(3.0), f32(1.0), f32(1.0), 16) == 0
    assert decision(f32(np.nan), f32(0.0), f32(1.0), 16) == 0
