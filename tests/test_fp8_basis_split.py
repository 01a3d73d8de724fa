"""The FP8 projection's basis format (Sec. 3.3 projection at e4m3 precision), modelled
on the CPU from the e4m3 definition (1 sign, 4 exponent bits with bias 7, 3
mantissa bits; normal exponents -6..8, subnormals in steps of 2^-9, largest finite
value 448; round to nearest even, saturating): a basis column scaled by a power of
two so that its largest entry is at most 448 loses up to 2^-4 of each normal
entry's magnitude when rounded once, and the hi + lo pair (hi = e4m3(b),
lo = e4m3(b - hi)) keeps every entry within 2^-8 of its magnitude (plus the
subnormal step of lo), which is why the kernel multiplies both parts into the
same FP32 accumulator."""
import numpy as np


def e4m3(x):
    """Round to the nearest e4m3 value (ties to even), saturating at +-448."""
    x = np.asarray(x, np.float64)
    a = np.minimum(np.abs(x), 448.0)
    e = np.floor(np.log2(np.where(a > 0, a, 1.0)))
    e = np.clip(e, -6, 8)                  # below 2^-6 the spacing stays 2^-9 (subnormals)
    step = 2.0 ** (e - 3)
    q = a / step
    r = np.floor(q)
    frac = q - r
    r = np.where((frac > 0.5) | ((frac == 0.5) & (r % 2 == 1)), r + 1, r)
    return np.sign(x) * np.minimum(r * step, 448.0)


def test_e4m3_model_grid():
    # every representable positive value round-trips; the grid has 8 values per binade
    vals = sorted({float(v) for v in e4m3(np.linspace(0, 448, 200001))})
    assert vals[0] == 0.0 and vals[1] == 2.0 ** -9 and vals[-1] == 448.0
    np.testing.assert_array_equal(e4m3(np.array(vals)), vals)
    assert len([v for v in vals if 1.0 <= v < 2.0]) == 8


def test_hi_lo_split_error():
    rng = np.random.default_rng(4)
    for _ in range(50):
        b = rng.standard_normal(256) * 2.0 ** rng.uniform(-8, 8)
        t = 2.0 ** np.floor(np.log2(448.0 / np.abs(b).max()))  # per-column power of two
        bs = b * t
        hi = e4m3(bs)
        lo = e4m3(bs - hi)
        normal = np.abs(bs) >= 2.0 ** -6
        one = np.abs(bs - hi)
        two = np.abs(bs - (hi + lo))
        assert (one[normal] <= 2.0 ** -4 * np.abs(bs[normal]) + 1e-300).all()
        assert (two <= 2.0 ** -8 * np.abs(bs) + 2.0 ** -10).all()
        assert one.max() > 8 * two.max()   # the pair is far more accurate than one rounding
