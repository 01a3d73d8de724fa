"""Host-side model of the FP32 bin decision of Sec. 3.1 (uniform bins between
lo and hi) and of its edge form, for tests: every IEEE-rounded step of
t = (y - lo) / (hi - lo), v = t B, q = clamp(trunc(v), 0, B - 1) is monotone
in y, so q is a step function of y and equals the number of edges
e_j = min{y : q(y) >= j} (j = 1..B-1) at or below y."""
import numpy as np

f32 = np.float32


def decision(y, lo, hi, B):
    """The FP32 decision, one value at a time (IEEE float32 arithmetic)."""
    y, lo, hi = f32(y), f32(lo), f32(hi)
    if not hi > lo:
        return 0
    with np.errstate(invalid="ignore", over="ignore"):
        v = (f32(y - lo) / f32(hi - lo)) * f32(B)
    if np.isnan(v) or v < 0:
        return 0
    return int(min(float(v), B - 1))


def key(f):
    u = int(np.array(f, dtype=np.float32).view(np.uint32))
    return (~u & 0xFFFFFFFF) if u & 0x80000000 else u | 0x80000000


def unkey(k):
    u = (k & 0x7FFFFFFF) if k & 0x80000000 else (~k & 0xFFFFFFFF)
    return np.array(u, dtype=np.uint32).view(np.float32)[()]


def edges(lo, hi, B):
    """e_1 .. e_{B-1} by bisection over the order-preserving keys of the floats."""
    out = []
    for j in range(1, B):
        a, b = key(f32(-np.inf)), key(f32(np.inf))
        while b - a > 1:
            m = a + (b - a) // 2
            if decision(unkey(m), lo, hi, B) >= j:
                b = m
            else:
                a = m
        out.append(unkey(b))
    return np.array(out, dtype=np.float32)
