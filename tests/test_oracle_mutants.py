"""The oracle's pins have teeth: each plausible mistake below is planted in a
temporary copy of the oracle's C source (on the CPU; the committed oracle is
untouched), the copy is built, and the CPU pin suites run against it in a
fresh interpreter.  Every mutant must fail at least one pin; the unmutated copy
must pass them all (a control for the harness itself).
"""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "qfca_oracle.c")
PIN_FILES = ["tests/test_oracle_golden.py", "tests/test_oracle_pins.py", "tests/test_oracle_assoc_pins.py",
             "tests/test_oracle_median_pins.py", "tests/test_oracle_residual_pins.py"]

# (name, text in the source, the mistake that replaces it; every occurrence is replaced)
MUTANTS = [
    ("alg1: signed instead of absolute bin distance",
     "int64_t dist = i > j ? i - j : j - i;", "int64_t dist = i - j;"),
    ("EMD: N_loc and N_ref swapped in the CDF difference",
     "int64_t diff = cumL * (int64_t)Nref - cumR * Nloc;", "int64_t diff = cumL * Nloc - cumR * (int64_t)Nref;"),
    ("EMD: unclipped window area at the borders",
     "int64_t Nloc = (int64_t)(y1 - y0 + 1) * (x1 - x0 + 1);", "int64_t Nloc = (int64_t)(2 * r + 1) * (2 * r + 1);"),
    ("score: component sum instead of mean",
     "score[(long)y * W + x] = s / (double)d;", "score[(long)y * W + x] = s;"),
    ("quantiser: B-1 instead of B bins across the range",
     "b = (long)floor((y[p] - lo) / (hi - lo) * (double)B);",
     "b = (long)floor((y[p] - lo) / (hi - lo) * (double)(B - 1));"),
    ("covariance: not centred",
     "s += (feat(X, layout, C, N, i, p) - mean[i]) * (feat(X, layout, C, N, j, p) - mean[j]);",
     "s += feat(X, layout, C, N, i, p) * feat(X, layout, C, N, j, p);"),
    ("projection: basis indexed transposed",
     "s += (feat(X, layout, C, N, c, p) - mean[c]) * V[(long)c * d + k];",
     "s += (feat(X, layout, C, N, c, p) - mean[c]) * V[(long)k * C + c];"),
    ("eigensolver: ascending order",
     "if (lj > lb || (lj == lb && order[j] < order[best]))", "if (lj < lb || (lj == lb && order[j] < order[best]))"),
    ("eigensolver: eigenvectors read as rows",
     "V[(long)c * d + k] = sgn * Q[(long)c * C + col];", "V[(long)c * d + k] = sgn * Q[(long)col * C + c];"),
    ("eigensolver: no sign normalisation",
     "double sgn = Q[(long)imax * C + col] < 0.0 ? -1.0 : 1.0;", "double sgn = 1.0;"),
    ("median reference: upper instead of lower median",
     "int med = col[(Np + 1) / 2 - 1];", "int med = col[Np / 2];"),
    ("residual: reconstruction added instead of subtracted",
     "Fres[(long)c * N + p] = (feat(X, layout, C, N, c, p) - mean[c]) - rec;",
     "Fres[(long)c * N + p] = (feat(X, layout, C, N, c, p) - mean[c]) + rec;"),
    ("association: divided by the full window area at the borders",
     "double a = s / (double)n;", "double a = s / (double)((2 * r + 1) * (2 * r + 1));"),
    ("smoothing: Gaussian exponent without the factor 2",
     "exp(-(double)t * t / (2.0 * sigma * sigma))", "exp(-(double)t * t / (sigma * sigma))"),
    ("smoothing: weights not renormalised over the taps inside the image",
     "out[(long)y * W + x] = s / w;", "out[(long)y * W + x] = s + 0.0 * w;"),
    ("single-pixel EMD: N_loc and N_ref swapped",
     "int64_t diff = cumL * (int64_t)Nref - cumR * (int64_t)Nloc;",
     "int64_t diff = cumL * (int64_t)Nloc - cumR * (int64_t)Nref;"),
    ("window histogram: last row of the window dropped",
     "for (int yy = y - r; yy <= y + r; yy++)\n        for (int xx = x - r; xx <= x + r; xx++)\n            if (yy >= 0",
     "for (int yy = y - r; yy < y + r; yy++)\n        for (int xx = x - r; xx <= x + r; xx++)\n            if (yy >= 0"),
    ("quantiser (FP32 decision): rounded instead of floored",
     "else b = (long)v;", "else b = (long)(v + 0.5f);"),
    ("quantiser: the maximum not clamped into the last bin",
     "if (b > B - 1) b = B - 1;", "if (b > B) b = B;"),
    ("reference histogram: first pixel skipped",
     "for (long p = 0; p < N; p++)\n            R[(long)k * B + q[(long)k * N + p]]++;",
     "for (long p = 1; p < N; p++)\n            R[(long)k * B + q[(long)k * N + p]]++;"),
    ("alg1: local masses scaled by N_loc instead of N_ref",
     "Pw[b] = P[b] * Nref;", "Pw[b] = P[b] * Nloc;"),
    ("median reference: last column of full windows skipped",
     "for (int x = r; x < W - r; x++, p++) {", "for (int x = r; x < W - r - 1; x++, p++) {"),
    ("residual: projections of uncentred features",
     "s += (feat(X, layout, C, N, c, p) - mean[c]) * V[(long)c * dres + k];",
     "s += feat(X, layout, C, N, c, p) * V[(long)c * dres + k];"),
    ("Jacobi: stopped at a loose off-diagonal tolerance",
     "if (off <= 1e-15 * frob || off == 0.0)", "if (off <= 1e-3 * frob || off == 0.0)"),
    ("alg1: the walk stops before the last local bin",
     "while (i < B && j < B)", "while (i < B - 1 && j < B)"),
    ("association: per-bin error normalised by N_loc instead of N_ref",
     "e[b] = L[b] > 0 ? (double)En[b] / ((double)L[b] * (double)Nref) : 0.0;",
     "e[b] = L[b] > 0 ? (double)En[b] / ((double)L[b] * (double)Nloc) : 0.0;"),
    ("association: each window's error of its centre's bin instead of the pixel's own bin",
     "s += E[((long)py * W + px) * B + bq];", "s += E[((long)py * W + px) * B + qk[(long)py * W + px]];"),
]

DRIVER = r"""
import sys
import oracle
oracle._SRC = sys.argv[1]
oracle._LIB_PATH = sys.argv[2]
import pytest
sys.exit(pytest.main(["-x", "-q", "-p", "no:cacheprovider", "-m", "not gpu"] + sys.argv[3:]))
"""


def run_pins(tmp_path, tag, text):
    src = tmp_path / f"{tag}.c"
    src.write_text(text)
    lib = tmp_path / f"{tag}.so"
    env = dict(os.environ)
    env["PYTHONPATH"] = ROOT + os.pathsep + env.get("PYTHONPATH", "")
    p = subprocess.run([sys.executable, "-c", DRIVER, str(src), str(lib)] + PIN_FILES, cwd=ROOT, env=env,
                       capture_output=True, text=True, timeout=900)
    return p


def test_unmutated_copy_passes(tmp_path):
    p = run_pins(tmp_path, "control", open(SRC).read())
    assert p.returncode == 0, p.stdout[-3000:]


@pytest.mark.parametrize("name,old,new", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_pins_reject_mutant(tmp_path, name, old, new):
    text = open(SRC).read()
    assert old in text, "the mutated line is no longer in the oracle: update the mutant"
    p = run_pins(tmp_path, "mutant", text.replace(old, new))
    assert p.returncode == 1, f"{name}: pins did not fail (rc {p.returncode})\n" + p.stdout[-3000:]
