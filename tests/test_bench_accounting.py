"""The bench's roofline accounting, on the CPU: the DRAM traffic it reports
per kernel equals the read + write bytes of the committed ncu summaries under
profiles/; the algorithmic work per launch follows the stated per-unit figures
on the 16-image 256x256xC256 batch; achieved/peak arithmetic; the ALU peaks
from unit counts and clocks; the measured peaks file is what the bench reads."""
import importlib.util
import json
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    m = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(m)
    return m


UNITS = {"byte": 1.0, "Kbyte": 1e3, "Mbyte": 1e6, "Gbyte": 1e9}


def profile_bytes(kernel):
    """Read + write DRAM bytes of the last capture in the kernel's summary."""
    txt = open(os.path.join(ROOT, "profiles", f"{kernel}_batch16_256_c256.md")).read()
    vals = {}
    for which in ("read", "write"):
        hits = re.findall(r"`dram__bytes_%s\.sum`\) \| ([0-9.]+) (\w+) \|" % which, txt)
        assert hits, (kernel, which)
        v, u = hits[-1]
        vals[which] = float(v) * UNITS[u]
    return vals["read"] + vals["write"]


def test_traffic_equals_profile_summaries(bench):
    assert bench.NCU_TRAFFIC
    for k, t in bench.NCU_TRAFFIC.items():
        assert abs(t - profile_bytes(k)) <= 1e3, k  # summaries print 6 decimals of their unit


def test_work_per_launch_on_the_batch(bench):
    H = W = 256
    C, d, B, r, n = 256, 32, 32, 7, 16
    N = H * W
    kw = lambda k: bench.kernel_work(k, H, W, C, d, B, r, n)["work"]
    assert kw("k_project_tma") == n * N * (4 * C + 4 * d)          # features read, components written
    assert kw("k_chan_absmax") == n * N * 4 * C
    assert kw("k_quantize") == n * N * 5 * d                       # components read, bins written
    assert kw("k_residual") == n * N * 8 * C
    assert kw("k_gram") == n * N * 3 * 10 * 2 * 128 * 128          # 3 tile pairs of 128 channels at C = 256
    assert kw("k_eig_ff") == n * (4 * 256 ** 3 // 3 + 2 * 256 * 256 * 32)
    assert kw("k_window_emd") == n * N * d * (2 * 15 + 4 * 31)     # 154 ops per (pixel, component)
    assert kw("k_median_ref") == n * (H - 14) * (W - 14) * d * (2 * 15 + 2 * 32)
    assert bench.kernel_work("k_gram", H, W, 512, d, B, r, 1)["work"] == N * 10 * 10 * 2 * 128 * 128


def test_roofline_arithmetic(bench):
    peaks = {"hbm_gbs": 8000.0, "bf16_tflops": 2000.0, "bf16_tflops_sustained": 1600.0, "source": "test"}
    e = bench.roofline_entry("k_project_tma", 2.0, 4, peaks, 256, 256, 256, 32, 32, 7, nimg=16)
    work = 16 * 65536 * (4 * 256 + 4 * 32)
    assert e["avg_launch_us"] == 500.0
    assert e["achieved"] == pytest.approx(work / 5e-4 / 1e9, rel=1e-6)
    assert e["frac"] == pytest.approx(e["achieved"] / 8000.0, abs=1e-4)
    g = bench.roofline_entry("k_gram", 1.0, 1, peaks, 256, 256, 256, 32, 32, 7, nimg=16)
    assert g["peak"] == 1600.0 and g["unit"] == "TFLOP/s"           # a kernel timed inside a long step


def test_alu_peaks_from_unit_counts(bench):
    assert bench.ALU_PEAKS["int32_tops"] == pytest.approx(40.27, abs=0.01)
    assert bench.ALU_PEAKS["fp32_tflops"] == pytest.approx(80.55, abs=0.01)
    assert bench.ALU_PEAKS["ff_tflops"] == pytest.approx(bench.ALU_PEAKS["int32_tops"] / 6)


def test_measured_peaks_are_read(bench):
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if not os.path.exists(path):  # written per machine, not part of the sources
        assert bench.measured_peaks()["source"] == "fallback"
        return
    m = json.load(open(path))
    p = bench.measured_peaks()
    assert p["source"] == "measured"
    assert p["hbm_gbs"] == m["hbm_gbs"] and p["bf16_tflops_sustained"] == m["bf16_tflops_sustained"]


def test_per_kind_auroc(bench):
    import numpy as np
    rng = np.random.default_rng(2)
    H = W = 20
    s1, s2 = rng.random((H, W)), rng.random((H, W))
    m1, m2 = np.zeros((H, W), np.uint8), np.zeros((H, W), np.uint8)
    ka, kb = np.zeros((H, W), np.uint8), np.zeros((H, W), np.uint8)
    ka[3:6, 3:6] = 1          # kind "a" scores high: perfectly separated
    s1[3:6, 3:6] = 2.0
    kb[10:14, 10:14] = 1      # kind "b" scores low: always below the normal pixels
    s2[10:14, 10:14] = -1.0
    m1 |= ka
    m2 |= kb
    out = bench.per_kind_auroc([s1, s2], [m1, m2], [{"a": ka}, {"b": kb}], border=2)
    assert out == {"a": 1.0, "b": 0.0}
    # a kind whose pixels all lie inside the discarded border has no positives
    kc = np.zeros((H, W), np.uint8)
    kc[0, :] = 1
    out = bench.per_kind_auroc([s1], [kc], [{"c": kc}], border=2)
    assert out == {"c": None}


def test_aniso_inputs_keep_the_anomalies(bench):
    import numpy as np
    (X0, m0), = bench.make_inputs([2])
    (X1, m1), = bench.make_inputs([2], aniso=True)
    np.testing.assert_array_equal(m0, m1)          # same anomalies, same places
    assert not np.allclose(X0, X1)
    # away from the anomalies the mixed field has the class's channel spectrum (0.9^k, mean 1)
    Z = X1[:, m1 == 0].astype(np.float64)
    lam = np.sort(np.linalg.eigvalsh(np.cov(Z)))[::-1]
    assert lam[0] > 5 * lam[len(lam) // 2]          # strongly anisotropic, unlike the unit field


def test_host_cpu(bench):
    h = bench.host_cpu()
    assert isinstance(h["cpu_model"], str) and h["cpu_model"]
    assert isinstance(h["cores_available"], int) and h["cores_available"] >= 1


def test_clock_sampler_summarises_the_timed_region(bench):
    import datetime

    class Proc:
        def terminate(self):
            pass

        def wait(self, timeout=None):
            pass

    class Thread:
        def join(self, timeout=None):
            pass

    base = datetime.datetime(2026, 1, 2, 3, 4, 5)

    def line(dt, sm, pcap="Not Active", hw="Not Active"):
        ts = (base + datetime.timedelta(seconds=dt)).strftime("%Y/%m/%d %H:%M:%S.%f")[:-3]
        return (0.0, f"{ts}, 0, {sm}, 2070, 900, 0x0, {hw}, Not Active, Not Active, {pcap}")

    c = bench.ClockSampler("0")
    c.proc, c.thread = Proc(), Thread()
    c.lines = [line(0.00, 1400), line(0.05, 2070, pcap="Active"), line(0.10, 2060), line(0.40, 900, hw="Active")]
    t0 = base.timestamp()
    out = c.stop(t0 + 0.04, t0 + 0.12)   # the nvidia-smi stamps decide, not the arrival times
    assert out["samples"] == 2 and out["samples_from"] == "inside the timed region"
    assert out["sm_mhz"] == 2065.0 and out["sm_max_mhz"] == 2070.0
    assert out["reasons"] == ["sw_power_cap"]          # the hw_slowdown sample lies outside
    out = c.stop(t0 + 0.20, t0 + 0.25)   # no sample inside: the nearest one is reported, and said so
    assert out["samples"] == 1 and out["sm_mhz"] == 2060.0 and "nearest" in out["samples_from"]
