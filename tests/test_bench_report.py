"""bench.py's report helpers on made-up timings (no GPU): the roofline of each
tridiagonalisation kernel is its algorithmic flops over the time of its own flop mix
at the peaks, and the dominant kernel is the roofline kernel with the most time."""
import os
import sys

import numpy as np

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402


def test_roofline_fp64_tridiag_at_peak():
    n = np.array([600, 700])
    flops = float(np.sum(4.0 * n.astype(float) ** 3 / 3.0))
    # a launch that runs exactly at the 1:1 mix of 1.0 and 2.0 TFLOP/s
    t = (flops / 2) / 1e12 + (flops / 2) / 2e12
    r = bench.roofline_report("k_tridiag", "fp64", n, t * 1e3, 1, 1.0, 2.0, 1700.0, "test")
    assert abs(r["frac"] - 1.0) < 1e-12
    assert abs(r["flops_per_launch"] - flops) < 1e-3 * flops


def test_roofline_mixed_band_and_chase():
    n = np.array([700])
    r = bench.roofline_report("k_band", "mixed", n, 100.0, 1, 1.0, 1.0, 1700.0, "test")
    gemm = 4.0 * 700.0 ** 3 / 3.0
    floor = 4.0 * 700 ** 2 * 32 / 1e12 + 36 * gemm / 1700e12
    assert abs(r["floor_ms"] - floor * 1e3) < 1e-9
    c = bench.roofline_report("k_chase", "mixed", n, 1.0, 1, 1.0, 1.0, 1700.0, "test")
    assert c["flops_per_launch"] == 6.0 * 700 ** 2 * 32


def test_dominant_and_fmin():
    times = {"k_tridiag": (5.0, 1), "k_band": (9.0, 1), "k_chase": (2.0, 1), "k_ql": (50.0, 1)}
    assert bench.dominant(times) == "k_band"
    assert bench.dominant({"k_ql": (1.0, 1)}) == "k_tridiag"
    n3 = np.array([700.0]) ** 3
    r64 = bench.step_fmin_report("fp64", n3, 1000.0, 1.0, 1.0, 1700.0)
    assert abs(r64["frac"] - (8.0 / 3.0 * 700 ** 3 / 1e12) / 1.0) < 1e-12
    r2 = bench.step_fmin_report("mixed", n3, 1000.0, 1.0, 1.0, 1700.0, two_stage=True)
    assert abs(r2["floor_ms"] - 36 * 8.0 / 3.0 * 700 ** 3 / 1700e12 * 1e3) < 1e-9
