"""Host logic of bench.py on the CPU: the clock-record summary that decides
whether a run is kept (median SM clock under load, throttle reasons), the
algorithmic flop count behind the roofline figure, and the derived FP32 peak."""

import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

bench = pytest.importorskip("bench")


def _row(sm, mx, hw="Not Active", hwt="Not Active", swt="Not Active", cap="Not Active"):
    # index, clocks.sm, clocks.max.sm, power.draw, reasons.active, hw_slowdown,
    # hw_thermal_slowdown, sw_thermal_slowdown, sw_power_cap (nounits csv)
    return ["0", sm, mx, "900.5", "0x0000000000000000", hw, hwt, swt, cap]


def test_clock_summary_median_and_reasons():
    s = bench.ClockSampler(0)
    s.rows = [_row("2070", "2070"), _row("2055", "2070", cap="Active"),
              _row("2070", "2040"), _row("[N/A]", "2070"), _row("2070", "2070")]
    out = s.summary()
    assert out["sm_mhz"] == 2070.0 and out["sm_max_mhz"] == 2070.0
    assert out["reasons"] == ["sw_power_cap"] and out["samples"] == 5


def test_clock_summary_flags_thermal_and_unsampled():
    s = bench.ClockSampler(0)
    s.rows = [_row("1500", "2070", hwt="Active"), _row("1490", "2070", swt="Active")]
    out = s.summary()
    assert out["sm_mhz"] == pytest.approx(1495.0)
    assert out["reasons"] == ["hw_thermal_slowdown", "sw_thermal_slowdown"]
    assert bench.ClockSampler(0).summary()["reasons"] == ["unsampled"]


def test_pass_b_flop_count_by_hand():
    """Pass B of one 16-direction launch at 256^2: per column (Py = 1024 of
    them) and field (3 per direction), a length-1024 FFT, two parity products,
    two inverse FFTs of 1024, the kernel-table product, two inverse FFTs of
    512 and the combination at the 257 nodes; 5 n log2 n flops per FFT,
    6 per complex product."""
    w = dict(nx=256, ny=256)
    f1024, f512 = 5 * 1024 * 10, 5 * 512 * 9
    per = 3 * f1024 + 6 * 2048 + 6 * 1024 + 2 * f512 + 8 * 257
    want = per * 1024 * 3 * 16
    assert bench.alg_flops_per_launch("tbc_B_fp32", w, 16) == pytest.approx(want, rel=1e-15)
    assert want == pytest.approx(10.82e9, rel=1e-3)
    # proportional to the directions, independent of the precision class
    assert bench.alg_flops_per_launch("tbc_B_pair32", w, 8) == pytest.approx(want / 2)
    assert bench.alg_flops_per_launch("field_y", w, 16) is None


def test_fp32_peak_is_units_times_clock():
    tf, src = bench.fp_peak_tflops("tbc_B_fp32", 2070.0)
    assert tf == pytest.approx(152 * 128 * 2 * 2.07e9 / 1e12) and "derived" in src
    tf64, src64 = bench.fp_peak_tflops("tbc_B_fp64", 2070.0)
    assert tf64 == bench.FP64_MEASURED_TFLOPS and "measured" in src64
    assert np.isclose(bench.fp_peak_tflops("tbc_B_fp32", None)[0], 80.54784)
