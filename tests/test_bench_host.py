"""Host-side logic of bench.py (no GPU): the clock-sample summary that decides
whether a run is rejected, the oracle CPU sample, and the byte counts behind
the roofline entry."""
import os
import sys

import numpy as np
import pytest

sys.path.insert(0, os.path.join(os.path.dirname(__file__), ".."))
import bench  # noqa: E402
import synth  # noqa: E402


def _line(sm, mx, hw="Not Active", therm="Not Active", swt="Not Active", cap="Not Active"):
    return ["0", str(sm), str(mx), "900.5", "0x0", hw, therm, swt, cap]


def test_clock_summary_reports_median_max_and_reasons():
    c = bench.ClockSampler()
    c.samples = [_line(1800, 2070), _line(1950, 2070, cap="Active"), _line(2000, 2070),
                 ["garbage"], _line(1900, 2070, hw="Active")]
    s = c.summary()
    assert s["sm_mhz"] == pytest.approx(np.median([1800, 1950, 2000, 1900]))
    assert s["sm_max_mhz"] == 2070
    assert s["reasons"] == ["hw_slowdown", "sw_power_cap"]
    assert s["samples"] == 5


def test_clock_summary_without_samples_says_unavailable():
    s = bench.ClockSampler().summary()
    assert s["sm_mhz"] is None and s["reasons"] == ["unavailable"]


def test_spmv_bytes_scale_with_the_matrix_and_vectors():
    base = {"nnzb": 1000, "n": 300}
    for prec, sm in (("fp64", 8), ("fp32", 4), ("bf16", 2)):
        b0 = bench.spmv_bytes(base, prec)
        # each extra block adds its 9 values and one 4-byte column index
        assert bench.spmv_bytes({"nnzb": 1001, "n": 300}, prec) - b0 == 9 * sm + 4
    # FP32 and BF16 share the vectors (float) and differ only in H's values
    assert bench.spmv_bytes(base, "fp32") - bench.spmv_bytes(base, "bf16") == 1000 * 9 * 2
    # FP64 doubles values and vectors against FP32; indices and row lengths stay
    idx = 1000 * 4 + 4 * 300
    assert bench.spmv_bytes(base, "fp64") - idx == 2 * (bench.spmv_bytes(base, "fp32") - idx)


def test_cpu_sample_on_a_small_scene():
    s = synth.tiny_scene(3, 2, 2, seed=2, contact=True, pinned=False)
    rate, desc, spent = bench.cpu_sample(s, newton_iters=3, pcg_iters_per_newton=40, cg_sample=10)
    assert rate > 0 and np.isfinite(rate) and spent > 0
    assert "3 Newton" in desc and "40 CG" in desc
    # more work per step: a lower rate
    rate2, _, _ = bench.cpu_sample(s, newton_iters=30, pcg_iters_per_newton=400, cg_sample=10)
    assert rate2 < rate
