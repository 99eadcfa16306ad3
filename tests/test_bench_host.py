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
    """The oracle sample: one full Newton iteration from the given state
    (threaded element loops, PCG to 1e-13, line search), scaled by the
    Newton count; a capped solve scales to a known iteration count."""
    s = synth.tiny_scene(3, 2, 2, seed=2, contact=True, pinned=False)
    res = bench.cpu_sample(s, s.x0, s.v0, newton_iters=3, threads=2)
    assert res["value"] > 0 and np.isfinite(res["value"]) and res["spent_s"] > 0
    assert res["cores"] == 2 and res["pcg_iters"] > 0
    assert "3 such iterations" in res["sample"] and "2 threads" in res["sample"]
    assert res["value"] == pytest.approx(1.0 / (3 * res["newton_iteration_s"]))
    # more Newton iterations per step: a lower rate
    res2 = bench.cpu_sample(s, s.x0, s.v0, newton_iters=30, threads=1)
    assert res2["value"] < res["value"]
    # a capped solve is scaled to the known count
    res3 = bench.cpu_sample(s, s.x0, s.v0, newton_iters=3, threads=1, pcg_iters_known=res["pcg_iters"], pcg_cap=2)
    assert res3["pcg_iters"] == res["pcg_iters"]


def test_threaded_oracle_evaluation_is_bitwise_serial():
    """The oracle's element loops on several threads (contiguous tet chunks,
    concatenated in order) give the serial results bit for bit."""
    from oracle import ip
    s = synth.tiny_scene(6, 4, 3, seed=5, contact=True, pinned=False)
    x = ip.Problem(s).x_tilde + 1e-3 * np.random.default_rng(1).normal(size=s.X.shape)
    x[:, 2] = np.maximum(x[:, 2], 2e-4)
    p1, p4 = ip.Problem(s), ip.Problem(s, threads=4)
    assert p1.energy(x) == p4.energy(x)
    assert np.array_equal(p1.gradient(x), p4.gradient(x))
    assert (p1.hessian(x) != p4.hessian(x)).nnz == 0


def test_oracle_error_estimate_is_zero_at_the_minimiser_and_scales():
    """The Newton-correction estimate of a step's error: ~0 at the oracle's
    minimiser, and for x* + e it recovers |e| / |x* + e - x^t| to the
    linearisation."""
    from oracle import ip, newton
    s = synth.tiny_scene(3, 2, 2, seed=4, pinned=True)
    p = ip.Problem(s)
    xs, _ = newton.timestep(p)
    assert bench.oracle_error_estimate(s, s.x0, s.v0, xs, threads=1) < 1e-9
    e = np.zeros_like(xs)
    e[~p.pinned] = 1e-6 * np.random.default_rng(0).normal(size=(int((~p.pinned).sum()), 3))
    est = bench.oracle_error_estimate(s, s.x0, s.v0, xs + e, threads=1)
    ref = np.linalg.norm(e) / np.linalg.norm(xs + e - s.x0)
    assert est == pytest.approx(ref, rel=2e-2)
