"""Host logic of bench.py (no GPU): the per-form summary of the JSON line, the roofline
entries and the profiled-traffic bookkeeping."""
import numpy as np
import pytest

import bench


def _res(ms, hist, charges, trace, herm=0.0):
    return {"ms": ms, "hist": np.asarray(hist), "obs": {"charges": np.asarray(charges),
                                                        "trace_re": trace, "herm_err": herm}}


def test_form_summary_against_the_fp64_form():
    res = {"fp64": _res([2.0, 2.0], [[0, 0, 0], [1, 0, 0]], [4.0, 4.0], 8.0),
           "fp16x6": _res([0.1, 0.1], [[0, 0, 0], [1, 2e-7, 0]], [4.0, 4.0 + 3e-8], 8.0 + 8e-9)}
    s = bench.form_summary(res, ["fp64", "fp16x6"], 8.0)
    assert s["fp64"]["steps_per_s"] == pytest.approx(500.0)
    assert s["fp64"]["max_dipole_err_vs_fp64_au"] == 0.0
    assert s["fp16x6"]["steps_per_s"] == pytest.approx(10000.0)
    assert s["fp16x6"]["max_dipole_err_vs_fp64_au"] == pytest.approx(2e-7)
    assert s["fp16x6"]["final_charge_err_vs_fp64"] == pytest.approx(3e-8)
    assert s["fp16x6"]["trace_rel_drift"] == pytest.approx(1e-9)
    assert s["fp16x6"]["herm_err"] == 0.0


def test_form_summary_without_the_fp64_form():
    s = bench.form_summary({"fp32": _res([1.0], [[0, 0, 0]], [1.0], 2.0)}, ["fp32"], 2.0)
    assert s["fp32"]["max_dipole_err_vs_fp64_au"] is None
    assert s["fp32"]["final_charge_err_vs_fp64"] is None
    assert s["fp32"]["trace_rel_drift"] == 0.0


def test_roofline_entries_follow_the_per_launch_counts():
    # X counts the method's 4N^3, delta M 2N^3, the update 64 B per element; the step is
    # judged against max(6N^3 / tensor peak, algorithmic bytes / HBM peak)
    N = 1024
    peaks = {"hbm_gbs": 6000.0, "bf16_tflops": 2000.0, "sm_max_mhz": 2070.0}
    x = bench.kernel_roofline("tc_gemm_X", 0.0343597383, "fp16x6", N, peaks, "measured")
    assert x["bound"] == "tensor" and x["achieved"] == pytest.approx(125.0, rel=1e-6)
    assert x["frac"] == pytest.approx(125.0 / 2000.0, rel=1e-6)
    assert x["executed_tflops"] == pytest.approx(6 * 6 * N ** 3 / 0.0343597383e-3 / 1e12)
    dm = bench.kernel_roofline("tc_gemm_dM", 0.02, "fp16x6", N, peaks, "measured")
    assert dm["achieved"] == pytest.approx(2 * N ** 3 / 0.02e-3 / 1e12)
    up = bench.kernel_roofline("update", 0.01, "fp16x6", N, peaks, "measured")
    assert up["bound"] == "hbm" and up["unit"] == "GB/s"
    assert up["achieved"] == pytest.approx(N * N * 60 / 0.01e-3 / 1e9)
    lv = bench.kernel_roofline("level", 0.005, "fp16x6", N, peaks, "measured")
    assert lv["bound"] == "latency" and lv["time_us"] == pytest.approx(5.0)
    r = bench.roofline({"tc_gemm_X": 0.03, "update": 0.02}, "fp16x6", N, peaks, "measured", 0.08)
    assert r["kernel"] == "tc_gemm_X" and set(r["kernels"]) == {"tc_gemm_X", "update"}
    floor = max(6 * N ** 3 / 2000e12, bench.step_bytes("fp16x6", N) / 6000e9)
    assert r["step"]["frac"] == pytest.approx(floor / 0.08e-3)


def test_profiled_traffic_is_dropped_when_a_source_changes(tmp_path, monkeypatch):
    src = tmp_path / "k.cu"
    src.write_text("kernel v1")
    import hashlib
    sha = hashlib.sha256(b"kernel v1").hexdigest()
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "PROFILED_TRAFFIC", {("tc_gemm_X", "fp16x6"): {"bytes": 123,
                                                    "sources": [("k.cu", sha)]}})
    assert bench._traffic("tc_gemm_X", "fp16x6") == 123
    assert bench._traffic("update", "fp16x6") is None
    src.write_text("kernel v2")
    assert bench._traffic("tc_gemm_X", "fp16x6") is None
