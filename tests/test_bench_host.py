"""Host logic of bench.py (no GPU): the per-form summary of the JSON line."""
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
