"""Host-side helpers of bench.py (no GPU): the strict-JSON sanitiser, the
clock-sample summary read from nvidia-smi lines, and the peak lookup with
its fallback."""
import json
import math
import os

import pytest

import bench


def test_nonfinite_values_become_null():
    line = {"a": 1.5, "b": float("nan"), "c": [1.0, float("inf"), {"d": -float("inf")}],
            "e": "x", "f": 3}
    out = bench._finite(line)
    assert out == {"a": 1.5, "b": None, "c": [1.0, None, {"d": None}], "e": "x", "f": 3}
    json.dumps(out, allow_nan=False)  # strict JSON


def test_clock_summary_parses_nvidia_smi_lines():
    c = bench.ClockSampler(0)
    c.lines = ["2070, 2070, 900.5, Not Active, Not Active, Not Active, Active",
               "2055, 2070, 950.0, Not Active, Not Active, Not Active, Not Active",
               "[N/A], 2070, 10, Not Active, Not Active, Not Active, Not Active",
               "garbage",
               "1980, 2070, 990.1, Active, Not Active, Not Active, Not Active"]
    s = c.summary()
    assert s["samples"] == 3 and s["sm_mhz"] == 2055.0 and s["sm_max_mhz"] == 2070.0
    assert s["reasons"] == ["hw_slowdown", "sw_power_cap"]
    assert bench.ClockSampler(0).summary() == {"sm_mhz": None, "sm_max_mhz": None,
                                               "reasons": [], "samples": 0}


def test_peaks_measured_or_fallback(tmp_path, monkeypatch):
    path = os.path.join(bench.ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as fh:
            want = float(json.load(fh)["hbm_gbs"])
        assert bench._peaks() == (want, "measured")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench._peaks() == (6800.0, "fallback")
    (tmp_path / "MEASURED_PEAKS.json").write_text(json.dumps({"hbm_gbs": 7000.5}))
    assert bench._peaks() == (7000.5, "measured")
    (tmp_path / "MEASURED_PEAKS.json").write_text("{not json")
    assert bench._peaks() == (6800.0, "fallback")


def test_reynolds_number_of_the_tau_sweep():
    # Re = u0 N / nu with nu = (tau - 1/2) / 3 (lattice units)
    assert bench._re(0.8) == pytest.approx(0.05 * 4096 / (0.3 / 3.0))
    assert math.isclose(bench._re(0.5005), 0.05 * 4096 / (0.0005 / 3.0), rel_tol=1e-9)
