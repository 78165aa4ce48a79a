"""Host logic of bench.py that needs no GPU: the clock record taken during the
timed region and the roofline denominator."""
import json
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _clocks(lines):
    c = bench.Clocks(0)
    c.out = "\n".join(lines)
    return c.summary()


def test_clock_summary_takes_the_median_and_the_active_reasons():
    s = _clocks([
        "0, 2070, 2070, 900.1, 0x0, Not Active, Not Active, Not Active, Not Active",
        "0, 1980, 2070, 1350.0, 0x4, Not Active, Not Active, Not Active, Active",
        "0, 2040, 2070, 1300.0, 0x0, Not Active, Not Active, Not Active, Not Active",
        "garbage line",
    ])
    assert s["samples"] == 3 and s["sm_mhz"] == 2040.0 and s["sm_max_mhz"] == 2070.0
    assert s["reasons"] == ["sw_power_cap"]


def test_clock_summary_reports_thermal_slowdown():
    s = _clocks(["0, 1500, 2070, 1400.0, 0x40, Not Active, Active, Not Active, Not Active"])
    assert s["reasons"] == ["hw_thermal_slowdown"]


def test_clock_summary_without_samples_says_so():
    s = _clocks([])
    assert s["samples"] == 0 and s["sm_mhz"] is None and s["reasons"] == ["nvidia-smi unavailable"]


def test_peak_comes_from_the_measured_file_else_the_fallback(tmp_path, monkeypatch):
    f = tmp_path / "peaks.json"
    f.write_text(json.dumps({"hbm_gbs": 6804.4, "bf16_tflops": 1864.0}))
    monkeypatch.setattr(bench, "PEAKS", str(f))
    assert bench.peaks() == (6804.4, "measured")
    monkeypatch.setattr(bench, "PEAKS", str(tmp_path / "absent.json"))
    assert bench.peaks() == (6800.0, "fallback")


def test_cores_used_is_cpu_time_over_wall_time():
    # unrounded: 4.8 s of CPU in 3.7 s of wall time is 1.3 cores, not 1
    assert bench.cores_used(4.8, 3.7) == 1.3
    assert bench.cores_used(31.0, 8.0) == 3.88
    assert bench.cores_used(0.1, 10.0) == 0.01
    assert bench.cores_used(1.0, 0.0) is None


def test_host_cpu_reports_count_and_model():
    n, model = bench.host_cpu()
    assert n == os.cpu_count() and n >= 1
    assert model is None or (isinstance(model, str) and model)


def test_effective_inner_tolerance_is_the_librarys_rule():
    # the library solves each float32 correction to sqrt(solve_tol), clamped to [1e-6, 1e-3]
    assert bench.effective_inner_tol(0.0, 1e-10) == pytest.approx(1e-5)
    assert bench.effective_inner_tol(0.0, 1e-14) == 1e-6
    assert bench.effective_inner_tol(0.0, 1e-4) == 1e-3
    assert bench.effective_inner_tol(3e-6, 1e-10) == 3e-6
