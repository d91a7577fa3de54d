"""Host logic of the measurement (no GPU): the clock record taken during the
timed region, the roofline denominator, and the workload's config object."""
import argparse
import json
import os

import pytest

import bench


def _sampler_with(tmp_path, lines):
    s = bench.ClockSampler(0)
    path = tmp_path / "clocks.csv"
    path.write_text("\n".join(lines) + "\n")
    s.path = str(path)
    return s


def test_clock_summary_median_max_and_reasons(tmp_path):
    rows = [
        "0, 2070, 2070, 900.1, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "0, 2055, 2070, 1300.4, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
        "0, 2070, 2070, 1000.0, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "garbage line",
        "0, [N/A], 2070, 1000.0, 0x0, Not Active, Not Active, Not Active, Not Active",
    ]
    s = _sampler_with(tmp_path, rows)
    out = s.summary()
    assert out == {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"], "samples": 3}
    assert not os.path.exists(s.path)  # the record is removed once read


def test_clock_summary_reports_thermal_slowdown(tmp_path):
    rows = ["0, 1500, 2070, 1390.0, 0x0000000000000040, Not Active, Active, Not Active, Not Active"] * 4
    out = _sampler_with(tmp_path, rows).summary()
    assert out["reasons"] == ["hw_thermal_slowdown"] and out["sm_mhz"] == 1500.0


def test_clock_summary_without_samples(tmp_path):
    assert _sampler_with(tmp_path, ["not, a, sample"]).summary() is None
    assert bench.ClockSampler(0).summary() is None


def test_peak_is_the_measured_copy_bandwidth():
    with open(os.path.join(bench.ROOT, "MEASURED_PEAKS.json")) as f:
        measured = float(json.load(f)["hbm_gbs"])
    assert bench._peaks() == (measured, "measured")


def test_workload_config_of_the_benchmark():
    cfg = {"n": 16, "n_omega": 256, "T": 64.0, "eta": 5.0 / 64.0, "aca_tol": 1e-5, "leaf": 64, "tol": 1e-5}
    args = argparse.Namespace(workload="cavity5120", guess="sem", precond="block3")
    out = bench.workload_config(args, cfg)
    assert out["triangles"] == 5120 and out["unknowns"] == 15360
    assert out["solves_per_step"] == 129
    assert out["workload"] == "cavity5120" and "flushed" in out["l2"]
    assert "model" not in out  # the config names a workload, not a model


@pytest.mark.parametrize("units,world,t_ms,rate", [(129, 1, 1000.0, 129.0), (129, 4, 500.0, 1032.0)])
def test_replica_rate_is_whole_job(units, world, t_ms, rate):
    assert bench.replica_throughput(units, world, t_ms) == pytest.approx(rate)
