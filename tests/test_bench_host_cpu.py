"""Host-side pieces of bench.py that shape its JSON line (no GPU): the clock-record summary and
its throttle reasons, the whole-step HBM fraction, and the benchmark case override used only for
profiling captures."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def sampler_with(lines):
    s = bench.ClockSampler(0)
    s.lines = list(lines)
    return s


def test_clock_summary_median_and_reasons():
    ok = "0, 2070, 2070, 900.5, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active"
    cap = "0, 1980, 2070, 1400.0, 0x0000000000000004, Not Active, Not Active, Not Active, Active"
    hot = "0, 1500, 2070, 1300.0, 0x0000000000000040, Not Active, Active, Not Active, Not Active"
    s = sampler_with([ok, ok, cap])
    out = s.summary()
    assert out["sm_mhz"] == 2070.0 and out["sm_max_mhz"] == 2070.0 and out["samples"] == 3
    assert out["reasons"] == ["sw_power_cap"]
    out = sampler_with([ok, hot, "garbage", ""]).summary()
    assert out["reasons"] == ["hw_thermal_slowdown"] and out["samples"] == 2
    assert sampler_with([]).summary() == {"sm_mhz": None, "sm_max_mhz": None, "reasons": [],
                                          "samples": 0}


def test_hbm_step_fraction():
    out = bench.hbm_step(272e6)
    assert out["bytes_per_point_stage"] == 160
    assert abs(out["achieved_gbs"] - 160 * 272e6 / 1e9) < 0.05
    if out["peak_gbs"]:
        assert abs(out["frac"] - out["achieved_gbs"] / out["peak_gbs"]) < 1e-3


def test_case_override_only_changes_the_grid():
    class A:
        grid = ""

    assert bench.bench_case(A()) is bench.CASE
    A.grid = "192x144x96"
    c = bench.bench_case(A())
    assert (c.nx, c.ny, c.nz) == (192, 144, 96) and c.name == "channel-192x144x96"
    assert (c.mach, c.reynolds, c.lx, c.ly, c.lz) == (bench.CASE.mach, bench.CASE.reynolds,
                                                      bench.CASE.lx, bench.CASE.ly, bench.CASE.lz)


def test_job_rate_counts_all_ranks():
    assert bench.job_rate(1000, 5, 2, 20.0) == 1000 * 3 * 5 * 2 / 0.02
