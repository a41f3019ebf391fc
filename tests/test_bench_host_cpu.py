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
    assert bench.CASE.name == "sbli-2048x384x256" and bench.CASE.shock
    A.grid = "512x192x64"
    c = bench.bench_case(A())
    assert (c.nx, c.ny, c.nz) == (512, 192, 64) and c.name == "sbli-512x192x64"
    # same spacing, gas, scheme and boundary kinds as the workload
    for a, b in ((c.lx / c.nx, bench.CASE.lx / bench.CASE.nx), (c.ly / c.ny, bench.CASE.ly / bench.CASE.ny),
                 (c.lz / c.nz, bench.CASE.lz / bench.CASE.nz)):
        assert abs(a - b) <= 1e-12 * b
    for k in ("mach", "reynolds", "t_wall", "shock", "shock_theta", "bc_xmin", "bc_xmax", "bc_ymin",
              "bc_ymax", "noise", "L", "weno_mode", "y_map", "beta"):
        assert getattr(c, k) == getattr(bench.CASE, k), k


def test_kernel_units_and_step_flops():
    """Units per kernel class from the timing record: WENO faces as counted, central faces as the
    direction's faces minus its WENO faces, nodes per launch otherwise; the step's flops are the
    sum over classes of flops per unit x units."""
    c = bench.inputs.Case(nx=4, ny=3, nz=2)
    kt = {"prims": (1.0, 3), "sensor": (1.0, 3), "faces_x": (1.0, 3), "faces_y": (1.0, 3),
          "faces_z": (1.0, 3), "weno_x": (1.0, 3), "weno_y": (1.0, 3), "weno_z": (2.0, 3),
          "assemble": (1.0, 3), "dt_finalize": (0.1, 1), "force_finalize": (0.0, 0)}
    wf = [10, 11, 12]
    u = bench.kernel_units(c, kt, wf)
    assert u["weno_z"] == 12 and u["faces_x"] == 5 * 3 * 2 * 3 - 10 and u["faces_z"] == 4 * 3 * 3 * 3 - 12
    assert u["assemble"] == 24 * 3 and u["rk_update"] == 24 * 3 and "force_finalize" not in u
    r = bench.roofline(c, kt, wf, 1.0, 1, 1.0, bench.FLOPS_PER_UNIT, {}, "fp64")
    assert r["kernel"] == "weno_z" and r["flops_per_unit"] == 900
    want = sum(bench.FLOPS_PER_UNIT.get(k, 0) * v for k, v in u.items())
    assert abs(r["step_flops"] - want) <= 1e-9 * want
    assert abs(r["weno_face_fraction"] - 33 / (3 * 3 * 24)) < 1e-4


def test_job_rate_counts_all_ranks():
    assert bench.job_rate(1000, 5, 2, 20.0) == 1000 * 3 * 5 * 2 / 0.02


def test_channel_workload_for_captures():
    class A:
        grid = ""
        workload = "channel"

    assert bench.bench_case(A()) is bench.CHANNEL
    A.grid = "192x144x96"
    c = bench.bench_case(A())
    assert (c.nx, c.ny, c.nz, c.kind) == (192, 144, 96, "channel") and c.name == "channel-192x144x96"
    assert (c.lx, c.ly, c.lz, c.reynolds) == (bench.CHANNEL.lx, bench.CHANNEL.ly, bench.CHANNEL.lz,
                                               bench.CHANNEL.reynolds)
