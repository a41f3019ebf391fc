#!/usr/bin/env python
"""Benchmark: grid-point RK-stage updates per second of the FP64 compressible-channel step.

Workload: the 256 x 192 x 128 plane channel (bulk Mach 1.5, bulk Re 7000, tanh-stretched walls,
6th-order central + WENO5 under the Ducros switch, power-law viscosity, CFL 0.8), seeded perturbed
laminar initial state. One benchmark step is one Wray RK3 step (three right-hand-side evaluations
and stage updates) over the whole grid; value = N * 3 * steps * ranks / time.

    python bench.py [--gpus N --steps K --warmup W] [--impl reference]

Prints one JSON line (rank 0). Multi-GPU runs are independent replicas (the method is not
decomposed across GPUs here): each rank advances its own copy, timing is the max over ranks.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

from paper_2004_02276_gb300 import inputs  # noqa: E402

METRIC = "grid-pt RK-stage updates/s, FP64 vs mixed, % HBM roofline at stated error"
UNIT = "grid-pt RK-stage updates/s"
CASE = inputs.C2

# Algorithmic FP64 flops per unit of work of each kernel (add/sub/mul = 1, FMA = 2, division and
# square root = 1), counted from the operations each kernel's formulation performs. Units: faces
# for the face kernels, interior nodes otherwise.
FLOPS_PER_UNIT = {
    "weno_x": 900, "weno_y": 900, "weno_z": 900,
    "faces_x": 151, "faces_y": 151, "faces_z": 151,
    "assemble": 430, "sensor": 105, "prims": 28,
}
# Mixed precision: FP64 flops of the projection into characteristic variables per WENO face
# (Roe state and eigen-scalars 30, acoustic-row scalars 25 per stencil node); the FP32 flux
# arithmetic (~700 flops per face) runs on the FP32 pipes at 62x the FP64 rate.
FLOPS_PER_UNIT_MIXED = {"weno_x": 180, "weno_y": 180, "weno_z": 180}
# DRAM bytes (read + write) per WENO face from one ncu capture of the current kernels on the
# 192x144x96 channel (dram__bytes_read.sum + dram__bytes_write.sum of the launch over its WENO
# faces), scaled to a launch by the faces it processes.
DRAM_BYTES_PER_UNIT = {"weno_x": 131.9, "weno_y": 190.8, "weno_z": 423.6}
DRAM_BYTES_PER_UNIT_MIXED = {"weno_x": 120.5, "weno_y": 160.6, "weno_z": 242.9}
# FP64 peak: 1.25 TFLOP/s nominal for GB300 (the profiling recipe's unit table); a probe of
# dependent-chain-free DFMA on a GB300 measured 1.20 TFLOP/s at ~1.97 GHz.
FP64_PEAK_TFLOPS = 1.25


# Algorithmic HBM bytes of one grid-point RK stage: read w and the residual register, write w
# and the new residual (5 FP64 each), the minimum of a fused stage.
STAGE_BYTES_PER_POINT = 160


def hbm_step(value):
    """The whole step against the HBM roofline: algorithmic bytes per grid-point stage times the
    measured rate, over the measured copy bandwidth. The FP64 path is bound by the FP64 pipe,
    so this fraction is small; it is reported for the metric's HBM roofline."""
    pk = peaks().get("hbm_gbs")
    gbs = STAGE_BYTES_PER_POINT * value / 1e9
    return {"bytes_per_point_stage": STAGE_BYTES_PER_POINT, "achieved_gbs": round(gbs, 1),
            "peak_gbs": pk, "frac": round(gbs / pk, 4) if pk else None,
            "peak_source": "MEASURED_PEAKS.json hbm_gbs (copy, measured)"}


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except OSError:
        return {}


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.t.join(timeout=5)

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx),
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist

        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        dist.init_process_group("gloo", rank=rank, world_size=world)
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist

        dist.barrier()


def max_over_ranks(world, v):
    if world == 1:
        return v
    import torch
    import torch.distributed as dist

    t = torch.tensor([v], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(points, steps, world, ms_max):
    """Whole-job grid-point RK-stage updates/s: every rank advances its own replica of
    `points` points by `steps` RK3 steps; the job time is the slowest rank's."""
    return points * 3 * steps * world / (ms_max / 1e3)


def cpu_sample(case):
    """The oracle on one full RK3 step of the workload (host cores): (rate, seconds, state)."""
    from oracle import oracle as O

    cfg = O.make_cfg(case)
    w0 = inputs.channel_state(case, seed=0)
    t0 = time.perf_counter()
    w1, dt = O.rk_step(cfg, w0, cfl=case.cfl)
    sec = time.perf_counter() - t0
    return case.npts * 3 / sec, sec, w1, O.threads()


def bench_case(args):
    """The benchmark workload, or (for profiling captures only) the same channel on another grid."""
    if not args.grid:
        return CASE
    nx, ny, nz = (int(v) for v in args.grid.lower().split("x"))
    return CASE.replace(name=f"channel-{nx}x{ny}x{nz}", nx=nx, ny=ny, nz=nz)


def measure(case, args, world, local, flops_per_unit, traffic_per_unit):
    """Warm-up, the timed region (K graph-replayed steps) and the per-kernel event timing of K
    eager steps, for one precision. Returns the figures, the solver and the state."""
    import torch

    from paper_2004_02276_gb300 import binding

    solver = binding.Solver(case, device=f"cuda:{local}")
    w0 = inputs.channel_state(case, seed=0)
    w = torch.from_numpy(w0).cuda()
    r_old = torch.zeros_like(w)
    stream = solver.stream
    solver.advance_n(w, r_old, args.warmup)  # also captures the step graph
    torch.cuda.synchronize()
    start, stop = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    n0 = solver.launch_count()
    with ClockSampler(local) as clk:
        barrier(world)
        torch.cuda.synchronize()
        start.record(stream)
        solver.advance_n(w, r_old, args.steps)
        stop.record(stream)
        torch.cuda.synchronize()
        barrier(world)
    launches = solver.launch_count() - n0
    ms_max = max_over_ranks(world, start.elapsed_time(stop))
    value = job_rate(case.npts, args.steps, world, ms_max)

    solver.timing(True)
    solver.advance_n(w, r_old, args.steps)
    ktimes, weno_faces = solver.timing_read()
    solver.timing(False)
    busy = {k: v for k, v in ktimes.items() if v[1] > 0}
    dom = max(busy, key=lambda k: busy[k][0])
    dom_ms, dom_n = busy[dom]
    avg_s = dom_ms / dom_n / 1e3
    if dom.startswith("weno"):
        units = weno_faces["xyz".index(dom[-1])] / dom_n
    elif dom.startswith("faces"):
        d = "xyz".index(dom[-1])
        units = (case.nx + (d == 0)) * (case.ny + (d == 1)) * (case.nz + (d == 2))
    else:
        units = case.npts
    achieved = flops_per_unit.get(dom, 0) * units / avg_s / 1e12
    total_ms = sum(v[0] for v in busy.values())
    roofline = {
        "bound": "alu", "kernel": dom, "achieved": round(achieved, 4),
        "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s", "frac": round(achieved / FP64_PEAK_TFLOPS, 4),
        "traffic": (traffic_per_unit[dom] * units if dom in traffic_per_unit else None),
        "traffic_source": "ncu dram__bytes_read+write per unit on the 192x144x96 channel, x units",
        "peak_source": "FP64 nominal 1.25 TFLOP/s (recipe); probe measured 1.20",
        "units_per_launch": units, "flops_per_unit": flops_per_unit.get(dom),
        "avg_launch_ms": round(dom_ms / dom_n, 4),
        "kernel_share": {k: round(v[0] / total_ms, 4) for k, v in sorted(busy.items())},
        "weno_face_fraction": round(sum(weno_faces) / (3 * args.steps * 3 * case.npts), 4),
    }
    return {"value": value, "ms": ms_max, "launches": launches, "clocks": clk.summary(),
            "roofline": roofline}, solver, w, w0


def run_ours(args, world, rank, local):
    import torch

    torch.cuda.set_device(local)
    case = bench_case(args)
    m64, solver, w, w0 = measure(case, args, world, local, FLOPS_PER_UNIT, DRAM_BYTES_PER_UNIT)

    # end to end through the C ABI with host buffers: per step H2D of the state, one RK3 step,
    # D2H of the new state
    w_host = torch.from_numpy(inputs.channel_state(case, seed=0)).pin_memory()
    wd = torch.empty_like(w)
    rd = torch.zeros_like(w)
    solver.advance_n_host(w_host, wd, rd, 1)  # warm (graph for these buffers)
    barrier(world)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        solver.advance_n_host(w_host, wd, rd, 1)
    e2e_s = max_over_ranks(world, time.perf_counter() - t0)
    nbytes = 5 * case.npts * 8
    e2e = {"value": case.npts * 3 * args.steps * world / e2e_s, "unit": UNIT,
           "h2d_bytes_per_step": nbytes, "d2h_bytes_per_step": nbytes}
    w64 = w.cpu().numpy()

    out = {
        "metric": METRIC, "value": m64["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": m64["ms"] / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": case.name, "grid": [case.nx, case.ny, case.nz],
                   "mach_b": case.mach, "re_b": case.reynolds, "scheme": "central6+WENO5 (Ducros 0.05)",
                   "cfl": case.cfl, "precision": "fp64", "parallelism": f"replicas x{world}",
                   "l2": "inputs larger than L2 (state %d MB + workspace %.1f GB vs 129 MB L2)"
                         % (5 * case.npts * 8 // 2**20, solver.workspace.numel() / 1e9)},
        "roofline": m64["roofline"], "e2e": e2e, "gpu_launches": m64["launches"],
        "clocks": m64["clocks"],
        "hbm_step": hbm_step(m64["value"]),
    }
    if rank == 0 and world == 1 and not args.no_cpu:  # the oracle baseline: N = 1 only
        rate, sec, w_ref, cores = cpu_sample(case)
        # the same first step on the GPU, for the error at which the figure holds
        wg = torch.from_numpy(w0).cuda()
        rg = torch.zeros_like(wg)
        solver.rk_step(wg, rg)
        wg = wg.cpu().numpy()
        err = [float(np.linalg.norm(wg[m] - w_ref[m]) / np.linalg.norm(w_ref[m])) for m in range(5)]
        out["cpu_baseline"] = {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle",
                               "sample": f"one RK3 step of the full {case.name} workload "
                                         f"({sec:.1f} s on the host)"}
        out["error"] = {"rel_l2_vs_oracle_first_step": err, "max": max(err)}
    solver.close()
    del solver, w, wd, rd

    if not args.no_mixed:
        # mixed precision: FP32 flux/sensor/WENO/viscous arithmetic, FP64 state and projection
        mcase = case.replace(precision="mixed")
        mm, msolver, wm, _ = measure(mcase, args, world, local, FLOPS_PER_UNIT_MIXED, DRAM_BYTES_PER_UNIT_MIXED)
        wmix = wm.cpu().numpy()
        msolver.close()
        steps_done = args.warmup + 2 * args.steps
        err = [float(np.linalg.norm(wmix[m] - w64[m]) / np.linalg.norm(w64[m])) for m in range(5)]
        out["variants"] = {"mixed": {
            "value": mm["value"], "ms_per_step": mm["ms"] / args.steps,
            "speedup_vs_fp64": mm["value"] / m64["value"], "dtype": "f32 flux / f64 state",
            "roofline": mm["roofline"], "gpu_launches": mm["launches"], "clocks": mm["clocks"],
            "error": {"rel_l2_vs_fp64_after_steps": err, "max": max(err), "steps": steps_done,
                      "note": "sensor-switched flux: the error is set by central/WENO choices that "
                              "flip at faces sitting at the threshold; with a continuous flux "
                              "the 100-step error is <= 1e-5 (tests/test_gpu_mixed.py)"},
        }}
    if not args.no_batched:
        out.setdefault("variants", {})["batched"] = run_batched(args, world, local, m64["value"])
        if not args.no_mixed:
            out["variants"]["batched_mixed"] = run_batched(args, world, local, mm["value"], "mixed")
    if rank == 0:
        print(json.dumps(out), flush=True)


def run_batched(args, world, local, large_grid_value, precision="fp64"):
    """The batched workload: 64 independent channels of uneven size, Mach and Reynolds number
    (44.7 M points in all), advanced by the ensemble kernels, one graph replay per step, launch
    shapes from the autotuner (run before the warm-up, outside the timed region). The per-point
    rate is compared with the large grid's rate in the same precision."""
    import torch

    from paper_2004_02276_gb300 import binding

    cases = inputs.ensemble_cases(seed=0, precision=precision)
    npts = sum(c.npts for c in cases)
    E = binding.Ensemble(cases, device=f"cuda:{local}")
    ws = [torch.from_numpy(inputs.channel_state(c)).cuda() for c in cases]
    rs = [torch.zeros_like(w) for w in ws]
    choice = E.tune(ws, rs)
    E.advance(ws, rs, args.warmup, cfl=0.8)
    torch.cuda.synchronize()
    start, stop = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        barrier(world)
        torch.cuda.synchronize()
        start.record(E.stream)
        E.advance(ws, rs, args.steps, cfl=0.8)
        stop.record(E.stream)
        torch.cuda.synchronize()
        barrier(world)
    ms = max_over_ranks(world, start.elapsed_time(stop))
    value = npts * 3 * args.steps * world / (ms / 1e3)
    tot = E.totals(ws)
    E.close()
    return {"value": value, "ms_per_step": ms / args.steps, "instances": len(cases),
            "points": npts, "dtype": "f64" if precision == "fp64" else "f32 flux / f64 state",
            "per_point_vs_large_grid": value / large_grid_value,
            "tuned": {"weno_block": choice[0], "weno_blocks_per_sm": choice[1],
                      "central_blocks_per_sm": choice[2]},
            "finite": bool(np.isfinite(np.array(tot)).all()), "clocks": clk.summary(),
            "workload": "64 channels, dims U{32..192}xU{32..128}xU{32..128}, M_b U[0.3,3], "
                        "Re_b U[2000,8000], seed 0"}


def run_reference(args, world, rank):
    """The FP64 C oracle timed on the host cores, each step a bounded sample of the workload:
    one RK3 step on a 256 x 192 x 16 slab of the channel (same x/y grid and scheme)."""
    if rank != 0:
        return
    from oracle import oracle as O

    case = CASE.replace(nz=16)
    cfg = O.make_cfg(case)
    w = inputs.channel_state(case, seed=0)
    for _ in range(args.warmup):
        w, _ = O.rk_step(cfg, w, cfl=case.cfl)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        w, _ = O.rk_step(cfg, w, cfl=case.cfl)
    sec = time.perf_counter() - t0
    value = case.npts * 3 * args.steps / sec
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": sec * 1e3 / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "impl": "reference",
        "config": {"workload": CASE.name, "grid": [CASE.nx, CASE.ny, CASE.nz], "precision": "fp64",
                   "sample": "each step: one RK3 step on a 256x192x16 slab of the workload"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": O.threads(), "kind": "oracle",
                         "sample": "one RK3 step on a 256x192x16 slab per benchmark step"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(out), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu", action="store_true", help="skip the oracle CPU baseline leg")
    ap.add_argument("--grid", default="", help="NXxNYxNZ override, for profiling captures only")
    ap.add_argument("--no-mixed", action="store_true", help="skip the mixed-precision variant")
    ap.add_argument("--no-batched", action="store_true", help="skip the batched-ensemble variant")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    world, rank, local = dist_setup()
    if args.impl == "reference":
        run_reference(args, world, rank)
    else:
        run_ours(args, world, rank, local)
    if world > 1:
        import torch.distributed as dist

        dist.destroy_process_group()


if __name__ == "__main__":
    main()
