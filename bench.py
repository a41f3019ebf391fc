#!/usr/bin/env python
"""Benchmark: grid-point RK-stage updates per second of the compressible Navier-Stokes step.

Headline workload: the oblique shock / boundary layer interaction of Section 3.3 on the
2048 x 384 x 256 grid (201 M points; Mach 2, Re_delta_in 10^4, 8-degree shock imposed at the
top, recycling inflow, characteristic outflow and top, isothermal wall at T_w/T_inf = 1.7,
6th-order central + WENO5 under the Ducros switch, power-law viscosity, CFL 0.8), FP64, from the
seeded synthetic initial state. One benchmark step is one Wray RK3 step (three right-hand sides
and stage updates) over the whole grid; value = N * 3 * steps * ranks / time.

Variants on the same line: the mixed-precision path on the same workload (with its error
against the FP64 path after 100 steps), the 256 x 192 x 128 channel in both precisions, and the
batched ensemble of 64 channels.

    python bench.py [--gpus N --steps K --warmup W] [--impl reference]

Prints one JSON line (rank 0). Multi-GPU runs are independent replicas (the method is not
decomposed across GPUs here): each rank advances its own copy, timing is the max over ranks.
"""
import argparse
import json
import math
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
CASE = inputs.C4          # the largest single-GPU workload: headline
CHANNEL = inputs.C2       # the 256 x 192 x 128 channel: variant
SMALL = inputs.C1         # the 64 x 48 x 32 channel: error against the oracle over 100 steps

# Algorithmic FP64 flops per unit of work of each kernel class (add/sub/mul = 1, FMA = 2,
# division and square root = 1), counted from each kernel's formulation. Units: WENO faces for
# weno_*, central faces for faces_*, interior nodes otherwise. rk_update also stands for the
# stage update fused into the assembly when there is no forcing.
FLOPS_PER_UNIT = {
    "weno_x": 900, "weno_y": 900, "weno_z": 900,
    "faces_x": 151, "faces_y": 151, "faces_z": 151,
    "assemble": 430, "sensor": 105, "prims": 28, "rk_update": 20,
}
# Mixed precision: FP64 flops per unit (the projection into characteristic variables of a WENO
# face: Roe state and eigen-scalars 30, acoustic-row scalars 25 per stencil node; the FP64
# primitives; the mass-flux difference of the assembly; the stage update) and FP32 flops per
# unit (the flux, WENO5, sensor and viscous arithmetic; the FP32 assembly derives the velocity
# gradients itself), each against its own pipe's measured rate.
FLOPS64_PER_UNIT_MIXED = {"weno_x": 180, "weno_y": 180, "weno_z": 180, "prims": 29, "assemble": 14,
                          "rk_update": 20}
FLOPS32_PER_UNIT_MIXED = {
    "weno_x": 700, "weno_y": 700, "weno_z": 700,
    "faces_x": 151, "faces_y": 151, "faces_z": 151,
    "assemble": 520, "sensor": 105,
}
# DRAM bytes (read + write) per node of the assembly, averaged over the three stages of its
# launches, from one ncu capture of dram__bytes_read.sum + dram__bytes_write.sum on a
# 1024 x 384 x 16 slice of the workload (profiles/dram-per-step_sbli-1024x384x16_fp64_mixed.md),
# scaled to a launch by its nodes; traffic per unit grows in proportion with the nodes.
DRAM_BYTES_PER_UNIT = {"assemble": 415.3}
DRAM_BYTES_PER_UNIT_MIXED = {"assemble": 238.1}
# Algorithmic HBM bytes per node of the mixed-precision assembly (stage update fused): FP64 w and
# the register in and out (160), the FP32 face fluxes of three directions (60), the FP32 node
# fields of the viscous stencils u, v, w, T, mu and the divergence (24).
ALG_BYTES_PER_UNIT_MIXED = {"assemble": 244}
# FP64 rate from the SM count and clock: 152 SMs x 2 DFMA per clock x 2 flops x 2.07 GHz.
FP64_UNITS_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12
FP32_UNITS_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12
PEAK_PROFILE = "profiles/fp64_fp32_fma_peak.md"

# Algorithmic HBM bytes of one grid-point RK stage: read w and the residual register, write w
# and the new residual (5 FP64 each), the minimum of a fused stage.
STAGE_BYTES_PER_POINT = 160
# DRAM bytes of all kernels per grid-point stage measured by ncu on a 1024 x 384 x 16 slice of
# the workload (its 16 planes make the ghost fill weigh more than on the full grid)
MEASURED_STEP_BYTES = 1622.3
MEASURED_STEP_BYTES_MIXED = 938.5


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except OSError:
        return {}


def hbm_step(value, copy_gbs=None, measured_bytes=MEASURED_STEP_BYTES):
    """The whole step against the HBM roofline: algorithmic bytes per grid-point stage times the
    measured rate, over the measured copy bandwidth (MEASURED_PEAKS.json when present, else the
    copy rate measured in this run). The FP64 path is bound by the FP64 pipe, so this fraction
    is small; it is reported for the metric's HBM roofline."""
    pk = peaks().get("hbm_gbs")
    src = "MEASURED_PEAKS.json hbm_gbs (copy, measured)"
    if not pk and copy_gbs:
        pk, src = copy_gbs, "device-to-device copy of 2 GiB measured in this run (peaks.copy_gbs)"
    gbs = STAGE_BYTES_PER_POINT * value / 1e9
    return {"bytes_per_point_stage": STAGE_BYTES_PER_POINT, "achieved_gbs": round(gbs, 1),
            "peak_gbs": pk, "frac": round(gbs / pk, 4) if pk else None,
            "peak_source": src,
            "measured_bytes_per_point_stage": measured_bytes,
            "measured_gbs": round(measured_bytes * value / 1e9, 1),
            "measured_frac": round(measured_bytes * value / 1e9 / pk, 4) if pk else None,
            "measured_source": "ncu dram__bytes_read+write of every kernel of 21 right-hand sides on a "
                               "1024x384x16 slice of the workload, per grid-point stage "
                               "(profiles/dram-per-step_sbli-1024x384x16_fp64_mixed.md)"}


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during a timed region."""

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


def initial_state(case, seed=0):
    return inputs.channel_state(case, seed=seed) if case.kind == "channel" else inputs.bl_state(case, seed=seed)


def sbli_grid(nx, ny, nz, **kw):
    """The shock/boundary-layer workload on another grid with the same spacing (profiling
    captures and CPU samples)."""
    c = CASE
    return inputs.bl_case(f"sbli-{nx}x{ny}x{nz}", nx, ny, nz, c.lx * nx / c.nx, c.ly * ny / c.ny,
                          c.lz * nz / c.nz, shock=True, noise=c.noise, **kw)


def bench_case(args):
    """The benchmark workload, or (for profiling captures only) the same workload on another
    grid of the same spacing, or the 256 x 192 x 128 channel (on another grid: the same domain)."""
    channel = getattr(args, "workload", "sbli") == "channel"
    if not args.grid:
        return CHANNEL if channel else CASE
    nx, ny, nz = (int(v) for v in args.grid.lower().split("x"))
    if channel:
        return CHANNEL.replace(name=f"channel-{nx}x{ny}x{nz}", nx=nx, ny=ny, nz=nz)
    return sbli_grid(nx, ny, nz)


# ------------------------------------------------------------------------------ FMA peaks

def measure_peaks(local):
    """The FP64 and FP32 FMA rates of this GPU (strm_peak_fma), with the clock seen meanwhile."""
    from paper_2004_02276_gb300 import binding

    with ClockSampler(local) as clk:
        f64, ms64 = binding.peak_fma("fp64", launches=12)
        f32, ms32 = binding.peak_fma("fp32", launches=6)
    return {"fp64_tflops": f64, "fp32_tflops": f32, "fp64_launch_ms": ms64, "fp32_launch_ms": ms32,
            "clocks": clk.summary(), "source": f"strm_peak_fma, measured in this run ({PEAK_PROFILE})",
            "fp64_from_units_tflops": round(FP64_UNITS_TFLOPS, 3),
            "fp32_from_units_tflops": round(FP32_UNITS_TFLOPS, 2), "copy_gbs": copy_bandwidth(local)}


def copy_bandwidth(local, nbytes=1 << 31, reps=6):
    """Device-to-device copy rate of a 2 GiB buffer (bytes read + written per second, best of
    the repeats): the HBM denominator when the measured-peaks file is absent."""
    import torch

    src = torch.empty(nbytes // 8, dtype=torch.float64, device=f"cuda:{local}").fill_(1.0)
    dst = torch.empty_like(src)
    st = torch.cuda.current_stream()
    best = None
    for _ in range(reps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(st)
        dst.copy_(src)
        b.record(st)
        b.synchronize()
        ms = a.elapsed_time(b)
        best = ms if best is None else min(best, ms)
    del src, dst
    torch.cuda.empty_cache()
    return round(2 * nbytes / (best * 1e-3) / 1e9, 1)


# ------------------------------------------------------------------------------ the GPU path

def kernel_units(case, ktimes, weno_faces):
    """Units processed per kernel class over the timing-mode run: WENO faces, central faces
    (every face of the direction minus its WENO faces) and nodes."""
    nf = [(case.nx + 1) * case.ny * case.nz, case.nx * (case.ny + 1) * case.nz,
          case.nx * case.ny * (case.nz + 1)]
    units = {}
    for k, (ms, n) in ktimes.items():
        if n == 0:
            continue
        if k.startswith("weno"):
            units[k] = weno_faces["xyz".index(k[-1])]
        elif k.startswith("faces"):
            d = "xyz".index(k[-1])
            units[k] = nf[d] * n - weno_faces[d]
        else:
            units[k] = case.npts * n
    n_rhs = ktimes["assemble"][1]
    units["rk_update"] = case.npts * n_rhs  # fused into the assembly or a kernel of its own
    return units


def roofline(case, ktimes, weno_faces, ms_step, steps_timed, peak, flops, traffic, pipe_name):
    """Dominant kernel's algorithmic flops per launch / its average launch time against the
    measured FMA rate, and the whole step's algorithmic flops / ms_per_step against the same."""
    busy = {k: v for k, v in ktimes.items() if v[1] > 0}
    units = kernel_units(case, busy, weno_faces)
    dom = max(busy, key=lambda k: busy[k][0])
    dom_ms, dom_n = busy[dom]
    per_launch = units[dom] / dom_n
    achieved = flops.get(dom, 0) * per_launch / (dom_ms / dom_n / 1e3) / 1e12
    step_flops = sum(flops.get(k, 0) * u for k, u in units.items()) / steps_timed
    step_tflops = step_flops / (ms_step / 1e3) / 1e12
    total_ms = sum(v[0] for v in busy.values())
    return {
        "bound": "alu", "pipe": pipe_name, "kernel": dom, "achieved": round(achieved, 4),
        "peak": round(peak, 4), "unit": "TFLOP/s", "frac": round(achieved / peak, 4),
        "traffic": (round(traffic[dom] * per_launch) if dom in traffic else None),
        "traffic_source": ("ncu dram__bytes_read+write per unit of the current kernel, x units per launch"
                           if dom in traffic else "no capture of the current kernel"),
        "peak_source": f"strm_peak_fma, measured in this run ({PEAK_PROFILE})",
        "units_per_launch": per_launch, "flops_per_unit": flops.get(dom),
        "avg_launch_ms": round(dom_ms / dom_n, 4),
        "step_flops": step_flops, "step_achieved": round(step_tflops, 4),
        "step_frac": round(step_tflops / peak, 4),
        "kernel_share": {k: round(v[0] / total_ms, 4) for k, v in sorted(busy.items())},
        "weno_face_fraction": round(sum(weno_faces) / (3 * busy["assemble"][1] * case.npts), 4),
        "weno_faces_per_rhs": [round(f / busy["assemble"][1]) for f in weno_faces],
    }


def timed_steps(solver, w, r_old, steps, world, local):
    """K graph-replayed steps on the library stream, an event after each; returns the total ms
    (max over ranks), the per-step ms, the kernel launches and the clock record."""
    import torch

    ev = [torch.cuda.Event(enable_timing=True) for _ in range(steps + 1)]
    n0 = solver.launch_count()
    with ClockSampler(local) as clk:
        barrier(world)
        torch.cuda.synchronize()
        ev[0].record(solver.stream)
        for k in range(steps):
            solver.advance_n(w, r_old, 1)
            ev[k + 1].record(solver.stream)
        torch.cuda.synchronize()
        barrier(world)
    per = [ev[k].elapsed_time(ev[k + 1]) for k in range(steps)]
    ms = max_over_ranks(world, ev[0].elapsed_time(ev[steps]))
    return ms, per, solver.launch_count() - n0, clk.summary()


def measure(case, args, world, local, peak, flops, traffic, pipe_name, extra_pipe=None):
    """Warm-up, the timed region and the per-kernel event timing of a few eager steps, for one
    precision. Returns the figures, the solver, the device state and the steps taken."""
    import torch

    from paper_2004_02276_gb300 import binding

    solver = binding.Solver(case, device=f"cuda:{local}")
    w = torch.from_numpy(initial_state(case)).cuda()
    r_old = torch.zeros_like(w)
    solver.advance_n(w, r_old, args.warmup)  # also captures the step graph
    torch.cuda.synchronize()
    ms, per, launches, clocks = timed_steps(solver, w, r_old, args.steps, world, local)
    value = job_rate(case.npts, args.steps, world, ms)
    solver.timing(True)
    solver.advance_n(w, r_old, args.timing_steps)
    ktimes, weno_faces = solver.timing_read()
    solver.timing(False)
    roof = roofline(case, ktimes, weno_faces, ms / args.steps, args.timing_steps, peak, flops, traffic,
                    pipe_name)
    if extra_pipe:
        p2, f2, name2 = extra_pipe
        r2 = roofline(case, ktimes, weno_faces, ms / args.steps, args.timing_steps, p2, f2, {}, name2)
        roof["other_pipe"] = {k: r2[k] for k in ("pipe", "kernel", "achieved", "peak", "frac",
                                                 "step_achieved", "step_frac")}
    med = statistics.median(per)
    return {"value": value, "ms": ms, "ms_step_median": med, "value_median": job_rate(case.npts, 1, world, med),
            "repeats": len(per), "launches": launches, "clocks": clocks, "roofline": roof}, solver, w, r_old, \
        args.warmup + args.steps + args.timing_steps


def host_page_locked(t):
    """Page-lock a host tensor in place (cudaHostRegister); the memory is then mapped into the
    device's address space, and strm_advance_n_host copies it with a kernel through that
    address (188-210 GB/s on the GB300 node, steady), not with the copy engines, whose
    device-to-host rate into page-locked buffers fell to 7-130 GB/s some seconds after the
    buffer was locked."""
    import torch

    rc = torch.cuda.cudart().cudaHostRegister(t.data_ptr(), t.numel() * t.element_size(), 0)
    if int(rc) != 0:
        raise RuntimeError(f"cudaHostRegister failed ({rc})")
    return t


def host_copy_rates(h, d):
    """H2D and D2H rates (GB/s, CUDA events) of one copy-engine copy (cudaMemcpyAsync through
    torch) of the page-locked host buffer h to and from the device tensor d; d is restored from
    h afterwards. For comparison with the library's kernel copies, which the e2e figure uses."""
    import torch

    st = torch.cuda.current_stream()
    out = {}
    for name, (dst, src) in (("d2h", (h, d)), ("h2d", (d, h))):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(st)
        dst.copy_(src, non_blocking=True)
        b.record(st)
        b.synchronize()
        out[name] = round(h.numel() * h.element_size() / (a.elapsed_time(b) * 1e-3) / 1e9, 1)
    return out


def field_errors(a, b):
    """Relative L2 difference per conserved field of two device states."""
    import torch

    return [float(torch.linalg.vector_norm(a[m] - b[m]) / torch.linalg.vector_norm(b[m])) for m in range(5)]


def z_profiles(w):
    """Spanwise (z) means per (x, y) column of u and the Reynolds stresses <u'u'>, <v'v'>,
    <w'w'>, <u'v'> (the homogeneous direction of the boundary layer), as a [5, ny, nx] tensor."""
    import torch

    rho = w[0]
    u, v, ww = w[1] / rho, w[2] / rho, w[3] / rho
    um, vm, wm = (a.mean(dim=0, keepdim=True) for a in (u, v, ww))
    up, vp, wp = u - um, v - vm, ww - wm
    return torch.stack([um[0], (up * up).mean(0), (vp * vp).mean(0), (wp * wp).mean(0), (up * vp).mean(0)])


def xz_profiles(w):
    """Channel: x-z means per wall-normal row of u and the Reynolds stresses <u'u'>, <v'v'>,
    <w'w'>, <u'v'>, as a [5, ny] tensor."""
    import torch

    rho = w[0]
    u, v, ww = w[1] / rho, w[2] / rho, w[3] / rho
    um, vm, wm = (a.mean(dim=(0, 2), keepdim=True) for a in (u, v, ww))
    up, vp, wp = u - um, v - vm, ww - wm
    return torch.stack([um[0, :, 0], (up * up).mean((0, 2)), (vp * vp).mean((0, 2)),
                        (wp * wp).mean((0, 2)), (up * vp).mean((0, 2))])


def profile_errors(pa, pb):
    """Largest difference of each profile relative to the profile's peak magnitude."""
    return [float((pa[q] - pb[q]).abs().max() / pb[q].abs().max().clamp_min(1e-300)) for q in range(pa.shape[0])]


def small_case_errors(case):
    """Mixed precision against the FP64 oracle on the 64 x 48 x 32 channel after 100 steps:
    in the configs' own sensor mode (free running: decisions may flip at the threshold), and
    with the decisions of the FP64 run prescribed to both at every step."""
    import torch

    from oracle import oracle as O
    from paper_2004_02276_gb300 import binding

    mc = case.replace(precision="mixed")
    cfg = O.make_cfg(case)
    w0 = inputs.channel_state(case, seed=0)
    out = {}
    wo, _, _ = O.advance(cfg, w0, 100, cfl=case.cfl)
    s = binding.Solver(mc)
    w = torch.from_numpy(w0).cuda()
    s.advance_n(w, torch.zeros_like(w), 100, cfl=case.cfl)
    wm = w.cpu().numpy()
    s.close()
    out["sensor_mode"] = [float(np.linalg.norm(wm[m] - wo[m]) / np.linalg.norm(wo[m])) for m in range(5)]
    # equal decisions: the FP64 oracle's sensor of its own state before each step, to both
    s = binding.Solver(mc)
    th_d = torch.empty((case.nz, case.ny, case.nx), dtype=torch.float64, device="cuda")
    s.set_theta(th_d)
    w = torch.from_numpy(w0).cuda()
    r = torch.zeros_like(w)
    wo = w0
    for _ in range(100):
        th = O.sensor(cfg, wo)[0]
        th_d.copy_(torch.from_numpy(th))
        s.advance_n(w, r, 1, cfl=case.cfl)
        wo, _ = O.rk_step(O.make_cfg(case, theta_fixed=th), wo, cfl=case.cfl)
    wm = w.cpu().numpy()
    s.close()
    out["equal_decisions"] = [float(np.linalg.norm(wm[m] - wo[m]) / np.linalg.norm(wo[m])) for m in range(5)]
    out["equal_decisions_profiles"] = profile_errors(xz_profiles(torch.from_numpy(wm)),
                                                     xz_profiles(torch.from_numpy(wo)))
    return out


def run_ours(args, world, rank, local):
    import torch

    from paper_2004_02276_gb300 import binding

    torch.cuda.set_device(local)
    case = bench_case(args)
    pk = measure_peaks(local)
    m64, solver, w, r_old, steps64 = measure(case, args, world, local, pk["fp64_tflops"], FLOPS_PER_UNIT,
                                             DRAM_BYTES_PER_UNIT, "fp64")

    # end to end through the C ABI with host buffers: per step H2D of the state from pinned
    # memory, one RK3 step, D2H of the new state. The host buffer carries the FP64 trajectory,
    # which continues from the device state (the register r_old is not read by stage 0).
    nbytes = 5 * case.npts * 8
    w_host = torch.empty(w.shape, dtype=torch.float64)
    w_host.fill_(0.0)  # first touch by the host's threads, before page-locking
    host_page_locked(w_host)
    w_host.copy_(w)
    wd = torch.empty_like(w)
    del r_old
    solver.advance_n_host(w_host, wd, w, 1)  # warm (graph for these buffers)
    copy_gbs = host_copy_rates(w_host, wd)
    barrier(world)
    t0 = time.perf_counter()
    calls = []
    for _ in range(args.steps):
        t1 = time.perf_counter()
        solver.advance_n_host(w_host, wd, w, 1)
        calls.append(time.perf_counter() - t1)
    e2e_s = max_over_ranks(world, time.perf_counter() - t0)
    steps64 += args.steps + 1
    wf = solver.weno_counts()
    calls.sort()
    e2e = {"value": case.npts * 3 * args.steps * world / e2e_s, "unit": UNIT,
           "h2d_bytes_per_step": nbytes, "d2h_bytes_per_step": nbytes,
           "host_buffer": "host memory page-locked with cudaHostRegister (mapped): the library "
                          "copies it with its k_copy_mapped kernel through the device address",
           "copy_engine_gbs": copy_gbs,
           "call_ms": {"min": round(calls[0] * 1e3, 1), "median": round(calls[len(calls) // 2] * 1e3, 1),
                       "max": round(calls[-1] * 1e3, 1)},
           "weno_face_fraction_last_rhs": round(sum(wf) / (3.0 * case.npts), 4)}
    ws_gb = solver.workspace.numel() / 1e9

    out = {
        "metric": METRIC, "value": m64["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": m64["ms"] / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": case.name, "grid": [case.nx, case.ny, case.nz], "points": case.npts,
                   "mach": case.mach, "re_delta_in": case.reynolds, "shock_deflection_deg": 8.0,
                   "scheme": "central6+WENO5 (Ducros 0.05)", "cfl": case.cfl, "precision": "fp64",
                   "parallelism": f"replicas x{world}",
                   "l2": "inputs larger than L2 (state %d MB + workspace %.1f GB vs 129 MB L2)"
                         % (nbytes // 2**20, ws_gb)},
        "ms_per_step_median": m64["ms_step_median"], "value_median": m64["value_median"],
        "timed_repeats": m64["repeats"],
        "roofline": m64["roofline"], "e2e": e2e, "gpu_launches": m64["launches"],
        "clocks": m64["clocks"], "hbm_step": hbm_step(m64["value"], pk.get("copy_gbs")), "peaks": pk,
    }
    # the FP64 trajectory on to the error leg's step count
    wd.copy_(w_host)
    torch.cuda.synchronize()
    torch.cuda.cudart().cudaHostUnregister(w_host.data_ptr())
    rest = max(args.error_steps - steps64, 0)
    if rest and not args.no_mixed:
        solver.advance_n(wd, w, rest)
    steps64 += rest
    w64 = wd
    solver.close()
    del solver, w, w_host
    torch.cuda.empty_cache()

    if not args.no_mixed:
        mcase = case.replace(precision="mixed")
        mm, msolver, wm, rm, stepsm = measure(mcase, args, world, local, pk["fp64_tflops"],
                                              FLOPS64_PER_UNIT_MIXED, DRAM_BYTES_PER_UNIT_MIXED, "fp64",
                                              extra_pipe=(pk["fp32_tflops"], FLOPS32_PER_UNIT_MIXED, "fp32"))
        mr = mm["roofline"]
        if mr["kernel"] in ALG_BYTES_PER_UNIT_MIXED and mr["avg_launch_ms"] > 0:
            hb = peaks().get("hbm_gbs") or pk.get("copy_gbs")
            gbs = ALG_BYTES_PER_UNIT_MIXED[mr["kernel"]] * mr["units_per_launch"] / (mr["avg_launch_ms"] * 1e-3) / 1e9
            mr["hbm_view"] = {"bound": "hbm", "kernel": mr["kernel"],
                              "bytes_per_unit": ALG_BYTES_PER_UNIT_MIXED[mr["kernel"]],
                              "achieved": round(gbs, 1), "peak": hb, "unit": "GB/s",
                              "frac": round(gbs / hb, 4) if hb else None,
                              "note": "algorithmic bytes of the mixed assembly per node (state and "
                                      "register in and out, FP32 face fluxes, FP32 node fields) over "
                                      "its launch time: the bound that applies to this kernel, whose "
                                      "FP64 and FP32 pipes are both far from busy"}
        if steps64 > stepsm:
            msolver.advance_n(wm, rm, steps64 - stepsm)
        err = field_errors(wm, w64)
        perr = profile_errors(z_profiles(wm), z_profiles(w64))
        msolver.close()
        del msolver, wm, rm
        torch.cuda.empty_cache()
        out["variants"] = {"mixed": {
            "value": mm["value"], "ms_per_step": mm["ms"] / args.steps,
            "ms_per_step_median": mm["ms_step_median"],
            "speedup_vs_fp64": mm["value"] / m64["value"], "dtype": "f32 flux / f64 state",
            "roofline": mm["roofline"], "gpu_launches": mm["launches"], "clocks": mm["clocks"],
            "hbm_step": hbm_step(mm["value"], pk.get("copy_gbs"), MEASURED_STEP_BYTES_MIXED),
            "error": {
                "vs": "the FP64 path on the same workload (itself within 1e-12 of the oracle)",
                "steps": steps64, "rel_l2_per_field": err, "max": max(err),
                "profiles": ["U", "u'u'", "v'v'", "w'w'", "u'v'"],
                "profile_rel_max": perr,
                "mode": "Ducros switch on (the workload's own), decisions free to flip at the threshold",
                "meets_1e-5": max(err) <= 1e-5},
        }}
    del w64
    torch.cuda.empty_cache()
    if rank == 0 and world == 1 and not args.no_cpu:
        if not args.no_mixed:
            sc = small_case_errors(SMALL)
            out["variants"]["mixed"]["error_64x48x32_vs_oracle_100_steps"] = {
                "sensor_mode_rel_l2": sc["sensor_mode"],
                "equal_decisions_rel_l2": sc["equal_decisions"],
                "equal_decisions_profile_rel_max": sc["equal_decisions_profiles"],
                "equal_decisions_meets_1e-5": max(sc["equal_decisions"]) <= 1e-5,
                "note": "equal decisions: the FP64 oracle's sensor of its state before each step "
                        "is prescribed to both runs (strm_set_theta)"}
        out["cpu_baseline"], out["error"] = cpu_baseline(local)
    if not args.no_variants:
        out.setdefault("variants", {})["channel_256x192x128"] = run_channel(args, world, local)
        out["variants"]["batched"] = run_batched(args, world, local,
                                                 out["variants"]["channel_256x192x128"]["fp64"])
        if not args.no_mixed:
            out["variants"]["batched_mixed"] = run_batched(
                args, world, local, out["variants"]["channel_256x192x128"]["mixed"], "mixed")
    if rank == 0:
        print(json.dumps(out), flush=True)


def cpu_baseline(local):
    """The oracle, unmodified, on the host cores: one RK3 step of a 2048 x 384 x 8 slab of the
    workload (same x/y grid and spacing, periodic z) on all cores, and of a 256 x 384 x 8 slab
    on one thread; the same all-core sample on the GPU gives the error at which the figures
    hold."""
    import torch

    from oracle import oracle as O
    from paper_2004_02276_gb300 import binding

    allc = O.threads()
    res = {}
    for name, case, nthr in (("all_cores", sbli_grid(CASE.nx, CASE.ny, 8), allc),
                             ("one_thread", sbli_grid(256, CASE.ny, 8), 1)):
        O.set_threads(nthr)
        cfg = O.make_cfg(case)
        w0 = initial_state(case)
        t0 = time.perf_counter()
        w1, _ = O.rk_step(cfg, w0, cfl=case.cfl)
        sec = time.perf_counter() - t0
        res[name] = (case, case.npts * 3 / sec, sec, w0, w1)
    O.set_threads(allc)
    case, rate, sec, w0, w1 = res["all_cores"]
    s = binding.Solver(case, device=f"cuda:{local}")
    wg = torch.from_numpy(w0).cuda()
    s.rk_step(wg, torch.zeros_like(wg))
    wg = wg.cpu().numpy()
    s.close()
    err = [float(np.linalg.norm(wg[m] - w1[m]) / np.linalg.norm(w1[m])) for m in range(5)]
    c1, rate1, sec1 = res["one_thread"][:3]
    base = {"value": rate, "unit": UNIT, "cores": allc, "kind": "oracle",
            "sample": f"one RK3 step of a {case.nx}x{case.ny}x{case.nz} slab of the workload "
                      f"({sec:.1f} s on {allc} host threads)",
            "one_thread": {"value": rate1, "cores": 1,
                           "sample": f"one RK3 step of a {c1.nx}x{c1.ny}x{c1.nz} slab ({sec1:.1f} s)"},
            "nproc": os.cpu_count()}
    return base, {"rel_l2_vs_oracle_one_step_of_the_sample": err, "max": max(err)}


def run_channel(args, world, local):
    """The 256 x 192 x 128 channel (bulk Mach 1.5, Re_b 7000) in both precisions: W warm-up
    and K timed graph-replayed steps each."""
    import torch

    from paper_2004_02276_gb300 import binding

    out = {"workload": CHANNEL.name}
    for prec in ("fp64",) + (() if args.no_mixed else ("mixed",)):
        c = CHANNEL.replace(precision=prec)
        s = binding.Solver(c, device=f"cuda:{local}")
        w = torch.from_numpy(initial_state(c)).cuda()
        r = torch.zeros_like(w)
        s.advance_n(w, r, args.warmup)
        ms, per, _, clk = timed_steps(s, w, r, args.steps, world, local)
        out[prec] = job_rate(c.npts, args.steps, world, ms)
        out[prec + "_ms_per_step"] = ms / args.steps
        s.close()
        del s, w, r
        torch.cuda.empty_cache()
    return out


def run_batched(args, world, local, large_grid_value, precision="fp64", schedule="tuned"):
    """The batched workload: 64 independent channels of uneven size, Mach and Reynolds number
    (44.7 M points in all), advanced by the ensemble kernels, one graph replay per step, launch
    shapes from the autotuner (run before the warm-up, outside the timed region). The per-point
    rate is compared with the 256 x 192 x 128 channel's rate in the same precision."""
    import torch

    from paper_2004_02276_gb300 import binding

    cases = inputs.ensemble_cases(seed=0, precision=precision)[:getattr(args, "ensemble_instances", 0) or None]
    npts = sum(c.npts for c in cases)
    E = binding.Ensemble(cases, device=f"cuda:{local}")
    ws = [torch.from_numpy(inputs.channel_state(c)).cuda() for c in cases]
    rs = [torch.zeros_like(w) for w in ws]
    if schedule == "tuned":
        choice = E.tune(ws, rs)
    else:  # a fixed schedule, for profiling captures
        choice = dict(weno_block=128, weno_per_sm=16, central_per_sm=16,
                      persistent=int(schedule == "persistent"), slab_cap=32)
        E.set_schedule(**choice)
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
    # both schedules with the tuned launch shapes and pencil tile, a few steps each (untimed by
    # the driver's contract; context for the tuner's choice)
    schedules = {}
    k = max(2, min(5, args.steps))
    for name, persistent in (("per_kernel_type", 0), ("persistent_stage", 1)):
        try:
            E.set_schedule(**dict(choice, persistent=persistent))
        except binding.StrmError as e:
            schedules[name] = str(e)
            continue
        E.advance(ws, rs, 1, cfl=0.8)
        torch.cuda.synchronize()
        start.record(E.stream)
        E.advance(ws, rs, k, cfl=0.8)
        stop.record(E.stream)
        torch.cuda.synchronize()
        schedules[name] = round(npts * 3 * k / (start.elapsed_time(stop) / 1e3) / 1e6, 1)
    schedules["unit"] = "M grid-pt RK-stage updates/s"
    schedules["steps"] = k
    E.close()
    return {"value": value, "ms_per_step": ms / args.steps, "instances": len(cases),
            "points": npts, "dtype": "f64" if precision == "fp64" else "f32 flux / f64 state",
            "per_point_vs_large_grid": value / large_grid_value if large_grid_value else None,
            "tuned": choice, "schedules": schedules,
            "schedule": "one cooperative launch per RK stage" if choice["persistent"] else
                        "one launch per kernel type, one graph per step",
            "finite": bool(np.isfinite(np.array(tot)).all()), "clocks": clk.summary(),
            "workload": "64 channels, dims U{32..192}xU{32..128}xU{32..128}, M_b U[0.3,3], "
                        "Re_b U[2000,8000], seed 0"}


def run_reference(args, world, rank):
    """The FP64 C oracle timed on the host cores, each benchmark step a bounded sample of the
    workload: one RK3 step of a 2048 x 384 x 8 slab (same x/y grid and spacing, periodic z)."""
    if rank != 0:
        return
    from oracle import oracle as O

    case = sbli_grid(CASE.nx, CASE.ny, 8)
    cfg = O.make_cfg(case)
    w = initial_state(case)
    for _ in range(args.warmup):
        w, _ = O.rk_step(cfg, w, cfl=case.cfl)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        w, _ = O.rk_step(cfg, w, cfl=case.cfl)
    sec = time.perf_counter() - t0
    value = case.npts * 3 * args.steps / sec
    sample = f"each step: one RK3 step on a {case.nx}x{case.ny}x{case.nz} slab of the workload"
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": sec * 1e3 / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "impl": "reference",
        "config": {"workload": CASE.name, "grid": [CASE.nx, CASE.ny, CASE.nz], "precision": "fp64",
                   "sample": sample},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": O.threads(), "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(out), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--timing-steps", type=int, default=2,
                    help="eager steps of the per-kernel event timing (roofline)")
    ap.add_argument("--error-steps", type=int, default=100,
                    help="steps after which the mixed path is compared with the FP64 path")
    ap.add_argument("--no-cpu", action="store_true", help="skip the oracle legs (CPU baseline, errors)")
    ap.add_argument("--grid", default="", help="NXxNYxNZ of the same workload, for profiling captures only")
    ap.add_argument("--workload", default="sbli", choices=["sbli", "channel"],
                    help="the timed workload: the shock/boundary layer (benchmark) or, for profiling "
                         "captures only, the channel")
    ap.add_argument("--no-mixed", action="store_true", help="skip the mixed-precision variant")
    ap.add_argument("--no-variants", action="store_true", help="skip the channel and batched variants")
    ap.add_argument("--ensemble-only", default="", choices=["", "fp64", "mixed"],
                    help="for profiling captures only: run the 64-channel ensemble alone in this "
                         "precision and print its figures")
    ap.add_argument("--ensemble-instances", type=int, default=0,
                    help="with --ensemble-only, for profiling captures: the first K instances only")
    ap.add_argument("--schedule", default="tuned", choices=["tuned", "per-kernel", "persistent"],
                    help="ensemble schedule with --ensemble-only (default: the autotuner's choice)")
    ap.add_argument("--peaks-only", action="store_true",
                    help="only measure and print the FP64/FP32 FMA rates (strm_peak_fma) and exit")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.steps < 1 or args.timing_steps < 1:
        ap.error("--steps and --timing-steps must be >= 1")
    world, rank, local = dist_setup()
    if args.peaks_only:
        import torch

        torch.cuda.set_device(local)
        print(json.dumps(measure_peaks(local)), flush=True)
        return
    if args.ensemble_only:
        import torch

        torch.cuda.set_device(local)
        out = run_batched(args, world, local, None, args.ensemble_only, args.schedule)
        if rank == 0:
            print(json.dumps(out), flush=True)
        return
    if args.impl == "reference":
        run_reference(args, world, rank)
    else:
        run_ours(args, world, rank, local)
    if world > 1:
        import torch.distributed as dist

        dist.destroy_process_group()


if __name__ == "__main__":
    main()
