"""Batched ensemble (many independent grids in one launch per kernel type, one CUDA graph per
RK step): every instance must compute what a context of its own computes, since both run the
same kernel bodies with the same per-instance reduction order. The only freedom left is the
compiler's choice of where to contract a multiply and an add into an FMA, which may differ
between the batched and the single-grid kernel that inline the same body; the comparison is
therefore to a few ulp (FP64) or FP32 round-off (mixed), through the C ABI, before and after the
autotuner picks launch shapes. Every instance is also checked against the FP64 oracle, so that a
defect shared by the batched and the single-grid kernels cannot pass unseen."""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2004_02276_gb300 import binding, inputs

pytestmark = pytest.mark.gpu

# max-norm difference per field relative to the field's max, after a few steps
TOL = {"fp64": 1e-13, "mixed": 1e-5}
# simulated time: the CFL step of mixed precision comes from FP32 wave speeds of a state that
# differs from the single context's by FP32 round-off (where the compiler fuses differently)
TIME_TOL = {"fp64": 1e-13, "mixed": 1e-6}


def rel_max(a, b):
    return max(np.abs(a[m] - b[m]).max() / max(np.abs(b[m]).max(), 1e-300) for m in range(5))


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__

    __graft_entry__.build()
    torch.cuda.set_device(0)


def mixed_bag(precision):
    return [
        inputs.Case(nx=40, ny=24, nz=18, mach=0.5, reynolds=2500.0, precision=precision),
        inputs.Case(nx=33, ny=37, nz=9, mach=2.4, reynolds=7000.0, precision=precision),
        inputs.Case(nx=64, ny=16, nz=30, y_wall=False, forcing=False, precision=precision),
        inputs.Case(nx=17, ny=21, nz=13, weno_mode="off", precision=precision),
        inputs.Case(nx=24, ny=12, nz=20, weno_mode="all", beta=0.0, precision=precision),
        inputs.Case(nx=50, ny=3, nz=7, mach=3.0, precision=precision),
    ]


def single_runs(cases, nsteps):
    out, times = [], []
    for c in cases:
        s = binding.Solver(c)
        w = torch.from_numpy(inputs.channel_state(c, seed=c.nx)).cuda()
        r = torch.zeros_like(w)
        s.advance_n(w, r, nsteps, cfl=0.8)
        out.append(w.cpu().numpy())
        times.append(s.time()[0])
        s.close()
    return out, times


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_ensemble_equals_independent_contexts(precision):
    cases = mixed_bag(precision)
    ref, tref = single_runs(cases, 4)
    E = binding.Ensemble(cases)
    ws = [torch.from_numpy(inputs.channel_state(c, seed=c.nx)).cuda() for c in cases]
    rs = [torch.zeros_like(w) for w in ws]
    E.advance(ws, rs, 4, cfl=0.8)
    torch.cuda.synchronize()
    errs = [rel_max(ws[e].cpu().numpy(), ref[e]) for e in range(len(cases))]
    print(precision, "ensemble vs independent contexts, max relative difference:", max(errs))
    assert max(errs) <= TOL[precision], errs
    np.testing.assert_allclose(E.times(), tref, rtol=TIME_TOL[precision])
    tot = E.totals(ws)
    assert all(np.isfinite(t).all() for t in tot)
    E.close()


def test_tuned_ensemble_still_exact():
    cases = mixed_bag("fp64")
    ref, _ = single_runs(cases, 3)
    E = binding.Ensemble(cases)
    ws = [torch.from_numpy(inputs.channel_state(c, seed=c.nx)).cuda() for c in cases]
    rs = [torch.zeros_like(w) for w in ws]
    choice = E.tune(ws, rs)
    assert choice["weno_block"] in (32, 64, 128) and choice["weno_per_sm"] in (4, 8, 16)
    assert choice["central_per_sm"] in (8, 16, 32) and choice["persistent"] in (0, 1)
    assert choice["slab_cap"] in (0, 8, 16, 32)
    E.advance(ws, rs, 3, cfl=0.8)
    errs = [rel_max(ws[e].cpu().numpy(), ref[e]) for e in range(len(cases))]
    assert max(errs) <= TOL["fp64"], errs
    E.close()


def test_ensemble_rejects_mixed_orders():
    cases = [inputs.Case(nx=8, ny=6, nz=4), inputs.Case(nx=8, ny=6, nz=4, L=2)]
    with pytest.raises(binding.StrmError):
        binding.Ensemble(cases)


def test_ensemble_workload_draws():
    cases = inputs.ensemble_cases(seed=0)
    assert len(cases) == 64
    assert all(32 <= c.nx <= 192 and 32 <= c.ny <= 128 and 32 <= c.nz <= 128 for c in cases)
    assert all(0.3 <= c.mach <= 3.0 and 2000 <= c.reynolds <= 8000 for c in cases)


def bl_bag(precision):
    """Channel and boundary-layer instances together: recycling inflow, oblique shock, digital-
    filter inflow, characteristic faces on every side."""
    return [
        inputs.Case(nx=40, ny=24, nz=18, mach=0.5, reynolds=2500.0, precision=precision),
        inputs.bl_case("bl-48x40x12", 48, 40, 12, 7.0, 6.0, 1.5, precision=precision),
        inputs.bl_case("sbli-64x40x12", 64, 40, 12, 12.0, 6.0, 1.5, shock=True, noise=0.003,
                       precision=precision),
        inputs.bl_case("bl-df-36x30x10", 36, 30, 10, 5.0, 6.0, 1.5, bc_xmin="df", df_ny=2, df_nz=2,
                       df_tau=0.3, df_seed=3, precision=precision),
        inputs.bl_case("open-40x24x10", 40, 24, 10, 6.0, 6.0, 1.5, bc_xmin="char", bc_ymin="char",
                       weno_mode="all", precision=precision),
    ]


def initial(c):
    return inputs.channel_state(c, seed=c.nx) if c.kind == "channel" else inputs.bl_state(c, seed=c.nx)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_ensemble_with_boundary_layer_instances(precision):
    cases = bl_bag(precision)
    inflows = {e: inputs.df_profiles(c) for e, c in enumerate(cases) if c.bc_xmin == "df"}
    ref, tref = [], []
    for e, c in enumerate(cases):
        s = binding.Solver(c, inflow=inflows.get(e))
        w = torch.from_numpy(initial(c)).cuda()
        s.advance_n(w, torch.zeros_like(w), 4, cfl=0.8)
        ref.append(w.cpu().numpy())
        tref.append(s.time()[0])
        s.close()
    E = binding.Ensemble(cases, inflows=inflows)
    ws = [torch.from_numpy(initial(c)).cuda() for c in cases]
    rs = [torch.zeros_like(w) for w in ws]
    E.advance(ws, rs, 4, cfl=0.8)
    errs = [rel_max(ws[e].cpu().numpy(), ref[e]) for e in range(len(cases))]
    print(precision, "boundary-layer ensemble vs independent contexts:", max(errs))
    assert max(errs) <= TOL[precision], errs
    np.testing.assert_allclose(E.times(), tref, rtol=TIME_TOL[precision])
    E.close()


# the oracle comparison: relative L2 per conserved field after the steps
ORACLE_TOL = {"fp64": 1e-12, "mixed": 1e-4}


def oracle_run(c, w0, nsteps):
    df = O.DFState(c, inputs.df_profiles(c)) if c.bc_xmin == "df" else None
    wo, to, _ = O.advance(O.make_cfg(c, df=df), w0, nsteps, cfl=0.8)
    return wo, to


def rel_l2(a, b):
    return np.array([np.linalg.norm(a[m] - b[m]) / max(np.linalg.norm(b[m]), 1e-300)
                     for m in range(5)])


@pytest.mark.parametrize("bag", ["channels", "boundary-layers"])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_ensemble_instances_match_oracle(bag, precision):
    """Every instance of the ensemble after 4 CFL steps against 4 oracle steps of that instance
    alone: relative L2 <= 1e-12 per field in FP64 (the FP64 target), <= 1e-4 in mixed precision
    (FP32 flux arithmetic over 12 stages); the same simulated time."""
    cases = mixed_bag(precision) if bag == "channels" else bl_bag(precision)
    w0s = [inputs.channel_state(c, seed=c.nx) if c.kind == "channel" else inputs.bl_state(c, seed=c.nx)
           for c in cases]
    inflows = {e: inputs.df_profiles(c) for e, c in enumerate(cases) if c.bc_xmin == "df"}
    E = binding.Ensemble(cases, inflows=inflows)
    ws = [torch.from_numpy(w0).cuda() for w0 in w0s]
    rs = [torch.zeros_like(w) for w in ws]
    E.advance(ws, rs, 4, cfl=0.8)
    times = E.times()
    got = [w.cpu().numpy() for w in ws]
    E.close()
    worst = 0.0
    for e, c in enumerate(cases):
        wo, to = oracle_run(c, w0s[e], 4)
        err = rel_l2(got[e], wo)
        worst = max(worst, err.max())
        assert err.max() <= ORACLE_TOL[precision], (c.name, err)
        assert abs(times[e] - to) <= (1e-13 if precision == "fp64" else 1e-5) * to, (c.name, times[e], to)
    print(bag, precision, "ensemble vs oracle, worst relative L2:", worst)


@pytest.mark.parametrize("bag", ["channels", "boundary-layers"])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_persistent_stage_matches_oracle(bag, precision):
    """The persistent schedule (one cooperative launch per RK stage, grid-wide barriers between
    the phases) with the natural traversal order, then with slab height 8: every instance after
    4 CFL steps against the oracle, as for the per-kernel-type schedule; no barrier gave up."""
    cases = mixed_bag(precision) if bag == "channels" else [c for c in bl_bag(precision) if c.bc_xmin != "df"]
    w0s = [initial(c) for c in cases]
    refs = [oracle_run(c, w0s[e], 4) for e, c in enumerate(cases)]
    for slab_cap in (0, 8):
        E = binding.Ensemble(cases)
        E.set_schedule(persistent=1, slab_cap=slab_cap)
        ws = [torch.from_numpy(w0).cuda() for w0 in w0s]
        rs = [torch.zeros_like(w) for w in ws]
        E.advance(ws, rs, 4, cfl=0.8)
        times = E.times()
        assert E.debug_flags() == 0
        got = [w.cpu().numpy() for w in ws]
        E.close()
        for e, c in enumerate(cases):
            wo, to = refs[e]
            err = rel_l2(got[e], wo)
            assert err.max() <= ORACLE_TOL[precision], (c.name, slab_cap, err)
            assert abs(times[e] - to) <= (1e-13 if precision == "fp64" else 1e-5) * to, (c.name, times[e], to)


def test_persistent_stage_equals_per_kernel_schedule():
    """FP64: the persistent stage and the per-kernel-type launches run the same bodies; after
    3 steps they agree to a few ulp (the forcing and CFL reductions may group their partial sums
    differently)."""
    cases = mixed_bag("fp64")
    out = []
    for persistent in (0, 1):
        E = binding.Ensemble(cases)
        E.set_schedule(persistent=persistent)
        ws = [torch.from_numpy(inputs.channel_state(c, seed=c.nx)).cuda() for c in cases]
        rs = [torch.zeros_like(w) for w in ws]
        E.advance(ws, rs, 3, cfl=0.8)
        out.append([w.cpu().numpy() for w in ws])
        E.close()
    errs = [rel_max(a, b) for a, b in zip(out[1], out[0])]
    assert max(errs) <= TOL["fp64"], errs


def test_schedule_checks():
    cases = bl_bag("fp64")
    inflows = {e: inputs.df_profiles(c) for e, c in enumerate(cases) if c.bc_xmin == "df"}
    E = binding.Ensemble(cases, inflows=inflows)
    with pytest.raises(binding.StrmError):  # a digital-filter inflow needs its own kernels per step
        E.set_schedule(persistent=1)
    for bad in (dict(weno_block=96), dict(slab_cap=12), dict(persistent=2), dict(central_per_sm=0)):
        with pytest.raises(binding.StrmError):
            E.set_schedule(**bad)
    E.set_schedule(slab_cap=0)
    E.close()


def test_persistent_barrier_gives_up_and_recovers():
    """Failure detection of the persistent stage without a GPU fault: with a barrier limit of 0
    the first block that has to wait gives up, every block leaves the kernel, and the ensemble
    reports bit 32 once (the report also resets the barrier). With the limit restored, the same
    ensemble advances a fresh state exactly as an ensemble that never failed."""
    cases = mixed_bag("fp64")
    fresh = lambda: [torch.from_numpy(inputs.channel_state(c, seed=c.nx)).cuda() for c in cases]
    ref = binding.Ensemble(cases)
    ref.set_schedule(persistent=1)
    wr = fresh()
    ref.advance(wr, [torch.zeros_like(w) for w in wr], 2, cfl=0.8)
    want = [w.cpu().numpy() for w in wr]
    ref.close()
    E = binding.Ensemble(cases)
    E.set_schedule(persistent=1)
    E.set_barrier_limit(0.0)
    ws = fresh()
    E.advance(ws, [torch.zeros_like(w) for w in ws], 1, cfl=0.8)
    assert E.debug_flags() & 32
    assert E.debug_flags() == 0  # reported once; the barrier is reset
    E.set_barrier_limit(10.0)
    ws = fresh()
    rs = [torch.zeros_like(w) for w in ws]
    E.advance(ws, rs, 2, cfl=0.8)
    assert E.debug_flags() == 0
    for e in range(len(cases)):
        assert np.array_equal(ws[e].cpu().numpy(), want[e]), e
    with pytest.raises(binding.StrmError):
        E.set_barrier_limit(-1.0)
    E.close()
