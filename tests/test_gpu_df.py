"""Digital-filter turbulent inflow (Section 3.2) on the GPU against the FP64 oracle: the same
counter-based random numbers are drawn on both sides, so the ghost states, the right-hand side
and the states after several steps (one new plane per step, blended in time) agree to
round-off."""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2004_02276_gb300 import binding, inputs

pytestmark = pytest.mark.gpu

TOL = 1e-12


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__

    __graft_entry__.build()
    torch.cuda.set_device(0)


def rel_max(a, b):
    return np.array([np.abs(a[m] - b[m]).max() / max(np.abs(b[m]).max(), 1e-300) for m in range(5)])


def rel_l2(a, b):
    return np.array([np.linalg.norm(a[m] - b[m]) / max(np.linalg.norm(b[m]), 1e-300) for m in range(5)])


DF_BL = inputs.bl_case("bl-df-48x40x16", 48, 40, 16, 7.0, 6.0, 1.5, bc_xmin="df", df_ny=3, df_nz=2,
                       df_tau=0.5, df_seed=12345)
DF_ODD = inputs.bl_case("bl-df-37x29x9", 37, 29, 9, 5.0, 6.0, 1.0, bc_xmin="df", df_ny=2, df_nz=4,
                        df_tau=0.2, df_seed=7, y_map="sinh1", beta=3.0)
# the paper's own boundary-layer settings together (Section 3.2): fourth-order stencils,
# Sutherland's law, hyperbolic-sine clustering and the digital-filter inflow
DF_PAPER = inputs.bl_case("bl-paper-48x40x12", 48, 40, 12, 7.0, 6.0, 1.5, bc_xmin="df", df_ny=3,
                          df_nz=3, df_tau=0.5, df_seed=11, L=2, visc_law="sutherland",
                          y_map="sinh1", beta=4.0)


def oracle_cfg(case):
    df = O.DFState(case, inputs.df_profiles(case))
    return O.make_cfg(case, df=df), df


@pytest.mark.parametrize("case", [DF_BL, DF_ODD, DF_PAPER], ids=lambda c: c.name)
def test_rhs_and_flags_match_oracle(case):
    w0 = inputs.bl_state(case, seed=2)
    cfg, _ = oracle_cfg(case)
    ref = O.rhs(cfg, w0)
    _, _, fx_o, fy_o, fz_o = O.sensor(cfg, w0)
    s = binding.Solver(case, inflow=inputs.df_profiles(case))
    w = torch.from_numpy(w0).cuda()
    r = s.compute_rhs(w).cpu().numpy()
    _, _, fx, fy, fz = (t.cpu().numpy() for t in s.sensor(w))
    s.close()
    assert np.array_equal(fx, fx_o) and np.array_equal(fy, fy_o) and np.array_equal(fz, fz_o)
    err = rel_max(r, ref)
    assert err.max() <= TOL, err


@pytest.mark.parametrize("case", [DF_BL, DF_ODD, DF_PAPER], ids=lambda c: c.name)
def test_ten_steps_match_oracle(case):
    w0 = inputs.bl_state(case, seed=3)
    cfg, df = oracle_cfg(case)
    wo, to, _ = O.advance(cfg, w0, 10, cfl=case.cfl)
    assert df.count[0] == 11
    s = binding.Solver(case, inflow=inputs.df_profiles(case))
    w = torch.from_numpy(w0).cuda()
    r_old = torch.zeros_like(w)
    s.advance_n(w, r_old, 10, cfl=case.cfl)
    t, _ = s.time()
    wg = w.cpu().numpy()
    s.close()
    err = rel_l2(wg, wo)
    assert err.max() <= TOL, err
    assert abs(t - to) <= 1e-13 * to


def test_graph_replay_equals_eager_steps():
    case = DF_BL
    w0 = torch.from_numpy(inputs.bl_state(case, seed=4)).cuda()
    outs = []
    for mode in ("graph", "eager"):
        s = binding.Solver(case, inflow=inputs.df_profiles(case))
        w = w0.clone()
        r_old = torch.zeros_like(w)
        if mode == "graph":
            s.advance_n(w, r_old, 6, cfl=case.cfl)
        else:
            for _ in range(6):
                s.rk_step(w, r_old, dt=0.0, cfl=case.cfl)
        outs.append(w.cpu().numpy())
        s.close()
    assert np.array_equal(outs[0], outs[1])


def test_mixed_precision_inflow():
    case = DF_BL.replace(precision="mixed")
    w0 = inputs.bl_state(case, seed=3)
    cfg, _ = oracle_cfg(case)
    wo, _, _ = O.advance(cfg, w0, 10, cfl=case.cfl)
    s = binding.Solver(case, inflow=inputs.df_profiles(case))
    w = torch.from_numpy(w0).cuda()
    r_old = torch.zeros_like(w)
    s.advance_n(w, r_old, 10, cfl=case.cfl)
    wg = w.cpu().numpy()
    s.close()
    err = rel_l2(wg, wo)
    assert np.isfinite(wg).all() and max(err[0], err[1], err[4]) <= 1e-4, err


def test_inflow_argument_errors():
    case = DF_BL
    s = binding.Solver(case.replace(bc_xmin="char"))
    L = binding.lib()
    df = binding.DF(case.ref[4], 0, 2, 0.5, 1)  # zero filter width
    assert L.strm_inflow_df_bytes(s.ctx, df) == 0
    prof = inputs.df_profiles(case)
    with pytest.raises(binding.StrmError):
        bad = prof.copy()
        bad[3, 5] = -1.0  # negative normal stress
        s.set_inflow_df(bad)
    assert L.strm_set_bc(s.ctx, binding.FACES["xmin"], binding.BC_KINDS["df"], None, 0) == -1
    s.close()
    with pytest.raises(ValueError):
        binding.Solver(case)  # profiles missing
