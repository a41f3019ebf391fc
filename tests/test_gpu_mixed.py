"""Mixed precision (FP32 flux, sensor, WENO and viscous arithmetic; FP64 state, projection into
characteristic variables, RK accumulation and reductions) against the FP64 oracle.

The stated error of the variant: with a continuous flux (central everywhere, or WENO everywhere)
the relative L2 error per conserved field after 100 RK3 steps of the 64x48x32 channel is <= 1e-5.
With the Ducros switch, FP32 rounding (~1e-7 after one step) eventually flips the central/WENO
choice at faces whose sensor value sits at the threshold, which the grid-scale noise of this
initial state makes common; each flip changes that face's flux by O(noise) and the difference
spreads. Those runs are checked for the error before the first flips, for exact conservation,
and the error reached after 100 steps is bounded and reported.
"""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2004_02276_gb300 import binding, inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__

    __graft_entry__.build()
    torch.cuda.set_device(0)


def rel_l2(a, b):
    return np.array([np.linalg.norm(a[m] - b[m]) / np.linalg.norm(b[m]) for m in range(5)])


def profiles(w):
    """Mean streamwise velocity and Reynolds stresses <u'u'>, <v'v'>, <w'w'>, <u'v'> over x, z."""
    rho = w[0]
    u, v, ww = w[1] / rho, w[2] / rho, w[3] / rho
    um, vm, wm = (a.mean(axis=(0, 2), keepdims=True) for a in (u, v, ww))
    up, vp, wp = u - um, v - vm, ww - wm
    return np.stack([um[0, :, 0], (up * up).mean(axis=(0, 2)), (vp * vp).mean(axis=(0, 2)),
                     (wp * wp).mean(axis=(0, 2)), (up * vp).mean(axis=(0, 2))])


def test_mixed_rhs_close_to_oracle():
    case = inputs.C1.replace(precision="mixed")
    w0 = inputs.channel_state(case, seed=0)
    ref = O.rhs(O.make_cfg(case), w0)
    s = binding.Solver(case)
    r = s.compute_rhs(torch.from_numpy(w0).cuda()).cpu().numpy()
    s.close()
    err = rel_l2(r, ref)
    assert err.max() < 1e-4, err


@pytest.mark.parametrize("name", ["paper-settings", "weno-all-L2"])
def test_mixed_l2_close_to_oracle(name):
    """Mixed precision with the 4th-order central scheme (L = 2: the paper's own settings with
    Sutherland's law and the erf map, and WENO at every face), which exercises the L = 2 deviation
    form of the x faces and the offset of the x WENO faces: the right-hand side within 1e-4 of
    the FP64 oracle, and within 1e-5 per field (relative L2) after 10 steps with WENO at every
    face (a continuous flux) and after 1 step under the switch (before any decision flips)."""
    base = inputs.PAPER_CHANNEL if name == "paper-settings" else inputs.C1.replace(L=2, weno_mode="all")
    case = base.replace(precision="mixed")
    w0 = inputs.channel_state(case, seed=0)
    ref = O.rhs(O.make_cfg(case), w0)
    s = binding.Solver(case)
    r = s.compute_rhs(torch.from_numpy(w0).cuda()).cpu().numpy()
    s.close()
    assert rel_l2(r, ref).max() < 1e-4, rel_l2(r, ref)
    nsteps = 10 if case.weno_mode == "all" else 1
    wm, wo, t, to = run_both(case, nsteps)
    err = rel_l2(wm, wo)
    print(name, f"mixed L = 2, relative L2 after {nsteps} steps:", err)
    assert err.max() <= 1e-5, err
    assert abs(t - to) <= 1e-6 * to


def run_both(case, nsteps):
    w0 = inputs.channel_state(case, seed=0)
    wo, to, _ = O.advance(O.make_cfg(case), w0, nsteps, cfl=case.cfl)
    s = binding.Solver(case)
    w = torch.from_numpy(w0).cuda()
    r_old = torch.zeros_like(w)
    s.advance_n(w, r_old, nsteps, cfl=case.cfl)
    t, _ = s.time()
    wm = w.cpu().numpy()
    s.close()
    return wm, wo, t, to


@pytest.mark.parametrize("mode", ["off", "all"])
def test_mixed_hundred_steps_continuous_flux(mode):
    case = inputs.C1.replace(precision="mixed", weno_mode=mode)
    wm, wo, t, to = run_both(case, 100)
    err = rel_l2(wm, wo)
    assert err.max() <= 1e-5, err
    assert abs(t - to) <= 1e-6 * to
    pm, po = profiles(wm), profiles(wo)
    perr = np.abs(pm - po).max(axis=1) / np.maximum(np.abs(po).max(axis=1), 1e-12)
    assert perr.max() <= 1e-4, perr


def test_mixed_sensor_switch():
    case = inputs.C1.replace(precision="mixed")
    wm, wo, _, _ = run_both(case, 1)
    assert rel_l2(wm, wo).max() <= 1e-6  # before any switch flip: FP32 rounding only
    wm, wo, t, to = run_both(case, 100)
    err = rel_l2(wm, wo)
    # the dense fields keep a small error; the velocity-noise fields (|rho v|, |rho w| ~ 0.01)
    # carry the local differences of the flipped faces
    assert max(err[0], err[1], err[4]) <= 2e-4, err
    assert max(err[2], err[3]) <= 2e-2, err
    print("mixed sensor-mode relative L2 error after 100 steps:", err)
    # the domain totals (metric-weighted sums) see only what crosses the walls and the forcing:
    # mass and bulk momentum are held exactly, total energy differs by the wall heat flux and
    # forcing work of the two runs, transverse momentum stays at rounding level of |rho u|
    cfg = O.make_cfg(case)
    tm, to_ = np.array(O.totals(cfg, wm)), np.array(O.totals(cfg, wo))
    terr = np.abs(tm - to_) / np.array([to_[0], to_[1], to_[1], to_[1], to_[4]])
    print("mixed sensor-mode conserved-total error after 100 steps:", terr)
    assert terr.max() <= 1e-5, terr
    # mean-velocity and Reynolds-stress profiles (x-z averages), relative to each profile's peak
    pm, po = profiles(wm), profiles(wo)
    perr = np.abs(pm - po).max(axis=1) / np.maximum(np.abs(po).max(axis=1), 1e-12)
    print("mixed sensor-mode profile error after 100 steps (U, u'u', v'v', w'w', u'v'):", perr)
    assert perr[0] <= 1e-5 and perr[1:].max() <= 5e-3, perr


def test_mixed_conserves_mass_and_bulk_flow():
    """Conservation does not depend on the arithmetic precision of the fluxes (telescoping and
    the staggered wall), and the forcing is reduced in FP64."""
    case = inputs.Case(nx=48, ny=32, nz=24, precision="mixed")
    s = binding.Solver(case)
    w = torch.from_numpy(inputs.channel_state(case, seed=2)).cuda()
    t0 = np.array(s.totals(w))
    r_old = torch.zeros_like(w)
    s.advance_n(w, r_old, 10, cfl=0.8)
    t1 = np.array(s.totals(w))
    s.close()
    assert abs(t1[0] - t0[0]) <= 1e-12 * t0[0]
    assert abs(t1[1] - t0[1]) <= 1e-12 * t0[1]


def theta_of_initial_state(case):
    """The FP64 Ducros sensor of the seeded initial state (from the oracle)."""
    w0 = inputs.channel_state(case, seed=0)
    th, _, _, _, _ = O.sensor(O.make_cfg(case.replace(precision="fp64")), w0)
    return w0, th


def run_prescribed(case, w0, th, nsteps):
    s = binding.Solver(case)
    th_d = torch.from_numpy(th).cuda()
    s.set_theta(th_d)
    w = torch.from_numpy(w0).cuda()
    s.advance_n(w, torch.zeros_like(w), nsteps, cfl=case.cfl)
    t, _ = s.time()
    out = w.cpu().numpy()
    s.close()
    return out, t


def test_prescribed_switch_fp64_matches_oracle():
    """FP64 with the switch reading a prescribed sensor field: the CUDA path and the oracle take
    the same decisions by construction; 20 steps agree within relative L2 1e-12 per field."""
    case = inputs.C1
    w0, th = theta_of_initial_state(case)
    wo, to, _ = O.advance(O.make_cfg(case, theta_fixed=th), w0, 20, cfl=case.cfl)
    wg, t = run_prescribed(case, w0, th, 20)
    err = rel_l2(wg, wo)
    assert err.max() <= 1e-12, err
    assert abs(t - to) <= 1e-13 * to


def test_mixed_hundred_steps_with_equal_decisions():
    """The mixed path's own arithmetic error under the switch. Both runs take the central/WENO
    decisions of the FP64 run: before each RK3 step the FP64 oracle's Ducros sensor of its
    current state is prescribed to the oracle and to the mixed-precision path for that step (the
    switch of the 64x48x32 channel goes from 98 % WENO faces to about 7 % over the 100 steps).
    After 100 steps the relative L2 error of every conserved field is within the 1e-5 target
    (measured 4.6e-8 rho, 6.9e-8 rho u, 3.8e-6 rho v, 2.4e-6 rho w, 5.3e-8 rho E). The
    transverse momenta are noise fields whose rms has decayed to 0.45 % and 0.56 % of rms(rho u),
    so their relative error is the dense fields' error seen against a small norm; it met the
    target once the x faces' central flux took the deviation form (it was 1.15e-5 in rho v with
    the flux formed from the FP32 values). The mean-velocity and Reynolds-stress profiles agree
    to 1e-5 of their peaks. What the free-running sensor mode adds beyond this is the effect of
    decisions that flip at the threshold."""
    case = inputs.C1.replace(precision="mixed")
    cfg64 = O.make_cfg(case.replace(precision="fp64"))
    w0 = inputs.channel_state(case, seed=0)
    s = binding.Solver(case)
    th_d = torch.empty((case.nz, case.ny, case.nx), dtype=torch.float64, device="cuda")
    s.set_theta(th_d)
    wm_d = torch.from_numpy(w0).cuda()
    r_old = torch.zeros_like(wm_d)
    wo, to, fracs = w0, 0.0, []
    for _ in range(100):
        th, _, fx, fy, fz = O.sensor(cfg64, wo)
        fracs.append(np.mean(np.concatenate([f.ravel() for f in (fx, fy, fz)])))
        th_d.copy_(torch.from_numpy(th))
        s.advance_n(wm_d, r_old, 1, cfl=case.cfl)
        wo, dt = O.rk_step(O.make_cfg(case, theta_fixed=th), wo, cfl=case.cfl)
        to += dt
    t, _ = s.time()
    wm = wm_d.cpu().numpy()
    s.close()
    assert fracs[0] > 0.9 and fracs[-1] < 0.2, (fracs[0], fracs[-1])  # a genuine mix over the run
    err = rel_l2(wm, wo)
    print("mixed, decisions of the FP64 run, relative L2 per field after 100 steps:", err)
    assert max(err[0], err[1], err[4]) <= 1e-6, err
    assert max(err[2], err[3]) <= 1e-5, err  # the target, for every field
    # absolute error of the transverse momenta against the momentum scale
    scale = np.linalg.norm(wo[1])
    for m in (2, 3):
        assert np.linalg.norm(wm[m] - wo[m]) <= 1e-7 * scale, (m, np.linalg.norm(wm[m] - wo[m]) / scale)
    assert abs(t - to) <= 1e-6 * to
    pm, po = profiles(wm), profiles(wo)
    perr = np.abs(pm - po).max(axis=1) / np.maximum(np.abs(po).max(axis=1), 1e-12)
    print("profile error (U, u'u', v'v', w'w', u'v'):", perr)
    assert perr.max() <= 1e-5, perr


def test_set_theta_rejected_outside_sensor_mode():
    s = binding.Solver(inputs.Case(nx=8, ny=6, nz=4, weno_mode="all"))
    th = torch.zeros((4, 6, 8), dtype=torch.float64, device="cuda")
    with pytest.raises(binding.StrmError):
        s.set_theta(th)
    s.close()
