"""Boundary-layer and shock/boundary-layer workloads on the GPU against the FP64 oracle:
recycling inflow, characteristic outflow and top, isothermal wall on a one-sided tanh grid,
and the oblique shock imposed at the top (Sections 3.2, 3.3)."""
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


BL = inputs.bl_case("bl-48x40x12", 48, 40, 12, 7.0, 6.0, 1.5)
SBLI = inputs.bl_case("sbli-64x40x12", 64, 40, 12, 12.0, 6.0, 1.5, shock=True, noise=0.003)
OPEN = inputs.bl_case("open-40x24x10", 40, 24, 10, 6.0, 6.0, 1.5, bc_xmin="char", bc_ymin="char",
                      weno_mode="all")
# the paper's boundary-layer clustering (hyperbolic sine, Section 3.2)
BL_SINH = inputs.bl_case("bl-sinh-48x40x12", 48, 40, 12, 7.0, 6.0, 1.5, y_map="sinh1", beta=4.0)


@pytest.mark.parametrize("case", [BL, SBLI, OPEN, BL_SINH], ids=lambda c: c.name)
def test_rhs_and_flags_match_oracle(case):
    w0 = inputs.bl_state(case, seed=4)
    cfg = O.make_cfg(case)
    ref = O.rhs(cfg, w0)
    _, _, fx_o, fy_o, fz_o = O.sensor(cfg, w0)
    s = binding.Solver(case)
    w = torch.from_numpy(w0).cuda()
    r = s.compute_rhs(w).cpu().numpy()
    _, _, fx, fy, fz = (t.cpu().numpy() for t in s.sensor(w))
    s.close()
    assert np.array_equal(fx, fx_o) and np.array_equal(fy, fy_o) and np.array_equal(fz, fz_o)
    err = rel_max(r, ref)
    assert err.max() <= TOL, err


@pytest.mark.parametrize("case", [BL, SBLI, BL_SINH], ids=lambda c: c.name)
def test_ten_steps_match_oracle(case):
    w0 = inputs.bl_state(case, seed=5)
    wo, to, _ = O.advance(O.make_cfg(case), w0, 10, cfl=case.cfl)
    s = binding.Solver(case)
    w = torch.from_numpy(w0).cuda()
    r_old = torch.zeros_like(w)
    s.advance_n(w, r_old, 10, cfl=case.cfl)
    t, _ = s.time()
    wg = w.cpu().numpy()
    s.close()
    err = rel_l2(wg, wo)
    assert err.max() <= TOL, err
    assert abs(t - to) <= 1e-13 * to


def test_mixed_precision_boundary_layer():
    case = SBLI.replace(precision="mixed")
    w0 = inputs.bl_state(case, seed=5)
    wo, _, _ = O.advance(O.make_cfg(case), w0, 10, cfl=case.cfl)
    s = binding.Solver(case)
    w = torch.from_numpy(w0).cuda()
    r_old = torch.zeros_like(w)
    s.advance_n(w, r_old, 10, cfl=case.cfl)
    wg = w.cpu().numpy()
    s.close()
    err = rel_l2(wg, wo)
    assert np.isfinite(wg).all()
    assert max(err[0], err[1], err[4]) <= 1e-4, err
    print("mixed SBLI relative L2 error after 10 steps:", err)


@pytest.mark.slow
def test_c3_full_size_rhs_matches_oracle():
    """The 1024x256x256 boundary layer: the full right-hand side, every element, and five GPU
    steps that stay finite."""
    case = inputs.C3
    w0 = inputs.bl_state(case, seed=0)
    s = binding.Solver(case)
    w = torch.from_numpy(w0).cuda()
    r = s.compute_rhs(w).cpu().numpy()
    ref = O.rhs(O.make_cfg(case), w0)
    err = rel_max(r, ref)
    del ref, r
    assert err.max() <= TOL, err
    r_old = torch.zeros_like(w)
    s.advance_n(w, r_old, 5, cfl=case.cfl)
    assert torch.isfinite(w).all()
    s.close()


@pytest.mark.slow
def test_c4_full_size_steps():
    """The 2048x384x256 shock/boundary-layer interaction on the GPU: the right-hand side at
    sampled wall-normal columns against the oracle, then finite after 5 steps with the shock
    entering through the top, WENO on a minority of the faces.

    The oracle cannot take the whole 201 M-point grid, but the right-hand side at a node depends
    only on the state within 6 nodes of it (WENO and central stencils of 3, the sensor window of
    the face flags and the ghost-filled divergence of the viscous terms, 3 more). So each sample
    column (i0, k0) is checked on a 24 x 384 x 24 block of the state around it, periodic in x and
    z, with the full wall-normal extent, metrics and wall: at its centre column the oracle's
    right-hand side equals the full grid's for every j at least 8 nodes below the top face
    (whose shock ghosts depend on x).

    The top rows, with the shock entering through the top boundary, are checked on a second
    block: the whole x extent and wall-normal extent with 24 planes around k0 = 128, periodic in
    z only, so that the inflow, outflow and shock ghosts see their own x positions. Its plane
    k0 equals the full grid's right-hand side at every node from i = 8 on (the recycled inflow
    ghosts take spanwise means over the block's 24 planes instead of 256, which reaches the
    first 6 nodes)."""
    case = inputs.C4
    w0 = inputs.bl_state(case, seed=0)
    s = binding.Solver(case)
    w = torch.from_numpy(w0).cuda()
    r = s.compute_rhs(w)
    h = 12
    dx, dz = case.lx / case.nx, case.lz / case.nz
    sub = case.replace(name="c4-block", nx=2 * h, nz=2 * h, lx=2 * h * dx, lz=2 * h * dz,
                       bc_xmin="periodic", bc_xmax="periodic", shock=False, shock_theta=0.0)
    cfg = O.make_cfg(sub)
    jmax = case.ny - 8
    cols = ((300, 40), (1229, 128), (1700, 200), (2000, 100))
    refs = {}
    for i0, k0 in cols:
        blk = np.ascontiguousarray(w0[:, k0 - h:k0 + h, :, i0 - h:i0 + h])
        refs[i0, k0] = O.rhs(cfg, blk)[:, h, :jmax, h]
        got = r[:, k0, :jmax, i0].cpu().numpy()
        err = rel_max(got, refs[i0, k0])
        assert err.max() <= TOL, ((i0, k0), err)
    kp, i_min = 128, 8
    plane = case.replace(name="c4-plane", nz=2 * h, lz=2 * h * dz)
    blk = np.ascontiguousarray(w0[:, kp - h:kp + h])
    ref_plane = O.rhs(O.make_cfg(plane), blk)[:, h, :, i_min:]
    del blk
    got = r[:, kp, :, i_min:].cpu().numpy()
    err = rel_max(got, ref_plane)
    print("C4 RHS error on the plane k = 128 (all j, i >= 8):", err)
    assert err.max() <= TOL, err
    # the rows next to the top boundary on their own (shock-top and characteristic ghosts)
    err_top = rel_max(got[:, -8:], ref_plane[:, -8:])
    assert err_top.max() <= TOL, err_top
    # the mixed-precision path at full size on the same columns: FP32 flux arithmetic, whose
    # rounding (~6e-8 of a flux) is amplified by the flux differences of the small wall-normal
    # and spanwise residuals (measured up to 1.2e-4 of the column's largest |R_rho v|)
    del r
    sm = binding.Solver(case.replace(precision="mixed"))
    rm = sm.compute_rhs(w)
    for i0, k0 in cols:
        err = rel_max(rm[:, k0, :jmax, i0].cpu().numpy(), refs[i0, k0])
        print("C4 mixed-precision RHS error at column", (i0, k0), err)
        assert err.max() <= 1e-3, ((i0, k0), err)
    err = rel_max(rm[:, kp, :, i_min:].cpu().numpy(), ref_plane)
    print("C4 mixed-precision RHS error on the plane k = 128:", err)
    assert err.max() <= 1e-3, err
    del ref_plane
    sm.close()
    del rm
    r_old = torch.zeros_like(w)
    s.advance_n(w, r_old, 5, cfl=case.cfl)
    s.compute_rhs(w)
    counts = s.weno_counts()
    frac = sum(counts) / (3.0 * case.npts)
    print("C4 WENO face fraction after 5 steps:", frac)
    assert torch.isfinite(w).all()
    assert 0.0 < frac < 0.5
    s.close()


# weak perturbations: 90 % of the y faces and 97 % of the z faces are central, so the y and z
# central fluxes come from the sweeps (chosen from 85 % in FP64, 50 % in mixed precision)
SWEEP = inputs.bl_case("sbli-64x40x24", 64, 40, 24, 12.0, 6.0, 3.0, shock=True, noise=0.001)


def test_central_sweeps_match_oracle():
    """The y/z central-flux sweeps (pair reuse along a column, every face written, the WENO
    faces overwritten afterwards) in sensor mode: the right-hand side element-wise within 1e-12
    of the oracle's, flags bit-equal, 10 CFL steps within relative L2 1e-12; the mixed right-hand
    side within 1e-4 of each field's largest value."""
    w0 = inputs.bl_state(SWEEP, seed=6)
    cfg = O.make_cfg(SWEEP)
    ref = O.rhs(cfg, w0)
    _, _, fx_o, fy_o, fz_o = O.sensor(cfg, w0)
    nf = [fx_o.size, fy_o.size, fz_o.size]
    s = binding.Solver(SWEEP)
    w = torch.from_numpy(w0).cuda()
    r = s.compute_rhs(w).cpu().numpy()
    counts = s.weno_counts()
    _, _, fx, fy, fz = (t.cpu().numpy() for t in s.sensor(w))
    assert all(1 - counts[dd] / nf[dd] >= 0.85 for dd in (1, 2)), counts  # the sweeps ran
    assert np.array_equal(fx, fx_o) and np.array_equal(fy, fy_o) and np.array_equal(fz, fz_o)
    err = rel_max(r, ref)
    assert err.max() <= TOL, err
    wo, to, _ = O.advance(cfg, w0, 10, cfl=SWEEP.cfl)
    r_old = torch.zeros_like(w)
    s.advance_n(w, r_old, 10, cfl=SWEEP.cfl)
    t, _ = s.time()
    wg = w.cpu().numpy()
    s.close()
    assert rel_l2(wg, wo).max() <= TOL
    assert abs(t - to) <= 1e-13 * to
    sm = binding.Solver(SWEEP.replace(precision="mixed"))
    rm = sm.compute_rhs(torch.from_numpy(w0).cuda()).cpu().numpy()
    sm.close()
    assert rel_max(rm, ref).max() <= 1e-4
