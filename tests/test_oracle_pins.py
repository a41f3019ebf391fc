"""Pins of the FP64 oracle against what the paper and the mathematics fix (no GPU).

Each test checks the oracle against something other than itself: closed forms, invariants the
method is designed to keep (Section 2.1: telescoping conservative fluxes, kinetic-energy
preservation of the split central flux, exact mass conservation with the staggered wall),
textbook reductions, exact solutions (isentropic vortex, Sod shock tube, manufactured
solutions by symbolic calculus) and the order of accuracy the paper states.
"""
import math
import os

import numpy as np
import pytest

import mms
import riemann
from paper_2004_02276_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def periodic_case(**kw):
    base = dict(nx=12, ny=10, nz=8, beta=1.5, y_wall=False, forcing=False)
    base.update(kw)
    return inputs.Case(**base)


def volumes(O, cfg, case):
    _, ye, _ = O.metrics(cfg)
    return (case.lx / case.nx) * (case.lz / case.nz) * (ye / case.ny)[None, :, None]


def central_coeffs_from_taylor(L):
    """First- and second-derivative central coefficients of order 2L from the Taylor
    conditions (independent of the oracle's tables)."""
    ls = np.arange(1, L + 1, dtype=float)
    A = np.array([2.0 * ls ** p for p in range(1, 2 * L, 2)])
    rhs = np.zeros(L)
    rhs[0] = 1.0
    a = np.linalg.solve(A, rhs)
    B = np.array([ls ** p for p in range(2, 2 * L + 1, 2)])
    b = np.linalg.solve(B, rhs)
    return a, b


def d1_periodic(f, a, h, axis):
    out = np.zeros_like(f)
    for l, al in enumerate(a, start=1):
        out += al * (np.roll(f, -l, axis=axis) - np.roll(f, l, axis=axis))
    return out / h


# ----------------------------------------------------------------------- grid metrics

def test_metrics_tanh_consistent(orc):
    c = inputs.Case(ny=400)
    cfg = orc.make_cfg(c)
    y, ye, yee = orc.metrics(cfg)
    assert np.all(np.diff(y) > 0)
    np.testing.assert_allclose(y, -y[::-1], atol=1e-15)
    assert -1.0 < y[0] < y[-1] < 1.0
    deta = 1.0 / c.ny
    # y_eta and y_etaeta agree with centred differences of the oracle's own node values
    np.testing.assert_allclose((y[2:] - y[:-2]) / (2 * deta), ye[1:-1], rtol=2e-4)
    np.testing.assert_allclose((ye[2:] - ye[:-2]) / (2 * deta), yee[1:-1], rtol=2e-3, atol=1e-3)
    # the node volumes tile the channel (midpoint rule in eta)
    assert abs(ye.sum() * deta - c.ly) < 1e-4


# ----------------------------------------------------------------------- free stream

@pytest.mark.parametrize("mode", ["off", "sensor", "all"])
@pytest.mark.parametrize("L", [2, 3])
def test_freestream_preservation_bitwise(orc, mode, L):
    """A uniform state has R = 0 exactly: every interface sees the same stencil values."""
    c = periodic_case(weno_mode=mode, L=L, viscous=True, forcing=True)
    w = inputs.primitive_state(c, 1.2, 0.3, -0.2, 0.1, 1.1)
    r = orc.rhs(orc.make_cfg(c), w)
    assert np.all(r == 0.0)


# ----------------------------------------------------------------------- conservation

@pytest.mark.parametrize("mode", ["off", "sensor", "all"])
def test_telescoping_conservation_periodic(orc, mode):
    """Locally conservative fluxes (Eq. num_flux): in a periodic box the volume integral of
    every convective residual vanishes to round-off, with any mix of central/WENO faces."""
    c = periodic_case(weno_mode=mode, viscous=False, theta_thr=0.6)
    cfg = orc.make_cfg(c)
    w = inputs.random_state(c, seed=3)
    r = orc.rhs(cfg, w)
    vol = volumes(orc, cfg, c)
    if mode == "sensor":
        _, _, fx, fy, fz = orc.sensor(cfg, w)
        frac = np.mean(np.concatenate([fx.ravel(), fy.ravel(), fz.ravel()]))
        assert 0.05 < frac < 0.95  # a genuine mix of both fluxes
    for m in range(5):
        s = (r[m] * vol).sum()
        scale = np.abs(r[m] * vol).sum()
        assert abs(s) <= 1e-14 * scale, (m, s, scale)


def test_viscous_mass_exact_momentum_not(orc):
    """With viscous terms on, mass stays exactly conserved (no viscous mass flux); momentum is
    not telescoping in the Laplacian form, but only at truncation level."""
    c = periodic_case(weno_mode="off", viscous=True, reynolds=50.0)
    cfg = orc.make_cfg(c)
    w = inputs.random_state(c, seed=4)
    r = orc.rhs(cfg, w)
    vol = volumes(orc, cfg, c)
    assert abs((r[0] * vol).sum()) <= 1e-14 * np.abs(r[0] * vol).sum()


def test_kinetic_energy_preservation(orc):
    """Energy-consistent split flux (Eqs. avg_operator, encflux): in a periodic inviscid box
    with uniform pressure the convective terms neither create nor destroy kinetic energy,
    sum_V (u . R_mom - |u|^2/2 R_rho) = 0 to round-off (Section 2.1)."""
    c = periodic_case(weno_mode="off", viscous=False)
    cfg = orc.make_cfg(c)
    s = 2.0 * inputs.uniform(11, (4, c.nz, c.ny, c.nx)) - 1.0
    rho = 1.0 + 0.3 * s[0]
    u, v, w = 0.5 * s[1], 0.5 * s[2], 0.5 * s[3]
    p = 0.7
    st = inputs.primitive_state(c, rho, u, v, w, p / (rho * c.r_gas))
    r = orc.rhs(cfg, st)
    vol = volumes(orc, cfg, c)
    ke = (u * r[1] + v * r[2] + w * r[3] - 0.5 * (u * u + v * v + w * w) * r[0]) * vol
    assert abs(ke.sum()) <= 1e-14 * np.abs(ke).sum()
    # the same state with WENO everywhere is dissipative: the identity is specific to the split flux
    r2 = orc.rhs(orc.make_cfg(c, weno_mode="all"), st)
    ke2 = (u * r2[1] + v * r2[2] + w * r2[3] - 0.5 * (u * u + v * v + w * w) * r2[0]) * vol
    assert ke2.sum() < -1e-6 * np.abs(ke2).sum()


def test_channel_mass_and_bulk_flow_constant(orc):
    """Staggered walls (zero convective mass flux through the wall) keep the total mass exact,
    and the forcing keeps the bulk x-momentum constant (Section 3.1: both exactly constant)."""
    c = inputs.Case(nx=16, ny=24, nz=8, reynolds=3000.0)
    cfg = orc.make_cfg(c)
    w = inputs.channel_state(c, seed=1)
    t0 = orc.totals(cfg, w)
    for _ in range(4):
        w, _ = orc.rk_step(cfg, w, cfl=c.cfl)
    t1 = orc.totals(cfg, w)
    assert abs(t1[0] - t0[0]) <= 1e-14 * abs(t0[0]) * 10
    assert abs(t1[1] - t0[1]) <= 1e-14 * abs(t0[1]) * 10
    # without forcing the walls decelerate the flow
    cfg_nf = orc.make_cfg(c, forcing=False)
    w2 = inputs.channel_state(c, seed=1)
    for _ in range(4):
        w2, _ = orc.rk_step(cfg_nf, w2, cfl=c.cfl)
    assert orc.totals(cfg_nf, w2)[1] < t0[1] - 1e-6


@pytest.mark.parametrize("mode", ["off", "sensor", "all"])
def test_wall_faces_carry_no_mass_tangential_momentum_or_energy(orc, mode):
    """Staggered isothermal walls (Section 3.1: the walls lie on interfaces, and no convective
    mass, tangential momentum or energy crosses them). Inviscid, unforced, periodic in x and z,
    random interior state: the x and z faces telescope, so sum_V R_m is the net flux through
    the two wall faces. It vanishes to round-off for rho, rho u, rho w and rho E; the wall-normal
    momentum keeps the pressure acting on the walls, so sum_V R_rhov does not."""
    c = inputs.Case(nx=12, ny=14, nz=10, forcing=False, viscous=False, weno_mode=mode,
                    theta_thr=0.6)
    cfg = orc.make_cfg(c)
    w = inputs.random_state(c, seed=5)
    r = orc.rhs(cfg, w)
    vol = volumes(orc, cfg, c)
    if mode == "sensor":
        _, _, _, fy, _ = orc.sensor(cfg, w)
        frac = fy.mean()
        assert 0.05 < frac < 0.95  # walls see both central and WENO faces
    for m in (0, 1, 3, 4):
        s = (r[m] * vol).sum()
        scale = np.abs(r[m] * vol).sum()
        assert abs(s) <= 1e-14 * scale, (m, s, scale)
    # rho v: the wall pressure. With the mirrored ghost (p_g = p) the central pressure flux at
    # a wall face is a positive combination of near-wall pressures, so the net force is O(p).
    s_v = (r[2] * vol).sum()
    assert abs(s_v) > 1e-3 * np.abs(r[2] * vol).sum()


@pytest.mark.parametrize("mode", ["off", "sensor"])
def test_forcing_adds_f_and_f_u(orc, mode):
    """Constant-mass-flow forcing (Eqs. 1b, 1c): f is the uniform x-momentum source that makes
    the volume integral of R_rhou vanish, and the energy equation gains the power f u.
    Comparing the right-hand sides with forcing on and off on the same state: R_rhou changes by
    f = -sum_V R_rhou(off) / V at every node, R_rhoE by f u (u = rho u / rho of that node), and
    rho, rho v, rho w are unchanged. (Viscous: without wall shear nothing decelerates the flow
    and f would vanish, as the wall-face pin shows.)"""
    c = inputs.Case(nx=12, ny=14, nz=10, reynolds=500.0, weno_mode=mode)
    # Poiseuille flow with density and temperature varying by +-20 % (so that u, rho u and
    # rho differ node by node)
    s = 2.0 * inputs.uniform(21, (2, c.nz, c.ny, c.nx)) - 1.0
    ch = inputs.channel_state(c, seed=2)
    u0, v0, w0 = ch[1], ch[2], ch[3]
    w = inputs.primitive_state(c, 1.0 + 0.2 * s[0], u0, v0, w0, 1.0 + 0.2 * s[1])
    on = orc.rhs(orc.make_cfg(c, forcing=True), w)
    off = orc.rhs(orc.make_cfg(c, forcing=False), w)
    cfg = orc.make_cfg(c)
    vol = np.broadcast_to(volumes(orc, cfg, c), w[0].shape)
    f = -(off[1] * vol).sum() / vol.sum()
    assert abs(f) > 1e-4  # the walls decelerate the unforced flow
    u = w[1] / w[0]
    for m in (0, 2, 3):
        assert np.array_equal(on[m], off[m])
    np.testing.assert_allclose(on[1] - off[1], f, rtol=1e-11, atol=0)
    ulp = 4 * np.finfo(float).eps * (np.abs(on[4]) + np.abs(off[4]))
    assert np.all(np.abs((on[4] - off[4]) - f * u) <= ulp + 1e-13 * abs(f))
    # the energy budget: the forcing's power integrates to f times the bulk velocity flux
    power = ((on[4] - off[4]) * vol).sum()
    assert abs(power - f * (u * vol).sum()) <= 1e-12 * abs(power)
    # and the forced x-momentum residual integrates to zero
    assert abs((on[1] * vol).sum()) <= 1e-13 * np.abs(on[1] * vol).sum()


# ----------------------------------------------------------------------- textbook reduction

@pytest.mark.parametrize("L", [2, 3])
def test_textbook_reduction_advection(orc, L):
    """Uniform velocity and pressure, varying density: the split flux reduces to the central
    derivative of order 2L, R_rho = -u0 D1(rho) and R_rhou = -u0^2 D1(rho) (the mass and
    momentum pair fluxes are linear in rho here), with coefficients from the Taylor
    conditions."""
    c = inputs.Case(nx=24, ny=4, nz=3, beta=0.0, y_wall=False, forcing=False, viscous=False,
                    weno_mode="off", L=L)
    cfg = orc.make_cfg(c)
    s = inputs.uniform(5, (c.nx,))
    rho1 = 1.0 + 0.3 * np.sin(2 * np.pi * np.arange(c.nx) / c.nx) + 0.1 * s
    rho = np.broadcast_to(rho1[None, None, :], (c.nz, c.ny, c.nx))
    u0, p0 = 0.7, 0.9
    w = inputs.primitive_state(c, rho, u0, 0.0, 0.0, p0 / (rho * c.r_gas))
    r = orc.rhs(cfg, w)
    a, _ = central_coeffs_from_taylor(L)
    d = d1_periodic(rho, a, c.lx / c.nx, axis=2)
    np.testing.assert_allclose(r[0], -u0 * d, atol=1e-13)
    np.testing.assert_allclose(r[1], -u0 * u0 * d, atol=1e-13)
    assert np.all(np.abs(r[2]) < 1e-14) and np.all(np.abs(r[3]) < 1e-14)


# ----------------------------------------------------------------------- design order

G_VORTEX = 1.4


def _vortex(X, Y, U=1.0, eps=5.0, g=G_VORTEX):
    """Isentropic vortex (Shu) in a uniform stream U, R = 1: an exact translating solution."""
    r2 = X * X + Y * Y
    f = np.exp(0.5 * (1 - r2))
    u = U - eps / (2 * np.pi) * Y * f
    v = eps / (2 * np.pi) * X * f
    T = 1 - (g - 1) * eps ** 2 / (8 * g * np.pi ** 2) * np.exp(1 - r2)
    rho = T ** (1 / (g - 1))
    p = rho * T
    return np.array([rho, rho * u, rho * v, 0 * rho, p / (g - 1) + 0.5 * rho * (u * u + v * v)])


def _vortex_rhs_error(orc, n, mode, L):
    c = inputs.Case(nx=n, ny=n, nz=1, lx=20.0, ly=20.0, lz=1.0, beta=0.0, y_wall=False,
                    forcing=False, viscous=False, weno_mode=mode, L=L, gamma=G_VORTEX)
    d = 20.0 / n
    xc = -10 + (np.arange(n) + 0.5) * d
    X, Y = np.meshgrid(xc, xc, indexing="xy")
    w = _vortex(X, Y)[:, None]
    h = 1e-30
    exact = -(_vortex(X + 1j * h, Y).imag / h)[:, None]  # R = -U dw/dx, complex step
    r = orc.rhs(orc.make_cfg(c, r_gas=1.0), w)
    return np.abs(r - exact).max() / np.abs(exact).max()


@pytest.mark.parametrize("mode,L,sizes,order", [
    ("off", 3, (64, 128), 5.0),
    ("off", 2, (64, 128), 3.5),
    ("all", 3, (256, 512), 4.5),
])
def test_design_order_isentropic_vortex(orc, mode, L, sizes, order):
    """Central flux of order 2L (Section 2.1) and WENO5 on a smooth exact Euler solution."""
    e = [_vortex_rhs_error(orc, n, mode, L) for n in sizes]
    assert math.log2(e[0] / e[1]) >= order, e


def test_time_order_rk3(orc):
    """Wray RK3 is third order in time: successive differences shrink by ~8 when dt halves."""
    n = 32
    c = inputs.Case(nx=n, ny=n, nz=1, lx=20.0, ly=20.0, lz=1.0, beta=0.0, y_wall=False,
                    forcing=False, viscous=False, weno_mode="off", L=3, gamma=G_VORTEX)
    cfg = orc.make_cfg(c, r_gas=1.0)
    xc = -10 + (np.arange(n) + 0.5) * (20.0 / n)
    X, Y = np.meshgrid(xc, xc, indexing="xy")
    w0 = _vortex(X, Y)[:, None]
    T = 0.8
    sols = []
    for nsteps in (8, 16, 32):
        w, _, _ = orc.advance(cfg, w0, nsteps, dt=T / nsteps)
        sols.append(w)
    d1 = np.abs(sols[0] - sols[1]).max()
    d2 = np.abs(sols[1] - sols[2]).max()
    assert 7.0 < d1 / d2 < 9.0, d1 / d2


# ----------------------------------------------------------------------- manufactured solutions

@pytest.mark.parametrize("conv,visc,L,law", [
    (False, True, 3, "power"),
    (False, True, 2, "power"),
    (False, True, 3, "sutherland"),
    (True, False, 3, "power"),
    (True, True, 3, "power"),
])
def test_manufactured_solution_order(orc, conv, visc, L, law):
    """Exact residual of the conservation form (Eqs. 1a-c, sigma_ij, q_j) by symbolic calculus
    on a tanh-stretched periodic grid: the Laplacian-form viscous terms and the split
    convective flux converge at order 2L. Nodes whose stencils reach across the periodic seam
    of the eta grid (where the tanh metric is not periodic-smooth) are excluded."""
    lx, lz, ly, beta = 2 * np.pi, np.pi, 2.0, 1.5
    c0 = inputs.Case(lx=lx, lz=lz, ly=ly, beta=beta, y_wall=False, forcing=False,
                     weno_mode="off", L=L, convective=conv, viscous=visc, reynolds=100.0,
                     visc_law=law)
    prims, exact_rhs = mms.build(lx, lz, ly, beta, c0.gamma, c0.r_gas, c0.mu_ref, c0.visc_exp,
                                 c0.prandtl, conv, visc, law, c0.suth_s)
    errs = []
    for n in (32, 64):
        c = c0.replace(nx=n, ny=n, nz=n // 2)
        X, E, Z = mms.grid(c.nx, c.ny, c.nz, lx, lz)
        rho, u, v, w, T = (np.broadcast_to(a, X.shape) for a in prims(X, E, Z))
        st = inputs.primitive_state(c, rho, u, v, w, T)
        rn = orc.rhs(orc.make_cfg(c), st)
        re = np.array([np.broadcast_to(a, X.shape) for a in exact_rhs(X, E, Z)])
        inner = slice(2 * L, c.ny - 2 * L)
        errs.append(max(np.abs(rn[m][:, inner] - re[m][:, inner]).max() / np.abs(re[m]).max()
                        for m in range(5) if np.abs(re[m]).max() > 0))
    assert math.log2(errs[0] / errs[1]) >= 2 * L - 0.7, errs
    assert errs[1] < 1e-5


# ----------------------------------------------------------------------- Sod shock tube

def _sod_l1(orc, n, mode="all", tend=0.2, cfl=0.5):
    g = 1.4
    c = inputs.Case(nx=n, ny=1, nz=1, lx=2.0, ly=1.0, lz=1.0, beta=0.0, y_wall=False,
                    forcing=False, viscous=False, weno_mode=mode, gamma=g, mach=1 / math.sqrt(g))
    cfg = orc.make_cfg(c)
    x = (np.arange(n) + 0.5) * 2.0 / n
    left = (x < 0.5) | (x > 1.5)
    rho = np.where(left, 1.0, 0.125)
    p = np.where(left, 1.0, 0.1)
    w = inputs.primitive_state(c, rho[None, None, :], 0.0, 0.0, 0.0, (p / rho)[None, None, :])
    t = 0.0
    while t < tend - 1e-14:
        dt = min(orc.cfl_dt(cfg, w, cfl), tend - t)
        w, _ = orc.rk_step(cfg, w, dt=dt)
        t += dt
    L_, R_ = (1.0, 0.0, 1.0), (0.125, 0.0, 0.1)
    # double tube: Sod at x = 0.5 and its mirror image at x = 1.5 (waves do not meet by t = 0.2)
    exact = np.where(x < 1.0, riemann.sample(L_, R_, (x - 0.5) / tend)[0],
                     riemann.sample(L_, R_, (1.5 - x) / tend)[0])
    return np.abs(w[0, 0, 0] - exact).mean() * 2.0, w


def test_exact_riemann_solver_matches_textbook():
    vals = np.loadtxt(os.path.join(GOLDEN, "sod_star_state.txt"))
    ps, us = riemann.star_state((1.0, 0.0, 1.0), (0.125, 0.0, 0.1))
    rl = riemann.sample((1.0, 0.0, 1.0), (0.125, 0.0, 0.1), np.array([us - 1e-9]))[0][0]
    rr = riemann.sample((1.0, 0.0, 1.0), (0.125, 0.0, 0.1), np.array([us + 1e-9]))[0][0]
    np.testing.assert_allclose([ps, us, rl, rr], vals, atol=6e-6)


@pytest.mark.slow
def test_sod_weno_converges_to_exact(orc):
    """Characteristic LF-WENO5 (Section 2.1) on the Sod problem: L1(rho) against the exact
    Riemann solution decreases at order >= 0.8 from 100 to 800 cells."""
    e = [_sod_l1(orc, n)[0] for n in (100, 800)]
    assert math.log2(e[0] / e[1]) / 3.0 >= 0.8, e
    assert e[1] < 5e-3


def test_sod_sensor_mode_bounded(orc):
    """Hybrid central/WENO with the Ducros switch stays non-oscillatory on Sod."""
    err, w = _sod_l1(orc, 200, mode="sensor")
    assert err < 2e-2
    assert w[0].max() < 1.0 + 2e-3 and w[0].min() > 0.125 - 2e-3


# ----------------------------------------------------------------------- time integration

def _rk_coeffs():
    rows = np.loadtxt(os.path.join(GOLDEN, "rk3_coefficients.txt"))
    return rows[:, 1] / rows[:, 2], rows[:, 3] / rows[:, 4]


def test_rk_coefficients_consistent():
    alpha, beta = _rk_coeffs()
    assert abs(alpha.sum() + beta.sum() - 1.0) < 1e-15
    # stage times 0, 8/15, 2/3
    c1 = beta[0]
    c2 = beta[0] + alpha[1] + beta[1]
    assert abs(c1 - 8 / 15) < 1e-15 and abs(c2 - 2 / 3) < 1e-15


def test_rk_linear_amplification(orc):
    """Through the oracle's stage update with R = lambda w: the amplification factor of a
    three-stage third-order scheme is 1 + z + z^2/2 + z^3/6."""
    for z in (-0.3, -1.0, 0.5 + 0.0):
        lam, dt = z, 1.0
        w = np.array([1.0])
        r_old = np.zeros(1)
        for stage in range(3):
            r = lam * w
            w = orc.rk_stage_update(stage, dt, w, r_old, r)
            r_old = r
        assert abs(w[0] - (1 + z + z * z / 2 + z ** 3 / 6)) < 1e-15


def test_rk_quadrature_exact_for_quadratic(orc):
    """R depending on time only, evaluated at the stage times (0, 8/15, 2/3) dt: a third-order
    scheme integrates 3 t^2 exactly."""
    dt = 0.7
    ct = [0.0, 8 / 15, 2 / 3]
    w = np.array([0.0])
    r_old = np.zeros(1)
    for stage in range(3):
        r = np.array([3.0 * (ct[stage] * dt) ** 2])
        w = orc.rk_stage_update(stage, dt, w, r_old, r)
        r_old = r
    assert abs(w[0] - dt ** 3) < 1e-15


# ----------------------------------------------------------------------- characteristic fields

def _euler_flux(wv, d, g):
    rho = wv[0]
    vel = wv[1:4] / rho
    p = (g - 1) * (wv[4] - 0.5 * rho * (vel * vel).sum())
    f = vel[d] * wv
    f[1 + d] = f[1 + d] + p
    f[4] = f[4] + p * vel[d]
    return f


@pytest.mark.parametrize("d", [0, 1, 2])
def test_eigenvectors_diagonalise_jacobian(orc, d):
    g = 1.4
    rng = inputs.uniform(7 + d, (4, 5))
    for s in rng:
        rho, u, v, w, p = 0.5 + s[0], s[1] - 0.5, s[2] - 0.5, s[3] - 0.5, 0.5 + s[4]
        H = g / (g - 1) * p / rho + 0.5 * (u * u + v * v + w * w)
        Lm, Rm = orc.eigvecs(d, g, u, v, w, H)
        np.testing.assert_allclose(Lm @ Rm, np.eye(5), atol=1e-13)
        wv = np.array([rho, rho * u, rho * v, rho * w, p / (g - 1) + 0.5 * rho * (u * u + v * v + w * w)])
        h = 1e-30
        A = np.empty((5, 5))
        for k in range(5):
            dw = wv.astype(complex)
            dw[k] += 1j * h
            A[:, k] = _euler_flux(dw, d, g).imag / h
        c = math.sqrt(g * p / rho)
        un = (u, v, w)[d]
        np.testing.assert_allclose(Lm @ A @ Rm, np.diag([un - c, un, un, un, un + c]), atol=1e-12)


def test_weno5_reconstruction(orc):
    # exact for quadratics: the interface value of the primitive-function reconstruction
    assert abs(orc.weno5([0.0, 0.0, 0.0, 0.0, 0.0]) - 0.0) == 0.0
    assert abs(orc.weno5([-2.0, -1.0, 0.0, 1.0, 2.0]) - 0.5) < 1e-15
    assert abs(orc.weno5([4.0, 1.0, 0.0, 1.0, 4.0]) - 1.0 / 6.0) < 1e-14
    # a jump between i and i+1: the smooth left stencil takes (almost) all the weight
    assert abs(orc.weno5([0.0, 0.0, 0.0, 1.0, 1.0])) < 1e-6
    assert abs(orc.weno5([1.0, 1.0, 1.0, 0.0, 0.0]) - 1.0) < 1e-6
    # fifth order on smooth data: flux difference of h(x) = sin with f = cell means of h
    errs = []
    for n in (40, 80):
        dx = 2 * np.pi / n
        xi = np.arange(n) * dx
        f = (np.cos(xi - dx / 2) - np.cos(xi + dx / 2)) / dx  # cell average of sin
        fh = np.array([orc.weno5([f[(i + q) % n] for q in range(-2, 3)]) for i in range(n)])
        errs.append(np.abs(fh - np.sin(xi + dx / 2)).max())
    assert math.log2(errs[0] / errs[1]) > 4.5, errs


# ----------------------------------------------------------------------- sensor

def test_sensor_zero_for_divergence_free(orc):
    """u independent of x, v of y, w of z: the discrete divergence is exactly zero, so
    theta = 0 (Eq. sensor) and no interface is flagged."""
    c = periodic_case(nx=16, ny=12, nz=10, weno_mode="sensor")
    nz, ny, nx = c.nz, c.ny, c.nx
    Y = (np.arange(ny) / ny)[None, :, None]
    Z = (np.arange(nz) / nz)[:, None, None]
    X = (np.arange(nx) / nx)[None, None, :]
    sh = (nz, ny, nx)
    u = np.broadcast_to(np.sin(2 * np.pi * Y) * np.cos(2 * np.pi * Z), sh)
    v = np.broadcast_to(np.cos(2 * np.pi * X + 2 * np.pi * Z), sh)
    w = np.broadcast_to(np.sin(2 * np.pi * X) * np.sin(2 * np.pi * Y), sh)
    st = inputs.primitive_state(c, 1.0, u, v, w, 1.0)
    th, dv, fx, fy, fz = orc.sensor(orc.make_cfg(c), st)
    assert np.all(dv == 0.0) and np.all(th == 0.0)
    assert not fx.any() and not fy.any() and not fz.any()


def test_sensor_closed_form_compression(orc):
    """1D velocity u(x): div = D1(u), curl = 0, theta = max(-div / sqrt(div^2 + (u0/L0)^2), 0),
    and the interface rule flags the faces whose node window holds theta > threshold."""
    L = 3
    c = inputs.Case(nx=32, ny=4, nz=3, beta=0.0, y_wall=False, forcing=False, L=L,
                    weno_mode="sensor", theta_thr=0.3, u0=0.5, l0=2.0)
    xs = np.arange(c.nx) * c.lx / c.nx
    u1 = 0.8 * np.sin(xs)
    st = inputs.primitive_state(c, 1.0, u1[None, None, :], 0.0, 0.0, 1.0)
    th, dv, fx, fy, fz = orc.sensor(orc.make_cfg(c), st)
    a, _ = central_coeffs_from_taylor(L)
    d = d1_periodic(u1, a, c.lx / c.nx, axis=0)
    expect = np.maximum(-d / np.sqrt(d * d + (c.u0 / c.l0) ** 2), 0.0)
    np.testing.assert_allclose(th[0, 0], expect, atol=1e-15)
    # face s sits between nodes s-1 and s; its window is nodes s-L .. s+L-1 (periodic)
    want = np.array([expect[[(s + q) % c.nx for q in range(-L, L)]].max() > c.theta_thr
                     for s in range(c.nx + 1)])
    assert np.array_equal(fx[0, 0].astype(bool), want)
    assert want.any() and not want.all()
    # theta is constant along y and z, so those faces are flagged where the column's theta is
    col = expect > c.theta_thr
    assert np.array_equal(fy.astype(bool), np.broadcast_to(col, fy.shape))
    assert np.array_equal(fz.astype(bool), np.broadcast_to(col, fz.shape))


# ----------------------------------------------------------------------- walls, CFL, totals

def test_wall_ghosts_mirror(orc):
    """Isothermal staggered wall: ghost velocity is mirrored with opposite sign, T_g = 2 T_w - T,
    p_g = p (Section 3.1); x and z ghosts are periodic copies; no corner is filled."""
    c = inputs.Case(nx=6, ny=8, nz=5, t_wall=1.3)
    cfg = orc.make_cfg(c)
    w = inputs.random_state(c, seed=9)
    G = orc.ghosts()
    wg = orc.fill_ghosts(cfg, w)
    cv = c.r_gas / (c.gamma - 1)

    def prim(a):
        rho = a[0]
        u, v, ww = a[1] / rho, a[2] / rho, a[3] / rho
        T = (a[4] / rho - 0.5 * (u * u + v * v + ww * ww)) / cv
        return rho, u, v, ww, T, rho * c.r_gas * T

    inner = wg[:, G:-G, :, G:-G]
    for q in range(G):
        lo_g, lo_i = prim(inner[:, :, G - 1 - q]), prim(inner[:, :, G + q])
        hi_g, hi_i = prim(inner[:, :, G + c.ny + q]), prim(inner[:, :, G + c.ny - 1 - q])
        for gh, it in ((lo_g, lo_i), (hi_g, hi_i)):
            np.testing.assert_allclose(gh[1], -it[1], atol=1e-14)
            np.testing.assert_allclose(gh[2], -it[2], atol=1e-14)
            np.testing.assert_allclose(gh[3], -it[3], atol=1e-14)
            np.testing.assert_allclose(gh[4], 2 * c.t_wall - it[4], rtol=1e-14)
            np.testing.assert_allclose(gh[5], it[5], rtol=1e-14)
    np.testing.assert_array_equal(wg[:, G:-G, G:-G, :G], w[:, :, :, -G:])
    np.testing.assert_array_equal(wg[:, :G, G:-G, G:-G], w[:, -G:, :, :])
    assert np.isnan(wg[:, 0, 0, 0]).all()


def test_cfl_closed_form(orc):
    c = inputs.Case(nx=8, ny=6, nz=4, beta=0.0, y_wall=False)
    cfg = orc.make_cfg(c)
    u0, v0, w0, T0 = 0.4, -0.3, 0.2, 1.2
    st = inputs.primitive_state(c, 1.1, u0, v0, w0, T0)
    cs = math.sqrt(c.gamma * c.r_gas * T0)
    h = (c.lx / c.nx, c.ly / c.ny, c.lz / c.nz)
    s = (abs(u0) + cs) / h[0] + (abs(v0) + cs) / h[1] + (abs(w0) + cs) / h[2]
    assert abs(orc.cfl_dt(cfg, st, 0.8) - 0.8 / s) < 1e-15


def test_totals_uniform(orc):
    c = inputs.Case(nx=8, ny=6, nz=4, beta=0.0, y_wall=False)
    cfg = orc.make_cfg(c)
    st = inputs.primitive_state(c, 1.1, 0.4, -0.3, 0.2, 1.2)
    np.testing.assert_allclose(orc.totals(cfg, st), st[:, 0, 0, 0] * c.lx * c.ly * c.lz,
                               rtol=1e-14)


def test_prescribed_switch_input(orc):
    """The prescribed sensor field (a test device that fixes the central/WENO decisions): given
    the sensor's own values it changes nothing; zero everywhere gives the central flux at every
    face (WENO off), one everywhere gives WENO at every face (the switch's two limits)."""
    c = inputs.Case(nx=16, ny=12, nz=10, reynolds=3000.0)
    w = inputs.channel_state(c, seed=7)
    cfg = orc.make_cfg(c)
    th, _, fx, fy, fz = orc.sensor(cfg, w)
    assert 0.05 < np.mean(np.concatenate([fx.ravel(), fy.ravel(), fz.ravel()])) < 0.95
    base = orc.rhs(cfg, w)
    assert np.array_equal(orc.rhs(orc.make_cfg(c, theta_fixed=th), w), base)
    zero, one = np.zeros_like(th), np.ones_like(th)
    assert np.array_equal(orc.rhs(orc.make_cfg(c, theta_fixed=zero), w),
                          orc.rhs(orc.make_cfg(c, weno_mode="off"), w))
    assert np.array_equal(orc.rhs(orc.make_cfg(c, theta_fixed=one), w),
                          orc.rhs(orc.make_cfg(c, weno_mode="all"), w))
    _, _, gx, gy, gz = orc.sensor(orc.make_cfg(c, theta_fixed=one), w)
    assert gx.all() and gy.all() and gz.all()
