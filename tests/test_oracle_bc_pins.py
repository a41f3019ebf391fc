"""Pins of the oracle's boundary-layer boundaries (no GPU): oblique shock (Section 3.3),
characteristic faces (Section 3.2), rescaled recycling inflow and the one-sided wall map.

The recycling inflow is not in the paper (its inflow is digital filtering from a DNS
Reynolds-stress database); its pins are the identity and rescaling properties the construction
must have. The characteristic faces are checked against their definition through the oracle's
eigenvectors, which are themselves pinned (test_oracle_pins.py)."""
import math

import numpy as np
import pytest

from paper_2004_02276_gb300 import inputs

G3 = 3


def small_bl(**kw):
    base = dict(nx=40, ny=32, nz=8)
    base.update(kw)
    return inputs.bl_case("bl-small", base.pop("nx"), base.pop("ny"), base.pop("nz"), 6.0, 6.0, 1.5, **base)


def prim(case, a):
    cv = case.r_gas / (case.gamma - 1.0)
    rho = a[0]
    u, v, w = a[1] / rho, a[2] / rho, a[3] / rho
    T = (a[4] / rho - 0.5 * (u * u + v * v + w * w)) / cv
    return rho, u, v, w, rho * case.r_gas * T, T


def cons(case, q):
    rho, u, v, w, p = q
    cv = case.r_gas / (case.gamma - 1.0)
    T = p / (rho * case.r_gas)
    return np.array([rho, rho * u, rho * v, rho * w, rho * (cv * T + 0.5 * (u * u + v * v + w * w))])


# ----------------------------------------------------------------------- oblique shock

@pytest.mark.parametrize("mach,theta_deg", [(2.0, 8.0), (2.28, 8.0), (3.0, 15.0)])
def test_oblique_shock_relations(orc, mach, theta_deg):
    g = 1.4
    theta = math.radians(theta_deg)
    beta, pr, rr, m2 = orc.oblique_shock(g, mach, theta)
    # theta-beta-M relation
    tb = 2.0 / math.tan(beta) * (mach ** 2 * math.sin(beta) ** 2 - 1.0) / (mach ** 2 * (g + math.cos(2 * beta)) + 2.0)
    assert abs(math.tan(theta) - tb) < 1e-12
    assert math.asin(1.0 / mach) < beta < math.radians(70.0)  # weak branch
    # Rankine-Hugoniot across the shock normal, upstream rho = p-scale = 1, c = 1
    rho1, p1 = 1.0, 1.0 / g
    u1 = mach
    un1, ut = u1 * math.sin(beta), u1 * math.cos(beta)
    rho2, p2 = rho1 * rr, p1 * pr
    un2 = rho1 * un1 / rho2
    assert abs(p1 + rho1 * un1 ** 2 - (p2 + rho2 * un2 ** 2)) < 1e-12
    h1 = g / (g - 1) * p1 / rho1 + 0.5 * un1 ** 2
    h2 = g / (g - 1) * p2 / rho2 + 0.5 * un2 ** 2
    assert abs(h1 - h2) < 1e-12
    # downstream Mach number and flow deflection
    V2 = math.hypot(ut, un2)
    c2 = math.sqrt(g * p2 / rho2)
    assert abs(V2 / c2 - m2) < 1e-12
    assert abs((beta - math.atan2(un2, ut)) - theta) < 1e-12


def test_recovery_temperature_matches_wall_ratio():
    """The wall temperature ratio of the boundary-layer workload is the recovery temperature
    1 + r (gamma-1)/2 M^2 with r = Pr^(1/3) at M = 2 (1.717)."""
    c = inputs.C3
    tr = 1.0 + c.prandtl ** (1.0 / 3.0) * 0.5 * (c.gamma - 1.0) * c.mach ** 2
    assert abs(tr - 1.717) < 1e-3 and abs(c.t_wall - tr) < 0.02


# ----------------------------------------------------------------------- one-sided map

def test_one_sided_map(orc):
    c = small_bl(ny=400)
    y, ye, yee = orc.metrics(orc.make_cfg(c))
    assert y[0] > 0 and y[-1] < c.ly and np.all(np.diff(y) > 0)
    assert np.all(np.diff(np.diff(y)) > 0)  # spacing grows away from the wall
    deta = 1.0 / c.ny
    np.testing.assert_allclose((y[2:] - y[:-2]) / (2 * deta), ye[1:-1], rtol=2e-4)
    np.testing.assert_allclose((ye[2:] - ye[:-2]) / (2 * deta), yee[1:-1], rtol=2e-3, atol=1e-3)
    assert abs(ye.sum() * deta - c.ly) < 1e-3


# ----------------------------------------------------------------------- characteristic faces

def test_char_outflow_supersonic_is_extrapolation(orc):
    """Every characteristic speed leaves through a supersonic outflow: ghosts equal the boundary
    node."""
    c = small_bl(bc_xmin="char", bc_ymin="char", noise=0.0)
    st = inputs.primitive_state(c, 1.0, 1.0, 0.0, 0.0, 1.0)  # M = 2 everywhere
    s = inputs.uniform(3, st.shape)
    st = st * (1.0 + 0.01 * (s - 0.5))
    wg = orc.fill_ghosts(orc.make_cfg(c), st)
    for q in range(G3):
        np.testing.assert_allclose(wg[:, G3:-G3, G3:-G3, G3 + c.nx + q], st[:, :, :, -1], rtol=1e-13)


def test_char_face_at_reference_is_reference(orc):
    c = small_bl(bc_xmin="char", bc_ymin="char", noise=0.0)
    ref = c.ref
    st = np.broadcast_to(cons(c, ref)[:, None, None, None], (5, c.nz, c.ny, c.nx)).copy()
    wg = orc.fill_ghosts(orc.make_cfg(c), st)
    np.testing.assert_allclose(wg[:, G3:-G3, G3 + c.ny, G3:-G3], st[:, :, -1, :], rtol=1e-13)
    np.testing.assert_allclose(wg[:, G3:-G3, G3:-G3, 0], st[:, :, :, 0], rtol=1e-13)


def test_char_top_partition(orc):
    """Top face: outgoing characteristic variables (speed > 0 along +y) keep the boundary
    node's values, incoming ones take the reference's, in the boundary node's eigenbasis."""
    c = small_bl(noise=0.0)
    cfg = orc.make_cfg(c)
    rng = inputs.uniform(5, (4, c.nz, c.nx))
    st = inputs.bl_state(c, 0)
    # give the top row a small upward or downward velocity so that both cases occur
    st = st.copy()
    rho_top = st[0, :, -1, :]
    v = 0.2 * (rng[0] - 0.5)
    st[4, :, -1, :] += 0.5 * rho_top * v * v
    st[2, :, -1, :] = rho_top * v
    wg = orc.fill_ghosts(cfg, st)
    wr = cons(c, c.ref)
    for k in range(c.nz):
        for i in range(0, c.nx, 7):
            wb = st[:, k, -1, i]
            rho, u, vv, w, p, T = prim(c, wb)
            H = (wb[4] + p) / rho
            Lm, Rm = orc.eigvecs(1, c.gamma, u, vv, w, H)
            cs = math.sqrt(c.gamma * p / rho)
            lam = np.array([vv - cs, vv, vv, vv, vv + cs])
            want = np.where(lam > 0, Lm @ wb, Lm @ wr)
            got = Lm @ wg[:, G3 + k, G3 + c.ny, G3 + i]
            np.testing.assert_allclose(got, want, rtol=1e-12, atol=1e-12)


def test_char_outflow_prescribes_pressure_only(orc):
    """At a subsonic outflow only the incoming acoustic variable changes, and it is the one of
    the boundary state at the reference pressure."""
    c = small_bl(noise=0.0)
    cfg = orc.make_cfg(c)
    st = inputs.bl_state(c, 0)
    wg = orc.fill_ghosts(cfg, st)
    for k in (0, 3):
        for j in (0, 5, 20):
            wb = st[:, k, j, -1]
            rho, u, v, w, p, T = prim(c, wb)
            H = (wb[4] + p) / rho
            Lm, Rm = orc.eigvecs(0, c.gamma, u, v, w, H)
            cs = math.sqrt(c.gamma * p / rho)
            lam = np.array([u - cs, u, u, u, u + cs])
            wref = cons(c, (rho, u, v, w, c.ref[4]))
            want = np.where(lam > 0, Lm @ wb, Lm @ wref)
            got = Lm @ wg[:, G3 + k, G3 + j, G3 + c.nx]
            np.testing.assert_allclose(got, want, rtol=1e-12, atol=1e-13)


def test_freestream_preserved_with_open_faces(orc):
    """A uniform free stream with characteristic faces on every side (inflow, outflow, bottom,
    top) stays steady. (Recycling assumes a no-slip wall below the profile and is pinned
    separately.)"""
    c = small_bl(bc_xmin="char", bc_ymin="char", noise=0.0)
    st = np.broadcast_to(cons(c, c.ref)[:, None, None, None], (5, c.nz, c.ny, c.nx)).copy()
    r = orc.rhs(orc.make_cfg(c), st)
    assert np.abs(r).max() < 1e-12


# ----------------------------------------------------------------------- recycling inflow

def test_recycling_identity_when_thickness_matches(orc):
    """With delta_in equal to the recycling plane's thickness (s = 1) the ghost planes are the
    planes upstream of the recycling plane (to the round-off of the primitive/conserved round
    trip)."""
    c = small_bl(noise=0.05)
    st = inputs.bl_state(c, 1)
    s = orc.recycle_scale(orc.make_cfg(c), st)
    assert 0.5 < s < 2.0 and s != 1.0
    c1 = c.replace(delta_in=c.delta_in * s)
    assert orc.recycle_scale(orc.make_cfg(c1), st) == 1.0
    wg = orc.fill_ghosts(orc.make_cfg(c1), st)
    for q in range(G3):
        np.testing.assert_allclose(wg[:, G3:-G3, G3:-G3, G3 - 1 - q], st[:, :, :, c.i_recycle - q],
                                   rtol=1e-14, atol=1e-15)


def test_recycling_rescales_thickness(orc):
    """The spanwise-mean inflow profile reaches 0.99 u_ref at delta_in (up to the grid
    spacing there) whatever the recycling plane's thickness."""
    c = small_bl(ny=96, noise=0.0, delta_in=0.8)
    cfg = orc.make_cfg(c)
    st = inputs.bl_state(c.replace(delta_in=1.0), 0)  # recycling plane thickness ~1.0
    wg = orc.fill_ghosts(cfg, st)
    y, ye, _ = orc.metrics(cfg)
    ub = (wg[1, G3:-G3, G3:-G3, G3 - 1] / wg[0, G3:-G3, G3:-G3, G3 - 1]).mean(axis=0)
    j = int(np.argmax(ub >= 0.99))
    d99 = y[j - 1] + (0.99 - ub[j - 1]) * (y[j] - y[j - 1]) / (ub[j] - ub[j - 1])
    assert abs(d99 - 0.8) < 2.0 * (y[j] - y[j - 1])
    # the wall side of the inflow keeps the wall temperature trend (no jump from interpolation)
    assert np.isfinite(wg[:, G3:-G3, G3:-G3, :G3]).all()


def test_boundary_layer_step_is_finite_and_bounded(orc):
    c = small_bl(noise=0.02)
    cfg = orc.make_cfg(c)
    st = inputs.bl_state(c, 0)
    m0 = st[0].sum()
    for _ in range(5):
        st, dt = orc.rk_step(cfg, st)
    assert np.isfinite(st).all() and dt > 0
    assert abs(st[0].sum() / m0 - 1.0) < 0.05  # open domain: mass changes only through the faces


# ----------------------------------------------------------------------- wall-normal maps

MAPS = ["tanh", "erf", "tanh1", "sinh1"]


def map_case(y_map, ny=400, beta=2.0):
    return inputs.Case(nx=4, ny=ny, nz=4, ly=2.0, beta=beta, y_map=y_map)


@pytest.mark.parametrize("y_map", MAPS)
def test_map_metrics_consistent(orc, y_map):
    """The analytic y_eta, y_etaeta agree with finite differences of y, the spacing integrates
    to L_y, and the map is monotone (Sections 3.1, 3.2 name the maps without formulas)."""
    c = map_case(y_map)
    y, ye, yee = orc.metrics(orc.make_cfg(c))
    deta = 1.0 / c.ny
    assert np.all(np.diff(y) > 0) and np.all(ye > 0)
    def d4(f):  # fourth-order central difference
        return (-f[4:] + 8 * f[3:-1] - 8 * f[1:-3] + f[:-4]) / (12 * deta)
    np.testing.assert_allclose(d4(y), ye[2:-2], rtol=1e-7)
    np.testing.assert_allclose(d4(ye), yee[2:-2], rtol=1e-6, atol=1e-7 * np.abs(yee).max())
    assert abs(ye.sum() * deta - c.ly) < 1e-4 * c.ly  # midpoint rule, O(deta^2)


@pytest.mark.parametrize("y_map", MAPS)
def test_map_clusters_at_walls(orc, y_map):
    c = map_case(y_map, ny=64)
    y, ye, yee = orc.metrics(orc.make_cfg(c))
    eta0 = 0.5 / c.ny
    # the wall sits at eta = 0: Taylor from the first node, remainder (eta0^2/2) y_etaeta
    wall = y[0] - eta0 * ye[0]
    tol = 1.5 * 0.5 * eta0 ** 2 * abs(yee[0]) + 1e-15
    if y_map in ("tanh", "erf"):
        assert ye[0] < ye[c.ny // 2] and ye[-1] < ye[c.ny // 2]
        np.testing.assert_allclose(y, -y[::-1], atol=1e-14)  # odd about the channel centre
        assert abs(wall + 0.5 * c.ly) < tol
    else:
        assert np.all(np.diff(ye) > 0)  # spacing grows away from the wall y = 0
        assert abs(wall) < tol


@pytest.mark.parametrize("y_map", MAPS)
def test_map_uniform_limit(orc, y_map):
    """As beta -> 0 every map tends to the uniform one (relative deviation O(beta^2))."""
    c = map_case(y_map, ny=16, beta=1e-4)
    y, ye, yee = orc.metrics(orc.make_cfg(c))
    eta = (np.arange(c.ny) + 0.5) / c.ny
    y_uniform = c.ly * (eta if y_map in ("tanh1", "sinh1") else eta - 0.5)
    np.testing.assert_allclose(y, y_uniform, atol=1e-7)
    np.testing.assert_allclose(ye, c.ly, rtol=1e-7)
    assert np.abs(yee).max() < 1e-6
