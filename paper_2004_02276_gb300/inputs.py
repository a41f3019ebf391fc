"""Seeded synthetic inputs and workload definitions.

This module is shared by the CUDA path's tests and benchmark and by the oracle's tests. It holds
no arithmetic of the method (no fluxes, derivatives, sensor or time stepping): only

* ``Case``: the parameters of a workload (grid, gas, scheme), with the non-dimensionalisation
  of the plane channel: rho_b = u_b = h = T_w = 1, R = 1/(gamma M_b^2) so that c_w = 1/M_b,
  mu_w = 2/Re_b (Re_b = 2 rho_b u_b h / mu_w, Section 3.1), mu = mu_w T^0.76;
* a counter-based SplitMix64 generator (Steele, Lea and Flood, 2014) indexed by
  (component, k, j, i), and
* initial states built from it (laminar Poiseuille profile plus uniform velocity noise).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, index: np.ndarray) -> np.ndarray:
    """SplitMix64 output number ``index`` (0-based) of the stream started at ``seed``."""
    with np.errstate(over="ignore"):
        z = np.uint64(seed) + (index.astype(np.uint64) + np.uint64(1)) * _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def uniform(seed: int, shape) -> np.ndarray:
    """Uniform doubles in [0, 1) with 53 random bits, C order over ``shape``."""
    n = int(np.prod(shape))
    z = splitmix64(seed, np.arange(n, dtype=np.uint64))
    return ((z >> np.uint64(11)).astype(np.float64) * 2.0**-53).reshape(shape)


@dataclasses.dataclass(frozen=True)
class Case:
    """A workload: grid, gas and scheme parameters (channel defaults).

    kind "channel": rho_b = u_b = h = T_w = 1, R = 1/(gamma M_b^2), mu_w = 2/Re_b.
    kind "bl" (boundary layer, optionally with an impinging oblique shock): free stream
    rho = u = T = 1, length delta_in = 1, R = 1/(gamma M^2), mu_inf = 1/Re_delta, T_w = t_wall.
    """

    name: str = "channel"
    kind: str = "channel"
    nx: int = 64
    ny: int = 48
    nz: int = 32
    lx: float = 2.0 * math.pi
    ly: float = 2.0
    lz: float = math.pi
    beta: float = 1.5            # tanh wall clustering; 0 gives a uniform y grid
    y_map: str = "tanh"          # "tanh", "erf": clustered at both walls; "tanh1", "sinh1": at y = 0 only
    y_wall: bool = True          # isothermal staggered walls in y (else periodic)
    bc_xmin: str = None          # face kinds ("periodic", "wall", "char", "recycle", "df"); None:
    bc_xmax: str = None          #   x periodic, y walls or periodic per y_wall
    bc_ymin: str = None
    bc_ymax: str = None
    shock: bool = False          # oblique shock imposed at the top (characteristic) face
    shock_theta: float = 0.0     # flow deflection of the shock (radians)
    shock_ximp: float = 0.0      # x where the incident shock reaches the wall
    i_recycle: int = 0           # recycling plane (x index) of a recycling inflow
    delta_in: float = 1.0        # inflow boundary-layer thickness
    df_ny: int = 0               # digital-filter inflow: filter half-widths n (grid points) in y, z,
    df_nz: int = 0               #   integral time scale and generator seed
    df_tau: float = 0.0
    df_seed: int = 0
    gamma: float = 1.4
    prandtl: float = 0.72
    mach: float = 1.5            # bulk Mach number u_b / c_w
    reynolds: float = 3000.0     # bulk Reynolds number 2 rho_b u_b h / mu_w
    visc_law: str = "power"
    visc_exp: float = 0.76
    suth_s: float = 110.4 / 288.15
    t_wall: float = 1.0
    forcing: bool = True
    L: int = 3                   # central scheme of order 2L
    weno_mode: str = "sensor"    # "off", "sensor" (Ducros switch) or "all"
    theta_thr: float = 0.05
    weno_eps: float = 1e-6
    u0: float = 1.0              # sensor velocity scale (bulk velocity)
    l0: float = 1.0              # sensor length scale (channel half height)
    convective: bool = True
    viscous: bool = True
    precision: str = "fp64"      # "fp64", or "mixed" (FP32 flux arithmetic, FP64 state)
    cfl: float = 0.8
    steps: int = 20
    noise: float = 0.05          # uniform velocity noise amplitude (fraction of u_b)
    seed: int = 0

    @property
    def r_gas(self) -> float:
        return 1.0 / (self.gamma * self.mach**2)

    @property
    def mu_ref(self) -> float:
        return 2.0 / self.reynolds if self.kind == "channel" else 1.0 / self.reynolds

    @property
    def t_ref(self) -> float:
        return self.t_wall if self.kind == "channel" else 1.0

    @property
    def ref(self):
        """Free-stream primitives (rho, u, v, w, p) of a boundary-layer case."""
        if self.kind == "channel":
            return None
        return (1.0, 1.0, 0.0, 0.0, self.r_gas)

    @property
    def npts(self) -> int:
        return self.nx * self.ny * self.nz

    def replace(self, **kw) -> "Case":
        return dataclasses.replace(self, **kw)


# The benchmark workloads: C1 is the small channel parity case, C2 the bench case, C3 the
# supersonic boundary layer and C4 the shock/boundary-layer interaction.
C1 = Case(name="channel-64x48x32", nx=64, ny=48, nz=32, reynolds=3000.0, steps=20)
C2 = Case(name="channel-256x192x128", nx=256, ny=192, nz=128, reynolds=7000.0, steps=200)
# The paper's own channel settings (Section 3.1) on the 64x48x32 grid: fourth-order central and
# viscous stencils (L = 2), Sutherland's law (T_w = 288.15 K), error-function clustering with
# beta = 1.4 (largest/smallest wall-normal spacing exp(beta^2) = 7.1, as 5.7/0.8 wall units in
# the paper), M_b = 1.5, Re_b = 14725 on a 6 pi x 2 x 2 pi box.
PAPER_CHANNEL = Case(name="paper-channel-64x48x32", nx=64, ny=48, nz=32, lx=6 * math.pi,
                     lz=2 * math.pi, reynolds=14725.0, L=2, visc_law="sutherland", y_map="erf",
                     beta=1.4, steps=20)


def bl_case(name, nx, ny, nz, lx, ly, lz, shock=False, **kw) -> Case:
    """Supersonic zero-pressure-gradient boundary layer (Section 3.2): M = 2, Re_delta_in =
    10000 (Re_theta ~ 1000), T_w/T_inf = 1.7, wall-clustered tanh grid, rescaled recycling
    inflow from 0.8 lx, characteristic outflow and top, isothermal wall; with shock=True an
    8-degree oblique shock imposed at the top (Section 3.3) reaching the wall at 0.6 lx."""
    base = dict(name=name, kind="bl", nx=nx, ny=ny, nz=nz, lx=lx, ly=ly, lz=lz, beta=2.5,
                y_map="tanh1", mach=2.0, reynolds=10000.0, t_wall=1.7, forcing=False,
                bc_xmin="recycle", bc_xmax="char", bc_ymin="wall", bc_ymax="char",
                i_recycle=int(0.8 * nx), delta_in=1.0, u0=1.0, l0=1.0, noise=0.05,
                shock=shock, shock_theta=math.radians(8.0) if shock else 0.0,
                shock_ximp=0.6 * lx)
    base.update(kw)
    return Case(**base)


C3 = bl_case("bl-1024x256x256", 1024, 256, 256, 26.25, 12.0, 5.0)
# The paper's own boundary-layer settings (Section 3.2) on the C3 grid: fourth-order stencils,
# Sutherland's law (T_inf = 288.15 K), hyperbolic-sine clustering (beta = 4, first node at
# y = 0.0034 delta_in) and the digital-filter inflow (profiles: df_profiles).
PAPER_BL = bl_case("paper-bl-1024x256x256", 1024, 256, 256, 26.25, 12.0, 5.0, L=2,
                   visc_law="sutherland", y_map="sinh1", beta=4.0, bc_xmin="df", df_ny=4, df_nz=4,
                   df_tau=0.5, df_seed=1)
C4 = bl_case("sbli-2048x384x256", 2048, 384, 256, 50.0, 12.0, 5.33, shock=True, noise=0.001)


def node_y(case: Case) -> np.ndarray:
    """Wall-normal node positions used to lay out the initial profile (nodes at the cell
    centres of a grid clustered toward both walls y = -ly/2 and y = ly/2, "tanh" or "erf", or
    toward the wall y = 0 up to y = ly, "tanh1" or "sinh1")."""
    eta = (np.arange(case.ny) + 0.5) / case.ny
    b = case.beta
    if not (b and b > 0):
        return case.ly * (eta - 0.5)
    if case.y_map == "tanh1":
        return case.ly * (1.0 - np.tanh(b * (1.0 - eta)) / math.tanh(b))
    if case.y_map == "sinh1":
        return case.ly * np.sinh(b * eta) / math.sinh(b)
    if case.y_map == "erf":
        return 0.5 * case.ly * np.array([math.erf(b * (2.0 * e - 1.0)) for e in eta]) / math.erf(b)
    return 0.5 * case.ly * np.tanh(b * (2.0 * eta - 1.0)) / math.tanh(b)


def df_profiles(case: Case) -> np.ndarray:
    """Inflow data of a digital-filter inflow, [7, ny]: mean U, V, T and the Reynolds stresses
    R11, R12, R22, R33 at the wall-normal nodes. Synthetic stand-in for a DNS Reynolds-stress
    profile: U and T as in bl_state (1/7 power law, Crocco-Busemann), and stresses of the shape
    g(h) = (h/h0) exp(1 - h/h0) with h0 = 0.1 delta_in, faded out above delta_in, amplitudes
    (0.1, 0.04, 0.06)^2 of u_inf^2 for R11, R22, R33 and a correlation R12 = -0.5 sqrt(R11 R22)."""
    yy = node_y(case)
    h = np.maximum(yy - (0.0 if one_sided(case) else -0.5 * case.ly), 0.0) / case.delta_in
    U = np.minimum(h ** (1.0 / 7.0), 1.0)
    tr = 1.0 + case.prandtl ** (1.0 / 3.0) * 0.5 * (case.gamma - 1.0) * case.mach ** 2
    T = case.t_wall + (tr - case.t_wall) * U + (1.0 - tr) * U * U
    g = (h / 0.1) * np.exp(1.0 - h / 0.1) * 0.5 * (1.0 - np.tanh((h - 1.0) / 0.1))
    R11, R22, R33 = 0.1 ** 2 * g, 0.04 ** 2 * g, 0.06 ** 2 * g
    R12 = -0.5 * np.sqrt(R11 * R22)
    return np.stack([U, np.zeros_like(U), T, R11, R12, R22, R33])


def one_sided(case: Case) -> bool:
    """True for maps with a single wall at y = 0."""
    return case.y_map in ("tanh1", "sinh1")


def channel_state(case: Case, seed: int | None = None) -> np.ndarray:
    """Initial channel state w = [rho, rho u, rho v, rho w, rho E], shape [5, nz, ny, nx].

    rho = 1, T = T_w; u = 1.5 u_b (1 - (2y/ly)^2) plus noise, v and w noise only; the noise is
    uniform in [-a, a] (a = ``case.noise``) from SplitMix64 over index (component, k, j, i).
    """
    seed = case.seed if seed is None else seed
    nz, ny, nx = case.nz, case.ny, case.nx
    r = uniform(seed, (3, nz, ny, nx))
    noise = case.noise * (2.0 * r - 1.0)
    yy = node_y(case)
    u = 1.5 * (1.0 - (2.0 * yy / case.ly) ** 2)[None, :, None] + noise[0]
    v = noise[1]
    w = noise[2]
    rho = np.ones((nz, ny, nx))
    T = np.full((nz, ny, nx), case.t_wall)
    cv = case.r_gas / (case.gamma - 1.0)
    out = np.empty((5, nz, ny, nx))
    out[0] = rho
    out[1] = rho * u
    out[2] = rho * v
    out[3] = rho * w
    out[4] = rho * (cv * T + 0.5 * (u * u + v * v + w * w))
    return out


def uniform_block(seed: int, start: int, count: int) -> np.ndarray:
    """Outputs start .. start + count - 1 of the stream of ``uniform`` (flat C order)."""
    z = splitmix64(seed, np.arange(start, start + count, dtype=np.uint64))
    return (z >> np.uint64(11)).astype(np.float64) * 2.0**-53


def bl_state(case: Case, seed: int | None = None, planes_per_chunk: int = 16) -> np.ndarray:
    """Initial boundary layer: u/u_inf = (h/delta_in)^(1/7) below delta_in and 1 above,
    temperature from the Crocco-Busemann relation T = T_w + (T_r - T_w) u + (1 - T_r) u^2 with
    the recovery temperature T_r = 1 + r (gamma-1)/2 M^2, r = Pr^(1/3), uniform pressure, and
    uniform velocity noise of amplitude ``case.noise`` inside the layer (SplitMix64 stream over
    (component, k, j, i)). Built a few z planes at a time (the values do not depend on
    ``planes_per_chunk``), so that large grids need little memory beyond the result."""
    seed = case.seed if seed is None else seed
    nz, ny, nx = case.nz, case.ny, case.nx
    yy = node_y(case)
    h = yy - (0.0 if one_sided(case) else -0.5 * case.ly)
    ub = np.minimum(np.maximum(h / case.delta_in, 0.0) ** (1.0 / 7.0), 1.0)
    tr = 1.0 + case.prandtl ** (1.0 / 3.0) * 0.5 * (case.gamma - 1.0) * case.mach ** 2
    T1 = case.t_wall + (tr - case.t_wall) * ub + (1.0 - tr) * ub * ub
    inside = (h < case.delta_in)[None, None, :, None]
    T = T1[None, :, None]
    p = case.r_gas  # p_inf = rho_inf R T_inf
    rho_row = p / (case.r_gas * T)
    cv = case.r_gas / (case.gamma - 1.0)
    plane = ny * nx
    out = np.empty((5, nz, ny, nx))
    for k0 in range(0, nz, max(1, planes_per_chunk)):
        k1 = min(nz, k0 + max(1, planes_per_chunk))
        nk = k1 - k0
        r = np.stack([uniform_block(seed, (c * nz + k0) * plane, nk * plane) for c in range(3)])
        noise = case.noise * (2.0 * r.reshape(3, nk, ny, nx) - 1.0) * inside
        u = ub[None, :, None] + noise[0]
        v = noise[1]
        w = noise[2]
        rho = np.broadcast_to(rho_row, (nk, ny, nx))
        out[0, k0:k1] = rho
        out[1, k0:k1] = rho * u
        out[2, k0:k1] = rho * v
        out[3, k0:k1] = rho * w
        out[4, k0:k1] = rho * (cv * T + 0.5 * (u * u + v * v + w * w))
    return out


def random_state(case: Case, seed: int, amp_u: float = 0.3, amp_rho: float = 0.2,
                 amp_t: float = 0.2) -> np.ndarray:
    """A rough random state (no structure) for conservation and parity checks:
    rho = 1 + amp_rho s, T = 1 + amp_t s, velocities amp_u s, s uniform in [-1, 1]."""
    nz, ny, nx = case.nz, case.ny, case.nx
    s = 2.0 * uniform(seed, (5, nz, ny, nx)) - 1.0
    rho = 1.0 + amp_rho * s[0]
    u, v, w = amp_u * s[1], amp_u * s[2], amp_u * s[3]
    T = case.t_wall * (1.0 + amp_t * s[4])
    cv = case.r_gas / (case.gamma - 1.0)
    out = np.empty((5, nz, ny, nx))
    out[0] = rho
    out[1] = rho * u
    out[2] = rho * v
    out[3] = rho * w
    out[4] = rho * (cv * T + 0.5 * (u * u + v * v + w * w))
    return out


def primitive_state(case: Case, rho, u, v, w, T) -> np.ndarray:
    """Conserved state from primitive fields given on the [nz, ny, nx] nodes."""
    cv = case.r_gas / (case.gamma - 1.0)
    shape = (case.nz, case.ny, case.nx)
    rho, u, v, w, T = (np.broadcast_to(np.asarray(a, dtype=np.float64), shape)
                       for a in (rho, u, v, w, T))
    out = np.empty((5,) + shape)
    out[0] = rho
    out[1] = rho * u
    out[2] = rho * v
    out[3] = rho * w
    out[4] = rho * (cv * T + 0.5 * (u * u + v * v + w * w))
    return out


def ensemble_cases(seed: int = 0, n: int = 64, precision: str = "fp64") -> list:
    """The batched workload: n independent channel instances with grid dimensions drawn from
    {32..192} x {32..128} x {32..128}, bulk Mach number from U[0.3, 3.0] and bulk Reynolds number
    from U[2000, 8000] (SplitMix64 stream ``seed``; same domain, walls and scheme as C1/C2)."""
    r = uniform(seed, (n, 5))
    cases = []
    for e in range(n):
        nx = 32 + int(r[e, 0] * 161)
        ny = 32 + int(r[e, 1] * 97)
        nz = 32 + int(r[e, 2] * 97)
        mach = 0.3 + 2.7 * r[e, 3]
        re = 2000.0 + 6000.0 * r[e, 4]
        cases.append(Case(name=f"ensemble-{e}", nx=nx, ny=ny, nz=nz, mach=mach, reynolds=re,
                          precision=precision, seed=seed * 1000 + e))
    return cases


def ensemble_bl_cases(seed: int = 0, n: int = 32, precision: str = "fp64") -> list:
    """Boundary-layer instances for a mixed ensemble: grid dimensions from {64..192} x {32..128}
    x {32..96} on a box of 3 x 12 x 3 delta_in per 64 x 128 x 64 nodes (the aspect of the
    1024x256x256 workload), free-stream Mach number from U[1.5, 3.0], and, in turn, a recycling
    inflow, a recycling inflow under the 8-degree shock, and a digital-filter inflow."""
    r = uniform(seed + 7, (n, 4))
    cases = []
    for e in range(n):
        nx = 64 + int(r[e, 0] * 129)
        ny = 32 + int(r[e, 1] * 97)
        nz = 32 + int(r[e, 2] * 65)
        mach = 1.5 + 1.5 * r[e, 3]
        kind = e % 3
        kw = dict(mach=mach, precision=precision, seed=seed * 1000 + 500 + e, noise=0.01)
        if kind == 1:
            kw.update(shock=True)
        if kind == 2:
            kw.update(bc_xmin="df", df_ny=3, df_nz=3, df_tau=0.5, df_seed=seed * 1000 + e)
        cases.append(bl_case(f"ensemble-bl-{e}", nx, ny, nz, 3.0 * nx / 64, 12.0, 3.0 * nz / 64, **kw))
    return cases
