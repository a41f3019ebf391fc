"""ctypes front end of the FP64 CPU oracle (test infrastructure only).

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may import
this module. It converts a workload description (``paper_2004_02276_gb300.inputs.Case``, or any
object with the same attributes) into the oracle's own configuration struct and calls the C
functions of ``strm_oracle.c``. Arrays are interior-only, SoA ``[5, nz, ny, nx]`` float64.
"""
import ctypes
import os

import numpy as np

from . import build as _build

_lib = None


class OrcCfg(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
        ("lx", ctypes.c_double), ("ly", ctypes.c_double), ("lz", ctypes.c_double),
        ("y_map", ctypes.c_int), ("beta", ctypes.c_double),
        ("bc_xmin", ctypes.c_int), ("bc_xmax", ctypes.c_int),
        ("bc_ymin", ctypes.c_int), ("bc_ymax", ctypes.c_int),
        ("ref", ctypes.c_double * 5), ("shock", ctypes.c_int),
        ("shock_theta", ctypes.c_double), ("shock_ximp", ctypes.c_double),
        ("i_recycle", ctypes.c_int), ("delta_in", ctypes.c_double),
        ("df_prof", ctypes.POINTER(ctypes.c_double)), ("df_psi", ctypes.POINTER(ctypes.c_double)),
        ("df_count", ctypes.POINTER(ctypes.c_longlong)), ("df_ny", ctypes.c_int),
        ("df_nz", ctypes.c_int), ("df_tau", ctypes.c_double), ("df_seed", ctypes.c_ulonglong),
        ("gamma", ctypes.c_double), ("prandtl", ctypes.c_double), ("r_gas", ctypes.c_double),
        ("visc_law", ctypes.c_int), ("mu_ref", ctypes.c_double), ("t_ref", ctypes.c_double),
        ("visc_exp", ctypes.c_double), ("suth_s", ctypes.c_double),
        ("t_wall", ctypes.c_double), ("forcing", ctypes.c_int),
        ("L", ctypes.c_int), ("weno_mode", ctypes.c_int), ("theta_thr", ctypes.c_double),
        ("weno_eps", ctypes.c_double), ("u0", ctypes.c_double), ("l0", ctypes.c_double),
        ("convective", ctypes.c_int), ("viscous", ctypes.c_int),
        ("theta_fixed", ctypes.POINTER(ctypes.c_double)),
    ]


WENO_MODES = {"off": 0, "sensor": 1, "all": 2}
BC_KINDS = {"periodic": 0, "wall": 1, "char": 2, "recycle": 3, "df": 4}
Y_MAPS = {"uniform": 0, "tanh": 1, "tanh1": 2, "erf": 3, "sinh1": 4}
VISC_LAWS = {"power": 0, "sutherland": 1}


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        _lib = ctypes.CDLL(path)
        P = ctypes.POINTER
        d, i = ctypes.c_double, ctypes.c_int
        dp = P(d)
        u8p = P(ctypes.c_ubyte)
        cp = P(OrcCfg)
        _lib.orc_rhs.argtypes = [cp, dp, dp]
        _lib.orc_rk_step.argtypes = [cp, dp, d, d, dp]
        _lib.orc_rk_stage_update.argtypes = [i, d, dp, dp, dp, ctypes.c_long]
        _lib.orc_rk_stage_update.restype = None
        _lib.orc_cfl_dt.argtypes = [cp, dp, d]
        _lib.orc_cfl_dt.restype = d
        _lib.orc_totals.argtypes = [cp, dp, dp]
        _lib.orc_sensor.argtypes = [cp, dp, dp, dp, u8p, u8p, u8p]
        _lib.orc_fill_ghosts.argtypes = [cp, dp, dp]
        _lib.orc_metrics.argtypes = [cp, dp, dp, dp]
        _lib.orc_metrics.restype = None
        _lib.orc_eigvecs.argtypes = [i, d, d, d, d, d, dp, dp]
        _lib.orc_eigvecs.restype = None
        _lib.orc_weno5.argtypes = [dp, d]
        _lib.orc_weno5.restype = d
        _lib.orc_ghosts.restype = i
        _lib.orc_oblique_shock.argtypes = [d, d, d, dp, dp, dp, dp]
        _lib.orc_recycle_scale.argtypes = [cp, dp]
        _lib.orc_recycle_scale.restype = d
        _lib.orc_stats.argtypes = [cp, dp, i, dp]
        _lib.orc_df_init.argtypes = [cp]
        _lib.orc_splitmix64.argtypes = [ctypes.c_ulonglong, ctypes.c_ulonglong]
        _lib.orc_splitmix64.restype = ctypes.c_ulonglong
        _lib.orc_df_plane.argtypes = [cp, ctypes.c_longlong, dp]
        _lib.orc_set_threads.argtypes = [i]
        _lib.orc_set_threads.restype = i
    return _lib


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _u8(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_ubyte))


class DFState:
    """The digital-filter inflow data the oracle configuration points to: the mean profiles and
    Reynolds stresses prof[7, ny] (U, V, T, R11, R12, R22, R33), the fluctuation plane
    psi[3, nz, ny] and the draw counter, kept alive by this object."""

    def __init__(self, case, prof):
        self.prof = np.ascontiguousarray(prof, dtype=np.float64)
        assert self.prof.shape == (7, case.ny)
        self.psi = np.zeros((3, case.nz, case.ny))
        self.count = np.zeros(1, dtype=np.int64)


def make_cfg(case, df=None, **over) -> OrcCfg:
    """Oracle configuration from a workload description; keyword overrides win. With a
    digital-filter inflow face, `df` is the DFState the configuration points to (and the first
    plane is drawn if its counter is still 0). ``theta_fixed=`` ([nz, ny, nx] array) makes the
    hybrid switch read that sensor field instead of the computed one."""
    get = lambda k, dflt=None: over.get(k, getattr(case, k, dflt))
    c = OrcCfg()
    c.nx, c.ny, c.nz = get("nx"), get("ny"), get("nz")
    c.lx, c.ly, c.lz = get("lx"), get("ly"), get("lz")
    beta = get("beta", 0.0)
    ymap = get("y_map", "tanh")
    c.y_map = Y_MAPS[ymap] if beta and beta > 0 else 0
    c.beta = beta if beta else 0.0
    ywall = get("y_wall", True)
    c.bc_xmin = BC_KINDS[get("bc_xmin", None) or "periodic"]
    c.bc_xmax = BC_KINDS[get("bc_xmax", None) or "periodic"]
    c.bc_ymin = BC_KINDS[get("bc_ymin", None) or ("wall" if ywall else "periodic")]
    c.bc_ymax = BC_KINDS[get("bc_ymax", None) or ("wall" if ywall else "periodic")]
    ref = get("ref", None)
    if ref is not None:
        for m in range(5):
            c.ref[m] = ref[m]
    c.shock = int(bool(get("shock", False)))
    c.shock_theta = get("shock_theta", 0.0)
    c.shock_ximp = get("shock_ximp", 0.0)
    c.i_recycle = get("i_recycle", 0)
    c.delta_in = get("delta_in", 1.0)
    c.df_ny, c.df_nz = get("df_ny", 0), get("df_nz", 0)
    c.df_tau, c.df_seed = get("df_tau", 0.0), get("df_seed", 0)
    c.gamma, c.prandtl = get("gamma"), get("prandtl")
    c.r_gas = get("r_gas")
    c.visc_law = VISC_LAWS[get("visc_law", "power")]
    c.mu_ref, c.t_ref = get("mu_ref"), get("t_ref", 1.0)
    c.visc_exp, c.suth_s = get("visc_exp", 0.76), get("suth_s", 0.0)
    c.t_wall = get("t_wall", 1.0)
    c.forcing = int(bool(get("forcing", False)))
    c.L = get("L", 3)
    wm = get("weno_mode", "sensor")
    c.weno_mode = WENO_MODES[wm] if isinstance(wm, str) else int(wm)
    c.theta_thr, c.weno_eps = get("theta_thr", 0.05), get("weno_eps", 1e-6)
    c.u0, c.l0 = get("u0", 1.0), get("l0", 1.0)
    c.convective = int(bool(get("convective", True)))
    c.viscous = int(bool(get("viscous", True)))
    th = over.get("theta_fixed")
    if th is not None:
        th = np.ascontiguousarray(th, dtype=np.float64)
        assert th.shape == (c.nz, c.ny, c.nx), th.shape
        c.theta_fixed = _dp(th)
        c._theta = th  # keep the array alive with the configuration
    if df is not None:
        c.df_prof = _dp(df.prof)
        c.df_psi = _dp(df.psi)
        c.df_count = df.count.ctypes.data_as(ctypes.POINTER(ctypes.c_longlong))
        c._df = df  # keep the arrays alive with the configuration
        if df.count[0] == 0 and c.bc_xmin == BC_KINDS["df"]:
            if lib().orc_df_init(ctypes.byref(c)):
                raise ValueError("orc_df_init: invalid digital-filter configuration")
    return c


def _state(cfg, w):
    w = np.ascontiguousarray(w, dtype=np.float64)
    assert w.shape == (5, cfg.nz, cfg.ny, cfg.nx), w.shape
    return w


def rhs(cfg, w):
    w = _state(cfg, w)
    r = np.empty_like(w)
    if lib().orc_rhs(ctypes.byref(cfg), _dp(w), _dp(r)):
        raise ValueError("orc_rhs: invalid configuration")
    return r


def rk_step(cfg, w, dt=0.0, cfl=0.8):
    """One RK3 step; returns (new state, dt used)."""
    w = _state(cfg, w).copy()
    used = ctypes.c_double(0.0)
    if lib().orc_rk_step(ctypes.byref(cfg), _dp(w), float(dt), float(cfl), ctypes.byref(used)):
        raise ValueError("orc_rk_step: invalid configuration")
    return w, used.value


def advance(cfg, w, nsteps, dt=0.0, cfl=0.8):
    """n RK3 steps; returns (state, elapsed time, list of dt)."""
    t, dts = 0.0, []
    for _ in range(nsteps):
        w, h = rk_step(cfg, w, dt, cfl)
        t += h
        dts.append(h)
    return w, t, dts


def rk_stage_update(stage, dt, w, r_old, r):
    w = np.ascontiguousarray(w, dtype=np.float64).copy()
    r_old = np.ascontiguousarray(r_old, dtype=np.float64)
    r = np.ascontiguousarray(r, dtype=np.float64)
    lib().orc_rk_stage_update(int(stage), float(dt), _dp(w), _dp(r_old), _dp(r), w.size)
    return w


def cfl_dt(cfg, w, cfl=0.8):
    w = _state(cfg, w)
    return lib().orc_cfl_dt(ctypes.byref(cfg), _dp(w), float(cfl))


def totals(cfg, w):
    w = _state(cfg, w)
    out = np.zeros(5)
    lib().orc_totals(ctypes.byref(cfg), _dp(w), _dp(out))
    return out


def sensor(cfg, w):
    """Returns (theta, div, flags_x, flags_y, flags_z); see strm_oracle.h for flag layout."""
    w = _state(cfg, w)
    nx, ny, nz = cfg.nx, cfg.ny, cfg.nz
    th = np.empty((nz, ny, nx))
    dv = np.empty((nz, ny, nx))
    fx = np.zeros((nz, ny, nx + 1), np.uint8)
    fy = np.zeros((nz, ny + 1, nx), np.uint8)
    fz = np.zeros((nz + 1, ny, nx), np.uint8)
    if lib().orc_sensor(ctypes.byref(cfg), _dp(w), _dp(th), _dp(dv), _u8(fx), _u8(fy), _u8(fz)):
        raise ValueError("orc_sensor: invalid configuration")
    return th, dv, fx, fy, fz


def fill_ghosts(cfg, w):
    w = _state(cfg, w)
    G = lib().orc_ghosts()
    out = np.empty((5, cfg.nz + 2 * G, cfg.ny + 2 * G, cfg.nx + 2 * G))
    lib().orc_fill_ghosts(ctypes.byref(cfg), _dp(w), _dp(out))
    return out


def ghosts():
    return lib().orc_ghosts()


def metrics(cfg):
    y, ye, yee = np.empty(cfg.ny), np.empty(cfg.ny), np.empty(cfg.ny)
    lib().orc_metrics(ctypes.byref(cfg), _dp(y), _dp(ye), _dp(yee))
    return y, ye, yee


def eigvecs(direction, gamma, u, v, w, H):
    Lm, Rm = np.empty(25), np.empty(25)
    lib().orc_eigvecs(int(direction), gamma, u, v, w, H, _dp(Lm), _dp(Rm))
    return Lm.reshape(5, 5), Rm.reshape(5, 5)


def oblique_shock(gamma, mach, theta):
    """(beta, p2/p1, rho2/rho1, M2) of the weak oblique shock; theta in radians."""
    out = [ctypes.c_double() for _ in range(4)]
    if lib().orc_oblique_shock(gamma, mach, theta, *[ctypes.byref(o) for o in out]):
        raise ValueError("deflection beyond the attached-shock limit")
    return tuple(o.value for o in out)


def recycle_scale(cfg, w):
    return lib().orc_recycle_scale(ctypes.byref(cfg), _dp(_state(cfg, w)))


STAT_NAMES = ["rho", "u", "v", "w", "p", "T", "rho_u", "rho_v", "rho_w", "rho_T", "rho_uu",
              "rho_vv", "rho_ww", "rho_uv", "rho_uw", "rho_vw", "uu", "vv", "ww", "uv", "pp", "TT",
              "rhorho", "mu"]


def stats(cfg, w, mode=0):
    """Means of the STAT_NAMES quantities of one state over x and z ([24, ny], mode 0) or over
    z ([24, ny, nx], mode 1)."""
    w = _state(cfg, w)
    shape = (len(STAT_NAMES), cfg.ny) if mode == 0 else (len(STAT_NAMES), cfg.ny, cfg.nx)
    out = np.empty(shape)
    if lib().orc_stats(ctypes.byref(cfg), _dp(w), int(mode), _dp(out)):
        raise ValueError("orc_stats: invalid configuration or mode")
    return out


def splitmix64(seed, k):
    return lib().orc_splitmix64(int(seed), int(k))


def df_plane(cfg, draw):
    """Filtered random plane psi[3, nz, ny] of draw number `draw` (no time correlation)."""
    out = np.empty((3, cfg.nz, cfg.ny))
    if lib().orc_df_plane(ctypes.byref(cfg), int(draw), _dp(out)):
        raise ValueError("orc_df_plane: invalid configuration")
    return out


def weno5(f, eps=1e-6):
    f = np.ascontiguousarray(f, dtype=np.float64)
    assert f.size == 5
    return lib().orc_weno5(_dp(f), float(eps))


def threads():
    """Threads the oracle's OpenMP loops use."""
    return lib().orc_set_threads(0)


def set_threads(n):
    """Use n threads in the oracle's OpenMP loops (timing only; results do not depend on it)."""
    return lib().orc_set_threads(int(n))
