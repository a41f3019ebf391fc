"""Pins of the oracle's per-sample statistics (Section 3: Reynolds averages over the homogeneous
directions, Favre averages rho phi / rho): closed-form means of a state whose fluctuations are
whole periods of cosines on the uniform directions, the identity of Favre and Reynolds means at
constant density, consistency of the two averaging modes, and brute force on a tiny state."""
import math

import numpy as np
import pytest

from paper_2004_02276_gb300 import inputs

NAMES = ["rho", "u", "v", "w", "p", "T", "rho_u", "rho_v", "rho_w", "rho_T", "rho_uu",
         "rho_vv", "rho_ww", "rho_uv", "rho_uw", "rho_vw", "uu", "vv", "ww", "uv", "pp", "TT",
         "rhorho", "mu"]


def cons(case, rho, u, v, w, T):
    cv = case.r_gas / (case.gamma - 1.0)
    return np.stack([rho, rho * u, rho * v, rho * w, rho * (cv * T + 0.5 * (u * u + v * v + w * w))])


def periodic_state(case, a=0.3, b=0.2, rho0=1.3):
    """rho = rho0, u = U(y) + a cos(kx x), v = b sin(kx x) cos(kz z), w = 0, T = T(y)."""
    nz, ny, nx = case.nz, case.ny, case.nx
    x = 2 * math.pi * np.arange(nx) / nx
    z = 2 * math.pi * np.arange(nz) / nz
    U = 1.0 + 0.5 * np.linspace(-1, 1, ny) ** 2
    Tj = 1.0 + 0.1 * np.linspace(0, 1, ny)
    shape = (nz, ny, nx)
    u = U[None, :, None] + a * np.cos(2 * x)[None, None, :]
    v = b * np.sin(x)[None, None, :] * np.cos(z)[:, None, None]
    w = np.zeros(shape)
    T = np.broadcast_to(Tj[None, :, None], shape)
    rho = np.full(shape, rho0)
    return cons(case, rho, u + 0 * w, v, w, T), U, Tj


def test_closed_form_means(orc):
    c = inputs.Case(nx=16, ny=7, nz=8, beta=0.0, y_wall=False)
    a, b, rho0 = 0.3, 0.2, 1.3
    st, U, Tj = periodic_state(c, a, b, rho0)
    s = dict(zip(NAMES, orc.stats(orc.make_cfg(c), st, 0)))
    mu = c.mu_ref * (Tj / c.t_ref) ** c.visc_exp
    want = {
        "rho": rho0, "u": U, "v": 0.0, "w": 0.0, "T": Tj, "p": rho0 * c.r_gas * Tj,
        "rho_u": rho0 * U, "rho_v": 0.0, "rho_T": rho0 * Tj,
        "uu": U ** 2 + a * a / 2, "vv": b * b / 4, "uv": 0.0, "ww": 0.0,
        "rho_uu": rho0 * (U ** 2 + a * a / 2), "rho_vv": rho0 * b * b / 4, "rho_uv": 0.0,
        "pp": (rho0 * c.r_gas * Tj) ** 2, "TT": Tj ** 2, "rhorho": rho0 ** 2, "mu": mu,
    }
    for k, v in want.items():
        np.testing.assert_allclose(s[k], np.broadcast_to(v, s[k].shape), atol=1e-13, rtol=1e-12,
                                   err_msg=k)
    # Favre mean of T equals its Reynolds mean at constant density
    np.testing.assert_allclose(s["rho_T"] / s["rho"], s["T"], rtol=1e-14)


def test_z_mode_means_and_mode_consistency(orc):
    c = inputs.Case(nx=6, ny=5, nz=12, beta=0.0, y_wall=False)
    st, U, Tj = periodic_state(c)
    cfg = orc.make_cfg(c)
    s1 = orc.stats(cfg, st, 1)
    assert s1.shape == (24, c.ny, c.nx)
    x = 2 * math.pi * np.arange(c.nx) / c.nx
    # over z only: v = b sin(x) cos(z) averages to 0, vv to b^2 sin^2(x) / 2
    np.testing.assert_allclose(s1[NAMES.index("v")], 0.0, atol=1e-15)
    np.testing.assert_allclose(s1[NAMES.index("vv")], np.broadcast_to(0.02 * np.sin(x) ** 2, (c.ny, c.nx)),
                               atol=1e-15)
    # the x-z mean is the x mean of the z means
    s0 = orc.stats(cfg, inputs.random_state(c, 3), 0)
    s1 = orc.stats(cfg, inputs.random_state(c, 3), 1)
    np.testing.assert_allclose(s0, s1.mean(axis=2), rtol=1e-13, atol=1e-15)


def test_brute_force_tiny(orc):
    c = inputs.Case(nx=4, ny=3, nz=5, beta=0.0, y_wall=False, visc_law="sutherland")
    st = inputs.random_state(c, 7)
    rho = st[0]
    u, v, w = st[1] / rho, st[2] / rho, st[3] / rho
    cv = c.r_gas / (c.gamma - 1.0)
    T = (st[4] / rho - 0.5 * (u * u + v * v + w * w)) / cv
    p = rho * c.r_gas * T
    tr = T / c.t_ref
    mu = c.mu_ref * tr ** 1.5 * (1 + c.suth_s) / (tr + c.suth_s)
    fields = [rho, u, v, w, p, T, rho * u, rho * v, rho * w, rho * T, rho * u * u, rho * v * v,
              rho * w * w, rho * u * v, rho * u * w, rho * v * w, u * u, v * v, w * w, u * v,
              p * p, T * T, rho * rho, mu]
    want = np.array([f.mean(axis=(0, 2)) for f in fields])
    np.testing.assert_allclose(orc.stats(orc.make_cfg(c), st, 0), want, rtol=1e-13)


def test_invalid_mode_rejected(orc):
    c = inputs.Case(nx=4, ny=3, nz=5, beta=0.0, y_wall=False)
    with pytest.raises(ValueError):
        orc.stats(orc.make_cfg(c), inputs.random_state(c, 0), 2)
