"""Manufactured solutions for the oracle pins: exact right-hand sides by symbolic calculus.

The exact residual is built from the conservation form of the Navier-Stokes equations
(Eqs. 1a-c with sigma_ij and q_j as defined in Section 2), not from the Laplacian form the
scheme uses, so a dropped term, a wrong sign or a transposed index in the discrete viscous
terms shows up as an O(1) error instead of an error that vanishes with the grid spacing.

Fields are smooth and periodic in (x, eta, z); the wall-normal coordinate is y(eta) with the
tanh map, and d/dy = (1/y_eta) d/deta with y_eta obtained by differentiating y(eta).
"""
import functools

import numpy as np
import sympy as sp

x, eta, z = sp.symbols("x eta z", real=True)


def _fields(lx, lz):
    kx, kz, ke = 2 * sp.pi / lx, 2 * sp.pi / lz, 2 * sp.pi
    rho = 1 + sp.Rational(1, 10) * sp.sin(kx * x + sp.Rational(3, 10)) * sp.cos(ke * eta) \
        + sp.Rational(1, 20) * sp.cos(kz * z)
    u = sp.Rational(1, 2) + sp.Rational(1, 5) * sp.sin(ke * eta + sp.Rational(1, 10)) * sp.cos(kz * z) \
        + sp.Rational(1, 10) * sp.cos(kx * x)
    v = sp.Rational(1, 10) * sp.cos(kx * x) * sp.sin(ke * eta) + sp.Rational(1, 20) * sp.sin(kz * z + 1)
    w = sp.Rational(3, 20) * sp.sin(kx * x + ke * eta) + sp.Rational(1, 10) * sp.cos(kz * z) * sp.sin(kx * x)
    T = 1 + sp.Rational(1, 10) * sp.cos(ke * eta) * sp.sin(kx * x) + sp.Rational(1, 20) * sp.sin(kz * z)
    return rho, u, v, w, T


@functools.lru_cache(maxsize=None)
def build(lx, lz, ly, beta, gamma, r_gas, mu_ref, visc_exp, prandtl, convective, viscous,
          visc_law="power", suth_s=0.0):
    """Return callables (prims(X, ETA, Z), rhs(X, ETA, Z)) for the manufactured state."""
    rho, u, v, w, T = _fields(sp.nsimplify(lx), sp.nsimplify(lz))
    g = sp.Float(gamma)
    R = sp.Float(r_gas)
    cv = R / (g - 1)
    cp = g * R / (g - 1)
    if beta > 0:
        b = sp.Float(beta)
        y = sp.Float(ly) / 2 * sp.tanh(b * (2 * eta - 1)) / sp.tanh(b)
    else:
        y = sp.Float(ly) * (eta - sp.Rational(1, 2))
    yeta = sp.diff(y, eta)

    def D(f, d):
        if d == 0:
            return sp.diff(f, x)
        if d == 1:
            return sp.diff(f, eta) / yeta
        return sp.diff(f, z)

    vel = [u, v, w]
    p = rho * R * T
    E = cv * T + (u * u + v * v + w * w) / 2
    H = E + p / rho
    if visc_law == "power":
        mu = sp.Float(mu_ref) * T ** sp.Float(visc_exp)
    else:
        s = sp.Float(suth_s)
        mu = sp.Float(mu_ref) * T ** sp.Rational(3, 2) * (1 + s) / (T + s)
    k = cp * mu / sp.Float(prandtl)
    div = sum(D(vel[a], a) for a in range(3))
    sigma = [[mu * (D(vel[i], j) + D(vel[j], i) - (sp.Rational(2, 3) * div if i == j else 0))
              for j in range(3)] for i in range(3)]
    res = [sp.Integer(0)] * 5
    for j in range(3):
        if convective:
            res[0] -= D(rho * vel[j], j)
            for i in range(3):
                res[1 + i] -= D(rho * vel[j] * vel[i] + (p if i == j else 0), j)
            res[4] -= D(rho * vel[j] * H, j)
        if viscous:
            for i in range(3):
                res[1 + i] += D(sigma[i][j], j)
            res[4] += D(sum(sigma[i][j] * vel[i] for i in range(3)) + k * D(T, j), j)
    prims = sp.lambdify((x, eta, z), [rho, u, v, w, T], "numpy")
    rhs = sp.lambdify((x, eta, z), res, "numpy")
    return prims, rhs


def grid(nx, ny, nz, lx, lz):
    """Node coordinates matching the oracle: x_i = i dx, eta_j = (j+1/2)/ny, z_k = k dz."""
    X = (np.arange(nx) * (lx / nx))[None, None, :]
    ETA = ((np.arange(ny) + 0.5) / ny)[None, :, None]
    Z = (np.arange(nz) * (lz / nz))[:, None, None]
    shape = (nz, ny, nx)
    return (np.broadcast_to(X, shape), np.broadcast_to(ETA, shape), np.broadcast_to(Z, shape))
