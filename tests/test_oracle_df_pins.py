"""Pins of the oracle's digital-filter inflow (Section 3.2 names a Klein-type digital filter
done as one-dimensional convolutions, the strong Reynolds analogy and prescribed Reynolds
stresses; the formulas are the cited methods'): the generator against its published test
vector, the moments and two-point correlations of the filtered planes against those of the
filter, the time blending, the Cholesky (Lund) transform against numpy's Cholesky factor, and
the strong Reynolds analogy and constant pressure of the ghost states."""
import math
import os

import numpy as np
import pytest

from paper_2004_02276_gb300 import inputs

G3 = 3
HERE = os.path.dirname(os.path.abspath(__file__))


def df_case(**kw):
    base = dict(bc_xmin="df", df_ny=3, df_nz=2, df_tau=0.4, df_seed=11)
    base.update(kw)
    return inputs.bl_case("bl-df", 12, 40, 32, 2.0, 6.0, 1.5, **base)


def filter_coefs(n):
    l = np.arange(-2 * n, 2 * n + 1)
    b = np.exp(-math.pi * l ** 2 / (2.0 * n * n))
    return b / np.sqrt((b * b).sum())


def test_generator_test_vector(orc):
    want = [int(l, 16) for l in open(os.path.join(HERE, "golden", "splitmix64_seed0.txt"))
            if not l.startswith("#") and l.strip()]
    assert [orc.splitmix64(0, k) for k in range(3)] == want


def test_plane_moments_and_correlations(orc):
    c = df_case()
    cfg = orc.make_cfg(c, df=orc.DFState(c, inputs.df_profiles(c)))
    planes = np.array([orc.df_plane(cfg, d) for d in range(60)])  # [draw, m, k(z), j(y)]
    n = planes.size
    assert abs(planes.mean()) < 5 / math.sqrt(n) * 4  # correlated samples: generous bound
    assert abs(planes.var() - 1.0) < 0.03
    # two-point correlation along y and z: the autocorrelation of the filter coefficients
    for axis, nf in ((3, c.df_ny), (2, c.df_nz)):
        b = filter_coefs(nf)
        for lag in (1, 2, 3):
            want = (b[:-lag] * b[lag:]).sum()
            x = np.moveaxis(planes, axis, -1)
            got = (x[..., :-lag] * x[..., lag:]).mean()
            assert abs(got - want) < 0.04, (axis, lag, got, want)
    # different components and different draws are uncorrelated
    assert abs((planes[:, 0] * planes[:, 1]).mean()) < 0.04
    assert abs((planes[:-1] * planes[1:]).mean()) < 0.04


def test_time_blending(orc):
    """Fixed dt: the blended plane keeps unit variance and has the lag-one correlation
    exp(-pi dt / (2 tau)) between steps."""
    c = inputs.bl_case("bl-df-t", 8, 12, 16, 2.0, 6.0, 1.5, bc_xmin="df", df_ny=1, df_nz=1,
                       df_tau=0.05, df_seed=5)
    df = orc.DFState(c, inputs.df_profiles(c))
    cfg = orc.make_cfg(c, df=df)
    w = inputs.bl_state(c, 0)
    dt = 0.01
    series = [df.psi.copy()]
    for _ in range(150):
        w, _ = orc.rk_step(cfg, w, dt)
        series.append(df.psi.copy())
    s = np.array(series)
    assert df.count[0] == 151
    want = math.exp(-math.pi * dt / (2 * c.df_tau))
    got = (s[:-1] * s[1:]).mean() / s.var()
    assert abs(got - want) < 0.05, (got, want)
    assert abs(s.var() - 1.0) < 0.1


def test_ghost_states_lund_and_strong_reynolds_analogy(orc):
    c = df_case()
    prof = inputs.df_profiles(c)
    df = orc.DFState(c, prof)
    cfg = orc.make_cfg(c, df=df)
    st = inputs.bl_state(c, 0)
    wg = orc.fill_ghosts(cfg, st)
    cv = c.r_gas / (c.gamma - 1.0)
    cp = cv + c.r_gas
    U, V, T, R11, R12, R22, R33 = prof
    for q in range(G3):
        g = wg[:, G3:-G3, G3:-G3, G3 - 1 - q]  # ghost plane i = -1-q, [5, nz, ny]
        rho = g[0]
        u, v, w = g[1] / rho, g[2] / rho, g[3] / rho
        Tg = (g[4] / rho - 0.5 * (u * u + v * v + w * w)) / cv
        p = rho * c.r_gas * Tg
        np.testing.assert_allclose(p, c.ref[4], rtol=1e-13)  # constant pressure
        up = u - U[None, :]
        np.testing.assert_allclose(cp * (Tg - T[None, :]), -U[None, :] * up, atol=1e-12)  # SRA
        for j in range(0, c.ny, 5):
            if R11[j] == 0.0:  # at the wall: no fluctuation
                np.testing.assert_allclose(up[:, j], 0.0, atol=1e-14)
                continue
            R = np.array([[R11[j], R12[j], 0.0], [R12[j], R22[j], 0.0], [0.0, 0.0, R33[j]]])
            Lc = np.linalg.cholesky(R)
            want = Lc @ df.psi[:, :, j]  # [3, nz]
            got = np.stack([up[:, j], v[:, j] - V[j], w[:, j]])
            np.testing.assert_allclose(got, want, rtol=1e-11, atol=1e-14)
