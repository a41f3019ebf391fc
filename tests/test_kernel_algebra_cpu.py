"""Algebraic identities behind the rewritten formulas of the CUDA kernels, checked symbolically
(no GPU): each rewrite must equal the textbook form it replaces, so that the kernels compute the
oracle's quantities up to rounding.

* WENO5 (Jiang-Shu, Section 2.1): the smoothness indicators as completed squares in the first
  differences a..d of the stencil, and the candidate numerators carried by the kernel;
* the acoustic difference rows of the characteristic projection written with the stored
  momentum rho u_n and normal momentum flux rho u_n^2 + p;
* the Laplacian with one shared centre term.
"""
import sympy as sp

f0, f1, f2, f3, f4 = sp.symbols("f0:5", real=True)
a, b, c, d = f1 - f0, f2 - f1, f3 - f2, f4 - f3
R = sp.Rational


def test_weno5_indicators_completed_squares():
    beta0 = R(13, 12) * (f0 - 2 * f1 + f2) ** 2 + R(1, 4) * (f0 - 4 * f1 + 3 * f2) ** 2
    beta1 = R(13, 12) * (f1 - 2 * f2 + f3) ** 2 + R(1, 4) * (f1 - f3) ** 2
    beta2 = R(13, 12) * (f2 - 2 * f3 + f4) ** 2 + R(1, 4) * (3 * f2 - 4 * f3 + f4) ** 2
    k = R(39, 64)
    q0 = (a - R(11, 8) * b) ** 2 + k * b ** 2
    q1 = (b - R(5, 8) * c) ** 2 + k * c ** 2
    q2 = (d - R(11, 8) * c) ** 2 + k * c ** 2
    for beta, q in ((beta0, q0), (beta1, q1), (beta2, q2)):
        assert sp.expand(R(3, 4) * beta - q) == 0


def test_weno5_candidate_numerators():
    p0 = (2 * f0 - 7 * f1 + 11 * f2) / 6
    p1 = (-f1 + 5 * f2 + 2 * f3) / 6
    p2 = (2 * f2 + 5 * f3 - f4) / 6
    e0 = a - R(5, 2) * b
    e1 = -3 * b - 6 * c
    e2 = R(3, 2) * d - 6 * c
    assert sp.expand(e0 + 3 * (p0 - f2)) == 0
    assert sp.expand(e1 + 18 * (p1 - f2)) == 0
    assert sp.expand(e2 + 9 * (p2 - f2)) == 0
    # with weights (w0, 6 v1, 3 v2) proportional to the normalised ones, the value is
    # f2 - num / (3 den)
    w0, v1, v2 = sp.symbols("w0 v1 v2", positive=True)
    den = w0 + 6 * v1 + 3 * v2
    num = w0 * e0 + v1 * e1 + v2 * e2
    value = (w0 * p0 + 6 * v1 * p1 + 3 * v2 * p2) / den
    assert sp.simplify(value - (f2 - num / (3 * den))) == 0


def test_acoustic_rows_from_stored_momentum_flux():
    rho, un, uan, p = sp.symbols("rho u_n ua_n p", real=True)
    m = rho * un               # stored rho u_n
    mflux = rho * un ** 2 + p  # stored rho u_n^2 + p
    cBw = rho * (uan - un)
    cBf = rho * un * (uan - un) - p
    assert sp.expand(cBw - (rho * uan - m)) == 0
    assert sp.expand(cBf - (m * uan - mflux)) == 0


def test_laplacian_shared_centre_term():
    L = 3
    bl = [R(-49, 18), R(3, 2), R(-3, 20), R(1, 90)]
    fx = sp.symbols("x_m3 x_m2 x_m1 c x_p1 x_p2 x_p3", real=True)
    fy = sp.symbols("y_m3 y_m2 y_m1 y_p1 y_p2 y_p3", real=True)
    fz = sp.symbols("z_m3 z_m2 z_m1 z_p1 z_p2 z_p3", real=True)
    f0 = fx[3]
    ix, iy, iz, c2 = sp.symbols("ix2 iy2 iz2 c2", positive=True)
    xp = {l: fx[3 + l] for l in range(1, L + 1)}
    xm = {l: fx[3 - l] for l in range(1, L + 1)}
    yp = {l: fy[2 + l] for l in range(1, L + 1)}
    ym = {l: fy[3 - l] for l in range(1, L + 1)}
    zp = {l: fz[2 + l] for l in range(1, L + 1)}
    zm = {l: fz[3 - l] for l in range(1, L + 1)}
    # difference form per direction: sum_l b_l (f_+l + f_-l - 2 f0)
    d2 = lambda P, M: sum(bl[l] * (P[l] + M[l] - 2 * f0) for l in range(1, L + 1))
    lap_ref = d2(xp, xm) * ix + d2(yp, ym) * c2 + d2(zp, zm) * iz
    # kernel form: cc f0 + sum bx (x pairs) + sum bz (z pairs) + c2 sum b (y pairs),
    # cc = b0 (1/dx^2 + 1/dz^2 + c2), b0 = -2 sum_l b_l
    assert bl[0] == -2 * sum(bl[1:])
    cc = bl[0] * ix + bl[0] * iz + bl[0] * c2
    lap = cc * f0 + sum(bl[l] * ix * (xp[l] + xm[l]) + bl[l] * iz * (zp[l] + zm[l])
                        for l in range(1, L + 1)) + c2 * sum(bl[l] * (yp[l] + ym[l]) for l in range(1, L + 1))
    assert sp.expand(lap - lap_ref) == 0


def _recip5_emulated(y, guard=True):
    """The WENO kernel's shared reciprocal of five positive doubles, emulated bit for bit in
    numpy: mantissas brought to [1, 2) by rewriting the exponent field, inverted together by
    prefix products and one division, exponents restored by an integer subtraction; with the
    guard, inputs outside the valid exponent range go through plain division."""
    import numpy as np

    y = np.asarray(y, dtype=np.float64)
    bits = y.view(np.uint64)
    hi = (bits >> np.uint64(32)).astype(np.uint64)
    field = hi >> np.uint64(20)
    if guard and not np.all((field >= 1) & (field <= 2044)):
        return 1.0 / y
    e = (field & np.uint64(0x7FF)).astype(np.int64) - 1023
    mbits = (bits & np.uint64(0x000FFFFFFFFFFFFF)) | np.uint64(0x3FF0000000000000)
    m = mbits.view(np.float64)
    p1 = m[0] * m[1]
    p2 = p1 * m[2]
    p3 = p2 * m[3]
    p4 = p3 * m[4]
    inv = 1.0 / p4
    i4 = inv * p3
    inv *= m[4]
    i3 = inv * p2
    inv *= m[3]
    i2 = inv * p1
    inv *= m[2]
    i1, i0 = inv * m[0], inv * m[1]
    im = np.array([i0, i1, i2, i3, i4]).view(np.uint64)
    out = (im - (e.astype(np.uint64) << np.uint64(52))) & np.uint64(0xFFFFFFFFFFFFFFFF)
    return out.view(np.float64)


def test_recip5_extreme_magnitudes():
    """Inside [2^-1022, 2^1022) the exponent-field reciprocal agrees with 1/y to a few ulp
    (three roundings of the prefix products); at 2^1022 and above, and for zeros and
    subnormals, the exponent subtraction wraps and gives a wrong value, which is why the kernel
    checks the range and divides plainly there. The guarded form is 1/y to a few ulp everywhere."""
    import numpy as np

    rng = np.random.default_rng(0)
    ok = np.exp2(rng.uniform(-1021.9, 1021.9, size=(200, 5)))
    for y in ok:
        np.testing.assert_allclose(_recip5_emulated(y, guard=False), 1.0 / y, rtol=8e-16, atol=0.0)
    extremes = [
        [1.5 * 2.0 ** 1022, 1.0, 3.0, 5.0, 7.0],    # reciprocal below 2^-1022
        [1.5 * 2.0 ** 1023, 1.0, 2.0, 3.0, 4.0],    # reciprocal subnormal
        [5e-324, 1.0, 2.0, 3.0, 4.0],               # subnormal input
        [0.0, 1.0, 2.0, 3.0, 4.0],
        [np.inf, 1.0, 2.0, 3.0, 4.0],
    ]
    with np.errstate(all="ignore"):
        wrong = [not np.allclose(_recip5_emulated(np.array(y), guard=False), 1.0 / np.array(y),
                                 rtol=1e-15, atol=0.0, equal_nan=True) for y in extremes]
        assert all(wrong)
        for y in extremes:
            y = np.array(y)
            np.testing.assert_allclose(_recip5_emulated(y), 1.0 / y, rtol=8e-16, atol=0.0)


def test_pow_19_25_series_and_accuracy():
    """The primitives kernel takes t^0.76 (t^(19/25), the power-law viscosity of the workloads) as an
    FP32 seed y0 corrected by y = y0 (1 + d)^(1/25), d = t^19 / y0^25 - 1, with the binomial series
    to third order. The coefficients are the series' own; emulated in numpy (FP32 seed, powers by
    repeated squaring, reciprocal to 2^-43) the result is within 2 ulp of t**0.76 over the range
    the kernel uses it in, [2^-6, 2^6], for seeds up to 1e-6 off."""
    import numpy as np

    d = sp.symbols("d")
    series = sp.series((1 + d) ** sp.Rational(1, 25), d, 0, 4).removeO()
    c1, c2, c3 = (series.coeff(d, n) for n in (1, 2, 3))
    assert (c1, c2, c3) == (sp.Rational(1, 25), sp.Rational(-12, 625), sp.Rational(196, 15625))
    rng = np.random.default_rng(1)
    t = np.exp(rng.uniform(np.log(2.0 ** -6), np.log(2.0 ** 6), 100000))
    ref = t ** 0.76
    for pert in (-1e-6, 0.0, 1e-6):
        seed32 = np.exp2(np.float32(0.76) * np.log2(t.astype(np.float32)))
        y0 = (seed32.astype(np.float64) * (1 + pert)).astype(np.float32).astype(np.float64)
        t2 = t * t
        t4 = t2 * t2
        t8 = t4 * t4
        t16 = t8 * t8
        t19 = (t16 * t2) * t
        y2 = y0 * y0
        y4 = y2 * y2
        y8 = y4 * y4
        y16 = y8 * y8
        y25 = (y16 * y8) * y0
        inv = (1.0 / y25) * (1 + rng.uniform(-2.0 ** -43, 2.0 ** -43, t.shape))
        dl = (t19 - y25) * inv
        y = y0 + (y0 * dl) * (float(c1) + dl * (float(c2) + float(c3) * dl))
        assert np.all(np.abs(y - ref) <= 2 * np.spacing(ref)), pert


def test_x_flux_deviation_form():
    """The mixed x faces' split flux in deviation form (central_flux_xdev): around a reference
    (rho_0, u_0, H_0) constant along the row, with v_0 = w_0 = 0, each pair's contribution
    q (phi_a + phi_b), q = a (rho_a + rho_b)(u_a + u_b), equals the kernel's
    K S_phi + q' (2 phi_0 + S_phi) for phi = u, H and (K + q') S_phi for v, w, plus the constant
    K (1, 2 u_0, 0, 0, 2 H_0) the kernel leaves out (K = 4 a rho_0 u_0, q' as in the kernel), and
    the left-out constants of a face add up to (rho_0 u_0)(1, u_0, 0, 0, H_0) times 8 sum_l l a_l
    (for f_rho: twice the sum of K over the pairs), the x WENO faces' offset."""
    a, r0, u0, H0 = sp.symbols("a rho0 u0 H0")
    dra, drb, dua, dub, dHa, dHb, va, vb = sp.symbols("dra drb dua dub dHa dHb va vb")
    Sr, Su, SH, Sv = dra + drb, dua + dub, dHa + dHb, va + vb
    q = a * (2 * r0 + Sr) * (2 * u0 + Su)
    K = 4 * a * r0 * u0
    qp = a * (Su * (2 * r0 + Sr) + 2 * u0 * Sr)
    assert sp.expand(q - (K + qp)) == 0
    assert sp.expand(q * (2 * u0 + Su) - (K * Su + qp * (2 * u0 + Su) + K * 2 * u0)) == 0
    assert sp.expand(q * (2 * H0 + SH) - (K * SH + qp * (2 * H0 + SH) + K * 2 * H0)) == 0
    assert sp.expand(q * Sv - (K + qp) * Sv) == 0
    # the constant per face: pairs (l, m), m < l, each with its own K_l = 4 a_l rho0 u0
    for L in (2, 3):
        al = sp.symbols(f"a1:{L + 1}")
        pairs = [(l, m) for l in range(1, L + 1) for m in range(l)]
        f_rho_const = 2 * sum(4 * al[l - 1] * r0 * u0 for l, m in pairs)
        f_u_const = sum(4 * al[l - 1] * r0 * u0 * 2 * u0 for l, m in pairs)
        s8 = 8 * sum(l * al[l - 1] for l in range(1, L + 1))
        assert sp.expand(f_rho_const - s8 * r0 * u0) == 0
        assert sp.expand(f_u_const - s8 * r0 * u0 * u0) == 0
