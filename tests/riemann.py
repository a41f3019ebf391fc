"""Exact solution of the Riemann problem for the 1D Euler equations of a perfect gas.

Pressure-function method with Newton iteration for the star pressure and the standard
sampling of the self-similar wave pattern (shock or rarefaction on each side). Used only by
the oracle's Sod shock-tube pin.
"""
import numpy as np


def _fk(p, rho, pk, ck, g):
    if p > pk:  # shock
        A = 2.0 / ((g + 1.0) * rho)
        B = (g - 1.0) / (g + 1.0) * pk
        f = (p - pk) * np.sqrt(A / (p + B))
        df = np.sqrt(A / (B + p)) * (1.0 - 0.5 * (p - pk) / (B + p))
    else:  # rarefaction
        f = 2.0 * ck / (g - 1.0) * ((p / pk) ** ((g - 1.0) / (2.0 * g)) - 1.0)
        df = 1.0 / (rho * ck) * (p / pk) ** (-(g + 1.0) / (2.0 * g))
    return f, df


def star_state(left, right, g=1.4, tol=1e-15):
    """(p*, u*) for left/right primitive states (rho, u, p)."""
    rl, ul, pl = left
    rr, ur, pr = right
    cl, cr = np.sqrt(g * pl / rl), np.sqrt(g * pr / rr)
    p = max(tol, 0.5 * (pl + pr))
    for _ in range(100):
        fl, dfl = _fk(p, rl, pl, cl, g)
        fr, dfr = _fk(p, rr, pr, cr, g)
        dp = (fl + fr + ur - ul) / (dfl + dfr)
        pn = max(tol, p - dp)
        if abs(pn - p) <= tol * 0.5 * (pn + p):
            p = pn
            break
        p = pn
    fl, _ = _fk(p, rl, pl, cl, g)
    fr, _ = _fk(p, rr, pr, cr, g)
    u = 0.5 * (ul + ur) + 0.5 * (fr - fl)
    return p, u


def sample(left, right, s, g=1.4):
    """Primitive state (rho, u, p) at similarity coordinate s = x/t (arrays allowed)."""
    rl, ul, pl = left
    rr, ur, pr = right
    cl, cr = np.sqrt(g * pl / rl), np.sqrt(g * pr / rr)
    ps, us = star_state(left, right, g)
    s = np.asarray(s, dtype=float)
    rho, u, p = np.empty_like(s), np.empty_like(s), np.empty_like(s)
    gm = (g - 1.0) / (g + 1.0)
    for idx, si in np.ndenumerate(s):
        if si <= us:  # left of the contact
            if ps > pl:  # left shock
                sl = ul - cl * np.sqrt((g + 1) / (2 * g) * ps / pl + (g - 1) / (2 * g))
                if si <= sl:
                    st = (rl, ul, pl)
                else:
                    st = (rl * (ps / pl + gm) / (gm * ps / pl + 1.0), us, ps)
            else:  # left rarefaction
                shl = ul - cl
                csl = cl * (ps / pl) ** ((g - 1) / (2 * g))
                stl = us - csl
                if si <= shl:
                    st = (rl, ul, pl)
                elif si >= stl:
                    st = (rl * (ps / pl) ** (1.0 / g), us, ps)
                else:
                    c = 2.0 / (g + 1) * (cl + (g - 1) / 2 * (ul - si))
                    uu = 2.0 / (g + 1) * (cl + (g - 1) / 2 * ul + si)
                    st = (rl * (c / cl) ** (2.0 / (g - 1)), uu, pl * (c / cl) ** (2 * g / (g - 1)))
        else:  # right of the contact
            if ps > pr:  # right shock
                sr = ur + cr * np.sqrt((g + 1) / (2 * g) * ps / pr + (g - 1) / (2 * g))
                if si >= sr:
                    st = (rr, ur, pr)
                else:
                    st = (rr * (ps / pr + gm) / (gm * ps / pr + 1.0), us, ps)
            else:  # right rarefaction
                shr = ur + cr
                csr = cr * (ps / pr) ** ((g - 1) / (2 * g))
                str_ = us + csr
                if si >= shr:
                    st = (rr, ur, pr)
                elif si <= str_:
                    st = (rr * (ps / pr) ** (1.0 / g), us, ps)
                else:
                    c = 2.0 / (g + 1) * (cr - (g - 1) / 2 * (ur - si))
                    uu = 2.0 / (g + 1) * (-cr + (g - 1) / 2 * ur + si)
                    st = (rr * (c / cr) ** (2.0 / (g - 1)), uu, pr * (c / cr) ** (2 * g / (g - 1)))
        rho[idx], u[idx], p[idx] = st
    return rho, u, p
