"""Exact solution of the Riemann problem for the 1D Euler equations (ideal gas).

Written from the textbook construction: the star-region pressure p* is the root
of f_L(p) + f_R(p) + (u_R - u_L) = 0, where f_K is the shock (Rankine-Hugoniot)
branch for p > p_K and the rarefaction (isentropic, Riemann invariant) branch
for p <= p_K; Newton iteration from the two-rarefaction guess.  The solution is
self-similar in x/t.  Used as a pin for the Sod shock-tube test of
arXiv:1705.03162 Appendix C (Eq. SodCond).
"""
from __future__ import annotations

import math

import numpy as np


def _fk(p, rho, pk, ck, g):
    """Pressure function f_K and its derivative for one side."""
    if p > pk:
        a = 2.0 / ((g + 1.0) * rho)
        b = (g - 1.0) / (g + 1.0) * pk
        s = math.sqrt(a / (p + b))
        return (p - pk) * s, s * (1.0 - 0.5 * (p - pk) / (p + b))
    e = (g - 1.0) / (2.0 * g)
    f = 2.0 * ck / (g - 1.0) * ((p / pk) ** e - 1.0)
    df = (p / pk) ** (-(g + 1.0) / (2.0 * g)) / (rho * ck)
    return f, df


def star_state(left, right, gamma=1.4, tol=1e-14, maxit=100):
    """(p*, u*) for primitive states left = (rho, u, p), right = (rho, u, p)."""
    rl, ul, pl = left
    rr, ur, pr = right
    cl = math.sqrt(gamma * pl / rl)
    cr = math.sqrt(gamma * pr / rr)
    z = (gamma - 1.0) / (2.0 * gamma)
    # two-rarefaction approximation as the starting guess
    p = ((cl + cr - 0.5 * (gamma - 1.0) * (ur - ul)) / (cl / pl ** z + cr / pr ** z)) ** (1.0 / z)
    for _ in range(maxit):
        fl, dfl = _fk(p, rl, pl, cl, gamma)
        fr, dfr = _fk(p, rr, pr, cr, gamma)
        pn = p - (fl + fr + ur - ul) / (dfl + dfr)
        pn = max(pn, 1e-14)
        if abs(pn - p) <= tol * 0.5 * (pn + p):
            p = pn
            break
        p = pn
    fl, _ = _fk(p, rl, pl, cl, gamma)
    fr, _ = _fk(p, rr, pr, cr, gamma)
    return p, 0.5 * (ul + ur) + 0.5 * (fr - fl)


def sample(x, t, x0, left, right, gamma=1.4):
    """Primitive (rho, u, p) arrays of the exact solution at positions x, time t."""
    rl, ul, pl = left
    rr, ur, pr = right
    g = gamma
    cl = math.sqrt(g * pl / rl)
    cr = math.sqrt(g * pr / rr)
    ps, us = star_state(left, right, g)
    g6 = (g - 1.0) / (g + 1.0)
    out = np.empty((3, len(x)))
    for i, xi in enumerate(x):
        s = (xi - x0) / t
        if s <= us:   # left of the contact
            if ps > pl:   # left shock
                sl = ul - cl * math.sqrt((g + 1.0) / (2.0 * g) * ps / pl + (g - 1.0) / (2.0 * g))
                if s <= sl:
                    w = (rl, ul, pl)
                else:
                    w = (rl * (ps / pl + g6) / (g6 * ps / pl + 1.0), us, ps)
            else:         # left rarefaction
                shl = ul - cl
                cstar = cl * (ps / pl) ** ((g - 1.0) / (2.0 * g))
                stl = us - cstar
                if s <= shl:
                    w = (rl, ul, pl)
                elif s > stl:
                    w = (rl * (ps / pl) ** (1.0 / g), us, ps)
                else:
                    u = 2.0 / (g + 1.0) * (cl + 0.5 * (g - 1.0) * ul + s)
                    c = 2.0 / (g + 1.0) * (cl + 0.5 * (g - 1.0) * (ul - s))
                    w = (rl * (c / cl) ** (2.0 / (g - 1.0)), u, pl * (c / cl) ** (2.0 * g / (g - 1.0)))
        else:         # right of the contact
            if ps > pr:   # right shock
                sr = ur + cr * math.sqrt((g + 1.0) / (2.0 * g) * ps / pr + (g - 1.0) / (2.0 * g))
                if s >= sr:
                    w = (rr, ur, pr)
                else:
                    w = (rr * (ps / pr + g6) / (g6 * ps / pr + 1.0), us, ps)
            else:         # right rarefaction
                shr = ur + cr
                cstar = cr * (ps / pr) ** ((g - 1.0) / (2.0 * g))
                str_ = us + cstar
                if s >= shr:
                    w = (rr, ur, pr)
                elif s <= str_:
                    w = (rr * (ps / pr) ** (1.0 / g), us, ps)
                else:
                    u = 2.0 / (g + 1.0) * (-cr + 0.5 * (g - 1.0) * ur + s)
                    c = 2.0 / (g + 1.0) * (cr - 0.5 * (g - 1.0) * (ur - s))
                    w = (rr * (c / cr) ** (2.0 / (g - 1.0)), u, pr * (c / cr) ** (2.0 * g / (g - 1.0)))
        out[:, i] = w
    return out
