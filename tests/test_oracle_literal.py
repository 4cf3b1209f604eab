"""The oracle's point updates against the paper's formulas as printed, in
exact arithmetic.

The oracle evaluates each scheme in one fixed rounding order, regrouped from
the printed formulas by exact identities (heat as T + Fo(T+ - 2T + T-), KS as
one five-point stencil sharing the factor v+ + v- with the nonlinear term,
Euler with reciprocals for its divisions).  Here one stage at one point is
evaluated from the formulas of Appendices A-C in the paper's own grouping,
without rounding (fractions for heat and KS, 60-digit arithmetic for Euler,
whose square roots are irrational), on a thousand seeded stencils, and the
oracle's FP64 stage must be within 4 ulp of it, the ulp taken at the scale of
the printed formula (the sum of the magnitudes of its terms, base value
included): random stencils can cancel the terms to a result near zero, and an
evaluation in any fixed order is only accurate relative to that scale.  A regrouping that is not an
identity of the printed formula (a dropped or changed term), or one that
loses accuracy, fails here even where the equation-level pins still pass;
every later change of the oracle's grouping must keep this test green."""
import math
from fractions import Fraction as Fr

import numpy as np
import pytest

import oracle as O
from helpers import oprob
from paper_1705_03162_gb300 import inputs as I

ULPS = 4
COUNT = 1000


def _ulps(got: float, exact: Fr, scale: Fr) -> float:
    """|got - exact| in ulps of the formula's scale."""
    return float(abs(Fr(got) - exact) / Fr(math.ulp(float(scale))))


@pytest.mark.parametrize("dx,alpha,r", [(1.0 / 1024, 1.0, 0.25), (0.37, 0.9, 0.31)])
def test_heat_stage_is_the_printed_ftcs_formula(dx, alpha, r):
    """Appendix A, Eq. heatdisc: T' = Fo (T_{i+1} + T_{i-1}) + (1 - 2 Fo) T_i."""
    dt = r * dx * dx / alpha
    spec = I.ProblemSpec("heat", "periodic", 64, dx, dt, alpha=alpha)
    prob = oprob(spec)
    rng = np.random.default_rng(11)
    fo = Fr(alpha) * Fr(dt) / (Fr(dx) * Fr(dx))
    worst = 0.0
    for _ in range(COUNT):
        v = rng.uniform(-1.0, 1.0, 3)
        got = O.stage(prob, 0, v[:, None], v[1:2])[0]
        tm, t0, tp = (Fr(float(x)) for x in v)
        exact = fo * (tp + tm) + (1 - 2 * fo) * t0
        scale = abs(fo) * (abs(tp) + abs(tm)) + abs(1 - 2 * fo) * abs(t0)
        worst = max(worst, _ulps(got, exact, scale))
    assert worst <= ULPS, worst


@pytest.mark.parametrize("dx,dt", [(0.5, 0.005), (0.37, 0.0021)])
@pytest.mark.parametrize("stage", [0, 1])
def test_ks_stage_is_the_printed_discretisation(dx, dt, stage):
    """Appendix B, Eq. KSDisc with the midpoint RK2 stages (Eqs. RKm, RKf):
    out = base + h f, h = dt/2 (predictor) or dt (final), with
    f = -[(u+^2 - u-^2)/(4dx) + (u+ - 2u + u-)/dx^2 + (u++ - 4u+ + 6u - 4u- + u--)/dx^4]."""
    spec = I.ProblemSpec("ks", "periodic", 64, dx, dt)
    prob = oprob(spec)
    rng = np.random.default_rng(17 + stage)
    X, T = Fr(dx), Fr(dt)
    h = T / 2 if stage == 0 else T
    worst = 0.0
    for _ in range(COUNT):
        v = rng.uniform(-1.0, 1.0, 5)
        base = rng.uniform(-2.0, 2.0, 1)
        got = O.stage(prob, stage, v[:, None], base)[0]
        vmm, vm, v0, vp, vpp = (Fr(float(x)) for x in v)
        f = -((vp * vp - vm * vm) / (4 * X) + (vp - 2 * v0 + vm) / (X * X)
              + (vpp - 4 * vp + 6 * v0 - 4 * vm + vmm) / (X ** 4))
        b0 = Fr(float(base[0]))
        exact = b0 + h * f
        a = [abs(x) for x in (vmm, vm, v0, vp, vpp)]
        scale = abs(b0) + h * ((a[3] ** 2 + a[1] ** 2) / (4 * X) + (a[3] + 2 * a[2] + a[1]) / (X * X)
                               + (a[4] + 4 * a[3] + 6 * a[2] + 4 * a[1] + a[0]) / (X ** 4))
        worst = max(worst, _ulps(got, exact, scale))
    assert worst <= ULPS, worst


def _euler_literal(mp, q, base, gamma, h_over_dx):
    """One Euler stage at the centre of five cells q (5 x 3, conserved), from
    Appendix C as printed, at mpmath precision: pressure Eq. EulerP, pressure
    ratio and limited states Eqs. Pratio / limitleft / limitright, flux
    F = (rho u, rho u^2 + P, u (E + P)), Rusanov interface flux with the
    spectral radius of the Roe-averaged state (sqrt(rho) weights on u and on
    e = E / rho), finite-volume update."""
    g = mp.mpf(gamma)
    Q = [[mp.mpf(float(x)) for x in cell] for cell in q]

    def pressure(c):
        r, m, E = c
        return (g - 1) * (E - m * m / (2 * r))

    P = [pressure(c) for c in Q]

    def limited(a):
        # interface between cells a and a+1
        qa, qb = Q[a], Q[a + 1]
        num, den = P[a + 1] - P[a], P[a] - P[a - 1]
        if num * den > 0:
            phi = min(num / den, 1)
            ql = [x + phi / 2 * (y - x) for x, y in zip(qa, qb)]
        else:
            ql = list(qa)
        num2, den2 = P[a + 2] - P[a + 1], P[a + 1] - P[a]   # ratio at cell a+1
        if num2 * den2 > 0:
            psi = min(den2 / num2, 1)                        # its inverse
            qr = [y + psi / 2 * (x - y) for x, y in zip(qa, qb)]
        else:
            qr = list(qb)
        return ql, qr

    def flux(c):
        r, m, E = c
        u = m / r
        p = pressure(c)
        return [m, m * u + p, u * (E + p)]

    def interface(a, mag=False):
        ql, qr = limited(a)
        rl, rr = ql[0], qr[0]
        ul, ur = ql[1] / rl, qr[1] / rr
        el, er = ql[2] / rl, qr[2] / rr
        sl, sr = mp.sqrt(rl), mp.sqrt(rr)
        usp = (sl * ul + sr * ur) / (sl + sr)
        esp = (sl * el + sr * er) / (sl + sr)
        rsp_rho = mp.sqrt(rl * rr)
        psp = (g - 1) * rsp_rho * (esp - usp * usp / 2)
        rsp = mp.sqrt(g * psp / rsp_rho) + abs(usp)
        fl, fr = flux(ql), flux(qr)
        if mag:   # magnitudes of the terms
            return [(abs(fr[k]) + abs(fl[k]) + rsp * (abs(ql[k]) + abs(qr[k]))) / 2 for k in range(3)]
        return [(fr[k] + fl[k] + rsp * (ql[k] - qr[k])) / 2 for k in range(3)]

    fm, fp = interface(1), interface(2)
    am, ap = interface(1, True), interface(2, True)
    b = [mp.mpf(float(base[k])) for k in range(3)]
    h = mp.mpf(h_over_dx)
    return ([b[k] - h * (fp[k] - fm[k]) for k in range(3)],
            [abs(b[k]) + h * (ap[k] + am[k]) for k in range(3)])


@pytest.mark.parametrize("stage", [0, 1])
def test_euler_stage_is_the_printed_scheme(stage):
    mpmath = pytest.importorskip("mpmath")
    mp = mpmath.mp
    mp.dps = 60
    gamma, N = 1.4, 1024
    spec = I.sod_spec(N, bc="periodic")
    prob = oprob(spec)
    h_over_dx = (Fr(spec.dt) / 2 if stage == 0 else Fr(spec.dt)) / Fr(spec.dx)
    rng = np.random.default_rng(23 + stage)
    worst = 0.0
    for _ in range(COUNT):
        rho = rng.uniform(1.0, 2.0, 5)
        u = rng.uniform(-0.8, 0.8, 5)
        p = rng.uniform(0.5, 2.0, 5)
        q = np.stack([rho, rho * u, p / (gamma - 1) + 0.5 * rho * u * u], axis=1)
        base = q[2] if stage == 0 else q[2] * rng.uniform(0.9, 1.1, 3)
        got = O.stage(prob, stage, q, base)
        exact, scale = _euler_literal(mp, q, base, gamma, mp.mpf(h_over_dx.numerator) / h_over_dx.denominator)
        for k in range(3):
            ulp = math.ulp(float(scale[k]))
            worst = max(worst, float(abs(mp.mpf(float(got[k])) - exact[k]) / ulp))
    assert worst <= ULPS, worst
