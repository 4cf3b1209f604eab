"""Pins of the CPU oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: closed-form
discrete solutions, invariants, textbook special cases, the exact Riemann
solution, brute-force equivalence of the swept and classic decompositions.
The schemes are those of arXiv:1705.03162 Appendices A-C; the swept rule is
Sections 4.2-4.3.  CPU only.
"""
import math

import numpy as np
import pytest

import oracle as O
import riemann_exact as R
from paper_1705_03162_gb300 import inputs as I

_EQ = {"heat": O.HEAT, "ks": O.KS, "euler": O.EULER}
_BC = {"periodic": O.PERIODIC, "reflective": O.REFLECTIVE, "dirichlet": O.DIRICHLET}


def oprob(spec: I.ProblemSpec) -> O.OracleProblem:
    return O.OracleProblem(_EQ[spec.eq], _BC[spec.bc], spec.n_points, spec.dx, spec.dt,
                           spec.alpha, spec.gamma, spec.left, spec.right)


def rel_max(a, b):
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


# --------------------------------------------------------------------------
# input generator
# --------------------------------------------------------------------------
def test_splitmix64_published_vector():
    # SplitMix64 from seed 0: first outputs of the reference generator
    out = I.splitmix64(0, 3)
    assert [int(v) for v in out] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


def test_uniform_field_is_counter_splitmix():
    # the vectorised counter form equals the sequential generator
    seq = I.uniform01(12345, 16)
    vec = (I.uniform_field(16, 12345, 0.0, 1.0))
    assert np.array_equal(seq, vec)


# --------------------------------------------------------------------------
# heat equation (Appendix A): FTCS amplification factor per Fourier mode
# --------------------------------------------------------------------------
@pytest.mark.parametrize("N,M", [(64, 100), (1024, 400)])
def test_heat_periodic_closed_form(N, M):
    """Mode sin(2 pi k x) evolves as G_k^M sin(2 pi k x), G_k = 1 - 4 r sin^2(pi k/N)."""
    spec = I.heat_spec(N, r=0.25)
    u = I.initial_state(spec)
    O.classic(oprob(spec), u, M)
    x = np.arange(N) / N
    G = lambda k: 1.0 - 4.0 * 0.25 * math.sin(math.pi * k / N) ** 2
    exact = np.sin(2 * math.pi * x) * G(1) ** M
    for k, a in zip(range(2, 10), I.heat_mode_amplitudes()):
        exact += a * np.sin(2 * math.pi * k * x) * G(k) ** M
    assert rel_max(u[0], exact) < 1e-12


@pytest.mark.parametrize("r", [0.1, 0.37, 0.5])
def test_heat_periodic_amplification_any_r(r):
    N, M, k = 48, 60, 5
    spec = I.heat_spec(N, r=r)
    x = np.arange(N) / N
    u = np.cos(2 * math.pi * k * x)[None, :].copy()
    O.classic(oprob(spec), u, M)
    G = 1.0 - 4.0 * r * math.sin(math.pi * k / N) ** 2
    assert np.max(np.abs(u[0] - G ** M * np.cos(2 * math.pi * k * x))) < 1e-12


def test_heat_reflective_cosine_mode():
    """With mirror ends T_{-1}=T_1, T_N=T_{N-2} (Eq. heatcond), cos(pi k i/(N-1)) is an
    eigenvector with factor 1 - 4 r sin^2(pi k / (2 (N-1)))."""
    N, M, k, r = 40, 80, 3, 0.3
    spec = I.heat_spec(N, r=r, bc="reflective")
    i = np.arange(N)
    theta = math.pi * k / (N - 1)
    u = np.cos(theta * i)[None, :].copy()
    O.classic(oprob(spec), u, M)
    G = 1.0 - 4.0 * r * math.sin(theta / 2) ** 2
    assert np.max(np.abs(u[0] - G ** M * np.cos(theta * i))) < 1e-12


def test_heat_reflective_trapezoid_sum_conserved():
    """Insulated ends conserve the trapezoid sum (end weights 1/2)."""
    N = 96
    spec = I.heat_spec(N, r=0.25, bc="reflective")
    u = I.initial_state(spec)
    w = np.ones(N)
    w[0] = w[-1] = 0.5
    s0 = float(np.dot(w, u[0]))
    O.classic(oprob(spec), u, 500)
    assert abs(float(np.dot(w, u[0])) - s0) < 1e-12


@pytest.mark.parametrize("bc", ["periodic", "reflective"])
def test_heat_constant_is_fixed_point(bc):
    spec = I.heat_spec(32, r=0.3, bc=bc)
    u = np.full((1, 32), 0.731)
    O.classic(oprob(spec), u, 50)
    assert np.all(u == 0.731)


def test_heat_fp32_tracks_fp64():
    spec = I.heat_spec(256)
    u64 = I.initial_state(spec)
    u32 = u64.astype(np.float32)
    O.classic(oprob(spec), u64, 200)
    O.classic(oprob(spec), u32, 200)
    assert rel_max(u32[0].astype(np.float64), u64[0]) < 1e-5


# --------------------------------------------------------------------------
# Kuramoto-Sivashinsky (Appendix B)
# --------------------------------------------------------------------------
def test_ks_constant_is_fixed_point():
    """Every stencil weight sums to zero (consistency): a constant stays constant
    up to the rounding of the combined weights."""
    spec = I.ks_spec(64)
    u = np.full((1, 64), -0.4321)
    O.classic(oprob(spec), u, 100)
    assert np.max(np.abs(u + 0.4321)) < 1e-13


def test_ks_mean_conserved():
    """Every central-difference term telescopes under periodic wrap: sum u is invariant."""
    spec = I.ks_spec(256)
    u = I.initial_state(spec)
    s0 = float(u.sum())
    O.classic(oprob(spec), u, 2000)
    assert abs(float(u.sum()) - s0) < 1e-10 * float(np.abs(u).sum())


@pytest.mark.parametrize("k,U", [(3, 0.7), (5, -0.4), (11, 0.0)])
def test_ks_linearised_mode(k, U):
    """Small mode on a constant background: linearised f has eigenvalue
    lam = 4s/dx^2 - 16 s^2/dx^4 - i U sin(theta)/dx (s = sin^2(theta/2)), and the
    midpoint RK2 multiplies the mode by 1 + z + z^2/2, z = dt lam, per step."""
    N, M, eps = 64, 200, 1e-7
    spec = I.ks_spec(N)
    dx, dt = spec.dx, spec.dt
    theta = 2 * math.pi * k / N
    j = np.arange(N)
    u = (U + eps * np.cos(theta * j))[None, :].copy()
    O.classic(oprob(spec), u, M)
    s = math.sin(theta / 2) ** 2
    lam = complex(4 * s / dx ** 2 - 16 * s * s / dx ** 4, -U * math.sin(theta) / dx)
    z = dt * lam
    g = (1 + z + z * z / 2) ** M
    expect = np.real(g * np.exp(1j * theta * j))
    got = (u[0] - U) / eps
    assert np.max(np.abs(got - expect)) < 1e-5 * np.max(np.abs(expect))


def test_ks_config_bounded_chaos():
    """The configuration's initial condition stays bounded and mean-preserving over
    the configuration's 10^4 steps (N = 2^11)."""
    spec = I.ks_spec(2048)
    u = I.initial_state(spec)
    s0 = float(u.sum())
    O.classic(oprob(spec), u, 10000)
    assert np.all(np.isfinite(u)) and np.max(np.abs(u)) < 10
    assert abs(float(u.sum()) - s0) < 1e-9 * float(np.abs(u).sum())


def test_ks_fp32_short_horizon_tracks_fp64():
    spec = I.ks_spec(256)
    u64 = I.initial_state(spec)
    u32 = u64.astype(np.float32)
    O.classic(oprob(spec), u64, 100)
    O.classic(oprob(spec), u32, 100)
    assert rel_max(u32[0].astype(np.float64), u64[0]) < 1e-5


# --------------------------------------------------------------------------
# Euler equations (Appendix C)
# --------------------------------------------------------------------------
def _cons(r, u, p, g=1.4):
    return np.array([r, r * u, p / (g - 1) + 0.5 * r * u * u])


def test_euler_pressure_worked_value():
    """Eq. EulerP with E total energy per volume: rho=2, rho u=3, E=5, gamma=1.4:
    P = 0.4 (5 - 3 * 1.5 / 2) = 0.4 * 2.75 = 1.1."""
    assert abs(O.euler_pressure(np.array([2.0, 3.0, 5.0])) - 1.1) < 1e-15


def _still(r, p, g=1.4):
    return np.array([r, 0.0, p / (g - 1)])


def test_euler_reconstruction_worked_values():
    """Eqs. Pratio / limitleft / limitright on hand-worked cells at rest
    (P = 0.4 E).  Cells a-1, a, b, b+1."""
    # P = 1, 2, 2.5, 2.75: ratio at a = 0.5 -> QL = Qa + 0.25 (Qb - Qa);
    # inverse ratio at b = 0.5 / 0.25 = 2 -> min(., 1) = 1 -> QR = (Qa + Qb) / 2
    q = np.array([_still(1, 1.0), _still(2, 2.0), _still(3, 2.5), _still(5, 2.75)])
    ql, qr = O.euler_reconstruct(q)
    assert np.allclose(ql, [2.25, 0.0, 5.3125], rtol=1e-14, atol=1e-15)
    assert np.allclose(qr, [2.5, 0.0, 5.625], rtol=1e-14, atol=1e-15)
    # P = 1, 1.5, 2.5, 4.5: ratio at a = 2 -> QL = (Qa + Qb) / 2;
    # inverse at b = 1 / 2 -> QR = Qb + 0.25 (Qa - Qb)
    q = np.array([_still(1, 1.0), _still(2, 1.5), _still(4, 2.5), _still(1, 4.5)])
    ql, qr = O.euler_reconstruct(q)
    assert np.allclose(ql, [3.0, 0.0, 5.0], rtol=1e-14, atol=1e-15)
    assert np.allclose(qr, [3.5, 0.0, 5.625], rtol=1e-14, atol=1e-15)
    # P = 1, 2, 1.5, 1.5: ratio at a < 0 and zero numerator at b -> first order
    q = np.array([_still(1, 1.0), _still(2, 2.0), _still(4, 1.5), _still(1, 1.5)])
    ql, qr = O.euler_reconstruct(q)
    assert np.array_equal(ql, q[1]) and np.array_equal(qr, q[2])


def test_euler_flux_roe_weights_worked_value():
    """Limiter inactive (left pair equal, right pair equal).  rho = 4 | 1,
    u = 1 | -2, p = 1.6 | 0.4 so E = 6 | 3 and e = E/rho = 1.5 | 3.
    sqrt(rho) weights 2 | 1: u_sp = (2 - 2)/3 = 0, e_sp = (3 + 3)/3 = 2,
    r_sp = sqrt(1.4 * 0.4 * 2) = sqrt(1.12).
    G = F(QR) + F(QL) + r_sp (QL - QR):
      mass     (-2) + 4 + 3 r_sp
      momentum (1 * 4 + 0.4) + (4 * 1 + 1.6) + 6 r_sp
      energy   -2 (3 + 0.4) + 1 (6 + 1.6) + 3 r_sp"""
    L = np.array([4.0, 4.0, 6.0])
    Rr = np.array([1.0, -2.0, 3.0])
    G = O.euler_interface(np.array([L, L, Rr, Rr]))
    r = math.sqrt(1.12)
    assert np.allclose(G, [2 + 3 * r, 10 + 6 * r, 0.8 + 3 * r], rtol=1e-14, atol=1e-14)


def test_euler_flux_consistency_worked_value():
    """Four equal cells: the flux is F(Q).  rho=1, u=2, p=3, gamma=1.4:
    E = 3/0.4 + 1/2 * 1 * 4 = 9.5, F = (2, 4 + 3, 2 (9.5 + 3)) = (2, 7, 25)."""
    q = np.tile(_cons(1.0, 2.0, 3.0), (4, 1))
    G = O.euler_interface(q)
    assert np.allclose(G, [4.0, 14.0, 50.0], rtol=1e-14, atol=0)


def test_euler_flux_spectral_radius_is_sound_speed():
    """Equal density and velocity, pressure step (limiter inactive at a step):
    the Roe average gives the largest eigenvalue |u| + c of the Jacobian with
    c^2 = gamma (pL + pR) / (2 rho), so G = F(QL) + F(QR) + (|u| + c)(QL - QR)."""
    g, r, u, pl, pr = 1.4, 0.8, -0.3, 1.2, 0.5
    ql, qr = _cons(r, u, pl), _cons(r, u, pr)
    G = O.euler_interface(np.array([ql, ql, qr, qr]))
    F = lambda q, p: np.array([q[1], q[1] * q[1] / q[0] + p, q[1] / q[0] * (q[2] + p)])
    c = math.sqrt(g * (pl + pr) / (2 * r))
    expect = F(ql, pl) + F(qr, pr) + (abs(u) + c) * (ql - qr)
    assert np.allclose(G, expect, rtol=1e-13, atol=1e-15)


def test_euler_uniform_state_is_fixed_point():
    N = 64
    spec = I.sod_spec(N, bc="periodic")
    q = np.tile(_cons(0.9, 0.35, 1.7)[:, None], (1, N)).copy()
    q0 = q.copy()
    O.classic(oprob(spec), q, 40)
    assert np.array_equal(q, q0)


def test_euler_mirror_symmetry():
    """Reflecting x and swapping the end states reflects rho and E and negates
    rho u (to rounding): catches exchanged left/right roles."""
    N, steps = 128, 100
    spec = I.sod_spec(N)
    q = I.initial_state(spec)
    O.classic(oprob(spec), q, steps)
    mspec = I.ProblemSpec("euler", "dirichlet", N, spec.dx, spec.dt, gamma=1.4,
                          left=spec.right, right=spec.left)
    qm = I.initial_state(mspec)
    O.classic(oprob(mspec), qm, steps)
    assert np.max(np.abs(qm[0, ::-1] - q[0])) < 1e-12
    assert np.max(np.abs(qm[1, ::-1] + q[1])) < 1e-12
    assert np.max(np.abs(qm[2, ::-1] - q[2])) < 1e-12


def test_euler_conservation_with_boundary_flux():
    """Finite-volume update: mass and energy are conserved while the waves stay
    inside; momentum grows by (pL - pR) dt per step through the uniform end states."""
    N = 256
    steps = N // 4
    spec = I.sod_spec(N)
    q = I.initial_state(spec)
    s0 = q.sum(axis=1)
    O.classic(oprob(spec), q, steps)
    s1 = q.sum(axis=1)
    lam = spec.dt / spec.dx
    assert abs(s1[0] - s0[0]) < 1e-12 * s0[0]
    assert abs(s1[2] - s0[2]) < 1e-12 * s0[2]
    assert abs(s1[1] - lam * (1.0 - 0.1) * steps) < 1e-11


def test_euler_periodic_conserves_all():
    N = 128
    spec = I.sod_spec(N, bc="periodic")
    x = (np.arange(N) + 0.5) / N
    q = np.stack([_cons(1 + 0.2 * math.sin(2 * math.pi * xi), 0.3, 1 + 0.1 * math.cos(2 * math.pi * xi))
                  for xi in x], axis=1).copy()
    s0 = q.sum(axis=1)
    O.classic(oprob(spec), q, 300)
    assert np.all(np.abs(q.sum(axis=1) - s0) < 1e-12 * np.abs(q).sum(axis=1))


def test_euler_rk2_temporal_order():
    """One step of dt against two of dt/2: the local error of a second-order
    scheme shrinks 8x when dt halves (4x if a stage were first order)."""
    g, N = 1.4, 64
    x = (np.arange(N) + 0.5) / N
    s = np.sin(2 * math.pi * x) + 0.3 * np.cos(4 * math.pi * x)
    q0 = np.stack([1 + 1e-2 * s, (1 + 1e-2 * s) * (0.5 + 0.0118 * s),
                   (1 + 0.014 * s) / (g - 1) + 0.5 * (1 + 1e-2 * s) * (0.5 + 0.0118 * s) ** 2])
    dx = 1.0 / N

    def adv(dt, k):
        q = q0.copy()
        O.classic(O.OracleProblem(O.EULER, O.PERIODIC, N, dx, dt, gamma=g), q, k)
        return q

    d1 = np.abs(adv(0.04 * dx, 1) - adv(0.02 * dx, 2)).max()
    d2 = np.abs(adv(0.02 * dx, 1) - adv(0.01 * dx, 2)).max()
    assert d1 / d2 > 6.5


def test_sod_exact_riemann_solver_textbook_values():
    ps, us = R.star_state((1.0, 0.0, 1.0), (0.125, 0.0, 0.1))
    assert abs(ps - 0.30313) < 1e-5 and abs(us - 0.92745) < 1e-5


def test_sod_converges_to_exact_solution():
    """L1(rho) against the exact Riemann solution decreases with N (discontinuous
    solution: observed order >= 0.6) and the star-region plateau matches p*, u*."""
    errs = []
    ps, us = R.star_state((1.0, 0.0, 1.0), (0.125, 0.0, 0.1))
    for N in (256, 512, 1024):
        spec = I.sod_spec(N)
        q = I.initial_state(spec)
        O.classic(oprob(spec), q, N)   # t = N dt = 0.2 at dt/dx = 0.2
        x = (np.arange(N) + 0.5) / N
        ex = R.sample(x, 0.2, 0.5, (1, 0, 1), (0.125, 0, 0.1))
        errs.append(np.abs(q[0] - ex[0]).mean())
        u = q[1] / q[0]
        p = 0.4 * (q[2] - 0.5 * q[1] * u)
        i = int(0.75 * N)   # between the contact (~0.686) and the shock (~0.850)
        assert abs(p[i] - ps) < 2e-3 and abs(u[i] - us) < 5e-3
    assert errs[0] > errs[1] > errs[2]
    assert math.log2(errs[0] / errs[2]) / 2 >= 0.6


# --------------------------------------------------------------------------
# swept == classic (Section 2: same operations in a different order)
# --------------------------------------------------------------------------
def _swept_cases():
    cases = []
    for n in (4, 8, 16, 32):
        for steps in (1, 2, 5, 8, 17, 40):
            cases.append(("heat", "periodic", 64, n, steps))
            cases.append(("heat", "reflective", 64, n, steps))
    for n in (8, 16, 32, 64):
        for steps in (1, 2, 3, 4, 7, 16, 21):
            cases.append(("ks", "periodic", 64, n, steps))
            cases.append(("euler", "dirichlet", 64, n, steps))
            cases.append(("euler", "periodic", 64, n, steps))
    cases.append(("ks", "periodic", 32, 32, 9))       # a single node
    cases.append(("heat", "periodic", 16, 16, 23))
    return cases


def _spec(eq, bc, N):
    if eq == "heat":
        return I.heat_spec(N, r=0.3, bc=bc)
    if eq == "ks":
        return I.ks_spec(N)
    return I.sod_spec(N, bc=bc)


@pytest.mark.parametrize("eq,bc,N,n,steps", _swept_cases())
def test_swept_equals_classic_bitwise(eq, bc, N, n, steps):
    spec = _spec(eq, bc, N)
    a = I.initial_state(spec)
    if eq == "ks":
        a = a + 0.1 * I.uniform_field(N, 99)[None, :]
    b = a.copy()
    O.classic(oprob(spec), a, steps)
    O.swept(oprob(spec), b, steps, n)
    assert np.array_equal(a, b)


@pytest.mark.parametrize("eq", ["heat", "ks"])
def test_swept_equals_classic_fp32(eq):
    spec = _spec(eq, "periodic", 128)
    a = I.initial_state(spec, np.float32)
    b = a.copy()
    O.classic(oprob(spec), a, 37)
    O.swept(oprob(spec), b, 37, 32)
    assert np.array_equal(a, b)


def test_swept_rejects_bad_node_width():
    spec = I.ks_spec(64)
    u = I.initial_state(spec)
    with pytest.raises(O.OracleError):
        O.swept(oprob(spec), u, 4, 24)     # N % n != 0
    spec48 = I.ks_spec(48)
    with pytest.raises(O.OracleError):
        O.swept(oprob(spec48), I.initial_state(spec48), 4, 12)   # H = n / 4 = 3 odd
    with pytest.raises(O.OracleError):
        O.classic(O.OracleProblem(O.KS, O.REFLECTIVE, 64, 0.5, 0.005), u, 1)


@pytest.mark.parametrize("n", [16, 32, 64, 128, 1024])
def test_swept_geometry_first_order_triangle_is_n_over_2(n):
    """Section 4.2: a first-order (heat) node of n points advances n/2
    timesteps per triangle, in a working array of two rows of n + k - 1 slots
    (stencil width k = 3)."""
    g = O.swept_geometry(O.HEAT, n, 1000)
    assert g["triangle_steps"] == n // 2
    assert g["W"] == n + 3 - 1


@pytest.mark.parametrize("eq", [O.KS, O.EULER])
@pytest.mark.parametrize("n", [32, 64, 256, 1024])
def test_swept_geometry_second_order_triangle_is_n_over_8(eq, n):
    """Sections 4.2 and 6: a second-order scheme (two sub-steps of a 5-point
    stencil) advances n/8 timesteps per triangle; the paper's example is
    n = 32 -> 4 timesteps.  Working array rows of n + 5 - 1 slots."""
    g = O.swept_geometry(eq, n, 1000)
    assert g["triangle_steps"] == n // 8
    assert g["W"] == n + 5 - 1
    if n == 32:
        assert g["triangle_steps"] == 4


def test_swept_geometry_rejects_odd_half_cycles():
    """H = n / (2 rad) must be even (the rows' level parity) and n a multiple
    of 2 rad."""
    assert O.swept_geometry(O.KS, 24, 10)["H"] == 6
    for eq, n in ((O.KS, 20), (O.HEAT, 30), (O.KS, 18)):
        with pytest.raises(O.OracleError):
            O.swept_geometry(eq, n, 10)
