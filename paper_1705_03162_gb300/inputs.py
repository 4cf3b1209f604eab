"""Seeded synthetic inputs shaped like the paper's test problems.

This module holds no arithmetic of the swept or classic schemes: it only
builds initial conditions and problem parameters, and is the one module the
CUDA path and the CPU oracle (tests) both use.

Random numbers come from SplitMix64 (Steele, Lea & Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014), mapped to [0, 1) as
(x >> 11) * 2^-53.

Problems (Appendices A-C of arXiv:1705.03162, sizes from Section 6):
  heat   u_t = alpha u_xx on [0, 1), N points x_i = i / N, Fourier number r,
         u0 = sin(2 pi x) + sum_{k=2..9} a_k sin(2 pi k x), a_k ~ U(-0.1, 0.1)
  ks     u_t + u u_x + u_xx + u_xxxx = 0, x_i = i dx, dx = 0.5, dt = 0.005,
         u0 = cos(x/16) (1 + sin(x/16))
  sod    Euler shock tube on [0, 1], N cells, centres (i + 1/2)/N, diaphragm at
         0.5, left (rho, u, p) = (1, 0, 1), right (0.125, 0, 0.1), gamma 1.4,
         dt/dx = 0.2
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

HEAT_SEED = 20170509
_MASK = (1 << 64) - 1


def splitmix64(seed: int, count: int) -> np.ndarray:
    """``count`` successive SplitMix64 outputs from ``seed`` (uint64)."""
    out = np.empty(count, dtype=np.uint64)
    s = seed & _MASK
    for i in range(count):
        s = (s + 0x9E3779B97F4A7C15) & _MASK
        z = s
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _MASK
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _MASK
        out[i] = z ^ (z >> 31)
    return out


def uniform01(seed: int, count: int) -> np.ndarray:
    """``count`` doubles in [0, 1): SplitMix64 output >> 11, times 2^-53."""
    return (splitmix64(seed, count) >> np.uint64(11)).astype(np.float64) * 2.0 ** -53


def uniform_field(n: int, seed: int, lo: float = -1.0, hi: float = 1.0) -> np.ndarray:
    """Vectorised seeded uniform field (counter-based SplitMix64 of seed + i)."""
    i = np.arange(1, n + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed & _MASK) + i * np.uint64(0x9E3779B97F4A7C15)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        z = z ^ (z >> np.uint64(31))
    u = (z >> np.uint64(11)).astype(np.float64) * 2.0 ** -53
    return lo + (hi - lo) * u


def heat_mode_amplitudes(seed: int = HEAT_SEED) -> np.ndarray:
    """a_2..a_9 of the heat initial condition, each 0.2 v - 0.1 with v ~ U[0,1)."""
    return 0.2 * uniform01(seed, 8) - 0.1


def heat_ic(n_points: int, seed: int = HEAT_SEED) -> np.ndarray:
    """Heat initial condition on x_i = i / N: sin(2 pi x) + sum a_k sin(2 pi k x)."""
    x = np.arange(n_points, dtype=np.float64) / n_points
    u = np.sin(2.0 * math.pi * x)
    for k, a in zip(range(2, 10), heat_mode_amplitudes(seed)):
        u += a * np.sin(2.0 * math.pi * k * x)
    return u


def ks_ic(n_points: int, dx: float = 0.5) -> np.ndarray:
    """KS initial condition cos(x/16) (1 + sin(x/16)) on x_i = i dx."""
    x = np.arange(n_points, dtype=np.float64) * dx
    return np.cos(x / 16.0) * (1.0 + np.sin(x / 16.0))


def sod_ic(n_points: int, gamma: float = 1.4, left=(1.0, 0.0, 1.0),
           right=(0.125, 0.0, 0.1)) -> np.ndarray:
    """Sod shock tube, conserved (rho, rho u, E) of shape (3, N); cells i < N/2 left."""
    q = np.empty((3, n_points), dtype=np.float64)
    half = n_points // 2
    for sl, (r, u, p) in ((slice(0, half), left), (slice(half, n_points), right)):
        q[0, sl] = r
        q[1, sl] = r * u
        q[2, sl] = p / (gamma - 1.0) + 0.5 * r * u * u
    return q


@dataclass(frozen=True)
class ProblemSpec:
    """Parameters of one problem instance (what a caller passes at create)."""
    eq: str            # "heat" | "ks" | "euler"
    bc: str            # "periodic" | "reflective" | "dirichlet"
    n_points: int
    dx: float
    dt: float
    alpha: float = 1.0
    gamma: float = 1.4
    left: tuple = (1.0, 0.0, 1.0)
    right: tuple = (0.125, 0.0, 0.1)

    @property
    def nv(self) -> int:
        return 3 if self.eq == "euler" else 1

    @property
    def substeps(self) -> int:
        return 1 if self.eq == "heat" else 2

    @property
    def radius(self) -> int:
        return 1 if self.eq == "heat" else 2


def heat_spec(n_points: int = 1024, r: float = 0.25, bc: str = "periodic",
              alpha: float = 1.0) -> ProblemSpec:
    dx = 1.0 / n_points
    return ProblemSpec("heat", bc, n_points, dx, r * dx * dx / alpha, alpha=alpha)


def ks_spec(n_points: int, dx: float = 0.5, dt: float = 0.005) -> ProblemSpec:
    return ProblemSpec("ks", "periodic", n_points, dx, dt)


def sod_spec(n_points: int, lam: float = 0.2, gamma: float = 1.4,
             bc: str = "dirichlet") -> ProblemSpec:
    dx = 1.0 / n_points
    return ProblemSpec("euler", bc, n_points, dx, lam * dx, gamma=gamma)


def initial_state(spec: ProblemSpec, dtype=np.float64) -> np.ndarray:
    """Initial state of shape (nv, N) for the problem's configuration."""
    if spec.eq == "heat":
        u = heat_ic(spec.n_points)[None, :]
    elif spec.eq == "ks":
        u = ks_ic(spec.n_points, spec.dx)[None, :]
    else:
        u = sod_ic(spec.n_points, spec.gamma, spec.left, spec.right)
    return np.ascontiguousarray(u.astype(dtype))
