"""Helpers shared by the tests: oracle problem from a ProblemSpec, error norms."""
import numpy as np

import oracle as O
from paper_1705_03162_gb300 import inputs as I

_EQ = {"heat": O.HEAT, "ks": O.KS, "euler": O.EULER}
_BC = {"periodic": O.PERIODIC, "reflective": O.REFLECTIVE, "dirichlet": O.DIRICHLET}


def oprob(spec: I.ProblemSpec) -> O.OracleProblem:
    return O.OracleProblem(_EQ[spec.eq], _BC[spec.bc], spec.n_points, spec.dx, spec.dt,
                           spec.alpha, spec.gamma, spec.left, spec.right)


def rel_max(a, b) -> float:
    """Relative max-norm max|a - b| / max|b|, per variable (max over variables)."""
    a = np.asarray(a, dtype=np.float64).reshape(-1, np.shape(a)[-1])
    b = np.asarray(b, dtype=np.float64).reshape(-1, np.shape(b)[-1])
    return max(float(np.max(np.abs(a[v] - b[v])) / max(float(np.max(np.abs(b[v]))), 1e-300))
               for v in range(a.shape[0]))


def spec_for(eq: str, bc: str, N: int) -> I.ProblemSpec:
    if eq == "heat":
        return I.heat_spec(N, r=0.25, bc=bc)
    if eq == "ks":
        return I.ks_spec(N)
    return I.sod_spec(N, bc=bc)


def state_for(spec: I.ProblemSpec, dtype=np.float64, seed: int = 7) -> np.ndarray:
    u = I.initial_state(spec)
    if spec.eq == "ks":
        u = u + 0.05 * I.uniform_field(spec.n_points, seed)[None, :]
    if spec.eq == "euler" and spec.bc == "periodic":
        x = (np.arange(spec.n_points) + 0.5) / spec.n_points
        rho = 1.0 + 0.3 * np.sin(2 * np.pi * x) + 0.05 * I.uniform_field(spec.n_points, seed)
        vel = 0.4 * np.cos(2 * np.pi * x)
        p = 1.0 + 0.2 * np.cos(4 * np.pi * x)
        u = np.stack([rho, rho * vel, p / (spec.gamma - 1) + 0.5 * rho * vel * vel])
    return np.ascontiguousarray(u.astype(dtype))
