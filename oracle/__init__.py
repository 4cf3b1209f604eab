"""CPU oracle for the swept time-space decomposition (arXiv:1705.03162).

TEST INFRASTRUCTURE.  A plain, slow, single-threaded C restatement of the
paper's classic and swept schemes (Sections 4-5, Appendices A-C), used only by
``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py``.  The CUDA library never imports, links or calls it; the two share
no code.  Only the seeded input generators (``paper_1705_03162_gb300.inputs``)
serve both.

Functions
---------
classic(problem, state, steps)        -- Section 5.1 classic decomposition
swept(problem, state, steps, n)       -- Sections 4.2-4.3 swept decomposition
euler_pressure(q, gamma)              -- Appendix C Eq. EulerP
euler_reconstruct(q4, gamma)          -- Appendix C limited reconstruction
euler_interface(q4, gamma)            -- Appendix C interface flux (x2)

``problem`` is an :class:`OracleProblem`; ``state`` is a numpy array of shape
(nv, N) (nv = 3 for Euler, else 1), float64 or float32, advanced in place.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = [os.path.join(_HERE, "swept_oracle.c"), os.path.join(_HERE, "scheme.inc")]
_BUILD_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None

HEAT, KS, EULER = 0, 1, 2
PERIODIC, REFLECTIVE, DIRICHLET = 0, 1, 2
_ERRORS = {1: "EINVAL", 2: "ENOMEM", 5: "EUNSUPPORTED"}


class OracleError(RuntimeError):
    pass


class _Problem(ctypes.Structure):
    _fields_ = [
        ("eq", ctypes.c_int32),
        ("bc", ctypes.c_int32),
        ("n_points", ctypes.c_int64),
        ("dx", ctypes.c_double),
        ("dt", ctypes.c_double),
        ("alpha", ctypes.c_double),
        ("gamma", ctypes.c_double),
        ("left", ctypes.c_double * 3),
        ("right", ctypes.c_double * 3),
    ]


@dataclass
class OracleProblem:
    eq: int
    bc: int
    n_points: int
    dx: float
    dt: float
    alpha: float = 1.0
    gamma: float = 1.4
    left: tuple = (1.0, 0.0, 1.0)
    right: tuple = (0.125, 0.0, 0.1)

    @property
    def nv(self) -> int:
        return 3 if self.eq == EULER else 1

    def _c(self) -> _Problem:
        p = _Problem()
        p.eq, p.bc, p.n_points = self.eq, self.bc, self.n_points
        p.dx, p.dt, p.alpha, p.gamma = self.dx, self.dt, self.alpha, self.gamma
        p.left = (ctypes.c_double * 3)(*self.left)
        p.right = (ctypes.c_double * 3)(*self.right)
        return p


def build(force: bool = False) -> str:
    """Compile the oracle into oracle/_build/liboracle.so (gcc, no FP contraction)."""
    with _lock:
        os.makedirs(_BUILD_DIR, exist_ok=True)
        stale = force or not os.path.exists(_LIB_PATH) or any(
            os.path.getmtime(s) > os.path.getmtime(_LIB_PATH) for s in _SRC)
        if stale:
            tmp = _LIB_PATH + f".tmp{os.getpid()}"
            cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
                   "-fno-fast-math", "-o", tmp, _SRC[0], "-lm"]
            subprocess.run(cmd, check=True, cwd=_HERE)
            os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        vp, i32, i64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
        lib.orc_classic.argtypes = [ctypes.POINTER(_Problem), i32, vp, i64]
        lib.orc_classic.restype = ctypes.c_int
        lib.orc_swept.argtypes = [ctypes.POINTER(_Problem), i32, vp, i64, i64]
        lib.orc_swept.restype = ctypes.c_int
        lib.orc_euler_interface_f64.argtypes = [vp, ctypes.c_double, vp]
        lib.orc_euler_interface_f64.restype = ctypes.c_int
        lib.orc_euler_reconstruct_f64.argtypes = [vp, ctypes.c_double, vp, vp]
        lib.orc_euler_reconstruct_f64.restype = ctypes.c_int
        lib.orc_swept_geometry.argtypes = [i32, i64, i64, vp]
        lib.orc_swept_geometry.restype = ctypes.c_int
        lib.orc_euler_pressure_f64.argtypes = [vp, ctypes.c_double]
        lib.orc_euler_pressure_f64.restype = ctypes.c_double
        _lib = lib
    return _lib


def _check(rc: int, what: str):
    if rc != 0:
        raise OracleError(f"{what}: {_ERRORS.get(rc, rc)}")


def _state(problem: OracleProblem, state: np.ndarray):
    if state.dtype not in (np.float64, np.float32):
        raise TypeError("state must be float64 or float32")
    if state.shape != (problem.nv, problem.n_points) or not state.flags.c_contiguous:
        raise ValueError(f"state must be C-contiguous of shape {(problem.nv, problem.n_points)}")
    return 0 if state.dtype == np.float64 else 1


def classic(problem: OracleProblem, state: np.ndarray, steps: int) -> np.ndarray:
    """Advance ``state`` in place by ``steps`` timesteps, classic decomposition."""
    dt = _state(problem, state)
    p = problem._c()
    _check(_load().orc_classic(ctypes.byref(p), dt, state.ctypes.data, int(steps)), "classic")
    return state


def swept(problem: OracleProblem, state: np.ndarray, steps: int, n: int) -> np.ndarray:
    """Advance ``state`` in place by ``steps`` timesteps, swept decomposition with
    nodes of ``n`` points."""
    dt = _state(problem, state)
    p = problem._c()
    _check(_load().orc_swept(ctypes.byref(p), dt, state.ctypes.data, int(steps), int(n)), "swept")
    return state


def swept_geometry(eq: int, n: int, steps: int) -> dict:
    """The swept plan the oracle runs for nodes of ``n`` points (Sections
    4.2-4.3): levels per half-cycle H, slots per working-array row W, full
    half-cycles Q, remaining levels r, kernels, and timesteps per triangle."""
    out = np.zeros(6, dtype=np.int64)
    _check(_load().orc_swept_geometry(int(eq), int(n), int(steps), out.ctypes.data), "geometry")
    return dict(zip(("H", "W", "Q", "r", "kernels", "triangle_steps"), (int(x) for x in out)))


def euler_interface(q4: np.ndarray, gamma: float = 1.4) -> np.ndarray:
    """2 x Flux at the interface between cells 1 and 2 of the 4 cells ``q4``
    (shape (4, 3), conserved (rho, rho u, E)), Appendix C."""
    q = np.ascontiguousarray(q4, dtype=np.float64).reshape(12)
    G = np.zeros(3)
    _check(_load().orc_euler_interface_f64(q.ctypes.data, float(gamma), G.ctypes.data), "flux")
    return G


def euler_pressure(q: np.ndarray, gamma: float = 1.4) -> float:
    """Pressure of one conserved state (rho, rho u, E), Appendix C Eq. EulerP."""
    q = np.ascontiguousarray(q, dtype=np.float64).reshape(3)
    return float(_load().orc_euler_pressure_f64(q.ctypes.data, float(gamma)))


def euler_reconstruct(q4: np.ndarray, gamma: float = 1.4):
    """Limited left and right states at the interface between cells 1 and 2 of
    the 4 cells ``q4`` (shape (4, 3)), Appendix C."""
    q = np.ascontiguousarray(q4, dtype=np.float64).reshape(12)
    ql, qr = np.zeros(3), np.zeros(3)
    _check(_load().orc_euler_reconstruct_f64(q.ctypes.data, float(gamma), ql.ctypes.data,
                                             qr.ctypes.data), "reconstruct")
    return ql, qr
