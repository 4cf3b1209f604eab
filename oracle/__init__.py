"""CPU oracle for the swept time-space decomposition (arXiv:1705.03162).

TEST INFRASTRUCTURE.  A plain, slow C restatement of the paper's classic and
swept schemes (Sections 4-5, Appendices A-C), used only by ``tests/``,
``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py``.  The
CUDA library never imports, links or calls it; the two share no code.  Only
the seeded input generators (``paper_1705_03162_gb300.inputs``) serve both.

It is built three times from the same sources: single-threaded, with OpenMP
(the classic loops split each sub-timestep's points over threads; same bits),
and with an operation-counting scalar type (``opcount.cpp``).

Functions
---------
classic(problem, state, steps, threads=1)  -- Section 5.1 classic decomposition
swept(problem, state, steps, n)       -- Sections 4.2-4.3 swept decomposition
euler_pressure(q, gamma)              -- Appendix C Eq. EulerP
euler_reconstruct(q4, gamma)          -- Appendix C limited reconstruction
euler_interface(q4, gamma)            -- Appendix C interface flux (x2)
opcounts(problem, state, steps)       -- operations per point-update (counting build)

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
_SRC = [os.path.join(_HERE, "swept_oracle.c"), os.path.join(_HERE, "scheme.inc"), os.path.join(_HERE, "oracle.h")]
_OPC_SRC = [os.path.join(_HERE, "opcount.cpp"), os.path.join(_HERE, "scheme.inc"), os.path.join(_HERE, "oracle.h")]
_BUILD_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD_DIR, "liboracle.so")
_OMP_PATH = os.path.join(_BUILD_DIR, "liboracle_omp.so")
_OPC_PATH = os.path.join(_BUILD_DIR, "liboracle_opcount.so")
_lock = threading.Lock()
_lib = None
_omp = None
_opc = None

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


def _compile(path, srcs, cmd_of):
    stale = not os.path.exists(path) or any(os.path.getmtime(s) > os.path.getmtime(path) for s in srcs)
    if stale:
        tmp = path + f".tmp{os.getpid()}"
        subprocess.run(cmd_of(tmp), check=True, cwd=_HERE)
        os.replace(tmp, path)


def build(force: bool = False) -> str:
    """Compile the oracle into oracle/_build/: liboracle.so (gcc, no FP
    contraction), liboracle_omp.so (the same with -fopenmp) and
    liboracle_opcount.so (g++, the counting build)."""
    with _lock:
        os.makedirs(_BUILD_DIR, exist_ok=True)
        if force:
            for p in (_LIB_PATH, _OMP_PATH, _OPC_PATH):
                if os.path.exists(p):
                    os.unlink(p)
        base = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off", "-fno-fast-math"]
        _compile(_LIB_PATH, _SRC, lambda t: base + ["-o", t, _SRC[0], "-lm"])
        _compile(_OMP_PATH, _SRC, lambda t: base + ["-fopenmp", "-o", t, _SRC[0], "-lm"])
        _compile(_OPC_PATH, _OPC_SRC, lambda t: ["g++", "-O1", "-std=c++17", "-fPIC", "-shared",
                                                 "-ffp-contract=off", "-fno-fast-math", "-o", t, _OPC_SRC[0]])
    return _LIB_PATH


def _declare(lib):
    vp, i32, i64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
    lib.orc_classic.argtypes = [ctypes.POINTER(_Problem), i32, vp, i64]
    lib.orc_classic.restype = ctypes.c_int
    lib.orc_set_threads.argtypes = [ctypes.c_int]
    lib.orc_set_threads.restype = ctypes.c_int
    return lib


def _load_omp():
    global _omp
    if _omp is None:
        build()
        _omp = _declare(ctypes.CDLL(_OMP_PATH))
    return _omp


def _load_opc():
    global _opc
    if _opc is None:
        build()
        lib = ctypes.CDLL(_OPC_PATH)
        vp, i64, ll = ctypes.c_void_p, ctypes.c_int64, ctypes.POINTER(ctypes.c_longlong)
        lib.orc_opcount_classic.argtypes = [ctypes.POINTER(_Problem), vp, i64, ll]
        lib.orc_opcount_classic.restype = ctypes.c_int
        lib.orc_opcount_euler_pressure.argtypes = [ll]
        lib.orc_opcount_euler_pressure.restype = ctypes.c_int
        lib.orc_opcount_euler_point.argtypes = [vp, vp, ctypes.c_double, ctypes.c_double, ll, ll]
        lib.orc_opcount_euler_point.restype = ctypes.c_int
        _opc = lib
    return _opc


def _load():
    global _lib
    if _lib is None:
        lib = _declare(ctypes.CDLL(build()))
        vp, i32, i64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
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
        lib.orc_stage_f64.argtypes = [ctypes.POINTER(_Problem), i32, vp, vp, vp]
        lib.orc_stage_f64.restype = ctypes.c_int
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


def classic(problem: OracleProblem, state: np.ndarray, steps: int, threads: int = 1) -> np.ndarray:
    """Advance ``state`` in place by ``steps`` timesteps, classic decomposition.
    ``threads`` > 1 runs the OpenMP build with that many threads (same bits)."""
    dt = _state(problem, state)
    p = problem._c()
    if threads > 1:
        lib = _load_omp()
        lib.orc_set_threads(int(threads))
    else:
        lib = _load()
    _check(lib.orc_classic(ctypes.byref(p), dt, state.ctypes.data, int(steps)), "classic")
    return state


def omp_threads(threads: int) -> int:
    """Threads the OpenMP build runs with after asking for ``threads``."""
    return int(_load_omp().orc_set_threads(int(threads)))


_OPS = ("add", "mul", "fma", "div", "sqrt")


def _ops_dict(c, scale: float = 1.0) -> dict:
    d = {k: float(c[i]) / scale for i, k in enumerate(_OPS)}
    d["ops"] = sum(d[k] for k in _OPS)
    d["flops"] = d["add"] + d["mul"] + 2 * d["fma"] + d["div"] + d["sqrt"]
    return d


def opcounts(problem: OracleProblem, state: np.ndarray, steps: int) -> dict:
    """Floating-point operations per point-update (one point, one timestep)
    of ``steps`` classic timesteps from ``state`` (FP64, not modified), from
    the counting build: additions (and subtractions), multiplications, FMAs,
    divisions, square roots, their sum ``ops`` and ``flops`` (an FMA is two).

    ``oracle`` is the count as the oracle evaluates the scheme.  For Euler
    that evaluates every interface flux twice and every pressure five times
    per cell; ``algorithmic`` is one pressure per cell, one flux per
    interface and the cell update, per sub-timestep (the work a scheme that
    keeps each value once must do).  For heat and KS the two agree."""
    _state(problem, state)
    st = np.ascontiguousarray(state, dtype=np.float64)
    lib = _load_opc()
    c = (ctypes.c_longlong * 5)()
    p = problem._c()
    _check(lib.orc_opcount_classic(ctypes.byref(p), st.ctypes.data, int(steps), c), "opcount")
    updates = float(problem.n_points) * steps
    out = {"oracle": _ops_dict(list(c), updates)}
    if problem.eq != EULER:
        out["algorithmic"] = dict(out["oracle"])
        return out
    pc = (ctypes.c_longlong * 5)()
    _check(lib.orc_opcount_euler_pressure(pc), "opcount pressure")
    # the cell update's own operations, from one stencil of the state
    q = np.ascontiguousarray(st[:, :5].T.reshape(15))
    base = np.ascontiguousarray(st[:, 2])
    pt, itf = (ctypes.c_longlong * 5)(), (ctypes.c_longlong * 5)()
    _check(lib.orc_opcount_euler_point(q.ctypes.data, base.ctypes.data, problem.gamma, -0.1, pt, itf),
           "opcount point")
    P = np.array(list(pc), dtype=np.float64)
    U = np.array(list(pt), dtype=np.float64) - 5 * P - np.array(list(itf), dtype=np.float64)
    cell_substeps = 2.0 * updates
    total = np.array(list(c), dtype=np.float64)
    # every interface is evaluated twice (right of one cell, left of the next)
    I_avg = (total - cell_substeps * (5 * P + U)) / (2 * cell_substeps)
    out["algorithmic"] = _ops_dict(list(2 * (P + I_avg + U)))
    out["pieces"] = {"pressure": _ops_dict(list(P)), "cell_update": _ops_dict(list(U)),
                     "interface_mean": _ops_dict(list(I_avg))}
    return out


def swept(problem: OracleProblem, state: np.ndarray, steps: int, n: int) -> np.ndarray:
    """Advance ``state`` in place by ``steps`` timesteps, swept decomposition with
    nodes of ``n`` points."""
    dt = _state(problem, state)
    p = problem._c()
    _check(_load().orc_swept(ctypes.byref(p), dt, state.ctypes.data, int(steps), int(n)), "swept")
    return state


def stage(problem: OracleProblem, stage_index: int, stencil: np.ndarray, base: np.ndarray) -> np.ndarray:
    """One sub-timestep at one point in FP64, as the classic scheme evaluates
    it: ``stencil`` is (2 rad + 1, nv) (points i - rad .. i + rad), ``base``
    the point's nv values at the start of the timestep; stage 0 is the
    predictor (heat: its only step), 1 the final RK2 stage."""
    st = np.ascontiguousarray(stencil, dtype=np.float64).reshape(-1)
    b = np.ascontiguousarray(base, dtype=np.float64).reshape(-1)
    out = np.zeros(problem.nv)
    p = problem._c()
    _check(_load().orc_stage_f64(ctypes.byref(p), int(stage_index), st.ctypes.data, b.ctypes.data,
                                 out.ctypes.data), "stage")
    return out


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
