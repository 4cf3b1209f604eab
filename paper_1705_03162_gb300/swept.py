"""Thin ctypes binding of libswept.so (C ABI in include/swept.h).

Argument marshalling only: every step of the classic and swept schemes runs in
the library's CUDA kernels.  Host buffers are numpy arrays; device buffers are
CUDA torch tensors (torch provides device memory and streams).  A missing or
unloadable library raises :class:`LibraryError`; there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading
from typing import Optional

import numpy as np

from .inputs import ProblemSpec

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libswept.so")

OK, EINVAL, ENOMEM, EBUDGET, ECUDA, EUNSUPPORTED, ETIMEOUT, EDEVICE = range(8)
HEAT, KS, EULER = 0, 1, 2
PERIODIC, REFLECTIVE, DIRICHLET = 0, 1, 2
F64, F32 = 0, 1
CLASSIC, SWEPT, SCHEME_AUTO = 0, 1, 2
LAUNCH_AUTO, LAUNCH_PER_PHASE, LAUNCH_PERSISTENT, LAUNCH_GRAPH, LAUNCH_REGISTER, LAUNCH_CLUSTER = 0, 1, 2, 3, 4, 5

_EQ = {"heat": HEAT, "ks": KS, "euler": EULER}
_BC = {"periodic": PERIODIC, "reflective": REFLECTIVE, "dirichlet": DIRICHLET}
_SCHEME = {"classic": CLASSIC, "swept": SWEPT, "auto": SCHEME_AUTO}
_SCHEME_NAME = {CLASSIC: "classic", SWEPT: "swept"}
_LAUNCH = {"auto": LAUNCH_AUTO, "per_phase": LAUNCH_PER_PHASE, "persistent": LAUNCH_PERSISTENT,
           "graph": LAUNCH_GRAPH, "register": LAUNCH_REGISTER, "cluster": LAUNCH_CLUSTER}
_DTYPE = {"f64": F64, "f32": F32}

# every symbol include/swept.h declares
ABI_SYMBOLS = (
    "swp_create", "swp_write", "swp_advance", "swp_advance_ex", "swp_read", "swp_synchronize",
    "swp_destroy", "swp_shape", "swp_kernel_launches", "swp_required_bytes",
    "swp_set_memory_budget", "swp_memory_in_use", "swp_debug_withhold_flags",
    "swp_status_str", "swp_last_error", "swp_swept_noalloc",
    "swp_batch_create", "swp_batch_advance", "swp_batch_synchronize", "swp_batch_destroy",
    "swp_batch_kernel_launches", "swp_autotune_width", "swp_tuned_width",
    "swp_batch_advance_ex", "swp_autotune", "swp_tuned", "swp_fit_width", "swp_batch_tune_width",
    "swp_server_create", "swp_server_submit", "swp_server_poll", "swp_server_wait",
    "swp_server_stats", "swp_server_destroy",
)


class LibraryError(RuntimeError):
    """libswept.so is missing or could not be loaded."""


class SweptError(RuntimeError):
    def __init__(self, status: int, what: str, detail: str):
        super().__init__(f"{what}: {_status_name(status)}: {detail}")
        self.status = status


class Desc(ctypes.Structure):
    _fields_ = [
        ("eq", ctypes.c_int32), ("bc", ctypes.c_int32), ("dtype", ctypes.c_int32),
        ("reserved", ctypes.c_int32), ("n_points", ctypes.c_int64),
        ("dx", ctypes.c_double), ("dt", ctypes.c_double), ("alpha", ctypes.c_double),
        ("gamma", ctypes.c_double), ("left", ctypes.c_double * 3), ("right", ctypes.c_double * 3),
    ]


class ServerConfig(ctypes.Structure):
    _fields_ = [("hbm_budget_bytes", ctypes.c_size_t), ("max_active", ctypes.c_int32),
                ("threads", ctypes.c_int32), ("round_target_ms", ctypes.c_double)]


class ServerStats(ctypes.Structure):
    _fields_ = [("completed", ctypes.c_int64), ("rounds", ctypes.c_int64),
                ("kernel_launches", ctypes.c_int64), ("pending", ctypes.c_int64),
                ("active", ctypes.c_int64), ("device_bytes_in_use", ctypes.c_size_t),
                ("point_updates", ctypes.c_double), ("busy_span_s", ctypes.c_double)]


class AdvanceOpts(ctypes.Structure):
    _fields_ = [("scheme", ctypes.c_int32), ("points_per_block", ctypes.c_int32),
                ("launch", ctypes.c_int32), ("threads", ctypes.c_int32)]


_lib = None
_lock = threading.Lock()


def load_library(path: str = LIB_PATH):
    """Load libswept.so and declare its C signatures (raises LibraryError)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(path):
            raise LibraryError(f"{path} not found: build it with "
                               "`python -m paper_1705_03162_gb300.build`")
        try:
            lib = ctypes.CDLL(path)
        except OSError as e:
            raise LibraryError(f"cannot load {path}: {e}") from e
        vp, i32, i64, sz = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_size_t
        P = ctypes.c_void_p
        sig = {
            "swp_create": ([ctypes.POINTER(Desc), vp, ctypes.c_int, vp, ctypes.POINTER(P)], ctypes.c_int),
            "swp_write": ([P, vp, sz, ctypes.c_int], ctypes.c_int),
            "swp_advance": ([P, i64, i32, i32], ctypes.c_int),
            "swp_advance_ex": ([P, i64, ctypes.POINTER(AdvanceOpts)], ctypes.c_int),
            "swp_read": ([P, vp, sz, ctypes.c_int], ctypes.c_int),
            "swp_synchronize": ([P], ctypes.c_int),
            "swp_destroy": ([P], ctypes.c_int),
            "swp_shape": ([P, ctypes.POINTER(i64), ctypes.POINTER(i32), ctypes.POINTER(i32)], ctypes.c_int),
            "swp_kernel_launches": ([P], i64),
            "swp_required_bytes": ([ctypes.POINTER(Desc), ctypes.POINTER(sz)], ctypes.c_int),
            "swp_set_memory_budget": ([sz], ctypes.c_int),
            "swp_memory_in_use": ([], sz),
            "swp_debug_withhold_flags": ([P, ctypes.c_int, i64], ctypes.c_int),
            "swp_swept_noalloc": ([ctypes.POINTER(Desc), vp, i64, i32, i32, vp], ctypes.c_int),
            "swp_batch_create": ([vp, ctypes.POINTER(P)], ctypes.c_int),
            "swp_batch_advance": ([P, ctypes.POINTER(P), ctypes.POINTER(i64), i32,
                                   ctypes.POINTER(i32), i32], ctypes.c_int),
            "swp_batch_advance_ex": ([P, ctypes.POINTER(P), ctypes.POINTER(i64), i32, ctypes.POINTER(i32),
                                      ctypes.POINTER(i32), i32, i32], ctypes.c_int),
            "swp_batch_synchronize": ([P], ctypes.c_int),
            "swp_batch_destroy": ([P], ctypes.c_int),
            "swp_batch_kernel_launches": ([P], i64),
            "swp_autotune_width": ([ctypes.POINTER(Desc), vp, i32, i64, ctypes.POINTER(i32)], ctypes.c_int),
            "swp_tuned_width": ([ctypes.POINTER(Desc), ctypes.POINTER(i32)], ctypes.c_int),
            "swp_autotune": ([ctypes.POINTER(Desc), vp, i32, i64, ctypes.POINTER(i32), ctypes.POINTER(i32)],
                             ctypes.c_int),
            "swp_tuned": ([ctypes.POINTER(Desc), ctypes.POINTER(i32), ctypes.POINTER(i32)], ctypes.c_int),
            "swp_fit_width": ([i32, i64, i32, ctypes.POINTER(i32)], ctypes.c_int),
            "swp_batch_tune_width": ([P, ctypes.POINTER(P), ctypes.POINTER(i64), i32, ctypes.POINTER(i32), i32, i32,
                                      ctypes.POINTER(i32), ctypes.POINTER(ctypes.c_float), ctypes.POINTER(i32)],
                                     ctypes.c_int),
            "swp_server_create": ([ctypes.POINTER(ServerConfig), vp, ctypes.POINTER(P)], ctypes.c_int),
            "swp_server_submit": ([P, ctypes.POINTER(Desc), vp, i64, ctypes.POINTER(i64)], ctypes.c_int),
            "swp_server_poll": ([P, i64, ctypes.POINTER(i32)], ctypes.c_int),
            "swp_server_wait": ([P, i64, vp, sz, ctypes.POINTER(ctypes.c_double)], ctypes.c_int),
            "swp_server_stats": ([P, ctypes.POINTER(ServerStats)], ctypes.c_int),
            "swp_server_destroy": ([P], ctypes.c_int),
            "swp_status_str": ([ctypes.c_int], ctypes.c_char_p),
            "swp_last_error": ([], ctypes.c_char_p),
        }
        for name, (args, res) in sig.items():
            fn = getattr(lib, name)
            fn.argtypes = args
            fn.restype = res
        _lib = lib
        return lib


def _status_name(s: int) -> str:
    names = ["SWP_OK", "SWP_EINVAL", "SWP_ENOMEM", "SWP_EBUDGET", "SWP_ECUDA",
             "SWP_EUNSUPPORTED", "SWP_ETIMEOUT", "SWP_EDEVICE"]
    return names[s] if 0 <= s < len(names) else f"status {s}"


def _check(status: int, what: str):
    if status != OK:
        raise SweptError(status, what, load_library().swp_last_error().decode())


def make_desc(spec: ProblemSpec, dtype: str = "f64") -> Desc:
    d = Desc()
    d.eq, d.bc, d.dtype, d.reserved = _EQ[spec.eq], _BC[spec.bc], _DTYPE[dtype], 0
    d.n_points, d.dx, d.dt = spec.n_points, spec.dx, spec.dt
    d.alpha, d.gamma = spec.alpha, spec.gamma
    d.left = (ctypes.c_double * 3)(*spec.left)
    d.right = (ctypes.c_double * 3)(*spec.right)
    return d


def _buffer(x):
    """(pointer, bytes, on_device) of a numpy array or a torch tensor."""
    if isinstance(x, np.ndarray):
        if not x.flags.c_contiguous:
            raise ValueError("array must be C-contiguous")
        return x.ctypes.data, x.nbytes, 0
    if hasattr(x, "data_ptr") and hasattr(x, "is_cuda"):
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        nbytes = x.numel() * x.element_size()
        if x.is_cuda:
            return x.data_ptr(), nbytes, 1
        return x.data_ptr(), nbytes, 0
    raise TypeError(f"unsupported buffer type {type(x)}")


def _host_state(spec: ProblemSpec, u0, dtype: str) -> np.ndarray:
    """u0 as a C-contiguous host array of the problem's dtype, checked to hold
    nv * N values: the library reads exactly that many from the pointer."""
    a = np.ascontiguousarray(u0, dtype=np.float64 if dtype == "f64" else np.float32)
    if a.size != spec.nv * spec.n_points:
        raise ValueError(f"u0 has {a.size} values, expected {spec.nv} x {spec.n_points}")
    return a


def required_bytes(spec: ProblemSpec, dtype: str = "f64") -> int:
    lib = load_library()
    out = ctypes.c_size_t(0)
    _check(lib.swp_required_bytes(ctypes.byref(make_desc(spec, dtype)), ctypes.byref(out)), "required_bytes")
    return out.value


def set_memory_budget(nbytes: int):
    _check(load_library().swp_set_memory_budget(int(nbytes)), "set_memory_budget")


def memory_in_use() -> int:
    return int(load_library().swp_memory_in_use())


class Problem:
    """One 1D problem whose state lives in the library's device memory.

    ``u0`` is a numpy array (host) or CUDA tensor (device) of shape (nv, N) in
    the problem's dtype; ``stream`` is a ``torch.cuda.Stream`` (or raw
    cudaStream_t handle) or None for the default stream.
    """

    def __init__(self, spec: ProblemSpec, u0, dtype: str = "f64", stream=None):
        self._lib = load_library()
        self.spec, self.dtype = spec, dtype
        self.nv, self.n_points = spec.nv, spec.n_points
        self.np_dtype = np.float64 if dtype == "f64" else np.float32
        self._h = ctypes.c_void_p(0)
        handle = getattr(stream, "cuda_stream", stream) if stream is not None else None
        ptr, nbytes, dev = _buffer(u0)
        if nbytes != self.nbytes:
            raise ValueError(f"u0 has {nbytes} bytes, expected {self.nbytes}")
        self._desc = make_desc(spec, dtype)
        _check(self._lib.swp_create(ctypes.byref(self._desc), ctypes.c_void_p(ptr), dev,
                                    ctypes.c_void_p(handle), ctypes.byref(self._h)), "create")

    @property
    def nbytes(self) -> int:
        return self.nv * self.n_points * (8 if self.dtype == "f64" else 4)

    def advance(self, steps: int, scheme: str = "swept", n: int = 0, launch: str = "auto",
                threads: int = 0):
        o = AdvanceOpts(_SCHEME[scheme], int(n), _LAUNCH[launch], int(threads))
        _check(self._lib.swp_advance_ex(self._h, int(steps), ctypes.byref(o)), "advance")
        return self

    def read(self, out=None):
        """Copy the state into ``out`` (numpy or CUDA tensor) or a new numpy array."""
        if out is None:
            out = np.empty((self.nv, self.n_points), dtype=self.np_dtype)
        ptr, nbytes, dev = _buffer(out)
        _check(self._lib.swp_read(self._h, ctypes.c_void_p(ptr), nbytes, dev), "read")
        return out

    def write(self, src):
        ptr, nbytes, dev = _buffer(src)
        _check(self._lib.swp_write(self._h, ctypes.c_void_p(ptr), nbytes, dev), "write")

    def synchronize(self):
        _check(self._lib.swp_synchronize(self._h), "synchronize")

    def kernel_launches(self) -> int:
        return int(self._lib.swp_kernel_launches(self._h))

    def debug_withhold_flags(self, withhold: bool, wait_limit_ns: int = 2_000_000_000):
        _check(self._lib.swp_debug_withhold_flags(self._h, int(bool(withhold)), int(wait_limit_ns)),
               "debug_withhold_flags")

    def close(self):
        if self._h and self._h.value:
            _check(self._lib.swp_destroy(self._h), "destroy")
            self._h = ctypes.c_void_p(0)

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def solve(spec: ProblemSpec, u0: np.ndarray, steps: int, scheme: str = "swept", n: int = 0,
          dtype: Optional[str] = None, launch: str = "auto", threads: int = 0) -> np.ndarray:
    """Create, advance ``steps`` timesteps and read back (host arrays)."""
    dtype = dtype or ("f32" if u0.dtype == np.float32 else "f64")
    with Problem(spec, np.ascontiguousarray(u0), dtype) as p:
        p.advance(steps, scheme, n, launch, threads)
        return p.read()


def swept_noalloc(spec: ProblemSpec, state, steps: int, n: int = 0, threads: int = 0,
                  stream=None, dtype: str = "f64"):
    """Advance the CUDA tensor ``state`` (shape (nv, N)) in place by ``steps``
    timesteps with the swept scheme through swp_swept_noalloc, which allocates
    no device memory (its scratch is a fixed 8 MiB array inside the library).
    Asynchronous on ``stream``; calls that overlap on the GPU race.

    swp_swept_noalloc takes no size argument, so the tensor is checked here
    before any call: it must hold exactly nv * N values of ``dtype`` and live
    on the current CUDA device."""
    lib = load_library()
    ptr, nbytes, dev = _buffer(state)
    if not dev:
        raise ValueError("state must be a CUDA tensor")
    if dtype not in _DTYPE:
        raise ValueError(f"unknown dtype {dtype!r}")
    esize = 8 if dtype == "f64" else 4
    want = spec.nv * spec.n_points * esize
    if nbytes != want:
        raise ValueError(f"state has {nbytes} bytes, expected {spec.nv} x {spec.n_points} x {esize} = {want}")
    tdt = str(getattr(state, "dtype", ""))
    if tdt != ("torch.float64" if dtype == "f64" else "torch.float32"):
        raise ValueError(f"state dtype {tdt} does not match the problem dtype {dtype!r}")
    index = getattr(getattr(state, "device", None), "index", None)
    import torch
    if index is None or index != torch.cuda.current_device():
        raise ValueError(f"state is on device {index}, not the current CUDA device")
    desc = make_desc(spec, dtype)
    handle = getattr(stream, "cuda_stream", stream) if stream is not None else None
    _check(lib.swp_swept_noalloc(ctypes.byref(desc), ctypes.c_void_p(ptr), int(steps), int(n),
                                 int(threads), ctypes.c_void_p(handle)), "swept_noalloc")
    return state


def _per_problem(name: str, values, count: int, ctype, convert=int):
    """ctypes array of one value per problem (None stays None); a list of
    another length is an error, not a silent zero fill."""
    if values is None:
        return None
    values = list(values)
    if len(values) != count:
        raise ValueError(f"{name} has {len(values)} entries for {count} problems")
    return (ctype * count)(*[convert(x) for x in values])


class Batch:
    """Batched advance: many problems (created with this batch's stream)
    advanced together in one persistent launch per (equation, dtype) group."""

    def __init__(self, stream=None):
        self._lib = load_library()
        self._h = ctypes.c_void_p(0)
        handle = getattr(stream, "cuda_stream", stream) if stream is not None else None
        _check(self._lib.swp_batch_create(ctypes.c_void_p(handle), ctypes.byref(self._h)), "batch_create")

    def advance(self, problems, steps, n=None, threads: int = 0):
        count = len(problems)
        hs = (ctypes.c_void_p * count)(*[p._h.value for p in problems])
        st = _per_problem("steps", steps, count, ctypes.c_int64)
        nn = _per_problem("n", n, count, ctypes.c_int32)
        _check(self._lib.swp_batch_advance(self._h, hs, st, count, nn, int(threads)), "batch_advance")

    def advance_ex(self, problems, steps, schemes=None, n=None, threads: int = 0, launch: str = "auto"):
        """Per-problem scheme ("swept", "classic" or "auto"; None = all auto)
        and width (node or chunk); launch "auto" or "graph"."""
        count = len(problems)
        hs = (ctypes.c_void_p * count)(*[p._h.value for p in problems])
        st = _per_problem("steps", steps, count, ctypes.c_int64)
        sc = _per_problem("schemes", schemes, count, ctypes.c_int32, lambda x: _SCHEME[x])
        nn = _per_problem("n", n, count, ctypes.c_int32)
        _check(self._lib.swp_batch_advance_ex(self._h, hs, st, count, sc, nn, int(threads), _LAUNCH[launch]),
               "batch_advance_ex")

    def tune_width(self, problems, steps, candidates=(256, 512, 1024, 2048), threads: int = 0):
        """swp_batch_tune_width: each candidate target width fitted to every
        problem's N and timed on one advance of the whole batch (states put
        back after each); returns (widths of the fastest, its index, the
        milliseconds of every candidate)."""
        count, nc = len(problems), len(candidates)
        hs = (ctypes.c_void_p * count)(*[p._h.value for p in problems])
        st = _per_problem("steps", steps, count, ctypes.c_int64)
        cand = (ctypes.c_int32 * nc)(*[int(c) for c in candidates])
        out = (ctypes.c_int32 * count)()
        ms = (ctypes.c_float * nc)()
        best = ctypes.c_int32(-1)
        _check(self._lib.swp_batch_tune_width(self._h, hs, st, count, cand, nc, int(threads), out, ms,
                                              ctypes.byref(best)), "batch_tune_width")
        return list(out), int(best.value), [float(x) for x in ms]

    def synchronize(self):
        _check(self._lib.swp_batch_synchronize(self._h), "batch_synchronize")

    def kernel_launches(self) -> int:
        return int(self._lib.swp_batch_kernel_launches(self._h))

    def close(self):
        if self._h and self._h.value:
            _check(self._lib.swp_batch_destroy(self._h), "batch_destroy")
            self._h = ctypes.c_void_p(0)

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def autotune_width(spec: ProblemSpec, u0: np.ndarray, count: int = 16, steps: int = 200,
                   dtype: str = "f64") -> int:
    """Time ``count`` copies of the problem in one batch for each node width and
    keep the fastest for later batches of this (equation, dtype, N)."""
    lib = load_library()
    u0 = _host_state(spec, u0, dtype)
    out = ctypes.c_int32(0)
    _check(lib.swp_autotune_width(ctypes.byref(make_desc(spec, dtype)), u0.ctypes.data, int(count),
                                  int(steps), ctypes.byref(out)), "autotune_width")
    return out.value


def fit_width(eq: str, n_points: int, target: int) -> int:
    """swp_fit_width: the node width for n_points from a target width (N in
    nearly equal nodes, none wider than target + 4 rad); 0 if none fits."""
    out = ctypes.c_int32(0)
    _check(load_library().swp_fit_width(_EQ[eq], int(n_points), int(target), ctypes.byref(out)), "fit_width")
    return int(out.value)


def tuned_width(spec: ProblemSpec, dtype: str = "f64") -> int:
    out = ctypes.c_int32(0)
    _check(load_library().swp_tuned_width(ctypes.byref(make_desc(spec, dtype)), ctypes.byref(out)),
           "tuned_width")
    return out.value


def autotune(spec: ProblemSpec, u0: np.ndarray, count: int = 16, steps: int = 200, dtype: str = "f64"):
    """Time the swept widths and the classic scheme in batches of ``count``
    copies; keep the faster for this (equation, dtype, N).  Returns
    (scheme name, width)."""
    lib = load_library()
    u0 = _host_state(spec, u0, dtype)
    sc, n = ctypes.c_int32(0), ctypes.c_int32(0)
    _check(lib.swp_autotune(ctypes.byref(make_desc(spec, dtype)), u0.ctypes.data, int(count), int(steps),
                            ctypes.byref(sc), ctypes.byref(n)), "autotune")
    return _SCHEME_NAME[sc.value], n.value


def tuned(spec: ProblemSpec, dtype: str = "f64"):
    sc, n = ctypes.c_int32(0), ctypes.c_int32(0)
    _check(load_library().swp_tuned(ctypes.byref(make_desc(spec, dtype)), ctypes.byref(sc), ctypes.byref(n)),
           "tuned")
    return _SCHEME_NAME[sc.value], n.value


class Server:
    """Serving loop with continuous batching (scheduler thread in libswept)."""

    def __init__(self, hbm_budget_bytes: int = 0, max_active: int = 256, round_target_ms: float = 5.0,
                 threads: int = 0, stream=None):
        self._lib = load_library()
        self._h = ctypes.c_void_p(0)
        cfg = ServerConfig(int(hbm_budget_bytes), int(max_active), int(threads), float(round_target_ms))
        handle = getattr(stream, "cuda_stream", stream) if stream is not None else None
        _check(self._lib.swp_server_create(ctypes.byref(cfg), ctypes.c_void_p(handle), ctypes.byref(self._h)),
               "server_create")
        self._shapes = {}

    def submit(self, spec: ProblemSpec, u0: np.ndarray, steps: int, dtype: str = "f64") -> int:
        u0 = _host_state(spec, u0, dtype)
        rid = ctypes.c_int64(0)
        _check(self._lib.swp_server_submit(self._h, ctypes.byref(make_desc(spec, dtype)), u0.ctypes.data,
                                           int(steps), ctypes.byref(rid)), "server_submit")
        self._shapes[rid.value] = (u0.shape, u0.dtype)
        return rid.value

    def done(self, rid: int) -> bool:
        d = ctypes.c_int32(0)
        _check(self._lib.swp_server_poll(self._h, int(rid), ctypes.byref(d)), "server_poll")
        return bool(d.value)

    def wait(self, rid: int):
        """(final state as numpy, latency in seconds); raises on a failed request."""
        shape, dt = self._shapes.pop(rid)
        out = np.empty(shape, dtype=dt)
        lat = ctypes.c_double(0.0)
        _check(self._lib.swp_server_wait(self._h, int(rid), out.ctypes.data, out.nbytes, ctypes.byref(lat)),
               f"server_wait (request {rid})")
        return out, lat.value

    def stats(self) -> dict:
        s = ServerStats()
        _check(self._lib.swp_server_stats(self._h, ctypes.byref(s)), "server_stats")
        return {f: getattr(s, f) for f, _ in ServerStats._fields_}

    def close(self):
        if self._h and self._h.value:
            self._lib.swp_server_destroy(self._h)
            self._h = ctypes.c_void_p(0)

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
