"""The C-ABI library builds, loads and exports every symbol include/swept.h
declares; host-side argument checks.  CPU only: no kernel runs here."""
import ctypes
import os
import re

import pytest

from paper_1705_03162_gb300 import build as B
from paper_1705_03162_gb300 import inputs as I
from paper_1705_03162_gb300 import swept as S

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    B.build()
    return S.load_library()


def _declared():
    text = open(os.path.join(ROOT, "include", "swept.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(swp_[a-z0-9_]+)\s*\(", text)))


def test_header_declares_binding_symbols():
    assert sorted(S.ABI_SYMBOLS) == _declared()


def test_library_exports_every_declared_symbol(lib):
    for name in _declared():
        assert hasattr(lib, name), name


def test_status_strings(lib):
    assert lib.swp_status_str(S.OK) == b"SWP_OK"
    assert lib.swp_status_str(S.ETIMEOUT) == b"SWP_ETIMEOUT"


def _create(lib, desc):
    h = ctypes.c_void_p(0)
    buf = (ctypes.c_double * 16)()
    return lib.swp_create(ctypes.byref(desc), buf, 0, None, ctypes.byref(h)), h


def test_create_rejects_bad_descriptions(lib):
    d = S.make_desc(I.ks_spec(64))
    d.eq = 7
    assert _create(lib, d)[0] == S.EINVAL
    d = S.make_desc(I.ks_spec(64))
    d.bc = S.REFLECTIVE
    assert _create(lib, d)[0] == S.EUNSUPPORTED
    d = S.make_desc(I.sod_spec(64), "f32")
    assert _create(lib, d)[0] == S.EUNSUPPORTED
    d = S.make_desc(I.heat_spec(64))
    d.dt = float("nan")
    assert _create(lib, d)[0] == S.EINVAL
    d = S.make_desc(I.heat_spec(64))
    d.n_points = 3
    assert _create(lib, d)[0] == S.EINVAL
    d = S.make_desc(I.heat_spec(64))
    d.reserved = 1
    assert _create(lib, d)[0] == S.EINVAL
    assert b"reserved" in lib.swp_last_error()


def test_create_null_arguments(lib):
    d = S.make_desc(I.heat_spec(64))
    assert lib.swp_create(ctypes.byref(d), None, 0, None, ctypes.byref(ctypes.c_void_p())) == S.EINVAL
    assert lib.swp_create(ctypes.byref(d), ctypes.c_void_p(1), 0, None, None) == S.EINVAL


def test_null_handles(lib):
    assert lib.swp_destroy(None) == S.OK
    assert lib.swp_advance(None, 1, S.SWEPT, 0) == S.EINVAL
    assert lib.swp_read(None, None, 0, 0) == S.EINVAL
    assert lib.swp_synchronize(None) == S.EINVAL
    assert lib.swp_kernel_launches(None) == -1


def test_required_bytes_and_budget(lib):
    assert S.required_bytes(I.sod_spec(1024)) == 2 * 3 * 1024 * 8
    assert S.required_bytes(I.heat_spec(1024), "f32") == 2 * 1024 * 4
    S.set_memory_budget(1000)
    try:
        d = S.make_desc(I.heat_spec(1024))
        st, _ = _create(lib, d)
        assert st == S.EBUDGET
        assert S.memory_in_use() == 0
    finally:
        S.set_memory_budget(0)


def test_missing_library_raises(tmp_path, monkeypatch):
    monkeypatch.setattr(S, "_lib", None)
    with pytest.raises(S.LibraryError):
        S.load_library(str(tmp_path / "nope.so"))


def test_tuned_choice_defaults_to_swept(lib):
    """With nothing measured for a key, SWP_SCHEME_AUTO means swept at the
    default width (no device needed to ask)."""
    d = S.make_desc(I.ks_spec(3 * 1024 + 512))
    sc, n = ctypes.c_int32(-1), ctypes.c_int32(-1)
    assert lib.swp_tuned(ctypes.byref(d), ctypes.byref(sc), ctypes.byref(n)) == S.OK
    assert (sc.value, n.value) == (S.SWEPT, 0)
    w = ctypes.c_int32(-1)
    assert lib.swp_tuned_width(ctypes.byref(d), ctypes.byref(w)) == S.OK and w.value == 0


def test_tuning_and_batch_entry_points_validate_on_the_host(lib):
    d = S.make_desc(I.ks_spec(1024))
    d.eq = 9
    sc, n = ctypes.c_int32(0), ctypes.c_int32(0)
    buf = (ctypes.c_double * 1024)()
    assert lib.swp_autotune(ctypes.byref(d), buf, 8, 10, ctypes.byref(sc), ctypes.byref(n)) == S.EINVAL
    d = S.make_desc(I.ks_spec(1024))
    assert lib.swp_autotune(ctypes.byref(d), None, 8, 10, ctypes.byref(sc), ctypes.byref(n)) == S.EINVAL
    assert lib.swp_autotune(ctypes.byref(d), buf, 0, 10, ctypes.byref(sc), ctypes.byref(n)) == S.EINVAL
    assert lib.swp_batch_advance_ex(None, None, None, 0, None, None, 0, 0) == S.EINVAL
    assert lib.swp_batch_kernel_launches(None) == -1
    assert lib.swp_batch_destroy(None) == S.OK


def test_fit_width_splits_n_into_nearly_equal_nodes(lib):
    """swp_fit_width (host arithmetic): at least two nodes, a multiple of
    4 rad, no wider than the target, the remainder widening nodes by at most
    4 rad; exact divisions keep the target; too-small N gives 0."""
    def fit(eq, N, w):
        out = ctypes.c_int32(-1)
        assert lib.swp_fit_width(eq, N, w, ctypes.byref(out)) == S.OK
        return out.value
    assert fit(S.KS, 1 << 20, 1024) == 1024 and fit(S.HEAT, 4096, 1024) == 1024
    assert fit(S.HEAT, 2049, 1024) == 680 and fit(S.KS, 3071, 1024) == 1016
    assert fit(S.HEAT, 7, 1024) == 0 and fit(S.KS, 15, 1024) == 0 and fit(S.KS, 16, 1024) == 8
    for eq, step in ((S.HEAT, 4), (S.KS, 8), (S.EULER, 8)):
        for N in list(range(2 * step, 700)) + [1023, 1025, 40001, 65535, (1 << 20) + 3]:
            for w in (step, 64, 100, 256, 1024, 2048):
                n = fit(eq, N, w)
                K, d = N // n, N % n
                assert n % step == 0 and step <= n <= max(w, step) and K >= 2, (eq, N, w, n)
                assert -(-d // K) <= step, (eq, N, w, n)
    out = ctypes.c_int32(0)
    assert lib.swp_fit_width(9, 1024, 256, ctypes.byref(out)) == S.EINVAL
    assert lib.swp_fit_width(S.KS, 0, 256, ctypes.byref(out)) == S.EINVAL
    assert lib.swp_fit_width(S.KS, 1024, 0, ctypes.byref(out)) == S.EINVAL
    assert lib.swp_fit_width(S.KS, 1024, 256, None) == S.EINVAL
    assert lib.swp_batch_tune_width(None, None, None, 0, None, 0, 0, None, None, None) == S.EINVAL


def test_scheme_enum_matches_header():
    text = open(os.path.join(ROOT, "include", "swept.h")).read()
    assert "SWP_CLASSIC = 0" in text and "SWP_SWEPT = 1" in text and "SWP_SCHEME_AUTO = 2" in text
    assert (S.CLASSIC, S.SWEPT, S.SCHEME_AUTO) == (0, 1, 2)


def test_batch_lists_must_match_problem_count():
    """A per-problem list shorter or longer than the problem list is an error
    in the binding (ctypes would zero-fill a short one: a silent 0-step
    advance)."""
    arr = S._per_problem("steps", [5, 6, 7], 3, ctypes.c_int64)
    assert list(arr) == [5, 6, 7]
    assert S._per_problem("n", None, 3, ctypes.c_int32) is None
    sc = S._per_problem("schemes", ["swept", "classic"], 2, ctypes.c_int32, lambda x: S._SCHEME[x])
    assert list(sc) == [S._SCHEME["swept"], S._SCHEME["classic"]]
    for bad in ([5, 6], [5, 6, 7, 8]):
        with pytest.raises(ValueError):
            S._per_problem("steps", bad, 3, ctypes.c_int64)


def test_host_state_checks_size_and_dtype():
    """Host initial states given by pointer (server submit, autotuners) are
    checked and converted in the binding: the library reads nv * N values."""
    import numpy as np
    spec = I.sod_spec(64)
    a = S._host_state(spec, np.zeros((3, 64)), "f64")
    assert a.dtype == np.float64 and a.flags.c_contiguous and a.size == 192
    b = S._host_state(I.ks_spec(64), np.zeros((1, 64)), "f32")
    assert b.dtype == np.float32
    with pytest.raises(ValueError):
        S._host_state(spec, np.zeros((1, 64)), "f64")
    with pytest.raises(ValueError):
        S._host_state(I.ks_spec(64), np.zeros(63), "f64")


def test_server_argument_errors_set_last_error(lib):
    """The serving entry points reject bad arguments on the host, before any
    device call, and say why through swp_last_error."""
    out = ctypes.c_void_p(0)
    cfg = S.ServerConfig(0, 0, 0, 5.0)   # max_active 0
    assert lib.swp_server_create(ctypes.byref(cfg), None, ctypes.byref(out)) == S.EINVAL
    assert b"max_active" in lib.swp_last_error()
    cfg = S.ServerConfig(0, 4, 0, 0.0)   # round_target_ms 0
    assert lib.swp_server_create(ctypes.byref(cfg), None, ctypes.byref(out)) == S.EINVAL
    assert lib.swp_server_create(None, None, ctypes.byref(out)) == S.EINVAL
    assert b"NULL" in lib.swp_last_error()
    rid = ctypes.c_int64(0)
    assert lib.swp_server_submit(None, None, None, 10, ctypes.byref(rid)) == S.EINVAL
    done = ctypes.c_int32(0)
    assert lib.swp_server_poll(None, 1, ctypes.byref(done)) == S.EINVAL
    assert b"server or done" in lib.swp_last_error()
    assert lib.swp_server_stats(None, None) == S.EINVAL
    assert lib.swp_server_destroy(None) == S.OK


class _FakeCudaTensor:
    """Stands in for a CUDA tensor on a machine without a GPU: the binding's
    checks of swept_noalloc run before any library or device call."""

    def __init__(self, numel, esize, dtype, index=0):
        self._numel, self._esize, self.dtype = numel, esize, dtype
        self.is_cuda = True
        self.device = type("Dev", (), {"index": index})()

    def data_ptr(self):
        return 0x10000

    def is_contiguous(self):
        return True

    def numel(self):
        return self._numel

    def element_size(self):
        return self._esize


def test_noalloc_binding_checks_size_dtype_and_device(monkeypatch):
    """swp_swept_noalloc takes no size argument, so the binding rejects a
    state of the wrong size, dtype or device before calling it."""
    torch = pytest.importorskip("torch")
    spec = I.sod_spec(64)
    calls = []
    lib = S.load_library()
    monkeypatch.setattr(S, "load_library", lambda: type("L", (), {
        "swp_swept_noalloc": lambda *a: calls.append(a) or 0})())
    with pytest.raises(ValueError, match="bytes"):
        S.swept_noalloc(spec, _FakeCudaTensor(3 * 63, 8, "torch.float64"), 10)
    with pytest.raises(ValueError, match="bytes"):   # float32 state passed as the default f64
        S.swept_noalloc(spec, _FakeCudaTensor(3 * 64, 4, "torch.float32"), 10)
    with pytest.raises(ValueError, match="dtype"):   # right size, wrong type
        S.swept_noalloc(spec, _FakeCudaTensor(3 * 64 * 2, 4, "torch.float32"), 10)
    monkeypatch.setattr(torch.cuda, "current_device", lambda: 0)
    with pytest.raises(ValueError, match="device"):
        S.swept_noalloc(spec, _FakeCudaTensor(3 * 64, 8, "torch.float64", index=1), 10)
    assert calls == []
    S.swept_noalloc(spec, _FakeCudaTensor(3 * 64, 8, "torch.float64"), 10)
    assert len(calls) == 1
    assert lib is not None
