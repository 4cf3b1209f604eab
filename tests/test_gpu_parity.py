"""GPU parity: the CUDA classic and swept paths against the CPU oracle, element
by element on the same seeded inputs, and against each other bit for bit.

Tolerances (relative max-norm per variable): 1e-12 for FP64, 1e-5 for FP32
(against the oracle run in the same precision).  Both CUDA paths evaluate the
same device point update with explicit round-to-nearest operations in the
oracle's order, so they are also checked to be bit-identical to the oracle.
Sizes span several classic tiles (512 points) and several swept nodes with a
ragged tail; step counts leave remainders of the swept half-cycle.
"""
import numpy as np
import pytest

import oracle as O
from helpers import oprob, rel_max, spec_for, state_for
from paper_1705_03162_gb300 import build as B
from paper_1705_03162_gb300 import inputs as I
from paper_1705_03162_gb300 import swept as S

pytestmark = pytest.mark.gpu

TOL = {"f64": 1e-12, "f32": 1e-5}


@pytest.fixture(scope="module", autouse=True)
def _lib():
    B.build()
    S.load_library()


def _np(dtype):
    return np.float64 if dtype == "f64" else np.float32


def _gpu(spec, u0, steps, dtype, scheme, n=0, launch="per_phase"):
    with S.Problem(spec, u0, dtype) as p:
        p.advance(steps, scheme, n, launch)
        return p.read()


def _oracle(spec, u0, steps):
    ref = u0.copy()
    O.classic(oprob(spec), ref, steps)
    return ref


CASES = [
    # eq, bc, N, dtype, steps, node widths
    ("heat", "periodic", 4992, "f64", 203, (32, 64, 128)),
    ("heat", "reflective", 4992, "f64", 157, (32, 64, 128)),
    ("heat", "periodic", 4992, "f32", 203, (32, 128)),
    ("heat", "reflective", 4992, "f32", 90, (64,)),
    ("ks", "periodic", 4992, "f64", 301, (32, 96, 128)),
    ("ks", "periodic", 4992, "f32", 301, (64, 128)),
    ("euler", "dirichlet", 4992, "f64", 333, (32, 64, 128)),
    ("euler", "periodic", 4992, "f64", 211, (32, 104)),
]


@pytest.mark.parametrize("eq,bc,N,dtype,steps,widths", CASES)
def test_classic_matches_oracle(eq, bc, N, dtype, steps, widths):
    spec = spec_for(eq, bc, N)
    u0 = state_for(spec, _np(dtype))
    ref = _oracle(spec, u0, steps)
    got = _gpu(spec, u0, steps, dtype, "classic")
    assert rel_max(got, ref) <= TOL[dtype]
    assert np.array_equal(got, ref), "classic is not bit-identical to the oracle"


@pytest.mark.parametrize("eq,bc,N,dtype", [("heat", "periodic", 4993, "f64"), ("heat", "reflective", 4993, "f32"),
                                           ("ks", "periodic", 4998, "f32"), ("ks", "periodic", 4999, "f64"),
                                           ("heat", "periodic", 64, "f32"), ("ks", "periodic", 130, "f64")])
def test_classic_sizes_off_the_vector_width(eq, bc, N, dtype):
    """N not a multiple of the 16-byte vector width (or too small) takes the
    shared-memory classic kernel; both forms must agree with the oracle."""
    spec = spec_for(eq, bc, N)
    u0 = state_for(spec, _np(dtype))
    ref = _oracle(spec, u0, 97)
    got = _gpu(spec, u0, 97, dtype, "classic")
    assert np.array_equal(got, ref)


@pytest.mark.parametrize("eq,bc,N,dtype,steps,widths", CASES)
@pytest.mark.parametrize("launch", ["per_phase", "persistent", "graph"])
def test_swept_matches_oracle_and_classic(eq, bc, N, dtype, steps, widths, launch):
    spec = spec_for(eq, bc, N)
    u0 = state_for(spec, _np(dtype))
    ref = _oracle(spec, u0, steps)
    classic = _gpu(spec, u0, steps, dtype, "classic")
    for n in widths:
        got = _gpu(spec, u0, steps, dtype, "swept", n, launch)
        assert rel_max(got, ref) <= TOL[dtype], f"n={n}"
        assert np.array_equal(got, classic), f"swept != classic bitwise at n={n}"


@pytest.mark.parametrize("eq,bc", [("heat", "periodic"), ("heat", "reflective"), ("ks", "periodic"),
                                   ("euler", "dirichlet")])
@pytest.mark.parametrize("steps", [0, 1, 2, 5, 16, 17, 33])
def test_swept_short_and_ragged_advances(eq, bc, steps):
    N, n = 512, 64
    spec = spec_for(eq, bc, N)
    u0 = state_for(spec)
    ref = _oracle(spec, u0, steps)
    for launch in ("per_phase", "persistent"):
        got = _gpu(spec, u0, steps, "f64", "swept", n, launch)
        assert np.array_equal(got, ref), (launch, steps)


@pytest.mark.parametrize("eq,bc,N,n", [
    ("ks", "periodic", 256, 256),        # a single node
    ("ks", "periodic", 512, 256),        # two nodes
    ("heat", "periodic", 128, 128),
    ("heat", "reflective", 256, 128),
    ("euler", "dirichlet", 256, 128),
    ("ks", "periodic", 65536, 8192),     # widest KS node in shared memory
    ("heat", "periodic", 65536, 8192),
    ("euler", "dirichlet", 16384, 2048),
])
def test_swept_node_count_extremes(eq, bc, N, n):
    spec = spec_for(eq, bc, N)
    u0 = state_for(spec)
    steps = 3 * n // (2 * spec.radius * spec.substeps) + 5
    steps = min(steps, 700)
    ref = _oracle(spec, u0, steps)
    for launch in ("per_phase", "persistent"):
        got = _gpu(spec, u0, steps, "f64", "swept", n, launch)
        assert np.array_equal(got, ref), launch


@pytest.mark.parametrize("launch", ["per_phase", "persistent"])
def test_split_advances_equal_one_advance(launch):
    """The state is complete after every advance (closing triangle), so
    advancing a then b steps equals advancing a + b (checkpoint / resume)."""
    spec = spec_for("ks", "periodic", 2048)
    u0 = state_for(spec)
    with S.Problem(spec, u0) as p:
        p.advance(37, "swept", 128, launch)
        mid = p.read()
        p.advance(85, "swept", 64, launch)
        end = p.read()
    with S.Problem(spec, mid) as q:
        q.advance(85, "classic")
        end2 = q.read()
    assert np.array_equal(mid, _oracle(spec, u0, 37))
    assert np.array_equal(end, end2)


def test_heat_config_closed_form_and_oracle():
    """Heat configuration: N = 1024, r = 0.25, 4096 steps, 64 points per node."""
    spec = I.heat_spec(1024, r=0.25)
    u0 = I.initial_state(spec)
    ref = _oracle(spec, u0, 4096)
    for launch in ("per_phase", "persistent"):
        got = _gpu(spec, u0, 4096, "f64", "swept", 64, launch)
        assert np.array_equal(got, ref)
    x = np.arange(1024) / 1024
    G = lambda k: 1.0 - np.sin(np.pi * k / 1024) ** 2
    exact = np.sin(2 * np.pi * x) * G(1) ** 4096
    for k, a in zip(range(2, 10), I.heat_mode_amplitudes()):
        exact += a * np.sin(2 * np.pi * k * x) * G(k) ** 4096
    assert rel_max(got[0], exact) < 1e-11


def test_sod_full_time_against_oracle():
    """Sod tube to t = 0.2 (N steps at dt/dx = 0.2), N = 2^12."""
    N = 4096
    spec = I.sod_spec(N)
    u0 = I.initial_state(spec)
    ref = _oracle(spec, u0, N)
    got_c = _gpu(spec, u0, N, "f64", "classic")
    got_s = _gpu(spec, u0, N, "f64", "swept", 256, "persistent")
    assert rel_max(got_c, ref) <= 1e-12 and rel_max(got_s, ref) <= 1e-12
    assert np.array_equal(got_s, got_c)


@pytest.mark.parametrize("eq,bc", [("heat", "periodic"), ("heat", "reflective"), ("ks", "periodic"),
                                   ("euler", "dirichlet")])
def test_graph_replay_matches_stream_launches(eq, bc):
    """Graph launches (captured once, replayed) give the stream launches' bits,
    on repeated identical advances and with the starting row alternating."""
    spec = spec_for(eq, bc, 2048)
    u0 = state_for(spec)
    with S.Problem(spec, u0) as a, S.Problem(spec, u0) as b:
        for steps, n in ((33, 64), (33, 64), (20, 128), (33, 64), (7, 64)):
            a.advance(steps, "swept", n, "per_phase")
            b.advance(steps, "swept", n, "graph")
            assert np.array_equal(a.read(), b.read())
        for steps in (5, 5, 6):
            a.advance(steps, "classic")
            b.advance(steps, "classic", launch="graph")
            assert np.array_equal(a.read(), b.read())


@pytest.mark.parametrize("eq,N,dtype,steps", [("ks", 4992, "f64", 301), ("ks", 4992, "f32", 150),
                                            ("heat", 4992, "f64", 203), ("heat", 96, "f32", 61),
                                            ("ks", 64, "f64", 9)])
def test_register_variant_matches_oracle(eq, N, dtype, steps):
    """The Register variant (one warp per node of 32 points, levels in
    registers) gives the oracle's bits, remainders and a two-node ring included."""
    spec = spec_for(eq, "periodic", N)
    u0 = state_for(spec, _np(dtype))
    ref = _oracle(spec, u0, steps)
    for threads in (32, 256):
        with S.Problem(spec, u0, dtype) as p:
            p.advance(steps, "swept", 0, "register", threads)
            assert np.array_equal(p.read(), ref)


def test_register_variant_rejects_unsupported():
    spec = spec_for("heat", "reflective", 256)
    with S.Problem(spec, state_for(spec)) as p:
        with pytest.raises(S.SweptError) as e:
            p.advance(5, "swept", 0, "register")
        assert e.value.status == S.EUNSUPPORTED
    spec = spec_for("ks", "periodic", 256)
    with S.Problem(spec, state_for(spec)) as p:
        with pytest.raises(S.SweptError) as e:
            p.advance(5, "swept", 64, "register")
        assert e.value.status == S.EINVAL


@pytest.mark.parametrize("eq", ["heat", "ks"])
def test_large_size_swept_equals_classic(eq):
    """At N = 2^24 (FP32 arrays of 64 MB, the bandwidth regime of the classic
    kernel) the swept and classic paths still agree bit for bit."""
    N = 1 << 24
    spec = spec_for(eq, "periodic", N)
    u0 = I.initial_state(spec, np.float32)
    steps = 600 if eq == "heat" else 150
    a = _gpu(spec, u0, steps, "f32", "classic")
    b = _gpu(spec, u0, steps, "f32", "swept", 4096 if eq == "heat" else 1024)
    assert np.array_equal(a, b)
    assert np.all(np.isfinite(a))


@pytest.mark.parametrize("eq,N,steps", [("ks", 1 << 26, 300), ("heat", 1 << 27, 1100)])
def test_large_fp64_dataflow_equals_classic(eq, N, steps):
    """FP64 grids of 0.5-1 GB per row through the default launch (the dataflow
    kernel from 2^17 points): bit-identical to classic, with several full
    half-cycles and a remainder."""
    spec = spec_for(eq, "periodic", N)
    u0 = I.initial_state(spec)
    a = _gpu(spec, u0, steps, "f64", "classic")
    b = _gpu(spec, u0, steps, "f64", "swept", 0, "auto")
    assert np.array_equal(a, b)
    assert np.all(np.isfinite(a))


@pytest.mark.parametrize("eq,n,steps", [("heat", 64, 4096), ("heat", 64, 100), ("ks", 128, 333), ("euler", 64, 50)])
def test_phase_count_matches_oracle_geometry(eq, n, steps):
    """The per-phase launch issues exactly the oracle's kernels: upright
    triangle, diamonds, closing triangle (and a truncated one for a
    remainder)."""
    bc = "dirichlet" if eq == "euler" else "periodic"
    spec = spec_for(eq, bc, 16 * n)
    g = O.swept_geometry({"heat": O.HEAT, "ks": O.KS, "euler": O.EULER}[eq], n, steps)
    with S.Problem(spec, state_for(spec)) as p:
        k0 = p.kernel_launches()
        p.advance(steps, "swept", n, "per_phase")
        assert p.kernel_launches() - k0 == g["kernels"]


def test_invalid_node_width_rejected():
    spec = spec_for("ks", "periodic", 1000)
    with S.Problem(spec, state_for(spec)) as p:
        for n in (12, 48 + 4, 2000, 1 << 20):
            with pytest.raises(S.SweptError) as e:
                p.advance(10, "swept", n)
            assert e.value.status == S.EINVAL


def test_device_buffers_roundtrip():
    torch = pytest.importorskip("torch")
    spec = spec_for("ks", "periodic", 4096)
    u0 = state_for(spec)
    dev = torch.from_numpy(u0).cuda()
    s = torch.cuda.Stream()
    with S.Problem(spec, dev, stream=s) as p:
        p.advance(50, "swept", 256)
        out = torch.empty_like(dev)
        p.read(out)
        s.synchronize()
    assert np.array_equal(out.cpu().numpy(), _oracle(spec, u0, 50))


@pytest.mark.parametrize("eq,bc", [("heat", "periodic"), ("heat", "reflective"), ("ks", "periodic")])
@pytest.mark.parametrize("n,threads", [(128, 64), (256, 64), (512, 64), (1024, 64), (256, 32), (512, 256)])
@pytest.mark.parametrize("launch", ["per_phase", "persistent"])
def test_fp32_register_blocked_levels(eq, bc, n, threads, launch):
    """FP32 heat / KS nodes run their levels register-blocked when the block
    splits the node into 2, 4, 8 or 16 slots per thread (the cases cover each);
    nodes next to a reflective end keep the shared-memory levels.  Several
    full cycles plus a remainder; bit-identical to the oracle and to classic."""
    N, steps = 3072, 2 * (n // 2) + 37
    spec = spec_for(eq, bc, N)
    u0 = state_for(spec, np.float32, seed=n + threads)
    ref = _oracle(spec, u0, steps)
    with S.Problem(spec, u0, "f32") as p:
        p.advance(steps, "swept", n, launch, threads)
        got = p.read()
    assert np.array_equal(got, ref), (eq, bc, n, threads, launch)
    assert np.array_equal(got, _gpu(spec, u0, steps, "f32", "classic"))


@pytest.mark.parametrize("eq,bc", [("heat", "periodic"), ("heat", "reflective"), ("ks", "periodic")])
@pytest.mark.parametrize("N,n,threads", [(10007, 1000, 96), (10007, 1000, 160), (8192, 2048, 64),
                                         (6151, 2048, 32), (4099, 64, 224)])
@pytest.mark.parametrize("launch", ["per_phase", "persistent"])
def test_fp32_shared_memory_level_runs(eq, bc, N, n, threads, launch):
    """FP32 heat / KS nodes beyond the register-blocked slot counts sweep
    their levels in shared memory, each thread a contiguous run: block sizes
    that are not powers of two (96, 160, 224: the run length by division),
    runs of 32 and 64 slots, prime and odd N (wider nodes from the
    remainder), and a block wider than the node.  Bit-identical to the oracle
    and to classic."""
    steps = 2 * (n // 2) + 37 if eq == "heat" else n + 37
    spec = spec_for(eq, bc, N)
    u0 = state_for(spec, np.float32, seed=N + n + threads)
    ref = _oracle(spec, u0, steps)
    with S.Problem(spec, u0, "f32") as p:
        p.advance(steps, "swept", n, launch, threads)
        got = p.read()
    assert np.array_equal(got, ref), (eq, bc, N, n, threads, launch)
    assert np.array_equal(got, _gpu(spec, u0, steps, "f32", "classic"))
