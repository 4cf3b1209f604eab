"""Any grid size N.  The paper's swept nodes all hold n points, so N must be a
multiple of n (Section 4.2); the classic scheme (Section 5.1) has no such
rule.  Here N = K n + d is split into K nodes with the remainder d spread over
them (some nodes wider), and an N too small for any node width runs the
classic scheme.  Either way the result must equal the CPU oracle's classic
result bit for bit, alone, in a batch and served."""
import numpy as np
import pytest

import oracle as O
from helpers import oprob, spec_for, state_for
from paper_1705_03162_gb300 import build as B
from paper_1705_03162_gb300 import inputs as I
from paper_1705_03162_gb300 import swept as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    B.build()
    S.load_library()


def _oracle(spec, u0, steps):
    ref = np.ascontiguousarray(u0.copy())
    O.classic(oprob(spec), ref, steps)
    return ref


def _gpu(spec, u0, steps, dtype, n, launch, threads=0):
    with S.Problem(spec, u0, dtype) as p:
        p.advance(steps, "swept", n, launch, threads)
        return p.read()


# (eq, bc, N, n): N prime or odd; K = floor(N / n) nodes, remainder d
RAGGED = [
    ("heat", "periodic", 1031, 64),        # K 16, d 7
    ("heat", "reflective", 1031, 64),
    ("ks", "periodic", 1031, 64),
    ("euler", "dirichlet", 1031, 64),
    ("euler", "periodic", 999, 128),       # K 7, d 103: every node wider by 14 or 15
    ("ks", "periodic", 2 * 256 + 1, 256),  # K 2, the fewest nodes a remainder allows
    ("heat", "reflective", 3 * 128 - 1, 128),   # K 2, d 127
    ("ks", "periodic", 40001, 128),
]


@pytest.mark.parametrize("eq,bc,N,n", RAGGED)
@pytest.mark.parametrize("launch", ["per_phase", "persistent", "graph"])
def test_ragged_nodes_match_oracle(eq, bc, N, n, launch):
    spec = spec_for(eq, bc, N)
    u0 = state_for(spec, seed=N)
    H = n // (2 * spec.radius)
    # a partial half-cycle, and several full ones with a remainder
    for steps in (H // spec.substeps // 2 + 1, 3 * H // spec.substeps + 5):
        steps = min(steps, 400)
        got = _gpu(spec, u0, steps, "f64", n, launch)
        assert np.array_equal(got, _oracle(spec, u0, steps)), (launch, steps)


@pytest.mark.parametrize("eq,bc", [("heat", "periodic"), ("heat", "reflective"), ("ks", "periodic")])
@pytest.mark.parametrize("launch", ["per_phase", "persistent"])
def test_ragged_nodes_fp32_register_blocked(eq, bc, launch):
    """FP32 nodes of n points run their levels in registers; the wider ones
    (and those at non-periodic ends) in shared memory, in the same launch."""
    N, n = 8191, 512
    spec = spec_for(eq, bc, N)
    u0 = state_for(spec, np.float32, seed=5)
    steps = 301
    got = _gpu(spec, u0, steps, "f32", n, launch, threads=64)
    assert np.array_equal(got, _oracle(spec, u0, steps))


def test_ragged_large_dataflow():
    """KS at 2^19 + 3 points, 1024-point nodes, the dataflow launch the
    benchmark uses for large problems."""
    spec = I.ks_spec((1 << 19) + 3)
    u0 = state_for(spec, seed=3)
    got = _gpu(spec, u0, 130, "f64", 1024, "persistent")
    assert np.array_equal(got, _oracle(spec, u0, 130))


@pytest.mark.parametrize("eq,bc,N", [("heat", "periodic", 7), ("heat", "reflective", 6), ("ks", "periodic", 9),
                                     ("ks", "periodic", 15), ("euler", "dirichlet", 11)])
def test_tiny_n_runs_classic(eq, bc, N):
    """N below two nodes of 4 rad points: swept with the default width and
    SWP_SCHEME_AUTO run the classic scheme; an explicit width is an error."""
    spec = spec_for(eq, bc, N)
    u0 = state_for(spec, seed=N)
    steps = 37
    ref = _oracle(spec, u0, steps)
    for scheme, launch in (("swept", "auto"), ("auto", "auto"), ("swept", "graph"), ("classic", "auto")):
        with S.Problem(spec, u0) as p:
            p.advance(steps, scheme, 0, launch)
            assert np.array_equal(p.read(), ref), (scheme, launch)
    with S.Problem(spec, u0) as p:
        with pytest.raises(S.SweptError) as e:
            p.advance(steps, "swept", 4 * spec.radius)
        assert e.value.status == S.EINVAL


def _any_n_cases():
    # prime, odd and power-of-two-plus-a-bit sizes; default and explicit widths
    return [("heat", "periodic", 1031, 0), ("ks", "periodic", 40001, 0), ("ks", "periodic", (1 << 19) + 3, 0),
            ("euler", "dirichlet", 4099, 0), ("heat", "reflective", 12345, 256), ("ks", "periodic", 9, 0),
            ("heat", "periodic", 7, 0), ("euler", "periodic", 2049, 128), ("heat", "periodic", 65537, 1024)]


def test_batch_any_n_matches_oracle():
    torch = pytest.importorskip("torch")
    stream = torch.cuda.Stream()
    cases = _any_n_cases()
    probs, inputs, steps = [], [], []
    for i, (eq, bc, N, n) in enumerate(cases):
        spec = spec_for(eq, bc, N)
        u0 = state_for(spec, seed=N)
        inputs.append((spec, u0))
        probs.append(S.Problem(spec, u0, stream=stream))
        steps.append(60 + 37 * i)
    with S.Batch(stream) as b:
        b.advance(probs, steps, [c[3] for c in cases])
        b.advance_ex(probs, steps, None, [c[3] for c in cases], launch="graph")
        b.synchronize()
    for (eq, bc, N, n), (spec, u0), st, p in zip(cases, inputs, steps, probs):
        got = p.read()
        p.close()
        assert np.array_equal(got, _oracle(spec, u0, 2 * st)), (eq, bc, N, n)


def test_served_any_n_matches_oracle():
    cases = _any_n_cases()
    with S.Server(max_active=4, round_target_ms=0.05) as srv:
        ids = []
        for i, (eq, bc, N, _) in enumerate(cases):
            spec = spec_for(eq, bc, N)
            u0 = state_for(spec, seed=N + 1)
            ids.append((srv.submit(spec, u0, 50 + 23 * i), spec, u0, 50 + 23 * i))
        for rid, spec, u0, st in ids:
            got, _ = srv.wait(rid)
            assert np.array_equal(got, _oracle(spec, u0, st)), (spec.eq, spec.n_points)


# sizes on each side of every boundary of the library's default launch choice
# (cluster, Register graph, Shared graph, dataflow; FP32 per-phase)
AUTO_CASES = [(eq, N, dt) for dt in ("f64", "f32") for eq in ("heat", "ks")
              for N in (64, 1024, 2048, 4096, 8192, 1 << 14, (1 << 15) + 32, 1 << 17, (1 << 18) + 96)]


@pytest.mark.parametrize("eq,N,dtype", AUTO_CASES)
def test_default_launch_matches_oracle(eq, N, dtype):
    spec = spec_for(eq, "periodic", N)
    u0 = state_for(spec, np.float64 if dtype == "f64" else np.float32, seed=N)
    steps = 61 if N <= (1 << 15) else 17
    with S.Problem(spec, u0, dtype) as p:
        p.advance(steps, "swept")          # SWP_LAUNCH_AUTO, default width
        got = p.read()
    assert np.array_equal(got, _oracle(spec, u0, steps))


@pytest.mark.parametrize("N", [1 << 12, 1 << 13, (1 << 16) + 5, 1 << 18])
def test_default_launch_euler_matches_oracle(N):
    spec = spec_for("euler", "dirichlet", N)
    u0 = state_for(spec, seed=N)
    steps = 40
    with S.Problem(spec, u0) as p:
        p.advance(steps, "swept")
        got = p.read()
    assert np.array_equal(got, _oracle(spec, u0, steps))
