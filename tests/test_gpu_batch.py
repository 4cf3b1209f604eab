"""Batched swept advance: every problem of a mixed batch (equations, sizes,
step counts, node widths, precisions) ends bit-identical to advancing it
alone, and to the CPU oracle."""
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


def _mix(seed=3, count=40):
    rng = np.random.default_rng(seed)
    cases = []
    for i in range(count):
        eq, bc = [("heat", "periodic"), ("heat", "reflective"), ("ks", "periodic"),
                  ("euler", "dirichlet")][i % 4]
        N = int(2 ** rng.integers(9, 13)) * (1 if i % 3 else 3)
        steps = int(rng.integers(1, 400))
        n = [0, 32, 64, 128][i % 4] if N % 128 == 0 else 32
        dtype = "f32" if (eq != "euler" and i % 5 == 0) else "f64"
        cases.append((eq, bc, N, steps, n, dtype))
    return cases


def test_batch_matches_single_and_oracle():
    torch = pytest.importorskip("torch")
    stream = torch.cuda.Stream()
    cases = _mix()
    probs, inputs = [], []
    for eq, bc, N, steps, n, dtype in cases:
        spec = spec_for(eq, bc, N)
        u0 = state_for(spec, np.float64 if dtype == "f64" else np.float32, seed=N + steps)
        inputs.append((spec, u0))
        probs.append(S.Problem(spec, u0, dtype, stream=stream))
    widths = [n for (_, _, _, _, n, _) in cases]
    with S.Batch(stream) as b:
        b.advance(probs, [c[3] for c in cases], widths)
        b.synchronize()
        assert b.kernel_launches() == 3   # heat+KS FP64, heat+KS FP32, Euler FP64
    for (eq, bc, N, steps, n, dtype), (spec, u0), p in zip(cases, inputs, probs):
        got = p.read()
        p.close()
        with S.Problem(spec, u0, dtype) as q:
            q.advance(steps, "swept", n if n else 0)
            alone = q.read()
        assert np.array_equal(got, alone), (eq, bc, N, steps, n, dtype)
        ref = u0.copy()
        O.classic(oprob(spec), ref, steps)
        assert np.array_equal(got, ref), (eq, bc, N, steps, n, dtype)


def test_batch_consecutive_advances_and_zero_steps():
    torch = pytest.importorskip("torch")
    stream = torch.cuda.Stream()
    spec = I.ks_spec(4096)
    u0 = state_for(spec)
    ps = [S.Problem(spec, u0, stream=stream) for _ in range(3)]
    with S.Batch(stream) as b:
        b.advance(ps, [50, 0, 7], [256, 256, 128])
        b.advance(ps, [25, 75, 68], [128, 256, 256])
        b.synchronize()
    ref = u0.copy()
    O.classic(oprob(spec), ref, 75)
    for p in ps:
        assert np.array_equal(p.read(), ref)
        p.close()


def test_batch_rejects_bad_input():
    torch = pytest.importorskip("torch")
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    spec = I.ks_spec(1024)
    p = S.Problem(spec, state_for(spec), stream=s1)
    with S.Batch(s2) as b:
        with pytest.raises(S.SweptError) as e:
            b.advance([p], [10])
        assert e.value.status == S.EINVAL
    with S.Batch(s1) as b:
        with pytest.raises(S.SweptError):
            b.advance([p, p], [10, 10])
        with pytest.raises(S.SweptError):
            b.advance([p], [10], [12])
    p.close()


def test_autotune_picks_a_valid_width():
    spec = I.ks_spec(8192)
    u0 = I.initial_state(spec)
    n = S.autotune_width(spec, u0, count=8, steps=64)
    assert n >= 32 and 8192 % n == 0 and n % 8 == 0
    assert S.tuned_width(spec) == n


def _classic_mix(seed=5, count=25):
    """Classic instances of every supported pairing, ragged sizes, chunk widths
    from the smallest (4) to the whole grid, FP64 and FP32."""
    rng = np.random.default_rng(seed)
    combos = [("heat", "periodic"), ("heat", "reflective"), ("ks", "periodic"), ("euler", "dirichlet"),
              ("euler", "periodic")]
    cases = []
    for i in range(count):
        eq, bc = combos[i % 5]
        N = int(rng.integers(100, 2500))
        steps = int(rng.integers(1, 90))
        m = [0, 4, 100, 256, N][(i // 5) % 5]
        dtype = "f32" if (eq != "euler" and i % 3 == 0) else "f64"
        cases.append((eq, bc, N, steps, m, dtype))
    return cases


def _solo_and_oracle(eq, bc, N, steps, dtype, spec, u0, got, scheme):
    with S.Problem(spec, u0, dtype) as q:
        q.advance(steps, scheme)
        alone = q.read()
    assert np.array_equal(got, alone), (eq, bc, N, steps, dtype, scheme)
    ref = u0.copy()
    O.classic(oprob(spec), ref, steps)
    assert np.array_equal(got, ref), (eq, bc, N, steps, dtype, scheme)


def test_batch_classic_items_match_single_and_oracle():
    """Classic instances (one phase per sub-timestep, chunks of the balanced
    partition) beside swept ones in the same launches."""
    torch = pytest.importorskip("torch")
    stream = torch.cuda.Stream()
    classic = _classic_mix()
    swept = _mix(seed=11, count=12)
    probs, inputs, schemes, widths, steps = [], [], [], [], []
    for kind, cases in (("classic", classic), ("swept", swept)):
        for eq, bc, N, st, n, dtype in cases:
            spec = spec_for(eq, bc, N)
            u0 = state_for(spec, np.float64 if dtype == "f64" else np.float32, seed=N + st)
            inputs.append((kind, eq, bc, N, st, dtype, spec, u0))
            probs.append(S.Problem(spec, u0, dtype, stream=stream))
            schemes.append(kind)
            widths.append(n)
            steps.append(st)
    with S.Batch(stream) as b:
        b.advance_ex(probs, steps, schemes, widths)
        b.synchronize()
        assert b.kernel_launches() == 3   # heat+KS FP64, heat+KS FP32, Euler FP64
    for (kind, eq, bc, N, st, dtype, spec, u0), p in zip(inputs, probs):
        got = p.read()
        p.close()
        _solo_and_oracle(eq, bc, N, st, dtype, spec, u0, got, kind)


def test_batch_classic_rejects_bad_chunks():
    torch = pytest.importorskip("torch")
    stream = torch.cuda.Stream()
    spec = I.heat_spec(200)
    p = S.Problem(spec, state_for(spec), stream=stream)
    with S.Batch(stream) as b:
        for m in (3, 201):
            with pytest.raises(S.SweptError) as e:
                b.advance_ex([p], [5], ["classic"], [m])
            assert e.value.status == S.EINVAL
        with pytest.raises(S.SweptError):
            b.advance_ex([p], [5], ["swept"], [12], launch="register")
    p.close()


def test_batch_graph_replays_match_oracle():
    """The same batch advance captured once per (rows, plans) and replayed:
    heat with an odd step count changes rows every advance, so two graphs
    alternate."""
    torch = pytest.importorskip("torch")
    stream = torch.cuda.Stream()
    cases = [("heat", "periodic", 1000, 7, 40, "swept"), ("heat", "reflective", 999, 5, 128, "classic"),
             ("ks", "periodic", 2048, 10, 256, "swept"), ("ks", "periodic", 1500, 3, 0, "classic"),
             ("euler", "dirichlet", 512, 6, 64, "swept"), ("euler", "periodic", 700, 4, 100, "classic")]
    probs, inputs = [], []
    for eq, bc, N, st, n, kind in cases:
        spec = spec_for(eq, bc, N)
        u0 = state_for(spec, seed=N)
        inputs.append((spec, u0))
        probs.append(S.Problem(spec, u0, stream=stream))
    reps = 5
    with S.Batch(stream) as b:
        for _ in range(reps):
            b.advance_ex(probs, [c[3] for c in cases], [c[5] for c in cases], [c[4] for c in cases],
                         launch="graph")
        b.synchronize()
        assert b.kernel_launches() == 2 * reps
    for (eq, bc, N, st, n, kind), (spec, u0), p in zip(cases, inputs, probs):
        ref = u0.copy()
        O.classic(oprob(spec), ref, reps * st)
        assert np.array_equal(p.read(), ref), (eq, bc, N, st, n, kind)
        p.close()


def test_autotune_scheme_and_auto_advances():
    torch = pytest.importorskip("torch")
    spec = I.heat_spec(2048)
    u0 = I.initial_state(spec)
    scheme, n = S.autotune(spec, u0, count=8, steps=64)
    assert (scheme, n) == S.tuned(spec)
    if scheme == "swept":
        assert 2048 % n == 0 and n % 4 == 0
    else:
        assert 4 <= n <= 2048
    ref = u0.copy()
    O.classic(oprob(spec), ref, 77)
    with S.Problem(spec, u0) as p:
        p.advance(77, "auto")
        assert np.array_equal(p.read(), ref)
    stream = torch.cuda.Stream()
    ps = [S.Problem(spec, u0, stream=stream) for _ in range(3)]
    with S.Batch(stream) as b:
        b.advance_ex(ps, [77, 77, 77])
        b.synchronize()
    for p in ps:
        assert np.array_equal(p.read(), ref)
        p.close()


def test_batch_graph_cache_after_problems_replaced():
    """Problems destroyed and new ones created between graph advances (the
    host may reuse their addresses): each advance runs on the live problems'
    rows, never on a cached graph of destroyed ones."""
    torch = pytest.importorskip("torch")
    stream = torch.cuda.Stream()
    spec = I.ks_spec(2048)
    u0 = state_for(spec)
    ref = u0.copy()
    O.classic(oprob(spec), ref, 9)
    with S.Batch(stream) as b:
        for _ in range(3):
            ps = [S.Problem(spec, u0, stream=stream) for _ in range(2)]
            b.advance_ex(ps, [9, 9], ["swept", "swept"], [256, 256], launch="graph")
            b.synchronize()
            for p in ps:
                assert np.array_equal(p.read(), ref)
                p.close()
        assert b.kernel_launches() == 3


def test_fp32_one_warp_batch_with_widths_off_the_block():
    """An FP32 batch of one-warp blocks whose instances mix node widths that
    split evenly over the warp (512: 16 register-blocked slots per lane, which
    makes the launch register-blocked) with widths that do not (528, 520, 1000,
    744: their levels stay in shared memory), with and without remainders:
    every instance bit-identical to the oracle and to its solo advance."""
    torch = pytest.importorskip("torch")
    stream = torch.cuda.Stream()
    cases = [("heat", "periodic", 1024, 512), ("heat", "periodic", 1061, 528), ("ks", "periodic", 1061, 528),
             ("heat", "reflective", 1583, 520), ("ks", "periodic", 2000, 1000), ("heat", "periodic", 1500, 744),
             ("ks", "periodic", 2048, 512), ("heat", "periodic", 3169, 1056)]
    probs, inputs, steps = [], [], []
    for i, (eq, bc, N, n) in enumerate(cases):
        spec = spec_for(eq, bc, N)
        u0 = state_for(spec, np.float32, seed=N + n)
        inputs.append((spec, u0))
        probs.append(S.Problem(spec, u0, "f32", stream=stream))
        steps.append(n + 61 + 17 * i)
    widths = [c[3] for c in cases]
    with S.Batch(stream) as b:
        b.advance_ex(probs, steps, ["swept"] * len(cases), widths, threads=32, launch="graph")
        b.synchronize()
    got = [p.read() for p in probs]
    for p in probs:
        p.close()
    for (eq, bc, N, n), (spec, u0), st, g in zip(cases, inputs, steps, got):
        ref = np.ascontiguousarray(u0.copy())
        O.classic(oprob(spec), ref, st)
        assert np.array_equal(g, ref), (eq, bc, N, n, st)
        with S.Problem(spec, u0, "f32") as q:
            q.advance(st, "swept", n)
            assert np.array_equal(q.read(), g), (eq, bc, N, n, st)


def test_batch_tune_width_restores_states_and_returns_fitted_widths():
    """swp_batch_tune_width times each candidate on the batch itself and puts
    every state back (heat advances that end in the odd row included): the
    states read after tuning equal those before, the widths returned are the
    best candidate's widths fitted to each N, and an advance with them equals
    the oracle bit for bit."""
    torch = pytest.importorskip("torch")
    stream = torch.cuda.Stream()
    cases = [("heat", "periodic", 1031, 501, "f64"), ("heat", "reflective", 2503, 377, "f64"),
             ("ks", "periodic", 4099, 211, "f64"), ("heat", "periodic", 3001, 333, "f32"),
             ("ks", "periodic", 2048, 150, "f32"), ("euler", "dirichlet", 1537, 97, "f64")]
    probs, inputs = [], []
    for eq, bc, N, steps, dtype in cases:
        spec = spec_for(eq, bc, N)
        u0 = state_for(spec, np.float64 if dtype == "f64" else np.float32, seed=N)
        inputs.append((spec, u0))
        probs.append(S.Problem(spec, u0, dtype, stream=stream))
    steps = [c[3] for c in cases]
    candidates = (64, 256, 1000)
    with S.Batch(stream) as b:
        # an odd first advance leaves some heat states in the other row
        b.advance(probs, [1] * len(probs))
        b.synchronize()
        before = [p.read() for p in probs]
        widths, best, ms = b.tune_width(probs, steps, candidates)
        assert 0 <= best < len(candidates) and len(ms) == len(candidates) and min(ms) > 0
        for p, x in zip(probs, before):
            assert np.array_equal(p.read(), x)
        for (eq, _, N, _, _), w in zip(cases, widths):
            assert w == S.fit_width(eq, N, candidates[best]), (eq, N, w)
        b.advance_ex(probs, steps, ["swept"] * len(probs), widths)
        b.synchronize()
    for (eq, bc, N, st, dtype), (spec, u0), p, x in zip(cases, inputs, probs, before):
        ref = np.ascontiguousarray(u0.copy())
        O.classic(oprob(spec), ref, 1 + st)
        assert np.array_equal(p.read(), ref), (eq, bc, N, st, dtype)
        p.close()


def test_batch_tune_width_errors_leave_states_unchanged():
    """A problem listed twice fails in the trial advance (SWP_EINVAL) after
    the states were saved, and they are put back; a candidate width <= 0
    fails before anything runs."""
    torch = pytest.importorskip("torch")
    stream = torch.cuda.Stream()
    specs = [spec_for("ks", "periodic", 2053), spec_for("heat", "periodic", 1501)]
    probs = [S.Problem(sp, state_for(sp, seed=3 + i), stream=stream) for i, sp in enumerate(specs)]
    with S.Batch(stream) as b:
        b.advance(probs, [3, 3])
        b.synchronize()
        before = [p.read() for p in probs]
        with pytest.raises(S.SweptError, match="EINVAL"):
            b.tune_width([probs[0], probs[1], probs[0]], [50, 50, 50], (256, 512))
        with pytest.raises(S.SweptError, match="EINVAL"):
            b.tune_width(probs, [50, 50], (256, 0))
        for p, x in zip(probs, before):
            assert np.array_equal(p.read(), x)
    for p in probs:
        p.close()
