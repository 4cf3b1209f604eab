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
