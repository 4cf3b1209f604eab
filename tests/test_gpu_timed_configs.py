"""Correctness at the sizes and in the launch forms the benchmark times.

- Sod tube at N = 2^20, 512-cell nodes, the dataflow launch: swept equals
  classic bit for bit, and sampled cells equal the CPU oracle exactly.  The
  value of a cell after M steps depends only on the cells within 4M of it
  (radius 2 per RK2 stage), so the oracle advances a window of 8M + 65 cells
  around it; Sod's ends are uniform there, so the window's own Dirichlet
  ends (the same states) change nothing inside.
- A batch drawn by the benchmark's own generator (heat and KS, N any integer
  on 2^10..2^16, 10^3..10^4 steps) with autotuned widths, in FP64 and FP32:
  every instance equals its single-problem advance bit for bit, and the
  instances of least work equal the CPU oracle."""
import numpy as np
import pytest

import bench
import oracle as O
from helpers import oprob
from paper_1705_03162_gb300 import build as B
from paper_1705_03162_gb300 import inputs as I
from paper_1705_03162_gb300 import swept as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    B.build()
    S.load_library()


def test_sod_full_size_dataflow_equals_classic_and_oracle():
    N, M = 1 << 20, 300
    spec = I.sod_spec(N)
    u0 = I.initial_state(spec)
    with S.Problem(spec, u0) as p:
        p.advance(M, "swept", 512, "persistent")
        swept = p.read()
    with S.Problem(spec, u0) as p:
        p.advance(M, "classic")
        classic = p.read()
    assert np.array_equal(swept, classic)
    half = 4 * M + 32
    # after M steps (t = 0.2 M dx) the rarefaction spans about -71..-10 cells
    # from the diaphragm, the contact sits near +56 and the shock near +105
    for centre in (N // 2 - 40, N // 2 + 56, N // 2 + 105, N // 2 + 400):
        win = np.ascontiguousarray(u0[:, centre - half:centre + half + 1])
        wspec = I.ProblemSpec("euler", "dirichlet", win.shape[1], spec.dx, spec.dt)
        O.classic(oprob(wspec), win, M)
        assert np.array_equal(win[:, half], swept[:, centre]), centre


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_bench_batched_workload_equals_solo_and_oracle(dtype):
    torch = pytest.importorskip("torch")
    npdt = np.float64 if dtype == "f64" else np.float32
    cases = bench.batched_cases(4096)[:384]
    tuned = {}
    for eq in ("heat", "ks"):
        for e in range(10, 17):
            spec, u0 = bench._spec_ic(eq, 2 ** e, npdt)
            tuned[(eq, e)] = S.autotune(spec, u0, count=32, steps=64, dtype=dtype)
    stream = torch.cuda.Stream()
    probs, schemes, widths, inputs = [], [], [], []
    for eq, N, steps in cases:
        spec, u0 = bench._spec_ic(eq, N, npdt)
        inputs.append((spec, u0))
        probs.append(S.Problem(spec, u0, dtype, stream=stream))
        scheme, n = tuned[(eq, bench.bucket(N))]
        schemes.append(scheme)
        widths.append(bench.fit_width(eq, N, n) if scheme == "swept" else min(n, N))
    steps = [c[2] for c in cases]
    assert any(N % n for (_, N, _), sc, n in zip(cases, schemes, widths) if sc == "swept")   # wider nodes occur
    with S.Batch(stream) as b:
        b.advance_ex(probs, steps, schemes, widths, launch="graph")
        b.synchronize()
    got = [p.read() for p in probs]
    for p in probs:
        p.close()
    for i, ((eq, N, st), (spec, u0)) in enumerate(zip(cases, inputs)):
        with S.Problem(spec, u0, dtype) as q:
            q.advance(st, schemes[i], widths[i] if schemes[i] == "swept" else 0)
            assert np.array_equal(got[i], q.read()), (i, eq, N, st, schemes[i], widths[i])
    # the instances of least work, against the oracle
    for i in sorted(range(len(cases)), key=lambda j: cases[j][1] * cases[j][2])[:4]:
        spec, u0 = inputs[i]
        ref = np.ascontiguousarray(u0.copy())
        O.classic(oprob(spec), ref, cases[i][2])
        assert np.array_equal(got[i], ref), (i, cases[i])
