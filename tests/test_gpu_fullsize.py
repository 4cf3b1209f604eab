"""Parity at the benchmark's full size, in the launch configuration bench.py
times: KS, N = 2^20, FP64, 10^4 steps.  The oracle cannot run the whole
problem in a test's time, so the full run is checked through properties that
hold at any size (swept == classic bit for bit, mean conservation, bounded
state) and sampled points are checked against the oracle: the value at point i
after M steps depends only on the initial values within 4M points (radius 2 per
RK2 stage), so the oracle advances a periodic window of 8M + 65 points around i
and its centre must equal the GPU's value exactly."""
import numpy as np
import pytest

import oracle as O
from helpers import oprob
from paper_1705_03162_gb300 import build as B
from paper_1705_03162_gb300 import inputs as I
from paper_1705_03162_gb300 import swept as S
import bench

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    B.build()
    S.load_library()


def _run(spec, u0, steps, scheme, n=0, launch="auto"):
    with S.Problem(spec, u0) as p:
        p.advance(steps, scheme, n, launch)
        return p.read()


def test_ks_full_size_bench_configuration():
    cfg = bench.DEFAULT_WORKLOAD
    spec = I.ks_spec(cfg["n_points"])
    u0 = I.initial_state(spec)
    steps = cfg["steps"]
    swept = _run(spec, u0, steps, "swept", cfg["points_per_block"], cfg["launch"])
    classic = _run(spec, u0, steps, "classic")
    assert np.array_equal(swept, classic)
    assert np.all(np.isfinite(swept)) and np.max(np.abs(swept)) < 10
    s0, s1 = float(u0.sum()), float(swept.sum())
    assert abs(s1 - s0) < 1e-9 * float(np.abs(swept).sum())


@pytest.mark.parametrize("centre", [0, 333_333, (1 << 20) - 1])
def test_ks_full_size_sampled_against_oracle(centre):
    cfg = bench.DEFAULT_WORKLOAD
    N, M = cfg["n_points"], 2500
    spec = I.ks_spec(N)
    u0 = I.initial_state(spec)
    got = _run(spec, u0, M, "swept", cfg["points_per_block"], cfg["launch"])
    half = 4 * M + 32
    idx = (np.arange(centre - half, centre + half + 1)) % N
    win = np.ascontiguousarray(u0[:, idx])
    wspec = I.ProblemSpec("ks", "periodic", win.shape[1], spec.dx, spec.dt)
    O.classic(oprob(wspec), win, M)
    assert win[0, half] == got[0, centre]
