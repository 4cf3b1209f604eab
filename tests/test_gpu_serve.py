"""Serving with continuous batching: every request's result is the same alone
and in the mix (bit-identical, hence within any tolerance), with requests
admitted under a device-memory budget and a slot limit, advanced in many small
rounds, and arriving while others are on the GPU."""
import threading
import time

import numpy as np
import pytest

import oracle as O
from helpers import oprob, spec_for, state_for
from paper_1705_03162_gb300 import build as B
from paper_1705_03162_gb300 import swept as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    B.build()
    S.load_library()


def _requests(count=12, seed=11):
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        eq, bc = [("heat", "periodic"), ("ks", "periodic"), ("euler", "dirichlet"),
                  ("heat", "reflective")][i % 4]
        N = int(2 ** rng.integers(9, 13))
        steps = int(rng.integers(20, 300))
        dtype = "f32" if (eq != "euler" and i % 5 == 1) else "f64"
        spec = spec_for(eq, bc, N)
        u0 = state_for(spec, np.float64 if dtype == "f64" else np.float32, seed=i)
        out.append((spec, u0, steps, dtype))
    return out


def _solo(spec, u0, steps, dtype):
    with S.Problem(spec, u0, dtype) as p:
        p.advance(steps, "swept")
        return p.read()


def test_served_results_equal_solo_and_oracle():
    reqs = _requests()
    budget = 3 * max(2 * u0.nbytes for _, u0, _, _ in reqs)   # a few requests at a time
    # a tiny round target: nearly every request is longer than a round, so
    # each runs a phase or a few per round and spans many rounds, with the
    # others in the same launches
    with S.Server(hbm_budget_bytes=budget, max_active=4, round_target_ms=0.0005) as srv:
        ids = [None] * len(reqs)

        def feed(lo, hi, delay):
            for i in range(lo, hi):
                spec, u0, steps, dtype = reqs[i]
                ids[i] = srv.submit(spec, u0, steps, dtype)
                time.sleep(delay)

        first = threading.Thread(target=feed, args=(0, 6, 0.0))
        later = threading.Thread(target=feed, args=(6, len(reqs), 0.01))   # arrive while others run
        first.start(); later.start(); first.join(); later.join()
        results = [srv.wait(i) for i in ids]
        stats = srv.stats()
    assert stats["completed"] == len(reqs) and stats["rounds"] > 2 * len(reqs)
    assert stats["device_bytes_in_use"] == 0
    for (spec, u0, steps, dtype), (got, lat) in zip(reqs, results):
        assert lat > 0
        assert np.array_equal(got, _solo(spec, u0, steps, dtype))
        ref = u0.copy()
        O.classic(oprob(spec), ref, steps)
        assert np.array_equal(got, ref)


def test_oversized_request_rejected_by_budget():
    spec = spec_for("ks", "periodic", 4096)
    u0 = state_for(spec)
    with S.Server(hbm_budget_bytes=4096, max_active=2) as srv:
        rid = srv.submit(spec, u0, 10)
        with pytest.raises(S.SweptError) as e:
            srv.wait(rid)
        assert e.value.status == S.EBUDGET
        assert "budget of 4096" in str(e.value)   # the scheduler's reason reaches the waiter
