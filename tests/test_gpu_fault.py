"""Failure detection of the persistent swept launch, without any GPU fault:
every neighbour wait is bounded by the device global timer.  The test hook
makes the waits wait for a flag value no node publishes; each wait then gives
up after its limit, the kernel returns, the host reports SWP_ETIMEOUT, and the
problem recovers once the hook is lifted and the state rewritten."""
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


def test_withheld_flags_time_out_and_recover():
    spec = spec_for("ks", "periodic", 4096)
    u0 = state_for(spec)
    ref = u0.copy()
    O.classic(oprob(spec), ref, 40)
    with S.Problem(spec, u0) as p:
        p.debug_withhold_flags(True, wait_limit_ns=200_000_000)
        t0 = time.perf_counter()
        p.advance(40, "swept", 256, "persistent")
        with pytest.raises(S.SweptError) as e:
            p.synchronize()
        assert e.value.status == S.ETIMEOUT
        assert time.perf_counter() - t0 < 30
        # recovery: lift the hook, restore the state, advance again
        p.debug_withhold_flags(False)
        p.write(u0)
        p.advance(40, "swept", 256, "persistent")
        assert np.array_equal(p.read(), ref)
        # the per-phase launch never waits on flags
        p.debug_withhold_flags(True, wait_limit_ns=200_000_000)
        p.write(u0)
        p.advance(40, "swept", 256, "per_phase")
        assert np.array_equal(p.read(), ref)


def test_wait_limit_validated():
    spec = spec_for("ks", "periodic", 256)
    with S.Problem(spec, state_for(spec)) as p:
        with pytest.raises(S.SweptError) as e:
            p.debug_withhold_flags(True, wait_limit_ns=0)
        assert e.value.status == S.EINVAL
