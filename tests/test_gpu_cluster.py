"""The Register variant on one thread-block cluster (SWP_LAUNCH_CLUSTER): the
whole advance in one launch, node windows through distributed shared memory,
a cluster barrier between phases.  Its levels are the per-phase Register
kernel's own device function, so its results must equal that kernel's and
the CPU oracle's bit for bit, for every cluster shape and step count."""
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


def _run(spec, u0, steps, dtype, launch, threads=0):
    with S.Problem(spec, u0, dtype) as p:
        p.advance(steps, "swept", 0, launch, threads)
        return p.read(), p.kernel_launches()


@pytest.mark.parametrize("eq", ["heat", "ks"])
@pytest.mark.parametrize("N,threads", [(64, 0), (1024, 0), (1024, 128), (1024, 256), (1536, 0), (2048, 0),
                                       (4096, 0), (4096, 256)])
@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_cluster_matches_register_and_oracle(eq, N, threads, dtype):
    spec = spec_for(eq, "periodic", N)
    u0 = state_for(spec, np.float64 if dtype == "f64" else np.float32, seed=N)
    for steps in (1, 7, 16, 33, 301):
        got, launches = _run(spec, u0, steps, dtype, "cluster", threads)
        assert launches == 1
        reg, _ = _run(spec, u0, steps, dtype, "register")
        assert np.array_equal(got, reg), steps
        ref = np.ascontiguousarray(u0.copy())
        O.classic(oprob(spec), ref, steps)
        assert np.array_equal(got, ref), steps


def test_cluster_heat_configuration():
    """The heat configuration: N = 1024, r = 0.25, 4096 steps (257 phases,
    one launch)."""
    spec = spec_for("heat", "periodic", 1024)
    u0 = state_for(spec)
    got, launches = _run(spec, u0, 4096, "f64", "cluster")
    assert launches == 1
    ref = np.ascontiguousarray(u0.copy())
    O.classic(oprob(spec), ref, 4096)
    assert np.array_equal(got, ref)


def test_cluster_rejects_what_it_cannot_hold():
    for eq, bc, N, n, threads, status in [("euler", "dirichlet", 1024, 0, 0, S.EUNSUPPORTED),
                                          ("heat", "reflective", 1024, 0, 0, S.EUNSUPPORTED),
                                          ("heat", "periodic", 1000, 0, 0, S.EINVAL),      # not 32 k
                                          ("ks", "periodic", 8192, 0, 0, S.EINVAL),        # 256 nodes
                                          ("ks", "periodic", 1024, 64, 0, S.EINVAL),       # node of 64
                                          ("ks", "periodic", 1024, 0, 96, S.EINVAL)]:      # 32 nodes, 3 per block
        spec = spec_for(eq, bc, N)
        with S.Problem(spec, state_for(spec)) as p:
            with pytest.raises(S.SweptError) as e:
                p.advance(10, "swept", n, "cluster", threads)
            assert e.value.status == status, (eq, bc, N, n, threads)
