"""swp_swept_noalloc: the swept advance for callers that cannot allocate device
memory (pool- or arena-owned memory, allocation-free loops, hosts that pass
only pre-allocated buffers).  Its scratch is a fixed array inside the library,
so its results must equal the allocating entry points' on the same inputs, on
consecutive calls that reuse that array.  This file is collected last so that a
run stopping at the first failure has already run every other test."""
import numpy as np
import pytest

from helpers import rel_max, spec_for, state_for
from paper_1705_03162_gb300 import build as B
from paper_1705_03162_gb300 import inputs as I
from paper_1705_03162_gb300 import swept as S

pytestmark = pytest.mark.gpu

TOL = {"f64": 1e-12, "f32": 1e-5}


@pytest.fixture(scope="module", autouse=True)
def _lib():
    B.build()
    S.load_library()


def _allocating(spec, u0, steps_list, n, dtype):
    out = []
    with S.Problem(spec, u0, dtype) as p:
        for steps in steps_list:
            p.advance(steps, "swept", n, "per_phase")
            out.append(p.read())
    return out


@pytest.mark.parametrize("eq,bc,N,n,dtype,steps_list", [
    ("ks", "periodic", 1 << 20, 512, "f64", (300, 177)),    # the full 8 MiB of scratch
    ("heat", "reflective", 4992, 64, "f64", (101, 57)),     # odd last level: result in scratch
    ("euler", "dirichlet", 4096, 128, "f64", (150, 93)),
    ("heat", "periodic", 8192, 128, "f32", (77, 200)),
])
def test_noalloc_matches_allocating_entry_points(eq, bc, N, n, dtype, steps_list):
    torch = pytest.importorskip("torch")
    spec = spec_for(eq, bc, N)
    u0 = state_for(spec, np.float64 if dtype == "f64" else np.float32)
    expect = _allocating(spec, u0, steps_list, n, dtype)
    state = torch.from_numpy(u0.copy()).cuda()
    stream = torch.cuda.Stream()
    for steps, ref in zip(steps_list, expect):
        S.swept_noalloc(spec, state, steps, n, stream=stream, dtype=dtype)
        stream.synchronize()
        got = state.cpu().numpy()
        assert rel_max(got, ref) <= TOL[dtype]
        assert np.array_equal(got, ref)


def test_noalloc_rejects_state_beyond_scratch():
    torch = pytest.importorskip("torch")
    spec = I.ks_spec((1 << 20) + 8)
    state = torch.zeros((1, spec.n_points), dtype=torch.float64, device="cuda")
    with pytest.raises(S.SweptError) as e:
        S.swept_noalloc(spec, state, 10, 8)
    assert e.value.status == S.EINVAL
    assert "scratch" in str(e.value)
