"""The oracle's counting build and its OpenMP build (CPU only).

The stored table oracle/opcounts.json, which bench.py reads for its roofline
figures, must equal a fresh count; the counts of heat and KS follow from the
formulas as the oracle writes them (heat: one addition and two FMAs; a KS
stage: three additions and four FMAs, two stages per timestep); and the
all-core OpenMP build of the classic scheme must give the single-threaded
oracle's bits."""
import json
import os
import sys

import numpy as np
import pytest

import oracle as O
from helpers import oprob, spec_for, state_for

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_stored_table_equals_a_fresh_count():
    sys.path.insert(0, os.path.join(ROOT, "oracle"))
    import write_opcounts as W
    with open(W.OUT) as f:
        stored = json.load(f)["counts"]
    fresh = json.loads(json.dumps(W.count_all()))
    assert stored == fresh


def test_heat_and_ks_counts_match_the_written_formulas():
    heat = O.opcounts(oprob(spec_for("heat", "periodic", 256)), state_for(spec_for("heat", "periodic", 256)), 3)
    assert heat["algorithmic"] == heat["oracle"]
    assert (heat["oracle"]["add"], heat["oracle"]["fma"], heat["oracle"]["mul"]) == (1, 2, 0)
    assert heat["oracle"]["flops"] == 5
    ks_spec = spec_for("ks", "periodic", 256)
    ks = O.opcounts(oprob(ks_spec), state_for(ks_spec), 3)
    assert (ks["oracle"]["add"], ks["oracle"]["fma"], ks["oracle"]["mul"]) == (6, 8, 0)
    assert ks["oracle"]["flops"] == 22 and ks["oracle"]["ops"] == 14


def test_euler_algorithmic_count_keeps_each_value_once():
    """Per cell and sub-timestep: one pressure (a division, three
    multiplications, an FMA), one interface and the update (three
    subtractions, three FMAs).  The plain oracle evaluates five pressures and
    two interfaces per cell; the algorithmic count is therefore well below
    half of it, and the uniform Sod regions need no limiter division."""
    spec = spec_for("euler", "dirichlet", 1024)
    c = O.opcounts(oprob(spec), state_for(spec), 4)
    assert c["pieces"]["pressure"]["ops"] == 5 and c["pieces"]["pressure"]["div"] == 1
    assert c["pieces"]["cell_update"]["ops"] == 6
    iface = c["pieces"]["interface_mean"]
    assert iface["sqrt"] == pytest.approx(3.0) and 3.0 <= iface["div"] <= 5.0
    alg, orc = c["algorithmic"]["ops"], c["oracle"]["ops"]
    assert alg == pytest.approx(2 * (5 + 6 + iface["ops"]))
    assert alg < 0.5 * orc


@pytest.mark.parametrize("eq,bc", [("heat", "reflective"), ("ks", "periodic"), ("euler", "dirichlet"),
                                   ("euler", "periodic")])
def test_openmp_build_gives_the_serial_bits(eq, bc):
    spec = spec_for(eq, bc, 3001)
    u = state_for(spec)
    a, b = u.copy(), u.copy()
    O.classic(oprob(spec), a, 40)
    O.classic(oprob(spec), b, 40, threads=4)
    assert O.omp_threads(4) == 4
    assert np.array_equal(a, b)
