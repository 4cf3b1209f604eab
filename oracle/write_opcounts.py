"""Write oracle/opcounts.json: floating-point operations per point-update of
each scheme, counted by the oracle's counting build (oracle.opcounts).

    python oracle/write_opcounts.py

TEST INFRASTRUCTURE: calls only the oracle (and the seeded input
generators).  bench.py reads the stored table for its roofline figures;
tests/test_oracle_opcounts.py checks that it equals a fresh count.  Heat and
KS counts do not depend on the data.  The Euler count does, through the
limiter (a limited interface costs a division and a few operations more than
a first-order one), so it is taken on the benchmark's Sod workload shape:
the waves cover a share of the tube proportional to steps / N, which is
1/256 for 4096 steps at N = 2^20 as for 16 steps at N = 4096; and on the
full Sod run to t = 0.2 (N steps) for reference.
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import oracle as O  # noqa: E402
from paper_1705_03162_gb300 import inputs as I  # noqa: E402

OUT = os.path.join(HERE, "opcounts.json")

WORKLOADS = {
    "heat": (I.heat_spec(1024), 8),
    "ks": (I.ks_spec(2048), 8),
    "euler_sod_steps_over_n_1_256": (I.sod_spec(4096), 16),
    "euler_sod_to_t_0.2": (I.sod_spec(1024), 1024),
}

_EQ = {"heat": O.HEAT, "ks": O.KS, "euler": O.EULER}
_BC = {"periodic": O.PERIODIC, "reflective": O.REFLECTIVE, "dirichlet": O.DIRICHLET}


def count_all() -> dict:
    out = {}
    for name, (spec, steps) in WORKLOADS.items():
        prob = O.OracleProblem(_EQ[spec.eq], _BC[spec.bc], spec.n_points, spec.dx, spec.dt, spec.alpha,
                               spec.gamma, spec.left, spec.right)
        c = O.opcounts(prob, I.initial_state(spec), steps)
        out[name] = {"n_points": spec.n_points, "timesteps": steps,
                     "oracle": c["oracle"], "algorithmic": c["algorithmic"]}
    return out


def main():
    table = {"what": "floating-point operations per point-update (one point, one timestep); "
                     "flops counts an FMA as two",
             "written_by": "python oracle/write_opcounts.py",
             "counts": count_all()}
    with open(OUT, "w") as f:
        json.dump(table, f, indent=1, sort_keys=True)
        f.write("\n")
    print(OUT)


if __name__ == "__main__":
    main()
