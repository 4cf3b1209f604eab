"""The oracle's pins catch plausible mistakes in it.

Each case plants one mistake, of the kind a restatement of the paper's
schemes could plausibly contain (a dropped term, a wrong sign, a wrong or
swapped index, a transposed operand), in a temporary copy of the oracle's
source on the CPU. It then runs the pins (test_oracle_pins.py, and
test_oracle_literal.py, the exact-arithmetic check of one stage against the
printed formulas) against that copy, and at least one pin must fail. An unmutated copy must pass. The
schemes are those of arXiv:1705.03162 Appendices A-C and Sections 4-5; each
case names the passage its mistake breaks. CPU only: nothing here touches a
GPU or the CUDA library.
"""
import concurrent.futures
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

# (name, passage, original text in oracle/scheme.inc, planted mistake)
MUTATIONS = [
    ("heat: neighbour index", "Appendix A Eq. heatdisc",
     "REAL s = v[2] + v[0];", "REAL s = v[2] + v[2];"),
    ("heat: centre weight sign", "Appendix A Eq. heatdisc",
     "REAL lap = FMA((REAL)-2, v[1], s);", "REAL lap = FMA((REAL)2, v[1], s);"),
    ("heat: Fourier number without dx^2", "Appendix A Eq. heatdisc",
     "double fo = pb->alpha * pb->dt / (pb->dx * pb->dx);", "double fo = pb->alpha * pb->dt / pb->dx;"),
    ("KS: advection difference reversed", "Appendix B Eq. KSDisc",
     "REAL d = v[3] - v[1];", "REAL d = v[1] - v[3];"),
    ("KS: fourth-difference index", "Appendix B Eq. KSDisc",
     "REAL s2 = v[4] + v[0];", "REAL s2 = v[4] + v[1];"),
    ("KS: fourth-difference term dropped", "Appendix B Eq. KSDisc",
     "acc = FMA(a4, s2, acc);", "acc = acc + (REAL)0 * s2;"),
    ("KS: centre weight sign of the Laplacian", "Appendix B Eq. KSDisc",
     "c->gam[s] = (REAL)(6.0 * a4 - 2.0 * a2);", "c->gam[s] = (REAL)(6.0 * a4 + 2.0 * a2);"),
    ("KS: advection coefficient 1/(2dx)", "Appendix B Eq. KSDisc",
     "double c1 = 1.0 / (4.0 * pb->dx);", "double c1 = 1.0 / (2.0 * pb->dx);"),
    ("RK2: full step in the predictor", "Appendix B Eqs. RKm, RKf",
     "double h = s == 0 ? 0.5 * pb->dt : pb->dt;", "double h = pb->dt;"),
    ("RK2: final stage based on the midpoint value", "Appendix B Eq. RKf",
     "            for (int v = 0; v < nv; ++v) base[v] = state[v * N + i];\n"
     "            SFX(point_update)(&c, 1, st, base, out);",
     "            for (int v = 0; v < nv; ++v) base[v] = half[v * N + i];\n"
     "            SFX(point_update)(&c, 1, st, base, out);"),
    ("Euler: kinetic-energy sign in the pressure", "Appendix C Eq. EulerP",
     "return gm1 * FMA((REAL)-0.5 * m, u, E);", "return gm1 * FMA((REAL)0.5 * m, u, E);"),
    ("Euler: pressure ratio inverted", "Appendix C Eq. Pratio",
     "REAL num = pb - pa, den = pa - pam;", "REAL num = pa - pam, den = pb - pa;"),
    ("Euler: limiter cap dropped", "Appendix C Eq. limitleft",
     "REAL phi = ratio < (REAL)1 ? ratio : (REAL)1;", "REAL phi = ratio;"),
    ("Euler: momentum flux without pressure", "Appendix C Eq. EulerF",
     "fl[1] = FMA(ql[1], ul, pl);", "fl[1] = ql[1] * ul;"),
    ("Euler: Roe weights swapped", "Appendix C Eq. Roe",
     "REAL usp = FMA(sl, ul, sr * ur) * iw;", "REAL usp = FMA(sr, ul, sl * ur) * iw;"),
    ("Euler: spectral radius without |u|", "Appendix C, the flux's spectral radius",
     "REAL rsp = SQRT(c2) + FABS(usp);", "REAL rsp = SQRT(c2);"),
    ("Euler: dissipation sign", "Appendix C, the interface flux",
     "G[c] = FMA(rsp, ql[c] - qr[c], fr[c] + fl[c]);", "G[c] = FMA(rsp, qr[c] - ql[c], fr[c] + fl[c]);"),
    ("Euler: update sign", "Appendix C, the finite-volume update",
     "c->kh[s] = (REAL)(-(0.5 * lamh));", "c->kh[s] = (REAL)(0.5 * lamh);"),
    ("Euler: ghost energy p/gamma", "Appendix C Eq. SodCond",
     "gh[s][2] = (REAL)(p / (g - 1.0) + 0.5 * r * u * u);", "gh[s][2] = (REAL)(p / g + 0.5 * r * u * u);"),
    ("reflective end mirrored about the half point", "Appendix A Eq. heatcond",
     "int64_t m = g < 0 ? -g : 2 * (N - 1) - g;", "int64_t m = g < 0 ? -g - 1 : 2 * N - 1 - g;"),
    ("swept: right neighbour's edge from the node itself", "Section 4.2, Fig. 2",
     "int64_t kr = odd ? k : (k + 1) % K;", "int64_t kr = k;"),
    ("swept: final-stage base from the source row", "Section 4.3 with Appendix B Eq. RKf",
     "base[v] = (stage == 0) ? src[v * W + q] : row0[v * W + q];", "base[v] = src[v * W + q];"),
    # rounding-level mistakes: the equation is kept, an exact regrouping is
    # replaced by a lossy one (only the exact-arithmetic pin sees these)
    ("KS: combined weight beta rounded to single precision", "Appendix B Eq. KSDisc",
     "c->beta[s] = (REAL)(a2 - 4.0 * a4);", "c->beta[s] = (REAL)(float)(a2 - 4.0 * a4);"),
    ("Euler: update coefficient rounded to single precision", "Appendix C, the finite-volume update",
     "c->kh[s] = (REAL)(-(0.5 * lamh));", "c->kh[s] = (REAL)(float)(-(0.5 * lamh));"),
]


def _run_pins(tmp_root: str, old: str, new: str):
    """Copy the oracle and its pins under tmp_root, plant old -> new in
    scheme.inc (nothing if old is None), run the pins; return (rc, tail)."""
    shutil.copytree(os.path.join(ROOT, "oracle"), os.path.join(tmp_root, "oracle"),
                    ignore=shutil.ignore_patterns("_build", "__pycache__"))
    os.makedirs(os.path.join(tmp_root, "tests"))
    for f in ("test_oracle_pins.py", "test_oracle_literal.py", "helpers.py", "riemann_exact.py", "conftest.py"):
        shutil.copy(os.path.join(ROOT, "tests", f), os.path.join(tmp_root, "tests", f))
    if old is not None:
        path = os.path.join(tmp_root, "oracle", "scheme.inc")
        text = open(path).read()
        assert text.count(old) == 1, f"mutation site not unique: {old!r}"
        open(path, "w").write(text.replace(old, new))
    # the copy's conftest puts tmp_root first on sys.path, so `oracle` is the
    # copy; the input generators come from the repository
    env = dict(os.environ, PYTHONPATH=ROOT)
    r = subprocess.run([sys.executable, "-m", "pytest", "tests/test_oracle_pins.py", "tests/test_oracle_literal.py",
                        "-x", "-q",
                        "-p", "no:cacheprovider"], cwd=tmp_root, env=env, capture_output=True,
                       text=True, timeout=600)
    lines = (r.stdout + r.stderr).strip().splitlines()
    return r.returncode, lines[-1] if lines else ""


def test_unmutated_copy_passes(tmp_path):
    rc, tail = _run_pins(str(tmp_path), None, None)
    assert rc == 0, tail


def test_every_planted_mistake_fails_a_pin(tmp_path):
    def one(i):
        name, _, old, new = MUTATIONS[i]
        d = tmp_path / f"m{i}"
        d.mkdir()
        return name, _run_pins(str(d), old, new)

    with concurrent.futures.ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 1)) as ex:
        results = list(ex.map(one, range(len(MUTATIONS))))
    survivors = [(name, tail) for name, (rc, tail) in results if not (rc == 1 and "failed" in tail)]
    assert not survivors, f"mistakes no pin catches (or runs that broke otherwise): {survivors}"


@pytest.mark.parametrize("name,passage,old,new", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_mutation_sites_exist(name, passage, old, new):
    """Each planted mistake replaces text that occurs exactly once in the oracle."""
    text = open(os.path.join(ROOT, "oracle", "scheme.inc")).read()
    assert text.count(old) == 1 and old != new, name
