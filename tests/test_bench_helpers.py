"""Host-side pieces of bench.py (no GPU): the traffic record matches the
committed kernel code for the timed configuration, the code-only hash ignores
comments, the workload generators are deterministic, and the reference arm
(the CPU oracle) prints the contract line."""
import os

import numpy as np

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_traffic_record_matches_the_timed_kernel_code():
    wl = bench.DEFAULT_WORKLOAD
    key = (f"{bench.KERNEL_OF_LAUNCH[wl['launch']]}<double,KS> "
           f"n={wl['points_per_block']} threads={wl['threads']}")
    rec = bench.NCU_TRAFFIC[key]
    assert rec["src"] == bench._kernel_src_hash(), "re-capture the traffic after a kernel code change"
    assert rec["bytes_per_launch"] > 0


def test_code_only_ignores_comments_and_blank_lines():
    a = "int f(int x)\n{\n    return x + 1;  // one more\n}\n"
    b = "/* header\n   text */\nint f(int x)\n{\n\n    return x + 1;\n}\n// trailing\n"
    assert bench._code_only(a) == bench._code_only(b)
    assert bench._code_only(a) != bench._code_only(a.replace("x + 1", "x + 2"))


def test_served_trace_is_seeded_and_ordered():
    t1 = bench._trace(48, 2000.0, 20170509)
    t2 = bench._trace(48, 2000.0, 20170509)
    assert t1 == t2
    times = [r[0] for r in t1]
    assert times == sorted(times) and times[0] > 0
    for _, eq, N, steps in t1:
        assert eq in ("heat", "ks", "euler")
        assert N % 1024 == 0 and 1024 <= N <= (1 << 20)
        assert 1000 <= steps <= 10000


def test_percentiles():
    lat = list(np.arange(1, 101, dtype=float))
    p = bench._percentiles(lat)
    assert abs(p["p50_s"] - np.percentile(lat, 50)) < 1e-12
    assert abs(p["p99_s"] - np.percentile(lat, 99)) < 1e-12
    assert p["max_s"] == 100.0


def test_reference_arm_prints_the_contract_line():
    """bench.py --impl reference (the CPU oracle on the host cores) prints one
    JSON line with the benchmark's metric, unit and configuration, its CPU
    baseline and an end-to-end figure with no device copies."""
    import json
    import subprocess
    import sys
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "3"], capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    line = json.loads(r.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference"
    assert line["metric"] == bench.METRIC and line["unit"] == bench.UNIT
    assert line["value"] > 0 and line["higher_is_better"] is True
    assert (line["n_gpus"], line["steps"], line["warmup"]) == (1, 1, 3)
    assert line["config"]["workload"] == bench.WORKLOAD.format("FP64")
    cb = line["cpu_baseline"]
    assert set(cb) >= {"value", "unit", "cores", "kind", "sample"} and cb["kind"] == "oracle"
    assert cb["value"] == line["value"] and cb["cores"] >= 1
    e2e = line["e2e"]
    assert e2e["value"] == line["value"] and e2e["unit"] == line["unit"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0


def test_bench_rejects_fewer_than_three_warmup_steps():
    import subprocess
    import sys
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--warmup", "2"], capture_output=True,
                       text=True, timeout=120, cwd=ROOT)
    assert r.returncode == 2 and "--warmup must be >= 3" in r.stderr
