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
        assert 1024 <= N <= (1 << 20)
        assert 100 <= steps <= 1000
    assert any(N % 1024 for _, _, N, _ in t1)   # any integer N, not rounded
    # the same request set at another rate: the arrival pattern rescaled
    t3 = bench._trace(48, 500.0, 20170509)
    assert [r[1:] for r in t3] == [r[1:] for r in t1]
    assert np.allclose([r[0] for r in t3], [4 * r[0] for r in t1])


def test_fifo_latencies():
    # arrivals 0, 1, 1.5; service 2, 1, 1: the second waits for the first
    lat = bench.fifo_latencies([0.0, 1.0, 1.5], [2.0, 1.0, 1.0])
    assert lat == [2.0, 2.0, 2.5]
    assert bench.fifo_latencies([0.0, 10.0], [1.0, 1.0]) == [1.0, 1.0]


def test_batched_cases_and_widths():
    from paper_1705_03162_gb300 import build as B
    B.build()
    cases = bench.batched_cases(512)
    assert cases == bench.batched_cases(512)
    assert [c[0] for c in cases[:4]] == ["heat", "ks", "heat", "ks"]
    assert all(1024 <= N <= 65536 and 1000 <= st <= 10000 for _, N, st in cases)
    assert any(N % 128 for _, N, _ in cases)
    for eq, N, _ in cases:
        step = 4 if eq == "heat" else 8
        for tuned in (256, 512, 1024):
            n = bench.fit_width(eq, N, tuned)
            K, d = N // n, N % n
            assert K >= 2 and n % step == 0 and n <= tuned
            assert n + -(-d // K) <= tuned + step   # the widest node
    assert bench.bucket(1024) == 10 and bench.bucket(65536) == 16 and bench.bucket(3000) == 12


def test_op_counts_table():
    assert bench.op_count("ks") == 22 and bench.op_count("ks", "ops") == 14
    assert bench.op_count("heat") == 5 and bench.op_count("heat", "ops") == 3
    assert 100 < bench.op_count("euler", "ops") < 200
    r = bench.alu_roofline(1e10, 1.0, "ks", "f64")
    assert abs(r["achieved"] - 0.22) < 1e-12 and r["peak"] == bench.FP64_PEAK_TFLOPS


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


def test_issue_record_matches_the_kernel_code():
    """The batched FP32 line's issue-slot figure comes from an ncu capture of
    the current kernel code (re-capture after a kernel change)."""
    assert bench.NCU_ISSUE_FP32_BATCH["src"] == bench._kernel_src_hash()
    assert 0 < bench.NCU_ISSUE_FP32_BATCH["issue_frac"] <= 1
