"""Host-side pieces of bench.py (no GPU): the traffic record matches the
committed kernel code for the timed configuration, the code-only hash ignores
comments, and the workload generators are deterministic."""
import numpy as np

import bench


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
