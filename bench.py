#!/usr/bin/env python3
"""Benchmark of the swept time-space decomposition on GB300.

Metric: G point-updates/s of the swept scheme (and, beside it, the classic
scheme) for the Kuramoto-Sivashinsky problem at N = 2^20 points, FP64,
10^4 timesteps (dx = 0.5, dt = 0.005, u0 = cos(x/16)(1 + sin(x/16))).
A point-update is one grid point advanced one full timestep.  One benchmark
step is one whole solve of 10^4 timesteps from the initial state.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl {gb300,reference}]

With --gpus N > 1 (under torch.distributed.run) every rank solves its own
instance: independent problems, no data exchange (weak scaling).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1705_03162_gb300 import inputs as I  # noqa: E402

DEFAULT_WORKLOAD = {
    "eq": "ks", "n_points": 1 << 20, "steps": 10_000, "dtype": "f64",
    "points_per_block": 1024, "launch": "persistent", "threads": 256,
}
METRIC = "G point-updates/s swept vs classic @2^20 pts (FP64); p50/p99 served solve latency"
WORKLOAD = "KS N=2^20 {} 10^4 steps (dx=0.5, dt=0.005, u0=cos(x/16)(1+sin(x/16)))"
UNIT = "G point-updates/s"

# Roofline denominators.  FP64 / FP32 pipes: measured on GB300 by a
# microbenchmark of independent FMA chains (626 G DFMA/s = 1.253 TFLOP/s;
# 78.3 TFLOP/s FFMA); the nominal 152 SMs x 2 DFMA/clk x 2 flop x 2.07 GHz is
# 1.259 TFLOP/s.  HBM: the measured copy bandwidth, read at run time.
FP64_PEAK_TFLOPS = 1.253
FP32_PEAK_TFLOPS = 78.3
HBM_FALLBACK_GBS = 6800.0

# Floating-point operations per point-update, counted by the CPU oracle's
# counting build and stored as data (oracle/opcounts.json, written by
# oracle/write_opcounts.py); read here as a table, never executed.
OPCOUNTS_PATH = os.path.join(ROOT, "oracle", "opcounts.json")


def _opcounts() -> dict:
    with open(OPCOUNTS_PATH) as f:
        return json.load(f)["counts"]


def op_count(eq: str, what: str = "flops") -> float:
    """Algorithmic flops (FMA = 2) or operations (FMA = 1) of one
    point-update; Euler on the Sod workload shape of the benchmark."""
    key = {"heat": "heat", "ks": "ks", "euler": "euler_sod_steps_over_n_1_256"}[eq]
    return float(_opcounts()[key]["algorithmic"][what])


def hbm_peak() -> tuple:
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "MEASURED_PEAKS.json hbm_gbs (measured)"
    except (OSError, KeyError, ValueError):
        return HBM_FALLBACK_GBS, "fallback 6.8 TB/s"


def alu_roofline(updates: float, seconds: float, eq: str, dtype: str) -> dict:
    """Algorithmic flops per second against the pipe of the working
    precision (every path here is bound by its FP pipe or by issue)."""
    peak = FP32_PEAK_TFLOPS if dtype == "f32" else FP64_PEAK_TFLOPS
    achieved = updates * op_count(eq) / seconds / 1e12
    ops = updates * op_count(eq, "ops") / seconds / 1e12
    return {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
            "flops_per_update": op_count(eq), "pipe_ops_frac": ops / (peak / 2),
            "peak_note": f"measured {'FP32' if dtype == 'f32' else 'FP64'} pipe"}

# DRAM traffic per launch of the dominant kernel from one ncu capture, keyed by
# a hash of the kernel sources it was taken on (code only: comments and blank
# lines do not count); reported as null once the code changes.
NCU_TRAFFIC = {
    # dram__bytes_read.sum + dram__bytes_write.sum of the whole 10^4-step solve in
    # one dataflow launch: a one-pass capture of the benchmark's own timed launch
    "swept_batch_kernel<double,KS> n=1024 threads=256": {"src": "3b6f26f5347ef8b7", "bytes_per_launch": 11734272},
}
# Issue-slot use of the batched FP32 launch from one ncu capture (the 4096
# instances of the batched workload, every node width 2048 fitted to N): warp
# instructions issued over 4 per SM per cycle, keyed like the traffic record
# and reported when the timed batch runs that width.
NCU_ISSUE_FP32_BATCH = {"src": "3b6f26f5347ef8b7", "width": 2048, "issue_frac": 0.70, "issue_active": 0.703,
                        "fma_pipe": 0.402}
KERNEL_OF_LAUNCH = {"per_phase": "swept_phase_kernel", "graph": "swept_phase_kernel",
                    "persistent": "swept_batch_kernel", "auto": "swept_batch_kernel"}


def _code_only(text: str) -> str:
    """Source without comments and blank lines (a comment edit does not change a kernel)."""
    import re
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    lines = (re.sub(r"//.*", "", ln).rstrip() for ln in text.splitlines())
    return "\n".join(ln for ln in lines if ln.strip())


def _kernel_src_hash() -> str:
    h = hashlib.sha256()
    for f in ("swept.cu", "geometry.cuh", "scheme.cuh", "launch.h"):
        with open(os.path.join(ROOT, "paper_1705_03162_gb300", "csrc", f), encoding="utf-8") as fh:
            h.update(_code_only(fh.read()).encode())
    return h.hexdigest()[:16]


# ---------------------------------------------------------------------------
# distributed helpers (one process per GPU; replicas, no data-path collective)
# ---------------------------------------------------------------------------
def _dist_init():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


class _Dist:
    def __init__(self, world, backend):
        self.world = world
        self.pg = None
        if world > 1:
            import torch.distributed as dist
            dist.init_process_group(backend=backend)
            self.pg = dist

    def barrier(self):
        if self.pg:
            self.pg.barrier()

    def max(self, x: float) -> float:
        if not self.pg:
            return x
        import torch
        dev = "cuda" if torch.cuda.is_available() and self.pg.get_backend() == "nccl" else "cpu"
        t = torch.tensor([x], dtype=torch.float64, device=dev)
        self.pg.all_reduce(t, op=self.pg.ReduceOp.MAX)
        return float(t.item())

    def close(self):
        if self.pg:
            self.pg.destroy_process_group()


# ---------------------------------------------------------------------------
# clocks sampled during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100", "-f", self.path], stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self) -> dict:
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        try:
            for line in open(self.path):
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    smax.append(float(parts[2]))
                except ValueError:
                    continue
                for nm, v in zip(names, parts[5:9]):
                    if v.lower().startswith("active"):
                        reasons.add(nm)
        finally:
            os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "samples": len(sm), "reasons": sorted(reasons)}


# ---------------------------------------------------------------------------
# CPU oracle baseline (test infrastructure, timed as it stands)
# ---------------------------------------------------------------------------
def _host_cpu() -> dict:
    """Core count and CPU model of the host the CPU baseline ran on."""
    import platform
    model = platform.processor() or platform.machine()
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                key = line.split(":")[0].strip().lower()
                if key in ("model name", "cpu model", "hardware") and ":" in line:
                    model = line.split(":", 1)[1].strip()
                    break
    except OSError:
        pass
    return {"nproc": os.cpu_count(), "model": model, "arch": platform.machine()}


def _oracle_ks_rate(n_points: int, threads: int, budget_s: float) -> tuple:
    """(G point-updates/s, timesteps, seconds) of the CPU oracle's classic KS
    from the initial state, about budget_s of work."""
    import oracle as O
    spec = I.ks_spec(n_points)
    u = I.initial_state(spec)
    prob = O.OracleProblem(O.KS, O.PERIODIC, spec.n_points, spec.dx, spec.dt)
    t0 = time.perf_counter()
    O.classic(prob, u, 2, threads=threads)
    probe = max(time.perf_counter() - t0, 1e-3) / 2
    steps = max(4, int(budget_s / probe))
    t0 = time.perf_counter()
    O.classic(prob, u, steps, threads=threads)
    el = time.perf_counter() - t0
    return spec.n_points * steps / el / 1e9, steps, el


def cpu_oracle_rate(wl: dict, budget_s: float = 8.0) -> dict:
    """The CPU oracle as it stands, on the host: its OpenMP build on all cores
    (the baseline) and its single-threaded build beside it."""
    import oracle as O
    cores = os.cpu_count() or 1
    used = O.omp_threads(cores)
    v_all, st_all, el_all = _oracle_ks_rate(wl["n_points"], used, budget_s)
    v_one, st_one, el_one = _oracle_ks_rate(wl["n_points"], 1, budget_s)
    return {"value": v_all, "unit": UNIT, "cores": used, "kind": "oracle", "host": _host_cpu(),
            "sample": f"KS N=2^20 FP64 classic oracle (OpenMP build, {used} threads), {st_all} timesteps from "
                      f"the initial state (of the workload's {wl['steps']}), {el_all:.1f} s",
            "single_thread": {"value": v_one, "unit": UNIT, "cores": 1,
                              "sample": f"the single-threaded oracle, {st_one} timesteps, {el_one:.1f} s"}}


def run_reference(args, wl):
    """The reference arm: the CPU oracle (OpenMP build) on all host cores,
    for the same metric and workload; rank 0 alone."""
    world, rank, _ = _dist_init()
    if rank != 0:
        return
    import oracle as O
    spec = I.ks_spec(wl["n_points"])
    u0 = I.initial_state(spec)
    prob = O.OracleProblem(O.KS, O.PERIODIC, spec.n_points, spec.dx, spec.dt)
    cores = O.omp_threads(os.cpu_count() or 1)
    sample_steps = 16
    for _ in range(args.warmup):
        O.classic(prob, u0.copy(), sample_steps, threads=cores)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        O.classic(prob, u0.copy(), sample_steps, threads=cores)
    el = time.perf_counter() - t0
    value = spec.n_points * sample_steps * args.steps / el / 1e9
    sample = (f"each step: KS N=2^20 FP64 classic oracle (OpenMP build) for {sample_steps} of the workload's "
              f"{wl['steps']} timesteps, {cores} threads")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": el / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": WORKLOAD.format("FP64"), "n_points": wl["n_points"],
                   "timesteps": wl["steps"], "sample_timesteps": sample_steps, "scheme": "classic (CPU oracle)",
                   "parallelism": f"{cores} host threads"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample,
                         "host": _host_cpu()},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# batched and served workloads, FP32 error (single GPU)
# ---------------------------------------------------------------------------
def _spec_ic(eq: str, N: int, dtype=np.float64):
    spec = I.heat_spec(N) if eq == "heat" else (I.ks_spec(N) if eq == "ks" else I.sod_spec(N))
    return spec, I.initial_state(spec, dtype)


def batched_cases(count: int = 4096, seed: int = 20170509):
    """(equation, N, timesteps) of the batched workload: heat and KS
    alternating, N log-uniform on [2^10, 2^16] (any integer), timesteps
    uniform on [10^3, 10^4]."""
    rng = np.random.default_rng(seed)
    cases = []
    for i in range(count):
        N = int(round(2 ** rng.uniform(10, 16)))
        cases.append(("heat" if i % 2 == 0 else "ks", N, int(rng.integers(1000, 10001))))
    return cases


def fit_width(eq: str, N: int, n: int) -> int:
    """The node width for an instance of N points from a target width n: the
    library's swp_fit_width (N split into max(2, ceil(N / n)) nearly equal
    nodes, none wider than n + 4 rad)."""
    from paper_1705_03162_gb300 import swept as S
    return S.fit_width(eq, N, n)


def bucket(N: int) -> int:
    import math
    return min(max(int(round(math.log2(N))), 10), 16)


def run_batched(count: int = 4096, seed: int = 20170509, dtypes=("f64", "f32"), width: int = 0,
                threads: int = 0) -> dict:
    """4096 independent heat + KS instances (batched_cases), one persistent
    launch per precision replayed from a CUDA graph, against advancing a
    sample of the same instances one by one, whose results must equal the
    batch's bit for bit.  Node widths (or `width` for every instance): the
    fastest, on one advance of the whole batch, of the library autotuner's
    choice per (equation, nearest power-of-two N) bucket and of one width for
    every instance (256, 512, 1024, 2048), each fitted to N (fit_width).  The
    autotuner measures each bucket alone; in the mixed batch every block is
    sized for the widest node, which can change the order."""
    import torch
    from paper_1705_03162_gb300 import swept as S
    cases = batched_cases(count, seed)
    out = {"instances": count, "workload": "heat+KS, N log-uniform 2^10..2^16 (any integer), steps U(1e3,1e4)"}
    steps = [c[2] for c in cases]
    upd = float(sum(c[1] * c[2] for c in cases))
    for dtype in dtypes:
        npdt = np.float64 if dtype == "f64" else np.float32
        stream = torch.cuda.Stream()
        probs, inputs = [], []
        for eq, N, _ in cases:
            spec, u0 = _spec_ic(eq, N, npdt)
            inputs.append((spec, u0))
            probs.append(S.Problem(spec, u0, dtype, stream=stream))

        def assign(choice):
            """(schemes, widths) of a candidate: a bucket table or one width."""
            sc, wd = [], []
            for eq, N, _ in cases:
                scheme, n = choice[(eq, bucket(N))] if isinstance(choice, dict) else ("swept", choice)
                sc.append(scheme)
                wd.append(fit_width(eq, N, n) if scheme == "swept" else min(n, N))
            return sc, wd

        def advance_ms(sc, wd, bt):
            ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            ev0.record(stream)
            bt.advance_ex(probs, steps, sc, wd, threads=threads, launch="persistent")
            ev1.record(stream)
            ev1.synchronize()
            return ev0.elapsed_time(ev1)

        t0 = time.perf_counter()
        tuning = {}
        if width:
            chosen = width
        else:
            tuned = {}
            for eq in ("heat", "ks"):
                for e in range(10, 17):
                    spec, u0 = _spec_ic(eq, 2 ** e, npdt)
                    # enough copies (at least 2^21 points) to fill the GPU
                    tuned[(eq, e)] = S.autotune(spec, u0, count=max(256, (1 << 21) >> e), steps=128, dtype=dtype)
            tuning["per_bucket_autotune"] = {f"{k[0]}2^{k[1]}": f"{v[0]} {v[1]}" for k, v in tuned.items()}
            uniform = (256, 512, 1024, 2048)
            with S.Batch(stream) as bt:
                # one width for every instance, fitted to each N, timed by the
                # library on the batch itself (states put back after each)
                _, best_u, ms_u = bt.tune_width(probs, steps, uniform, threads=threads)
                # and the per-bucket autotuner's choice, timed the same way
                ms_b = advance_ms(*assign(tuned), bt)
            for p, (_, u0) in zip(probs, inputs):   # back to the initial states
                p.write(u0)
            times = {"per-bucket autotune": ms_b, **{str(w): m for w, m in zip(uniform, ms_u)}}
            tuning["one_advance_ms"] = {k: round(v, 2) for k, v in times.items()}
            chosen = tuned if ms_b < ms_u[best_u] else uniform[best_u]
            tuning["chosen"] = "per-bucket autotune" if isinstance(chosen, dict) else str(chosen)
        tune_s = time.perf_counter() - t0
        schemes, widths = assign(chosen)
        with S.Batch(stream) as bt:
            # warm-up: two advances captured as CUDA graphs (an instance whose
            # advance ends in its other row alternates between two); the timed
            # third advance replays the first graph
            for _ in range(2):
                bt.advance_ex(probs, steps, schemes, widths, threads=threads, launch="graph")
            bt.synchronize()
            l0 = bt.kernel_launches()
            ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            ev0.record(stream)
            bt.advance_ex(probs, steps, schemes, widths, threads=threads, launch="graph")
            ev1.record(stream)
            bt.synchronize()
            ms = ev0.elapsed_time(ev1)
            launches = bt.kernel_launches() - l0
        # a sample advanced one problem at a time (the first advance timed),
        # the sample advanced one by one with the library defaults (scheme,
        # launch and width chosen per problem), three advances like the
        # batch's: every decomposition computes the same point updates, so the
        # results must be the batch's bits
        sample = range(min(32, count))
        su = float(sum(cases[i][1] * cases[i][2] for i in sample))
        solo_s, mismatches = 0.0, 0
        for i in sample:
            spec, u0 = inputs[i]
            with S.Problem(spec, u0, dtype) as q:
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                q.advance(steps[i], "auto")
                q.synchronize()
                solo_s += time.perf_counter() - t0
                q.advance(steps[i], "auto")
                q.advance(steps[i], "auto")
                mismatches += int(not np.array_equal(q.read(), probs[i].read()))
        for p in probs:
            p.close()
        if mismatches:
            raise AssertionError(f"batched {dtype}: {mismatches} sampled instances differ from solo advances")
        eqs = [c[0] for c in cases]
        flops = sum(c[1] * c[2] * op_count(c[0]) for c in cases)
        ops = sum(c[1] * c[2] * op_count(c[0], "ops") for c in cases)
        peak = FP32_PEAK_TFLOPS if dtype == "f32" else FP64_PEAK_TFLOPS
        out[dtype] = {"value": upd / ms / 1e6, "unit": UNIT, "ms": ms, "kernel_launches": launches,
                      "launch": "persistent kernel replayed from a CUDA graph",
                      "per_instance_value": su / solo_s / 1e9, "autotune_s": tune_s,
                      "swept_instances": sum(1 for x in schemes if x == "swept"),
                      "instances_with_wider_nodes": sum(1 for (e, N, _), sc, n in zip(cases, schemes, widths)
                                                        if sc == "swept" and N % n),
                      "sample_equals_solo_bitwise": f"{len(sample)} of {count} instances",
                      "roofline": {"bound": "alu", "achieved": flops / ms / 1e9, "peak": peak, "unit": "TFLOP/s",
                                   "frac": flops / ms / 1e9 / peak, "pipe_ops_frac": ops / ms / 1e9 / (peak / 2),
                                   "flops": f"heat {op_count('heat'):g}, KS {op_count('ks'):g} per update "
                                            f"({eqs.count('heat')} heat, {eqs.count('ks')} KS)",
                                   "peak_note": f"measured {'FP32' if dtype == 'f32' else 'FP64'} pipe",
                                   "issue": (dict(NCU_ISSUE_FP32_BATCH, bound="issue",
                                                  note="ncu capture of this workload at that width")
                                             if dtype == "f32" and NCU_ISSUE_FP32_BATCH["src"] == _kernel_src_hash()
                                             and chosen == NCU_ISSUE_FP32_BATCH["width"] else None)},
                      "widths": tuning if tuning else f"every instance {width}, fitted to N"}
    return out


def served_requests(count: int, seed: int, steps_lo: int = 100, steps_hi: int = 1000):
    """(unit-rate arrival gap, equation, N, timesteps) of the served mix:
    heat, KS and Euler with equal probability, N log-uniform on [2^10, 2^20]
    (any integer), timesteps uniform on [steps_lo, steps_hi]; the arrival
    times of a trace at rate lam are the cumulative gaps / lam."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        gap = float(rng.exponential(1.0))
        eq = ("heat", "ks", "euler")[int(rng.integers(0, 3))]
        N = int(round(2 ** rng.uniform(10, 20)))
        out.append((gap, eq, N, int(rng.integers(steps_lo, steps_hi + 1))))
    return out


def _trace(count: int, lam: float, seed: int):
    """(arrival time, equation, N, timesteps) of a Poisson trace at rate lam."""
    t, reqs = 0.0, []
    for gap, eq, N, st in served_requests(count, seed):
        t += gap / lam
        reqs.append((t, eq, N, st))
    return reqs


def _percentiles(lat):
    lat = np.sort(np.asarray(lat))
    return {"p50_s": float(np.percentile(lat, 50)), "p99_s": float(np.percentile(lat, 99)),
            "mean_s": float(lat.mean()), "max_s": float(lat.max()), "samples": int(lat.size)}


def fifo_latencies(arrivals, service):
    """Latency of each request of a single FIFO server: it starts when it has
    arrived and the previous request has finished, and takes its own
    service time."""
    t, lat = 0.0, []
    for a, s in zip(arrivals, service):
        start = max(a, t)
        t = start + s
        lat.append(t - a)
    return lat


def _digest(a: np.ndarray) -> str:
    return hashlib.sha1(np.ascontiguousarray(a).tobytes()).hexdigest()


def _serve(reqs, inputs, budget):
    """Submit reqs (arrival, eq, N, steps) at their arrival times to a server
    with continuous batching; latencies, span, server statistics and a digest
    of every result."""
    import threading
    from paper_1705_03162_gb300 import swept as S
    with S.Server(hbm_budget_bytes=budget, max_active=256, round_target_ms=20.0) as srv:
        ids = [None] * len(reqs)
        t_start = time.perf_counter()

        def feed():
            for i, (t_arr, eq, N, st) in enumerate(reqs):
                d = t_start + t_arr - time.perf_counter()
                if d > 0:
                    time.sleep(d)
                spec, u0 = inputs[i]
                ids[i] = srv.submit(spec, u0, st)

        th = threading.Thread(target=feed)
        th.start()
        th.join()
        lat, digests = [], []
        for i in ids:
            out, lt = srv.wait(i)
            lat.append(lt)
            digests.append(_digest(out))
        span = time.perf_counter() - t_start
        stats = srv.stats()
    return lat, span, stats, digests


def run_served(count: int = 1000, seed: int = 20170509, budget: int = 1 << 30) -> dict:
    """Serving with continuous batching against one request at a time.

    One request set (served_requests, FP64) at three offered loads: an
    overload trace (lam = 2000/s), then Poisson traces at 0.95 and 0.7 of the
    device's capacity for this mix solved one request at a time, C = count /
    (the sum of the solo solve times), the same arrival pattern rescaled.  The
    server's own capacity is its completion rate under overload.  The
    per-instance baseline is a FIFO queue over each request's own solo solve
    (create, advance with the library default, read back), timed once on the
    host clock and replayed against every trace."""
    from paper_1705_03162_gb300 import swept as S
    base = served_requests(count, seed)
    inputs = [_spec_ic(eq, N) for _, eq, N, _ in base]
    upd = float(sum(N * st for _, _, N, st in base))
    unit_arrivals = np.cumsum([g for g, _, _, _ in base])
    res = {"requests": count, "hbm_budget_bytes": budget,
           "mix": "heat/KS/Euler uniform, N log-uniform 2^10..2^20 (any integer), steps U(1e2,1e3), FP64",
           "per_instance_baseline": "FIFO over each request's measured solo solve (create, advance, read)",
           "loads": []}

    def trace(lam):
        return [(float(a / lam), eq, N, st) for a, (_, eq, N, st) in zip(unit_arrivals, base)]

    # per-instance service times, one solve at a time (and each result's
    # digest: every served result must equal its solo solve bit for bit)
    service, solo = [], []
    for (_, eq, N, st), (spec, u0) in zip(base, inputs):
        t0 = time.perf_counter()
        with S.Problem(spec, u0) as p:
            p.advance(st, "swept")
            out = p.read()
        service.append(time.perf_counter() - t0)
        solo.append(_digest(out))
    cap = count / sum(service)
    res["per_instance_capacity_req_per_s"] = cap
    for label, lam in (("overload", 2000.0), ("0.95 of capacity", 0.95 * cap), ("0.7 of capacity", 0.7 * cap)):
        reqs = trace(lam)
        lat, span, stats, digests = _serve(reqs, inputs, budget)
        differ = sum(1 for x, y in zip(digests, solo) if x != y)
        if differ:
            raise AssertionError(f"served ({label}): {differ} results differ from their solo solves")
        if label == "overload":
            res["capacity_req_per_s"] = count / span
        lat_b = fifo_latencies([r[0] for r in reqs], service)
        span_b = max(r[0] + l for r, l in zip(reqs, lat_b))
        res["loads"].append({
            "label": label, "lambda_per_s": lam, "offered_load": lam / cap,
            "served": dict(_percentiles(lat), throughput=upd / span / 1e9, unit=UNIT, rounds=stats["rounds"],
                           kernel_launches=stats["kernel_launches"],
                           results_equal_solo_bitwise=f"{count - differ} of {count}"),
            "per_instance": dict(_percentiles(lat_b), throughput=upd / span_b / 1e9, unit=UNIT)})
    return res


def other_configs(which=("heat", "sod")) -> dict:
    """The heat configuration (N = 1024, r = 0.25, 4096 steps) and the Sod
    tube at N = 2^20 (4096 steps, dt/dx = 0.2): swept against classic, FP64,
    device-timed, with the swept result checked bit for bit against the
    classic one.  Heat reports both swept forms, Shared (64-point nodes, CUDA
    graph) and the paper's Register variant (32-point warp nodes, graph), and
    the faster as `swept`; and the Register variant on one thread-block
    cluster (the whole advance in one launch)."""
    import torch
    from paper_1705_03162_gb300 import swept as S
    out = {}
    for name, eq, N, steps in (("heat N=1024 r=0.25 4096 steps", "heat", 1024, 4096),
                               ("Sod Euler N=2^20 4096 steps n=512 dataflow", "euler", 1 << 20, 4096)):
        if ("heat" if eq == "heat" else "sod") not in which:
            continue
        spec, u0 = _spec_ic(eq, N)
        u0d = torch.from_numpy(u0).cuda()
        rec, results = {}, {}
        with S.Problem(spec, u0d) as p:
            if eq == "heat":
                t_sh = _time_solve(p, u0d, steps, "swept", 64, "graph")
                results["swept_shared"] = p.read()
                t_reg = _time_solve(p, u0d, steps, "swept", 32, "register")
                results["swept_register"] = p.read()
                t_cl = _time_solve(p, u0d, steps, "swept", 32, "cluster")
                results["swept_cluster"] = p.read()
                rec["swept_shared_n64_graph"] = N * steps / t_sh / 1e9
                rec["swept_register_graph"] = N * steps / t_reg / 1e9
                rec["swept_register_cluster"] = N * steps / t_cl / 1e9
                t_sw = min(t_sh, t_reg, t_cl)
            else:
                t_sw = _time_solve(p, u0d, steps, "swept", 512, "persistent")
                results["swept"] = p.read()
            rec["swept"] = N * steps / t_sw / 1e9
            t_cl = _time_solve(p, u0d, steps, "classic", launch="graph")
            classic = p.read()
            rec["classic_graph"] = N * steps / t_cl / 1e9
        for k, v in results.items():
            if not np.array_equal(v, classic):
                raise AssertionError(f"{name}: {k} differs from classic")
        rec.update(unit=UNIT, swept_speedup=rec["swept"] / rec["classic_graph"],
                   swept_equals_classic_bitwise=True,
                   roofline=alu_roofline(float(N) * steps, t_sw, eq, "f64"))
        out[name] = rec
    return out


def fp32_error() -> dict:
    """FP32 heat / KS against the FP64 oracle (reported, not gated)."""
    import oracle as O
    from paper_1705_03162_gb300 import swept as S
    out = {}
    for name, spec, steps in (("heat N=1024 r=0.25 4096 steps", I.heat_spec(1024), 4096),
                              ("KS N=2^11 10^4 steps", I.ks_spec(2048), 10_000)):
        u64 = I.initial_state(spec)
        ref = u64.copy()
        eq = O.HEAT if spec.eq == "heat" else O.KS
        O.classic(O.OracleProblem(eq, O.PERIODIC, spec.n_points, spec.dx, spec.dt, spec.alpha), ref, steps)
        with S.Problem(spec, u64.astype(np.float32), "f32") as p:
            p.advance(steps, "swept")
            got = p.read().astype(np.float64)
        out[name] = float(np.max(np.abs(got - ref)) / np.max(np.abs(ref)))
    return out


def sweep_line(steps: int = 500) -> dict:
    """Swept at the library default (SWP_LAUNCH_AUTO and the default width)
    against classic replayed as a CUDA graph, heat and KS FP64 at
    N = 2^11..2^20 (the paper's size range, Section 6) and at 2^22 and 2^24,
    where the two level rows no longer fit in L2, with each one's fraction of
    the FP64 pipe."""
    import torch
    from paper_1705_03162_gb300 import swept as S
    pts = []
    for eq in ("heat", "ks"):
        for e in list(range(11, 21)) + [22, 24]:
            N = 1 << e
            spec, u0 = _spec_ic(eq, N)
            u0d = torch.from_numpy(u0).cuda()
            with S.Problem(spec, u0d) as p:
                t_cl = _time_solve(p, u0d, steps, "classic", launch="graph")
                t_sw = _time_solve(p, u0d, steps, "swept", 0, "auto")
            pts.append({"eq": eq, "n_points": N, "classic_graph": N * steps / t_cl / 1e9,
                        "swept": N * steps / t_sw / 1e9, "speedup": t_cl / t_sw,
                        "swept_frac": alu_roofline(float(N) * steps, t_sw, eq, "f64")["frac"],
                        "classic_frac": alu_roofline(float(N) * steps, t_cl, eq, "f64")["frac"]})
    return {"timesteps": steps, "dtype": "f64", "unit": UNIT,
            "swept": "library default (SWP_LAUNCH_AUTO, default node width)", "classic": "CUDA graph",
            "frac": "algorithmic flops / time / measured FP64 pipe", "points": pts,
            "swept_beats_classic_at": f"{sum(1 for q in pts if q['speedup'] > 1)} of {len(pts)} sizes"}


def bandwidth_line(steps: int = 200) -> dict:
    """Classic FP32 heat and KS at N = 2^26 (arrays far beyond L2), replayed as
    a CUDA graph: achieved algorithmic HBM bandwidth against the measured copy
    peak (heat reads and writes one value per update, 8 B; a KS timestep
    reads u, writes the predictor, reads it and u and writes u, 20 B)."""
    import torch
    from paper_1705_03162_gb300 import swept as S
    peak, src = hbm_peak()
    N = 1 << 26
    out = {"n_points": N, "dtype": "f32", "hbm_peak_gbs": peak, "peak_source": src, "lines": []}
    for eq, bytes_per_update, st in (("heat", 8, steps), ("ks", 20, steps // 2)):
        spec, u0 = _spec_ic(eq, N, np.float32)
        u0d = torch.from_numpy(u0).cuda()
        with S.Problem(spec, u0d, "f32") as p:
            t = _time_solve(p, u0d, st, "classic", launch="graph")
        gbs = bytes_per_update * N * st / t / 1e9
        out["lines"].append({"eq": eq, "timesteps": st, "value": N * st / t / 1e9, "unit": UNIT,
                             "roofline": {"bound": "hbm", "achieved": gbs, "peak": peak, "unit": "GB/s",
                                          "frac": gbs / peak, "bytes_per_update": bytes_per_update}})
        del u0d
    return out


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------
def run_gpu(args, wl):
    import torch
    from paper_1705_03162_gb300 import swept as S

    world, rank, local = _dist_init()
    torch.cuda.set_device(local)
    dist = _Dist(world, "nccl")
    S.load_library()

    spec = I.ks_spec(wl["n_points"])
    f32 = wl["dtype"] == "f32"
    u0_host = I.initial_state(spec).astype(np.float32 if f32 else np.float64)
    u0_dev = torch.from_numpy(u0_host).cuda()
    steps = wl["steps"]
    N = spec.n_points
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")   # > 126 MB L2
    prob = S.Problem(spec, u0_dev, wl["dtype"])

    def one(scheme):
        if scheme == "classic":
            return prob.advance(steps, "classic")
        return prob.advance(steps, "swept", wl["points_per_block"], wl["launch"], wl["threads"])

    def timed(scheme, k):
        """k solves, each from the initial state with L2 flushed before it;
        device time of the solves only (CUDA events on the problem's stream)."""
        total = 0.0
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(k)]
        for i in range(k):
            flush.fill_(i & 0xFF)
            prob.write(u0_dev)
            ev[i][0].record()
            one(scheme)
            ev[i][1].record()
        torch.cuda.synchronize()
        for a, b in ev:
            total += a.elapsed_time(b) / 1e3
        return total

    # warm-up (also builds per-width shared-memory attributes)
    for _ in range(args.warmup):
        prob.write(u0_dev)
        one("swept")
        prob.write(u0_dev)
        one("classic")
    torch.cuda.synchronize()

    clocks = ClockSampler(local)
    dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    launches0 = prob.kernel_launches()
    t_swept = timed("swept", args.steps)
    launches_swept = prob.kernel_launches() - launches0
    torch.cuda.synchronize()
    dist.barrier()
    t_swept = dist.max(t_swept)
    swept_result = prob.read()     # outside the timed regions
    l1 = prob.kernel_launches()
    t_classic = timed("classic", args.steps)
    launches_classic = prob.kernel_launches() - l1
    torch.cuda.synchronize()
    dist.barrier()
    t_classic = dist.max(t_classic)
    classic_result = prob.read()
    if not np.array_equal(swept_result, classic_result):
        raise AssertionError("the timed swept solve differs from the classic solve")
    # classic with its launch sequence as a CUDA graph (captured in warm-up)
    prob.write(u0_dev)
    prob.advance(steps, "classic", launch="graph")
    torch.cuda.synchronize()
    t_classic_graph = 0.0
    for _ in range(args.steps):
        flush.fill_(1)
        prob.write(u0_dev)
        a, b2 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        prob.advance(steps, "classic", launch="graph")
        b2.record()
        torch.cuda.synchronize()
        t_classic_graph += a.elapsed_time(b2) / 1e3
    t_classic_graph = dist.max(t_classic_graph)
    clk = clocks.stop()

    # end to end through the C ABI with host buffers (pinned): H2D of the
    # initial state, the solve, D2H of the result, every step
    pinned_in = torch.from_numpy(u0_host).pin_memory()
    pinned_out = torch.empty_like(pinned_in).pin_memory()
    dist.barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        prob.write(pinned_in)
        one("swept")
        prob.read(pinned_out)
    t_e2e = dist.max(time.perf_counter() - t0)
    prob.close()
    del flush

    upd = float(N) * steps * args.steps * world
    value = upd / t_swept / 1e9
    classic_value = upd / t_classic / 1e9
    classic_graph_value = upd / t_classic_graph / 1e9
    e2e_value = upd / t_e2e / 1e9

    # roofline of the dominant kernel (the dataflow kernel, FP64-pipe bound):
    # algorithmic flops of one launch / its average duration
    launches_per_solve = launches_swept / args.steps
    avg_launch_s = t_swept / args.steps / launches_per_solve
    roof = alu_roofline(float(N) * steps / launches_per_solve, avg_launch_s, "ks", wl["dtype"])
    key = (f"{KERNEL_OF_LAUNCH[wl['launch']]}<{'float' if f32 else 'double'},KS> "
           f"n={wl['points_per_block']} threads={wl['threads']}")
    traffic = None
    rec = NCU_TRAFFIC.get(key)
    if rec and rec.get("src") == _kernel_src_hash():
        traffic = rec["bytes_per_launch"]
    roof.update(traffic=traffic, kernel=key)

    if rank != 0:
        dist.close()
        return
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_swept / args.steps * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": wl["dtype"], "data": "synthetic",
        "config": {"workload": WORKLOAD.format("FP32" if f32 else "FP64"),
                   "n_points": N, "timesteps": steps, "scheme": "swept",
                   "points_per_block": wl["points_per_block"], "launch": wl["launch"],
                   "parallelism": f"replicas x{world}",
                   "l2": "256 MB buffer written before every timed solve (state 16 MB is L2-resident within a solve)"},
        "classic": {"value": classic_value, "ms_per_step": t_classic / args.steps * 1e3,
                    "kernel_launches_per_solve": launches_classic / args.steps,
                    "swept_speedup": classic_value and value / classic_value,
                    "graph_value": classic_graph_value,
                    "swept_speedup_vs_graph": value / classic_graph_value},
        "parity": {"swept_equals_classic_bitwise": True, "checked": "final states of the timed solves"},
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(u0_host.nbytes),
                "d2h_bytes_per_step": int(u0_host.nbytes)},
        "roofline": roof,
        "gpu_launches": int(launches_swept),
        "clocks": clk,
    }
    if world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_oracle_rate(wl)
    if world == 1 and not args.no_extras:
        line["sweep"] = sweep_line()
        line["bandwidth"] = bandwidth_line()
        line["other_configs"] = other_configs()
        line["fp32_rel_error_vs_fp64_oracle"] = fp32_error()
        line["batched"] = run_batched()
        line["served"] = run_served()
    print(json.dumps(line), flush=True)
    dist.close()


# ---------------------------------------------------------------------------
# optional modes: full size sweep (every width and launch), Sod sweep
# ---------------------------------------------------------------------------
def _time_solve(prob, u0d, steps, scheme, n=0, launch="per_phase", threads=0, reps=2):
    """Best of reps device-timed solves from u0d (after a short warm-up that
    also captures any graph); the state is the last solve's result."""
    import torch
    prob.write(u0d)
    prob.advance(min(steps, 20), scheme, n, launch, threads)
    torch.cuda.synchronize()
    best = float("inf")
    for _ in range(reps):
        prob.write(u0d)
        a, b2 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        prob.advance(steps, scheme, n, launch, threads)
        b2.record()
        torch.cuda.synchronize()
        best = min(best, a.elapsed_time(b2) / 1e3)
    return best


def run_sweep(steps: int = 2000):
    """Swept (shared, every node width and launch: per-phase, graph or
    dataflow), the library default, the Register variant and classic (CUDA
    graph) for heat and KS at N = 2^11..2^20, FP64: one JSON line each."""
    import torch
    from paper_1705_03162_gb300 import swept as S
    for eq in ("ks", "heat"):
        for e in range(11, 21):
            N = 1 << e
            spec, u0 = _spec_ic(eq, N)
            u0d = torch.from_numpy(u0).cuda()
            runs = []
            with S.Problem(spec, u0d) as p:
                classic = N * steps / _time_solve(p, u0d, steps, "classic", launch="graph") / 1e9
                reg = N * steps / _time_solve(p, u0d, steps, "swept", 0, "register", 64) / 1e9
                auto = N * steps / _time_solve(p, u0d, steps, "swept", 0, "auto") / 1e9
                cluster = N * steps / _time_solve(p, u0d, steps, "swept", 0, "cluster") / 1e9 if N <= 4096 else None
                best, cfg = 0.0, None
                for n in (64, 128, 256, 512, 1024):
                    if N % n or N // n < 2:
                        continue
                    for launch in ("per_phase", "graph", "persistent"):
                        r = N * steps / _time_solve(p, u0d, steps, "swept", n, launch) / 1e9
                        runs.append((n, launch, round(r, 3)))
                        if r > best:
                            best, cfg = r, {"points_per_block": n, "launch": launch}
            print(json.dumps({"sweep": eq, "n_points": N, "timesteps": steps, "dtype": "f64", "unit": UNIT,
                              "classic_graph": classic, "swept": best, "swept_config": cfg, "auto": auto,
                              "register": reg, "cluster": cluster, "swept_speedup": best / classic,
                              "runs": runs}), flush=True)


def run_sod(exps, steps: int, widths=None, threads=None):
    """Sod shock tube (dt/dx = 0.2, Dirichlet ends), FP64, fixed step count:
    swept at each node width, block size and launch (per-phase, graph,
    dataflow) and at the library default, against classic on a stream and as
    a CUDA graph; one JSON line per N."""
    import torch
    from paper_1705_03162_gb300 import swept as S
    for e in exps:
        N = 1 << e
        spec, u0 = _spec_ic("euler", N)
        u0d = torch.from_numpy(u0).cuda()
        with S.Problem(spec, u0d) as p:
            classic = N * steps / _time_solve(p, u0d, steps, "classic") / 1e9
            classic_graph = N * steps / _time_solve(p, u0d, steps, "classic", launch="graph") / 1e9
            auto = N * steps / _time_solve(p, u0d, steps, "swept", 0, "auto") / 1e9
            runs = []
            for n in widths or (64, 128, 256, 512):
                if N % n or N // n < 2:
                    continue
                for t in threads or (128, 256):
                    for launch in ("per_phase", "graph", "persistent"):
                        r = N * steps / _time_solve(p, u0d, steps, "swept", n, launch, t) / 1e9
                        runs.append({"points_per_block": n, "threads": t, "launch": launch, "swept": r})
        best = max(runs, key=lambda x: x["swept"])
        print(json.dumps({"sod": f"N=2^{e}", "timesteps": steps, "dtype": "f64", "unit": UNIT,
                          "classic": classic, "classic_graph": classic_graph, "swept_auto": auto, "swept_best": best,
                          "swept_speedup_vs_graph": best["swept"] / classic_graph, "swept_runs": runs}),
              flush=True)


def main():
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["gb300", "reference"], default="gb300")
    ap.add_argument("--points-per-block", type=int, default=None)
    ap.add_argument("--launch", choices=["per_phase", "persistent", "auto"], default=DEFAULT_WORKLOAD["launch"])
    ap.add_argument("--threads", type=int, default=None)
    ap.add_argument("--timesteps", type=int, default=None)
    ap.add_argument("--dtype", choices=["f64", "f32"], default=DEFAULT_WORKLOAD["dtype"],
                    help="precision of the timed KS workload (FP64 is the benchmark; FP32 is the variant)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--sweep", action="store_true", help="print the full per-size sweep lines instead")
    ap.add_argument("--bandwidth", action="store_true", help="print the classic FP32 bandwidth line instead")
    ap.add_argument("--sod", type=int, nargs="*", metavar="LOG2N",
                    help="print Sod swept-vs-classic lines for N = 2^LOG2N (default 11 14 17 20) instead; "
                         "--timesteps defaults to 4096 here, and --points-per-block / --threads, when given, "
                         "fix the swept configuration")
    ap.add_argument("--batched", type=int, metavar="COUNT",
                    help="print the batched heat+KS line for COUNT instances in the --dtype precision instead; "
                         "--points-per-block, when given, replaces the autotuned widths, and --threads sets "
                         "the batch's block size")
    ap.add_argument("--served", type=int, metavar="COUNT", help="print the served line for COUNT requests instead")
    ap.add_argument("--other", choices=["heat", "sod"], nargs="+",
                    help="print the heat-configuration and / or Sod line instead")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the sweep, bandwidth, other-configuration, batched, served and FP32-error lines")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    wl = dict(DEFAULT_WORKLOAD, launch=args.launch, dtype=args.dtype)
    if args.dtype == "f32":
        # per-phase launches of the register-blocked FP32 levels (8 slots per thread)
        wl.update(points_per_block=1024, launch="per_phase", threads=128)
    for key, val in (("points_per_block", args.points_per_block), ("threads", args.threads),
                     ("steps", args.timesteps)):
        if val is not None:
            wl[key] = val
    if args.impl == "reference":
        run_reference(args, wl)
        return
    if args.batched is not None or args.sod is not None or args.sweep or args.bandwidth or args.served or args.other:
        from paper_1705_03162_gb300 import swept as S
        S.load_library()
    if args.batched is not None:
        if args.batched < 1:
            ap.error("--batched needs COUNT >= 1")
        print(json.dumps({"batched": run_batched(args.batched, dtypes=(args.dtype,),
                                                 width=args.points_per_block or 0, threads=args.threads or 0)}))
    elif args.sod is not None:
        run_sod(args.sod or [11, 14, 17, 20], args.timesteps or 4096,
                [args.points_per_block] if args.points_per_block else None,
                [args.threads] if args.threads else None)
    elif args.served:
        print(json.dumps({"served": run_served(args.served)}))
    elif args.other:
        print(json.dumps({"other_configs": other_configs(tuple(args.other))}))
    elif args.sweep or args.bandwidth:
        if args.sweep:
            run_sweep()
        if args.bandwidth:
            print(json.dumps({"bandwidth": bandwidth_line()}))
    else:
        run_gpu(args, wl)


if __name__ == "__main__":
    main()
