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
    "points_per_block": 512, "launch": "per_phase", "threads": 0,
}
METRIC = "G point-updates/s swept vs classic @2^20 pts (FP64); p50/p99 served solve latency"
UNIT = "G point-updates/s"

# Floating-point operations of one KS point-update (two RK2 stages of eight
# FP64 operations: five FMAs, two adds, one multiply = 13 flops each).
KS_FLOPS_PER_UPDATE = 26
KS_FP64_OPS_PER_UPDATE = 16
# FP64 pipe of GB300: 152 SMs x 2 DFMA/clk x 2 flop x 2.07 GHz (the nominal
# 1.25 TFLOP/s dense FP64 at the maximum SM clock).
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12

# DRAM traffic per launch of the dominant kernel from one ncu capture, keyed by
# a hash of the kernel sources it was taken on; reported as null once the
# sources change.
NCU_TRAFFIC = {
    # profiles/swept_phase_kernel_ks_n512.md: dram__bytes_read.sum + dram__bytes_write.sum of a
    # full-diamond launch (16.78 MB + 0), cold caches
    "swept_phase_kernel<double,KS> n=512": {"src": "cc59ea96f376ed8e", "bytes_per_launch": 16784384},
}


def _kernel_src_hash() -> str:
    h = hashlib.sha256()
    for f in ("swept.cu", "scheme.cuh", "launch.h"):
        with open(os.path.join(ROOT, "paper_1705_03162_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
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
def cpu_oracle_rate(wl: dict, budget_s: float = 12.0) -> dict:
    import oracle as O
    spec = I.ks_spec(wl["n_points"])
    u = I.initial_state(spec)
    prob = O.OracleProblem(O.KS, O.PERIODIC, spec.n_points, spec.dx, spec.dt)
    t0 = time.perf_counter()
    O.classic(prob, u, 4)
    probe = max(time.perf_counter() - t0, 1e-3) / 4
    steps = max(4, int(budget_s / probe))
    t0 = time.perf_counter()
    O.classic(prob, u, steps)
    el = time.perf_counter() - t0
    return {"value": spec.n_points * steps / el / 1e9, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"KS N=2^20 FP64 classic oracle, {steps} timesteps from the initial state "
                      f"(of the workload's {wl['steps']}), single thread, {el:.1f} s"}


def run_reference(args, wl):
    world, rank, _ = _dist_init()
    if rank != 0:
        return
    import oracle as O
    spec = I.ks_spec(wl["n_points"])
    u0 = I.initial_state(spec)
    prob = O.OracleProblem(O.KS, O.PERIODIC, spec.n_points, spec.dx, spec.dt)
    sample_steps = 16
    for _ in range(args.warmup):
        O.classic(prob, u0.copy(), sample_steps)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        O.classic(prob, u0.copy(), sample_steps)
    el = time.perf_counter() - t0
    value = spec.n_points * sample_steps * args.steps / el / 1e9
    sample = (f"each step: KS N=2^20 FP64 classic oracle for {sample_steps} of the workload's "
              f"{wl['steps']} timesteps, single thread")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": el / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": "KS N=2^20 FP64 10^4 steps (dx=0.5, dt=0.005)", "n_points": wl["n_points"],
                   "timesteps": wl["steps"], "sample_timesteps": sample_steps},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


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
    u0_host = I.initial_state(spec)
    u0_dev = torch.from_numpy(u0_host).cuda()
    steps = wl["steps"]
    N = spec.n_points
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")   # > 126 MB L2
    prob = S.Problem(spec, u0_dev)

    def one(scheme):
        return prob.advance(steps, scheme, wl["points_per_block"] if scheme == "swept" else 0,
                            wl["launch"], wl["threads"])

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
    l1 = prob.kernel_launches()
    t_classic = timed("classic", args.steps)
    launches_classic = prob.kernel_launches() - l1
    torch.cuda.synchronize()
    dist.barrier()
    t_classic = dist.max(t_classic)
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

    upd = float(N) * steps * args.steps * world
    value = upd / t_swept / 1e9
    classic_value = upd / t_classic / 1e9
    e2e_value = upd / t_e2e / 1e9

    # roofline of the dominant kernel (the swept phase kernel, FP64-pipe bound)
    launches_per_solve = launches_swept / args.steps
    avg_launch_s = t_swept / args.steps / launches_per_solve
    flops_per_launch = float(N) * steps * KS_FLOPS_PER_UPDATE / launches_per_solve
    achieved = flops_per_launch / avg_launch_s / 1e12
    ops_rate = float(N) * steps * args.steps * KS_FP64_OPS_PER_UPDATE / t_swept / 1e12
    key = f"swept_phase_kernel<double,KS> n={wl['points_per_block']}"
    traffic = None
    rec = NCU_TRAFFIC.get(key)
    if rec and rec.get("src") == _kernel_src_hash():
        traffic = rec["bytes_per_launch"]

    if rank != 0:
        dist.close()
        return
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_swept / args.steps * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "KS N=2^20 FP64 10^4 steps (dx=0.5, dt=0.005, u0=cos(x/16)(1+sin(x/16)))",
                   "n_points": N, "timesteps": steps, "scheme": "swept",
                   "points_per_block": wl["points_per_block"], "launch": wl["launch"],
                   "parallelism": f"replicas x{world}",
                   "l2": "256 MB buffer written before every timed solve (state 16 MB is L2-resident within a solve)"},
        "classic": {"value": classic_value, "ms_per_step": t_classic / args.steps * 1e3,
                    "kernel_launches_per_solve": launches_classic / args.steps,
                    "swept_speedup": classic_value and value / classic_value},
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(u0_host.nbytes),
                "d2h_bytes_per_step": int(u0_host.nbytes)},
        "roofline": {"bound": "alu", "achieved": achieved, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                     "frac": achieved / FP64_PEAK_TFLOPS, "traffic": traffic,
                     "kernel": key, "flops_per_update": KS_FLOPS_PER_UPDATE,
                     "fp64_ops_per_update": KS_FP64_OPS_PER_UPDATE,
                     "fp64_pipe_frac": ops_rate / (FP64_PEAK_TFLOPS / 2),
                     "peak_note": "FP64 pipe derived: 152 SMs x 2 DFMA/clk x 2 flop x 2.07 GHz"},
        "gpu_launches": int(launches_swept),
        "clocks": clk,
    }
    if world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_oracle_rate(wl)
    print(json.dumps(line), flush=True)
    dist.close()


def main():
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["gb300", "reference"], default="gb300")
    ap.add_argument("--points-per-block", type=int, default=DEFAULT_WORKLOAD["points_per_block"])
    ap.add_argument("--launch", choices=["per_phase", "persistent", "auto"], default=DEFAULT_WORKLOAD["launch"])
    ap.add_argument("--threads", type=int, default=0)
    ap.add_argument("--timesteps", type=int, default=DEFAULT_WORKLOAD["steps"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    wl = dict(DEFAULT_WORKLOAD, points_per_block=args.points_per_block, launch=args.launch,
              threads=args.threads, steps=args.timesteps)
    if args.impl == "reference":
        run_reference(args, wl)
    else:
        run_gpu(args, wl)


if __name__ == "__main__":
    main()
