"""Build and run the GB300 peaks probe (csrc/peaks_probe.cu).

    python -m paper_1705_03162_gb300.peaks

Prints FP64 / FP32 FMA throughput, the cost of masked lanes, DDIV / DSQRT
throughput, a shared-memory load rate and kernel-launch latency.  These set the
FP64-pipe roofline of the stencil kernels (all FP64 paths here are bound by it).
"""
import os
import subprocess
import sys

from .build import ARCH, BUILD, CSRC, _nvcc


def main() -> int:
    os.makedirs(BUILD, exist_ok=True)
    exe = os.path.join(BUILD, "peaks_probe")
    src = os.path.join(CSRC, "peaks_probe.cu")
    if not os.path.exists(exe) or os.path.getmtime(src) > os.path.getmtime(exe):
        subprocess.run([_nvcc(), *ARCH, "-O3", "-o", exe, src], check=True)
    return subprocess.run([exe]).returncode


if __name__ == "__main__":
    sys.exit(main())
