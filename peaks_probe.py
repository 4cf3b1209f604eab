"""Build and run the GB300 peaks probe (peaks_probe.cu), a measurement tool
beside bench.py and not part of the library: FP64 / FP32 FMA throughput, the
cost of masked lanes, DDIV / DSQRT throughput, a barrier loop and kernel-launch
latency.  Its FP64 and FP32 FMA rates are the pipe peaks bench.py divides by.

    python peaks_probe.py
"""
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.abspath(__file__))


def main() -> int:
    sys.path.insert(0, ROOT)
    from paper_1705_03162_gb300.build import ARCH, _nvcc
    out = os.path.join(ROOT, "_build")
    os.makedirs(out, exist_ok=True)
    exe = os.path.join(out, "peaks_probe")
    src = os.path.join(ROOT, "peaks_probe.cu")
    if not os.path.exists(exe) or os.path.getmtime(src) > os.path.getmtime(exe):
        subprocess.run([_nvcc(), *ARCH, "-O3", "-o", exe, src], check=True)
    return subprocess.run([exe]).returncode


if __name__ == "__main__":
    sys.exit(main())
