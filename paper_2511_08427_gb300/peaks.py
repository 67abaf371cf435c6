"""On-chip throughput micro-benchmarks (roofline denominators of the projector kernels).

    python -m paper_2511_08427_gb300.peaks

Builds peaks.cu (beside this file) for sm_103a and prints one JSON line: int32 and FP32 shared-memory reductions,
conflict-free 32-bit shared-memory loads, FP32 FMAs, and L1-resident 32-bit global loads (read-only path) and
texture point fetches, each per clock per SM (clock = the device's reported maximum SM clock; a run at a
lower clock reads proportionally lower).
"""
from __future__ import annotations

import os
import subprocess
import sys

from .build import ARCH, OUT, _nvcc

HERE = os.path.dirname(os.path.abspath(__file__))


def main() -> int:
    os.makedirs(OUT, exist_ok=True)
    exe = os.path.join(OUT, "peaks")
    src = os.path.join(HERE, "peaks.cu")
    subprocess.run([_nvcc(), *ARCH, "-O3", "-o", exe, src], check=True)
    return subprocess.run([exe]).returncode


if __name__ == "__main__":
    sys.exit(main())
