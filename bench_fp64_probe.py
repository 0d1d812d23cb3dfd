"""Build and run the FP64 / FP32 throughput probe (bench_fp64_probe.cu).

Measures FMA issue rates and the throughput of CUDA's math-library calls
(exp, log, erfcx, erfc, reciprocal, sqrt, normcdfinv, expm1, log1p, and their
FP32 forms), of the library's own table-driven FP64 erfcx, log and exp, of an
FP64 -> FP32 -> FP64 conversion pair and of an FP64 division: the numbers that
decide which steps of the implied-volatility path are affordable in FP64 on
this GPU.

Usage: python bench_fp64_probe.py
"""
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_2604_27210_gb300 import build as _build  # noqa: E402


def main():
    src = os.path.join(ROOT, "bench_fp64_probe.cu")
    exe = os.path.join(_build.OUT_DIR, "bench_fp64_probe")
    os.makedirs(os.path.dirname(exe), exist_ok=True)
    subprocess.run([_build.nvcc()] + _build.ARCH + ["-O3", "-std=c++17", "--extended-lambda",
                                                   "-I", _build.CSRC, src, "-o", exe],
                   check=True)
    r = subprocess.run([exe])
    sys.exit(r.returncode)


if __name__ == "__main__":
    main()
