"""Build and run the FP64 / FP32 throughput probe (csrc/throughput_probe.cu).

Measures FMA issue rates and the throughput of CUDA's math-library calls
(exp, log, erfcx, erfc, reciprocal, sqrt, normcdfinv, expm1, log1p, and their
FP32 forms), of the library's own table-driven FP64 erfcx, log and exp, of an
FP64 -> FP32 -> FP64 conversion pair and of an FP64 division: the numbers that
decide which steps of the implied-volatility path are affordable in FP64 on
this GPU.

Usage: python -m paper_2604_27210_gb300.throughput_probe
"""
import os
import subprocess
import sys

from . import build as _build

HERE = os.path.dirname(os.path.abspath(__file__))


def main():
    src = os.path.join(HERE, "csrc", "throughput_probe.cu")
    exe = os.path.join(HERE, "_build", "throughput_probe")
    os.makedirs(os.path.dirname(exe), exist_ok=True)
    subprocess.run([_build.nvcc()] + _build.ARCH + ["-O3", "-std=c++17", "--extended-lambda",
                                                   "-I", os.path.join(HERE, "csrc"), src, "-o", exe],
                   check=True)
    r = subprocess.run([exe])
    sys.exit(r.returncode)


if __name__ == "__main__":
    main()
