"""Compile the C oracle into ``oracle/_build/liboracle.so`` (test infrastructure).

Plain gcc, no FMA contraction, so that every FP64 operation in the oracle is
the rounded operation written in the source.
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "liboracle.so")
SRC = [os.path.join(HERE, "fv_oracle.c")]
HDR = [os.path.join(HERE, "fv_oracle.h"), os.path.join(HERE, "lbr_steps.h")]


def up_to_date() -> bool:
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(f) <= t for f in SRC + HDR)


def compile_library(sources, out: str) -> None:
    """gcc the given C sources into the shared library ``out``."""
    cmd = ["gcc", "-std=gnu11", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
           "-Wall", "-Wextra", "-Wno-unused-parameter", "-o", out] + list(sources) + ["-lm",
                                                                                       "-lpthread"]
    subprocess.run(cmd, check=True)


def build(force: bool = False) -> str:
    if not force and up_to_date():
        return LIB
    os.makedirs(OUT_DIR, exist_ok=True)
    tmp = LIB + ".tmp%d" % os.getpid()
    compile_library(SRC, tmp)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
