"""Build the FP64 CPU oracle (test infrastructure) into oracle/_build/libstp_oracle.so.

Plain gcc, no CUDA: the oracle shares nothing with the CUDA library. OpenMP is used only to
spread independent tiles over host cores when the oracle is timed as the CPU baseline.
"""
from __future__ import annotations

import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "libstp_oracle.so")
SRC = os.path.join(HERE, "stp_oracle.c")


def gcc_command(src: str, out: str) -> list:
    """The compile line of the oracle library (FP64, no contraction, no fast math)."""
    return ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
            "-fno-fast-math", "-Wall", "-o", out, src, "-lm"]


def build(force: bool = False) -> str:
    os.makedirs(OUT_DIR, exist_ok=True)
    if (not force and os.path.exists(LIB)
            and os.path.getmtime(LIB) >= max(os.path.getmtime(SRC),
                                             os.path.getmtime(os.path.join(HERE, "stp_oracle.h")))):
        return LIB
    tmp = LIB + ".tmp.%d" % os.getpid()
    subprocess.run(gcc_command(SRC, tmp), check=True)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force=True))
