"""Compile the FP64 CPU oracle into oracle/liborc.so (test infrastructure only).

The oracle is plain C99 built with -O2 -ffp-contract=off and no fast-math, so that x86-64
and aarch64 hosts give the same results; OpenMP only splits independent node loops.
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "strm_oracle.c")
LIB = os.path.join(HERE, "liborc.so")


def build(force: bool = False) -> str:
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= max(
        os.path.getmtime(SRC), os.path.getmtime(os.path.join(HERE, "strm_oracle.h"))
    ):
        return LIB
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = [
        "gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
        "-fPIC", "-shared", "-Wall", "-Wno-unknown-pragmas", "-o", tmp, SRC, "-lm",
    ]
    subprocess.run(cmd, check=True, cwd=HERE)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
