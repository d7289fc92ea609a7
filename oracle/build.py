"""Compile the FP64 CPU oracle into oracle/liboracle.so.

Test infrastructure only: the oracle is the correctness reference for the
CUDA path and is never linked or loaded by the product library.
Flags: -O2 -ffp-contract=off (no FMA contraction, IEEE round-to-nearest),
OpenMP over elements.
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SOURCES = ["lgl.c", "thermo.c", "dg.c", "cases.c", "mlp.c", "filter.c", "hevi.c", "closure.c"]
LIB = os.path.join(HERE, "liboracle.so")


def build(force=False):
    srcs = [os.path.join(HERE, s) for s in SOURCES]
    deps = srcs + [os.path.join(HERE, h) for h in ("oracle.h", "oracle_internal.h")]
    if not force and os.path.exists(LIB):
        t = os.path.getmtime(LIB)
        if all(os.path.getmtime(d) <= t for d in deps):
            return LIB
    cmd = ["gcc", "-O2", "-std=gnu11", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
           "-fPIC", "-shared", "-Wall", "-Wno-unused-function", "-o", LIB] + srcs + ["-lm"]
    subprocess.check_call(cmd)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
