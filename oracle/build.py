"""Compile the FP64 CPU oracle (test infrastructure) with gcc.

Builds oracle/liboracle.so from harp_oracle.c. Portable flags only (the
same source builds on x86_64 and aarch64); OpenMP splits independent outer
loops. Usage: python oracle/build.py
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "harp_oracle.c")
LIB = os.path.join(HERE, "liboracle.so")


def build(force: bool = False, quiet: bool = False) -> str:
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(SRC):
        return LIB
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-fno-fast-math",
           "-ffp-contract=off", SRC, "-o", LIB + ".tmp", "-lm"]
    if not quiet:
        print(" ".join(cmd), file=sys.stderr)
    subprocess.check_call(cmd)
    os.replace(LIB + ".tmp", LIB)
    return LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv)
