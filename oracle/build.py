"""Compile the CPU oracle (oracle.c) into oracle/_oracle.so with gcc.

Test infrastructure: the oracle is the checker, not the product.  It is built
with -ffp-contract=off so that x86-64 and aarch64 hosts evaluate the same
expressions without fused multiply-adds.
"""
from __future__ import annotations

import os
import platform
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "oracle.c")
LIB = os.path.join(HERE, "_oracle.so")


def needs_quadmath() -> bool:
    # long double is IEEE binary128 on aarch64 Linux; x86-64 needs libquadmath.
    return platform.machine() not in ("aarch64", "arm64")


LIB_OMP = os.path.join(HERE, "_oracle_omp.so")


def build(force: bool = False, openmp: bool = False) -> str:
    """The single-threaded parity library (_oracle.so), or with openmp=True
    the same source with its grid loops on all host cores (_oracle_omp.so,
    -O3 -fopenmp), which only times the CPU baseline."""
    lib = LIB_OMP if openmp else LIB
    if not force and os.path.exists(lib) and os.path.getmtime(lib) >= os.path.getmtime(SRC):
        return lib
    opt = ["-O3", "-fopenmp"] if openmp else ["-O2"]
    cmd = ["gcc", "-std=c11", *opt, "-ffp-contract=off", "-fPIC", "-shared", SRC, "-o", lib + ".tmp", "-lm"]
    if needs_quadmath():
        cmd.append("-lquadmath")
    subprocess.run(cmd, check=True)
    os.replace(lib + ".tmp", lib)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
    print(build(force="--force" in sys.argv, openmp=True))
