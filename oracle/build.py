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


def build(force: bool = False, openmp: bool = False) -> str:
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(SRC):
        return LIB
    cmd = ["gcc", "-std=c11", "-O2", "-ffp-contract=off", "-fPIC", "-shared", SRC, "-o", LIB + ".tmp", "-lm"]
    if needs_quadmath():
        cmd.append("-lquadmath")
    subprocess.run(cmd, check=True)
    os.replace(LIB + ".tmp", LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
