"""Build the engine's shared library (_lexgb.so) in-tree with nvcc for sm_103a."""
from __future__ import annotations

import os
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
LIB = os.path.join(PKG, "_lexgb.so")
SOURCES = ["lexgb_capi.cu", "lexgb_noalloc.cu", "lexgb_mlp.cu", "lexgb_vertical.cu", "lexgb_rhs.cu", "lexgb_df2x.cu",
           "lexgb_df2bx.cu", "lexgb_batch_df.cu",
           "lexgb_up3z.cu", "lexgb_up3x.cu", "leja_host.cpp"]
HEADERS = ["leja_kernels.cuh", "leja_df64.cuh", "leja_df64_2step.cuh", "leja_vertical.cuh", "leja_batch.cuh",
           "leja_upwind.cuh", "leja_upwind_2step.cuh", "lexgb_internal.h", "lexgb_vertical.h",
           "leja_df64_2step_x.cuh", "lexgb_df2x.h", "leja_df64_2step_bx.cuh", "leja_batch_state.h",
           "leja_upwind_z.cuh", "leja_upwind_2step_x.cuh",
           "leja_vertical_2x.cuh", "leja_vertical_2bx.cuh"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _inputs():
    files = [os.path.join(CSRC, s) for s in SOURCES + HEADERS]
    files.append(os.path.join(INCLUDE, "lexgb.h"))
    files.append(os.path.abspath(__file__))
    return files


def up_to_date() -> bool:
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(f) <= t for f in _inputs() if os.path.exists(f))


def _threads() -> int:
    """Translation units compiled at once: one per core, at most one per source."""
    return max(1, min(os.cpu_count() or 4, len(SOURCES)))


def nvcc_command(out: str, extra=()):
    nvcc = os.environ.get("NVCC", "nvcc")
    return [nvcc, "-O3", "-std=c++17", *ARCH, "-lineinfo", "-Xcompiler", "-fPIC,-O2", "-shared",
            "--threads", str(_threads()), "-diag-suppress", "177", f"-I{INCLUDE}", *extra, *[os.path.join(CSRC, s) for s in SOURCES], "-o", out]


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and up_to_date():
        return LIB
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = nvcc_command(tmp)
    if verbose:
        print(" ".join(cmd))
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
