"""Compile the CUDA kernels and the C ABI into libinspirit.so (sm_103a).

With INSP_CHECK=1 in the environment the debug variant libinspirit_check.so is
built (and loaded by the binding) instead: internal bounds checks record
INSP_ECHECK in the DAG's status word rather than touching memory out of range.
"""
from __future__ import annotations

import glob
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CHECK = os.environ.get("INSP_CHECK", "") not in ("", "0")
SO = os.path.join(HERE, "libinspirit_check.so" if CHECK else "libinspirit.so")
ARCH = "-gencode=arch=compute_103a,code=sm_103a"


def sources() -> list[str]:
    return sorted(glob.glob(os.path.join(HERE, "csrc", "*.cu")))


def deps() -> list[str]:
    return sources() + glob.glob(os.path.join(HERE, "csrc", "*.cuh")) + glob.glob(os.path.join(HERE, "csrc", "*.h")) \
        + [os.path.join(ROOT, "include", "inspirit.h")]


def stale() -> bool:
    if not os.path.exists(SO):
        return True
    t = os.path.getmtime(SO)
    return any(os.path.getmtime(p) > t for p in deps())


def build(force: bool = False, verbose: bool = False, extra: list[str] | None = None) -> str:
    if not force and not stale():
        return SO
    nvcc = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
    tmp = SO + f".tmp{os.getpid()}"
    cmd = [nvcc, ARCH, "-O3", "-lineinfo", "-std=c++17", "--expt-relaxed-constexpr",
           "-Xcompiler", "-fPIC,-fvisibility=hidden", "-shared", "-o", tmp, *sources()] + (extra or []) + \
        (["-DINSP_CHECK"] if CHECK else [])
    if verbose:
        print(" ".join(cmd), file=sys.stderr)
    subprocess.check_call(cmd, cwd=HERE)
    os.replace(tmp, SO)
    return SO


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True,
                extra=["-Xptxas", "-v"] if "--ptxas" in sys.argv else None))
