"""Compile the CUDA library ``libemt.so`` in-tree for sm_103a (B300)."""
from __future__ import annotations

import glob
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libemt.so")
# the checks build: every device-data index into a global array tested against the array's length (a bad one
# latches an error that emt_sync reports, and the access is kept in bounds); loaded when EMT_CHECKS=1
CHECKS_LIB_PATH = os.path.join(HERE, "libemt_checks.so")
# the phase-clock build: clock64 cycles per phase of every step of the single-network kernel, read by
# emt_phase_clocks (bench.py --leg phases); loaded when EMT_PHASES=1
PHASES_LIB_PATH = os.path.join(HERE, "libemt_phases.so")
ARCH = "-gencode=arch=compute_103a,code=sm_103a"


def sources():
    return sorted(glob.glob(os.path.join(HERE, "csrc", "*.cu")))


def headers():
    return sorted(glob.glob(os.path.join(HERE, "csrc", "*.h")) + glob.glob(os.path.join(HERE, "csrc", "*.cuh")) +
                  glob.glob(os.path.join(os.path.dirname(HERE), "include", "*.h")))


def needs_build(path: str = LIB_PATH) -> bool:
    if not os.path.exists(path):
        return True
    t = os.path.getmtime(path)
    return any(os.path.getmtime(f) > t for f in sources() + headers())


def build(force: bool = False, verbose: bool = False, checks: bool = False, phases: bool = False) -> str:
    """Build ``libemt.so`` (``libemt_checks.so`` with checks=True,
    ``libemt_phases.so`` with phases=True) with nvcc if it is missing or
    stale; return its path."""
    path = CHECKS_LIB_PATH if checks else (PHASES_LIB_PATH if phases else LIB_PATH)
    if not force and not needs_build(path):
        return path
    nvcc = os.environ.get("NVCC", "nvcc")
    tmp = path + f".tmp{os.getpid()}"
    # warnings are errors: one (a host-only constexpr call in __host__ __device__ code) once compiled to
    # device code that silently did nothing
    cmd = [nvcc, "-shared", "-Xcompiler", "-fPIC", ARCH, "-lineinfo", "-O3", "-std=c++17", "-Werror", "all-warnings",
           "-cudart", "shared", "-Xlinker", "-rpath,/usr/local/cuda/lib64", "-o", tmp] + sources()
    if checks:
        cmd.insert(1, "-DEMT_CHECKS")
    if phases:
        cmd.insert(1, "-DEMT_PHASE_CLOCKS")
    if verbose:
        cmd.insert(1, "-Xptxas=-v")
    subprocess.check_call(cmd)
    os.replace(tmp, path)
    return path


if __name__ == "__main__":
    print(build(force=True, verbose=True))
    print(build(force=True, checks=True))
    print(build(force=True, phases=True))
