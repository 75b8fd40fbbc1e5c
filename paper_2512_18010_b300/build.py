"""Builds the CUDA library ``libscff.so`` in-tree with nvcc for sm_103a.

The library is a plain C-ABI shared object (include/scff.h); the Python
binding in ``scff.py`` loads it with ctypes.  Run ``python -m
paper_2512_18010_b300.build`` or call :func:`build`.
"""
from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
LIB = os.path.join(HERE, "libscff.so")
SOURCES = ["scff_host.cpp", "kernels_direct.cu", "kernels_tc.cu", "kernels_separable.cu", "static_entry.cu",
           "server.cpp"]
HEADERS = ["scff_internal.h", "tc_internal.h", "device_common.cuh", "scff_objects.h"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    deps = [os.path.join(CSRC, f) for f in SOURCES + HEADERS]
    deps.append(os.path.join(os.path.dirname(HERE), "include", "scff.h"))
    return any(os.path.getmtime(d) > t for d in deps if os.path.exists(d))


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and not _stale():
        return LIB
    nvcc = os.environ.get("NVCC", "nvcc")
    cmd = [nvcc, *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-shared",
           "-cudart", "shared", "--expt-relaxed-constexpr", "-Xptxas", "-v" if verbose else "-O3",
           "-o", LIB + ".tmp", *[os.path.join(CSRC, f) for f in SOURCES],
           "-Xlinker", "-rpath,/usr/local/cuda/lib64"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        sys.stderr.write(r.stdout + r.stderr)
        raise RuntimeError("nvcc failed building libscff.so")
    if verbose:
        sys.stderr.write(r.stderr)
    os.replace(LIB + ".tmp", LIB)
    return LIB


if __name__ == "__main__":
    build(force=True, verbose="-v" in sys.argv)
    print(LIB)
