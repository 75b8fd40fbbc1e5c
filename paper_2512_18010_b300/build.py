"""Builds the CUDA library ``libscff.so`` in-tree with nvcc for sm_103a.

The library is a plain C-ABI shared object (include/scff.h); the Python
binding in ``scff.py`` loads it with ctypes.  Run ``python -m
paper_2512_18010_b300.build`` or call :func:`build`.

Each source compiles to its own relocatable object under ``_build/`` (in
parallel, and only when it or a header is newer than its object); one nvcc
link step then writes the shared object.
"""
from __future__ import annotations

import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OBJ = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libscff.so")
SOURCES = ["scff_host.cpp", "kernels_direct.cu", "kernels_tc.cu", "kernels_separable.cu", "kernels_peaks.cu", "static_entry.cu",
           "server.cpp", "kernels_sph.cu", "spherical.cpp", "kernels_fft.cu", "fft_method.cpp"]
HEADERS = ["scff_internal.h", "tc_internal.h", "tc_schedule.h", "device_common.cuh", "scff_objects.h", "sph_common.h",
           "sph_internal.h", "fft_internal.h"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = [*ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr"]


def _headers_mtime() -> float:
    deps = [os.path.join(CSRC, f) for f in HEADERS]
    deps.append(os.path.join(os.path.dirname(HERE), "include", "scff.h"))
    return max(os.path.getmtime(d) for d in deps if os.path.exists(d))


def _obj(src: str) -> str:
    return os.path.join(OBJ, src + ".o")


def _obj_stale(src: str, hdr_t: float) -> bool:
    o = _obj(src)
    if not os.path.exists(o):
        return True
    t = os.path.getmtime(o)
    return os.path.getmtime(os.path.join(CSRC, src)) > t or hdr_t > t


def _stale() -> bool:
    if not os.path.exists(LIB):
        return True
    hdr_t = _headers_mtime()
    t = os.path.getmtime(LIB)
    return any(_obj_stale(s, hdr_t) or os.path.getmtime(_obj(s)) > t for s in SOURCES)


def _compile(nvcc: str, src: str, verbose: bool) -> tuple:
    cmd = [nvcc, *FLAGS, "-Xptxas", "-v" if verbose else "-O3", "-c",
           "-o", _obj(src) + ".tmp", os.path.join(CSRC, src)]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode == 0:
        os.replace(_obj(src) + ".tmp", _obj(src))
    return src, r


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and not _stale():
        return LIB
    nvcc = os.environ.get("NVCC", "nvcc")
    os.makedirs(OBJ, exist_ok=True)
    hdr_t = _headers_mtime()
    todo = [s for s in SOURCES if force or _obj_stale(s, hdr_t)]
    with ThreadPoolExecutor(max_workers=max(1, min(len(todo), os.cpu_count() or 4))) as ex:
        results = list(ex.map(lambda s: _compile(nvcc, s, verbose), todo))
    failed = False
    for src, r in results:
        if r.returncode != 0:
            failed = True
            sys.stderr.write(f"--- {src}\n" + r.stdout + r.stderr)
        elif verbose:
            sys.stderr.write(f"--- {src}\n" + r.stderr)
    if failed:
        raise RuntimeError("nvcc failed building libscff.so")
    link = [nvcc, *ARCH, "-shared", "-cudart", "shared", "-o", LIB + ".tmp", *[_obj(s) for s in SOURCES],
            "-Xlinker", "-rpath,/usr/local/cuda/lib64", "-Xlinker", "--no-undefined"]
    r = subprocess.run(link, capture_output=True, text=True)
    if r.returncode != 0:
        sys.stderr.write(r.stdout + r.stderr)
        raise RuntimeError("nvcc failed linking libscff.so")
    os.replace(LIB + ".tmp", LIB)
    return LIB


if __name__ == "__main__":
    build(force="--incremental" not in sys.argv, verbose="-v" in sys.argv)
    print(LIB)
