"""Compile the native library ``libdq.so`` in-tree for sm_103a.

Each translation unit under ``csrc/`` is compiled by nvcc in parallel (one ``-gencode`` for
compute_103a / sm_103a), then linked into ``paper_2407_14591_gb300/libdq.so``. Objects go to
``paper_2407_14591_gb300/_build/``. Both are git-ignored. No cmake.

``build(checked=True)`` makes ``libdq_checked.so`` with ``-DDQ_CHECKED``: every rank used to
gather x is compared with the sector dimension on the device, and an out-of-range rank raises
the sector's error word instead of reading outside x (a debugging aid where no memory checker
can run). The binding loads it when the environment sets ``DQ_CHECKED=1``.

    python -m paper_2407_14591_gb300.build
"""

from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(PKG, "csrc")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(PKG, "libdq.so")
LIB_CHECKED = os.path.join(PKG, "libdq_checked.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-Wall", "--expt-relaxed-constexpr"]


def _nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found; the CUDA toolkit is required to build libdq.so")


def sources() -> list[str]:
    return sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cu", ".cpp")))


def _compile(nvcc: str, src: str, extra: list[str], objdir: str) -> str:
    obj = os.path.join(objdir, os.path.basename(src) + ".o")
    cmd = [nvcc, *ARCH, *FLAGS, *extra, "-I", os.path.join(PKG, "..", "include"), "-c", src, "-o", obj]
    res = subprocess.run(cmd, capture_output=True, text=True)
    if res.returncode != 0:
        raise RuntimeError(f"nvcc failed for {src}:\n{res.stdout}\n{res.stderr}")
    return obj


def build(verbose: bool = False, extra: list[str] | None = None, checked: bool = False) -> str:
    """Build libdq.so (or libdq_checked.so) if any source or header is newer than it; returns
    its path."""
    extra = list(extra or [])
    lib, objdir = (LIB_CHECKED, os.path.join(BUILD, "checked")) if checked else (LIB, BUILD)
    if checked:
        extra.append("-DDQ_CHECKED")
    srcs = sources()
    headers = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".h", ".cuh"))]
    headers.append(os.path.join(PKG, "..", "include", "dq.h"))
    if os.path.exists(lib) and extra == (["-DDQ_CHECKED"] if checked else []):
        t_lib = os.path.getmtime(lib)
        if all(os.path.getmtime(p) < t_lib for p in srcs + headers + [__file__]):
            return lib
    os.makedirs(objdir, exist_ok=True)
    nvcc = _nvcc()
    with cf.ThreadPoolExecutor(max_workers=min(8, len(srcs))) as ex:
        objs = list(ex.map(lambda s: _compile(nvcc, s, extra, objdir), srcs))
    tmp = lib + ".tmp"
    cmd = [nvcc, *ARCH, "-shared", "-o", tmp, *objs, "-lcudart_static", "-lrt", "-ldl", "-lpthread"]
    res = subprocess.run(cmd, capture_output=True, text=True)
    if res.returncode != 0:
        raise RuntimeError(f"link failed:\n{res.stdout}\n{res.stderr}")
    os.replace(tmp, lib)
    if verbose:
        print(f"built {lib}")
    return lib


if __name__ == "__main__":
    build(verbose=True, extra=sys.argv[1:])
