"""Builds the sm_103a shared library ``lib/libchordal_admm.so`` in the source tree.

Each translation unit compiles in its own nvcc process (in parallel), then one nvcc call links the
shared library against the shared CUDA runtime (the same one PyTorch loads).
"""

from __future__ import annotations

import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
LIBDIR = os.path.join(PKG, "lib")
LIB = os.path.join(LIBDIR, "libchordal_admm.so")
OBJDIR = os.path.join(ROOT, "_build")

SOURCES = ["setup.cpp", "chordal.cpp", "project.cu", "kernels.cu", "adjoint.cu", "api.cu", "noalloc.cu", "kkt.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
COMMON = ["-std=c++17", "-O3", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-O3",
          "-I" + os.path.join(ROOT, "include")]


def _nvcc() -> str:
    cand = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(cand):
        raise RuntimeError("nvcc not found; the CUDA toolkit is required to build the library")
    return cand


def _run(cmd, verbose):
    if verbose:
        print(" ".join(cmd), flush=True)
    res = subprocess.run(cmd, capture_output=True, text=True)
    if res.returncode != 0:
        sys.stderr.write(res.stdout + res.stderr)
        raise RuntimeError(f"command failed ({res.returncode}): {' '.join(cmd)}")
    return res.stdout + res.stderr


def build(verbose: bool = False, ptxas_info: bool = False) -> str:
    """Compile every source for sm_103a and link the shared library; returns its path."""
    nvcc = _nvcc()
    os.makedirs(OBJDIR, exist_ok=True)
    os.makedirs(LIBDIR, exist_ok=True)
    objs = []
    cmds = []
    for src in SOURCES:
        obj = os.path.join(OBJDIR, os.path.splitext(src)[0] + ".o")
        objs.append(obj)
        cmd = [nvcc, *COMMON, *ARCH, "-c", os.path.join(CSRC, src), "-o", obj]
        if ptxas_info and src.endswith(".cu"):
            cmd += ["-Xptxas", "-v"]
        cmds.append(cmd)
    with ThreadPoolExecutor(max_workers=len(cmds)) as ex:
        outs = list(ex.map(lambda c: _run(c, verbose), cmds))
    if ptxas_info:
        for o in outs:
            sys.stdout.write(o)
    tmp = LIB + ".tmp"
    rpaths = []
    for cand in (nvcc, os.path.realpath(nvcc)):
        d = os.path.join(os.path.dirname(os.path.dirname(cand)), "lib64")
        if d not in rpaths:
            rpaths.append(d)
    _run([nvcc, "-shared", *ARCH, "-cudart", "shared", "-o", tmp, *objs, "-lpthread",
          "-Xlinker", "-rpath=" + ":".join(rpaths)], verbose)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(verbose=True, ptxas_info="-v" in sys.argv))
