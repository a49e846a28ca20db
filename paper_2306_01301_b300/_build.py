"""Build the nhplan shared library for sm_103a (B300) in-tree.

Produces paper_2306_01301_b300/_lib/libnhplan.so from csrc/*.cu with nvcc.
Objects are cached per source in _build/ next to the package root and the
library is relinked only when a source or header changed.
"""
from __future__ import annotations

import glob
import os
import shutil
import subprocess

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
LIBDIR = os.path.join(PKG, "_lib")
LIB = os.path.join(LIBDIR, "libnhplan.so")
OBJDIR = os.path.join(ROOT, "_build", "nhplan")
# the bounds-check build: every index of the plain plan path's kernels is
# checked on the device; the host reports a failure as PLAN_EINTERNAL
LIB_CHECKED = os.path.join(LIBDIR, "libnhplan_checked.so")
OBJDIR_CHECKED = os.path.join(ROOT, "_build", "nhplan_checked")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-Wall",
         "--expt-relaxed-constexpr", "-I" + os.path.join(ROOT, "include")]


def nvcc() -> str:
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", shutil.which("nvcc")):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found: the CUDA library cannot be built")


def _headers():
    return (glob.glob(os.path.join(CSRC, "*.h")) + glob.glob(os.path.join(CSRC, "*.cuh")) +
            glob.glob(os.path.join(ROOT, "include", "*.h")))


def build(force: bool = False, verbose: bool = False, extra_flags=(), checked: bool = False) -> str:
    lib, objdir = (LIB_CHECKED, OBJDIR_CHECKED) if checked else (LIB, OBJDIR)
    if checked:
        extra_flags = tuple(extra_flags) + ("-DPLAN_BOUNDS_CHECK",)
    os.makedirs(LIBDIR, exist_ok=True)
    os.makedirs(objdir, exist_ok=True)
    srcs = sorted(glob.glob(os.path.join(CSRC, "*.cu")))
    hdr_time = max(os.path.getmtime(h) for h in _headers())
    objs, relink = [], force or not os.path.exists(lib)
    for src in srcs:
        obj = os.path.join(objdir, os.path.basename(src)[:-3] + ".o")
        objs.append(obj)
        if force or not os.path.exists(obj) or os.path.getmtime(obj) < max(os.path.getmtime(src), hdr_time):
            cmd = [nvcc()] + ARCH + FLAGS + list(extra_flags) + ["-c", src, "-o", obj + ".tmp"]
            if verbose:
                print(" ".join(cmd))
            subprocess.check_call(cmd)
            os.replace(obj + ".tmp", obj)
            relink = True
    if not relink and os.path.getmtime(lib) < max(os.path.getmtime(o) for o in objs):
        relink = True
    if relink:
        tmp = lib + f".tmp{os.getpid()}"
        cmd = [nvcc()] + ARCH + ["-shared", "-o", tmp] + objs
        if verbose:
            print(" ".join(cmd))
        subprocess.check_call(cmd)
        os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    import sys
    print(build(force="--force" in sys.argv, verbose=True, checked="--checked" in sys.argv))
