"""Build the fmmcph shared library in-tree with nvcc for sm_103a.

``python -m paper_2410_01626_b300.build`` or ``build()``; objects and the
library go to ``paper_2410_01626_b300/_build/``.  Rebuilds only what changed.
``build(checked=True)`` builds the bounds-checked variant (``-DFMM_BOUNDS_CHECK``:
index checks that report through the status word instead of accessing out of
range) into ``_build/checked/libfmmcph_checked.so``; ``--checked`` on the
command line builds both.
"""
from __future__ import annotations

import glob
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")
OUT = os.path.join(HERE, "_build")
LIB = os.path.join(OUT, "libfmmcph.so")
OUT_CHECKED = os.path.join(OUT, "checked")
LIB_CHECKED = os.path.join(OUT_CHECKED, "libfmmcph_checked.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-I" + INCLUDE, "-I" + CSRC]


def _nvcc():
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if c and (os.path.isabs(c) and os.path.exists(c) or not os.path.isabs(c)):
            return c
    return "nvcc"


def build(force: bool = False, verbose: bool = False, checked: bool = False) -> str:
    out = OUT_CHECKED if checked else OUT
    lib_path = LIB_CHECKED if checked else LIB
    flags = NVCC_FLAGS + (["-DFMM_BOUNDS_CHECK"] if checked else [])
    os.makedirs(out, exist_ok=True)
    headers = (glob.glob(os.path.join(CSRC, "*.h")) + glob.glob(os.path.join(CSRC, "*.cuh")) +
               glob.glob(os.path.join(INCLUDE, "*.h")))
    hdr_time = max(os.path.getmtime(h) for h in headers)
    objs = []
    for src in sorted(glob.glob(os.path.join(CSRC, "*.cu")) + glob.glob(os.path.join(CSRC, "*.cpp"))):
        obj = os.path.join(out, os.path.basename(src) + ".o")
        objs.append(obj)
        if not force and os.path.exists(obj) and os.path.getmtime(obj) >= max(os.path.getmtime(src), hdr_time):
            continue
        cmd = [_nvcc(), *flags, *ARCH, "-c", src, "-o", obj]
        if src.endswith(".cpp"):
            cmd = [_nvcc(), "-x", "cu", *flags, *ARCH, "-c", src, "-o", obj]
        if verbose:
            print(" ".join(cmd), file=sys.stderr)
        subprocess.check_call(cmd)
    if force or not os.path.exists(lib_path) or os.path.getmtime(lib_path) < max(os.path.getmtime(o) for o in objs):
        tmp = lib_path + f".{os.getpid()}.tmp"
        subprocess.check_call([_nvcc(), *ARCH, "-shared", "-o", tmp, *objs, "-lcuda"])
        os.replace(tmp, lib_path)
    return lib_path


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
    if "--checked" in sys.argv:
        print(build(force="--force" in sys.argv, verbose=True, checked=True))
