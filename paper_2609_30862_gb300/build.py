"""In-tree build of the CUDA library (libqieo.so) for sm_103a with nvcc.

One -gencode; the translation units compile in parallel and are linked into one shared
object. The library is rebuilt when a source or the public header is newer than it.
"""
from __future__ import annotations

import glob
import os
import shutil
import subprocess

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(BUILD, "libqieo.so")
GENCODE = "arch=compute_103a,code=sm_103a"


def nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the QIEO CUDA library cannot be built")


def sources() -> list[str]:
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def deps() -> list[str]:
    return sources() + sorted(glob.glob(os.path.join(CSRC, "*.cuh"))) + \
        [os.path.join(ROOT, "include", "qieo.h")]


def stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    return any(os.path.getmtime(d) > t for d in deps())


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile every translation unit to an object in parallel, then link the library."""
    if not force and not stale():
        return LIB
    from concurrent.futures import ThreadPoolExecutor
    os.makedirs(BUILD, exist_ok=True)
    tag = "%d" % os.getpid()
    common = [nvcc(), "-gencode", GENCODE, "-O3", "-lineinfo", "-std=c++17",
              "-Xcompiler", "-fPIC", "-I", os.path.join(ROOT, "include"),
              *(["-Xptxas", "-v"] if verbose else [])]
    objs = [os.path.join(BUILD, os.path.basename(src)[:-3] + ".%s.o" % tag) for src in sources()]

    def compile_one(pair):
        src, obj = pair
        subprocess.check_call(common + ["-c", src, "-o", obj])

    try:
        with ThreadPoolExecutor(max_workers=max(1, len(objs))) as ex:
            list(ex.map(compile_one, zip(sources(), objs)))
        tmp = LIB + ".tmp" + tag
        subprocess.check_call([nvcc(), "-gencode", GENCODE, "-shared", *objs, "-o", tmp])
        os.replace(tmp, LIB)
    finally:
        for obj in objs:
            if os.path.exists(obj):
                os.remove(obj)
    return LIB


if __name__ == "__main__":
    import sys
    print(build(force=True, verbose="-v" in sys.argv))
