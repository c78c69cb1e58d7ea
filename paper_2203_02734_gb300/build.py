"""Compile the CUDA library (csrc/) into libpywolf_gb.so next to this file, for sm_103a.

One translation unit, one -gencode, no cmake: a single nvcc call.  Rebuilds only when a
source or the public header is newer than the library (or when forced).
"""
import glob
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
LIB = os.path.join(HERE, "libpywolf_gb.so")
SRC = os.path.join(HERE, "csrc", "pywolf_gb.cu")
SRCS = [SRC, os.path.join(HERE, "csrc", "noalloc.cu"), os.path.join(HERE, "csrc", "batch.cu")]
ARCH = "-gencode=arch=compute_103a,code=sm_103a"


def _nvcc():
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libpywolf_gb.so")


def _deps():
    return SRCS + glob.glob(os.path.join(HERE, "csrc", "*.cuh")) + [os.path.join(ROOT, "include", "pywolf_gb.h")]


def up_to_date():
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(p) <= t for p in _deps())


def build(force=False, verbose=False):
    """Build libpywolf_gb.so if needed; returns its path.  Raises on a compiler error."""
    if not force and up_to_date():
        return LIB
    tmp = LIB + ".tmp%d" % os.getpid()
    cmd = [_nvcc(), "-std=c++17", "-O3", ARCH, "-lineinfo", "-Xptxas", "-v" if verbose else "-O3",
           "-shared", "-Xcompiler", "-fPIC", "-o", tmp] + SRCS
    res = subprocess.run(cmd, capture_output=True, text=True)
    if res.returncode != 0:
        raise RuntimeError("nvcc failed (%d):\n%s\n%s" % (res.returncode, " ".join(cmd), res.stderr[-4000:]))
    os.replace(tmp, LIB)
    if verbose:
        print(res.stderr)
    return LIB


if __name__ == "__main__":
    import sys
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
