"""Builds the CUDA shared library behind include/gheap.h, in-tree.

nvcc -gencode arch=compute_103a,code=sm_103a (GB300) -> libgheap.so next to
this file: every .cu file of csrc/ -- gheap.cu (the heap and its C ABI),
sssp.cu and knapsack.cu (the applications built on that ABI) -- compiled in
parallel and linked once.  Rebuilds when a source is newer than the library.
"""
import glob
import os
import shutil
import subprocess

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
LIB = os.path.join(PKG, "libgheap.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
COMPILE = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC"]


def sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _deps():
    return (sources() + glob.glob(os.path.join(CSRC, "*.cuh"))
            + glob.glob(os.path.join(INCLUDE, "*.h")))


def nvcc():
    exe = shutil.which("nvcc")
    if exe is None and os.path.exists("/usr/local/cuda/bin/nvcc"):
        exe = "/usr/local/cuda/bin/nvcc"
    if exe is None:
        raise RuntimeError("nvcc not found: cannot build libgheap.so")
    return exe


def up_to_date():
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(f) <= t for f in _deps())


def build(force=False, verbose=False):
    """Compiles libgheap.so: every .cu file in csrc/ to an object, in parallel,
    then one link."""
    if not force and up_to_date():
        return LIB
    tag = "%d" % os.getpid()
    objs, procs = [], []
    for src in sources():
        obj = os.path.join(PKG, "." + os.path.basename(src) + "." + tag + ".o")
        cmd = [nvcc()] + ARCH + COMPILE + ["-I" + INCLUDE, "-I" + CSRC, "-c", "-o", obj, src]
        if verbose:
            print(" ".join(cmd))
        objs.append(obj)
        procs.append((cmd, subprocess.Popen(cmd)))
    try:
        for cmd, p in procs:
            if p.wait() != 0:
                raise subprocess.CalledProcessError(p.returncode, cmd)
        tmp = LIB + "." + tag + ".tmp"
        cmd = [nvcc()] + ARCH + ["-shared", "-o", tmp] + objs
        if verbose:
            print(" ".join(cmd))
        subprocess.check_call(cmd)
        os.replace(tmp, LIB)
    finally:
        for cmd, p in procs:
            if p.poll() is None:
                p.kill()
                p.wait()
        for obj in objs:
            if os.path.exists(obj):
                os.remove(obj)
    return LIB


if __name__ == "__main__":
    print(build(force=True, verbose=True))
