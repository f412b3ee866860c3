"""Builds libspk.so in-tree with nvcc for sm_103a (GB300).  No CPU fallback exists.

The translation units (the scan kernels and C ABI, the refiner) compile in parallel and
link into one shared library.
"""
from __future__ import annotations

import os
import subprocess
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
SRC = [os.path.join(CSRC, "spk.cu"), os.path.join(CSRC, "refiner.cu")]
DEPS = SRC + [os.path.join(CSRC, "spk_scan.cuh"), os.path.join(os.path.dirname(HERE), "include", "spk.h")]
LIB = os.path.join(HERE, "libspk.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ARCH + ["-lineinfo", "-O3", "-std=c++17", "-Xcompiler", "-fPIC"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (os.path.sep not in cand or os.path.exists(cand)):
            return cand
    return "nvcc"


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile libspk.so unless it is newer than every source."""
    if not force and os.path.exists(LIB):
        t = os.path.getmtime(LIB)
        if all(os.path.getmtime(d) <= t for d in DEPS):
            return LIB
    tag = f"{os.getpid()}"
    objs = [os.path.join(CSRC, os.path.basename(s)[:-3] + f".{tag}.o") for s in SRC]
    cmds = [[nvcc(), *NVCC_FLAGS, "-c", s, "-o", o] for s, o in zip(SRC, objs)]
    if verbose:
        for c in cmds:
            print(" ".join(c))
    with ThreadPoolExecutor(len(cmds)) as ex:
        for f in [ex.submit(subprocess.check_call, c) for c in cmds]:
            f.result()
    tmp = LIB + f".{tag}.tmp"
    subprocess.check_call([nvcc(), *ARCH, "-shared", *objs, "-o", tmp])
    for o in objs:
        os.remove(o)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force=True, verbose=True))
