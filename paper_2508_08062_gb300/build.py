"""Compile the CUDA library (sm_103a) in-tree: ``libaapdhg.so`` next to this file."""
from __future__ import annotations

import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
SRC_DIR = os.path.join(HERE, "csrc")
LIB = os.path.join(HERE, "libaapdhg.so")
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _sources():
    out = []
    for f in sorted(os.listdir(SRC_DIR)):
        if f.endswith((".cu", ".cuh", ".h")):
            out.append(os.path.join(SRC_DIR, f))
    out.append(os.path.join(ROOT, "include", "aapdhg.h"))
    return out


def stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    return any(os.path.getmtime(s) > t for s in _sources())


UNITS = ("aapdhg.cu", "batch.cu", "serve.cu", "kkt_noalloc.cu")


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile each translation unit in parallel (one nvcc per unit), then link."""
    if not force and not stale():
        return LIB
    obj_dir = os.path.join(HERE, "_build")
    os.makedirs(obj_dir, exist_ok=True)
    flags = ["-O3", "-std=c++17", *ARCH, "-lineinfo", "-Xcompiler", "-fPIC"]
    if verbose:
        flags.insert(0, "-Xptxas=-v")
    procs, objs = [], []
    for u in UNITS:
        obj = os.path.join(obj_dir, u.replace(".cu", f".{os.getpid()}.o"))
        objs.append(obj)
        procs.append((u, subprocess.Popen([NVCC, *flags, "-c", "-o", obj, os.path.join(SRC_DIR, u)])))
    failed = [u for u, p in procs if p.wait() != 0]
    if failed:
        raise RuntimeError(f"nvcc failed on {failed}")
    tmp = LIB + f".{os.getpid()}.tmp"
    subprocess.check_call([NVCC, *ARCH, "-shared", "-o", tmp, *objs])
    for o in objs:
        os.remove(o)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force=True, verbose=True))
