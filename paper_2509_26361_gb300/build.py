"""Build libebit.so in-tree with nvcc for sm_103a (GB300).

The library is built from three CUDA translation units (the context-based ABI,
the allocation-free sweep and the batched persistent sweep), compiled in
parallel with --fmad=false so that every
floating-point operation of the EBIT kernels rounds separately in the written
order.  Output: ``paper_2509_26361_gb300/_build/libebit.so``.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "libebit.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _nvcc() -> str:
    cand = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(cand):
        raise RuntimeError("nvcc not found: the EBIT CUDA library cannot be built")
    return cand


def sources():
    out = []
    for d in (CSRC, os.path.join(ROOT, "include")):
        for f in sorted(os.listdir(d)):
            if f.endswith((".cu", ".cuh", ".h")):
                out.append(os.path.join(d, f))
    return out


def up_to_date() -> bool:
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(s) <= t for s in sources())


UNITS = ("ebit_abi.cu", "ebit_noalloc.cu", "ebit_batch.cu")


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile the translation units in parallel (one nvcc each), then link."""
    if not force and up_to_date():
        return LIB
    os.makedirs(OUT_DIR, exist_ok=True)
    tag = f".tmp{os.getpid()}"
    flags = ["-O3", "-std=c++17", *ARCH, "-lineinfo", "--fmad=false", "-Xcompiler", "-fPIC",
             "-I", os.path.join(ROOT, "include")]
    if verbose:
        flags.insert(0, "-Xptxas=-v")
    objs, procs = [], []
    for u in UNITS:
        obj = os.path.join(OUT_DIR, u.replace(".cu", tag + ".o"))
        objs.append(obj)
        procs.append(subprocess.Popen([_nvcc(), *flags, "-c", "-o", obj, os.path.join(CSRC, u)],
                                      stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True))
    failed = False
    for pr in procs:
        out, err = pr.communicate()
        if pr.returncode != 0:
            failed = True
            sys.stderr.write(out + err)
        elif verbose:
            sys.stderr.write(err)
    tmp = LIB + tag
    if not failed:
        r = subprocess.run([_nvcc(), *ARCH, "-shared", "-o", tmp, *objs], capture_output=True, text=True)
        if r.returncode != 0:
            failed = True
            sys.stderr.write(r.stdout + r.stderr)
    for obj in objs:
        if os.path.exists(obj):
            os.remove(obj)
    if failed:
        raise RuntimeError("nvcc failed building libebit.so")
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose="-v" in sys.argv)
    print(LIB)
