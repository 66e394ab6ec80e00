"""Build the in-tree SND library ``libsnd.so`` for sm_103a (GB300).

Each CUDA translation unit is compiled by nvcc in parallel, the host-only plan builder by
g++, and the objects are linked into one shared library with the static CUDA runtime. Host
code is compiled with -ffp-contract=off: the delay rounding and the encoder/matched-filter
decisions are FP64 expressions with a fixed operation order.
"""
from __future__ import annotations

import os
import shutil
import subprocess
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "csrc")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libsnd.so")
CU_SOURCES = ["encode.cu", "tree.cu", "tree_direct.cu", "ztree.cu", "mf.cu", "ccl.cu", "runtime.cu", "noalloc.cu", "multirate.cu",
              "sifter.cu", "batch.cu"]
CPP_SOURCES = ["plan.cpp"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _nvcc() -> str:
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", shutil.which("nvcc")):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _cuda_home(nvcc: str) -> str:
    return os.path.dirname(os.path.dirname(os.path.realpath(nvcc)))


def _run(cmd):
    r = subprocess.run(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)
    if r.returncode != 0:
        raise RuntimeError("build step failed:\n" + " ".join(cmd) + "\n" + r.stdout)
    return r.stdout


def build(verbose: bool = False, extra_nvcc=()) -> str:
    nvcc = _nvcc()
    cuda = _cuda_home(nvcc)
    os.makedirs(OUT_DIR, exist_ok=True)
    cmds = []
    objs = []
    for f in CU_SOURCES:
        obj = os.path.join(OUT_DIR, f + ".o")
        objs.append(obj)
        cmds.append([nvcc, "-c", os.path.join(SRC, f), "-o", obj, *ARCH, "-O3", "-lineinfo", "-std=c++17",
                     "-Xcompiler", "-fPIC,-ffp-contract=off", "-Xptxas", "-v" if verbose else "-O3",
                     *extra_nvcc])
    for f in CPP_SOURCES:
        obj = os.path.join(OUT_DIR, f + ".o")
        objs.append(obj)
        cmds.append(["g++", "-c", os.path.join(SRC, f), "-o", obj, "-O2", "-std=c++17", "-fPIC",
                     "-ffp-contract=off", "-I", os.path.join(cuda, "include")])
    with ThreadPoolExecutor(max_workers=len(cmds)) as ex:
        logs = list(ex.map(_run, cmds))
    if verbose:
        for log in logs:
            if log.strip():
                print(log)
    tmp = LIB + ".tmp"
    _run([nvcc, "-shared", *ARCH, "-o", tmp, *objs, "-cudart", "static", "-Xcompiler", "-fPIC"])
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    import sys
    print(build(verbose="-v" in sys.argv))
