"""Build the CUDA library ``_build/libpf.so`` in-tree with nvcc for sm_103a.

The translation units are compiled in parallel and linked into one shared
library that exports the C ABI of ``include/pf.h``.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libpf.so")
SOURCES = ("pf_step.cu", "pf_step_staged.cu", "pf_step_bc.cu", "pf_step3d.cu", "pf_step3f.cu", "pf_step3f_bc.cu",
           "pf_step3f_wide.cu", "pf_adjoint.cu",
           "pf_kernels.cu", "pf_capi.cu", "pf_noalloc.cu")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _nvcc() -> str:
    exe = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(exe):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libpf.so")
    return exe


def _inputs():
    deps = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    deps.append(os.path.join(ROOT, "include", "pf.h"))
    return deps


def build(force: bool = False, verbose: bool = False) -> str:
    os.makedirs(BUILD, exist_ok=True)
    if not force and os.path.exists(LIB):
        newest = max(os.path.getmtime(p) for p in _inputs())
        if os.path.getmtime(LIB) >= newest:
            return LIB
    nvcc = _nvcc()
    flags = ["-std=c++17", "-O3", "-lineinfo", *ARCH, "-Xcompiler", "-fPIC",
             f"-I{os.path.join(ROOT, 'include')}"]
    if verbose:
        flags += ["-Xptxas", "-v"]

    def compile_one(src):
        obj = os.path.join(BUILD, src.replace(".cu", f".{os.getpid()}.o"))
        subprocess.run([nvcc, *flags, "-c", os.path.join(CSRC, src), "-o", obj], check=True)
        return obj

    with cf.ThreadPoolExecutor(len(SOURCES)) as ex:
        objs = list(ex.map(compile_one, SOURCES))
    tmp = LIB + f".tmp{os.getpid()}"
    subprocess.run([nvcc, "-shared", *ARCH, "-o", tmp, *objs, "-lcudart"], check=True)
    os.replace(tmp, LIB)
    for o in objs:
        os.remove(o)
    return LIB


if __name__ == "__main__":
    print(build(force=True, verbose=True))
