"""Builds the FSZ CUDA library (libfsz.so) in-tree for sm_103a with nvcc.

Each translation unit compiles in parallel; the shared object links the CUDA runtime
statically, so it loads next to any PyTorch build.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
LIBDIR = os.path.join(PKG, "_lib")
LIB = os.path.join(LIBDIR, "libfsz.so")
SOURCES = ["fsz_stats.cu", "fsz_compress.cu", "fsz_decompress.cu", "fsz_api.cu",
           "fsz_noalloc.cu", "fsz_serve.cu", "fsz_multipass.cu", "fsz_quality.cu",
           "fsz_tiled.cu"]
HEADERS = [os.path.join(CSRC, "fsz_internal.cuh"), os.path.join(ROOT, "include", "fsz.h")]

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
# --fmad=false: no multiply-add contraction anywhere; the quantizer and the
# reconstruction are defined as separately rounded multiplies and adds.
NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++17", "--fmad=false", "-Xcompiler", "-fPIC",
              "-Xcompiler", "-Wall", "-I", os.path.join(ROOT, "include")]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the FSZ CUDA library cannot be built")


def _stale(out: str, deps) -> bool:
    if not os.path.exists(out):
        return True
    t = os.path.getmtime(out)
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose_ptxas: bool = False) -> str:
    os.makedirs(os.path.join(LIBDIR, "obj"), exist_ok=True)
    cc = nvcc()
    objs = []
    jobs = []
    for src in SOURCES:
        spath = os.path.join(CSRC, src)
        obj = os.path.join(LIBDIR, "obj", src.replace(".cu", ".o"))
        objs.append(obj)
        if force or _stale(obj, [spath, *HEADERS]):
            cmd = [cc, *ARCH, *NVCC_FLAGS, "-c", spath, "-o", obj + ".tmp"]
            if verbose_ptxas:
                cmd.insert(1, "-Xptxas=-v")
            jobs.append((cmd, obj))
    if jobs:
        with cf.ThreadPoolExecutor(max_workers=len(jobs)) as ex:
            futs = [ex.submit(subprocess.run, cmd, capture_output=True, text=True) for cmd, _ in jobs]
            for (cmd, obj), fut in zip(jobs, futs):
                res = fut.result()
                if res.returncode != 0:
                    raise RuntimeError(f"nvcc failed: {' '.join(cmd)}\n{res.stdout}\n{res.stderr}")
                if verbose_ptxas and res.stderr:
                    print(res.stderr)
                os.replace(obj + ".tmp", obj)
    if force or jobs or _stale(LIB, objs):
        tmp = LIB + f".tmp{os.getpid()}"
        subprocess.run([cc, *ARCH, "-shared", "-cudart", "static", "-o", tmp, *objs], check=True)
        os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    import sys
    print(build(force="--force" in sys.argv, verbose_ptxas="-v" in sys.argv))
