"""Builds the CUDA library libadc_gb300.so in-tree for sm_103a (GB300).

Each translation unit under ``csrc/`` is compiled by nvcc in parallel and the
objects are linked into ``paper_2511_21640_gb300/libadc_gb300.so``. Objects go
to ``_build/`` (git-ignored). No CMake; the CUDA runtime is linked statically
and the driver's tensor-map encoder is fetched at run time, so the library
needs no -lcuda at link time.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(os.path.dirname(HERE), "_build")
LIB = os.path.join(HERE, "libadc_gb300.so")
SOURCES = ["tensor.cu", "setup.cu", "sigma.cu", "sigma_tc.cu", "tc_gemm.cu", "eig.cu",
           "davidson.cu", "fns.cu", "api.cu", "diag.cu", "noalloc.cu", "blockops.cu", "terms.cu", "ee.cu",
           "batch.cu", "adjoint.cu", "ee_struct.cu", "tc_slice.cu", "ssfns.cu", "properties.cu", "cholesky.cu", "ladder.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-std=c++17", "-O3", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2"]


def nvcc():
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _compile(src):
    obj = os.path.join(BUILD, os.path.splitext(src)[0] + ".o")
    cmd = [nvcc(), *ARCH, *FLAGS, "-c", os.path.join(CSRC, src), "-o", obj]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
    return obj


def build(force=False, verbose=False):
    os.makedirs(BUILD, exist_ok=True)
    srcs = [os.path.join(CSRC, s) for s in SOURCES]
    headers = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith(".cuh")]
    headers += [os.path.join(os.path.dirname(HERE), "include", f)
                for f in os.listdir(os.path.join(os.path.dirname(HERE), "include"))]
    if not force and os.path.exists(LIB):
        t = os.path.getmtime(LIB)
        if all(os.path.getmtime(p) < t for p in srcs + headers + [__file__]):
            return LIB
    with cf.ThreadPoolExecutor(max_workers=min(len(SOURCES), os.cpu_count() or 4)) as ex:
        objs = list(ex.map(_compile, SOURCES))
    tmp = LIB + ".tmp"
    cmd = [nvcc(), *ARCH, "-shared", "-o", tmp, *objs, "-lpthread"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB)
    if verbose:
        print("built", LIB, file=sys.stderr)
    return LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose=True)
