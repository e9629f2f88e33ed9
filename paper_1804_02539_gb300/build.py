"""Builds libigamg.so in-tree for sm_103a (nvcc + g++, translation units compiled in
parallel, no cmake).  Usage: python -m paper_1804_02539_gb300.build"""
from __future__ import annotations

import concurrent.futures as cf
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "libigamg.so")
ARCH = "-gencode=arch=compute_103a,code=sm_103a"

CU_SOURCES = ["kernels.cu", "igamg.cu", "noalloc.cu", "tc_gemm.cu", "batch.cu", "server.cu", "micro.cu"]
CPP_SOURCES = ["host_math.cpp", "topology.cpp"]


def _nvcc():
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (os.path.isabs(cand) and os.path.exists(cand) or not os.path.isabs(cand)):
            return cand
    return "nvcc"


def _run(cmd):
    r = subprocess.run(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)
    if r.returncode != 0:
        raise RuntimeError("build step failed: " + " ".join(cmd) + "\n" + r.stdout)
    return r.stdout


def build(verbose: bool = False) -> str:
    os.makedirs(OUT_DIR, exist_ok=True)
    nvcc = _nvcc()
    jobs = []
    objs = []
    for src in CU_SOURCES:
        obj = os.path.join(OUT_DIR, src + ".o")
        objs.append(obj)
        jobs.append([nvcc, "-std=c++17", "-O3", ARCH, "-lineinfo", "-Xcompiler", "-fPIC",
                     "-c", os.path.join(CSRC, src), "-o", obj])
    for src in CPP_SOURCES:
        obj = os.path.join(OUT_DIR, src + ".o")
        objs.append(obj)
        jobs.append(["g++", "-std=c++17", "-O3", "-fPIC", "-fopenmp", "-c", os.path.join(CSRC, src), "-o", obj])
    with cf.ThreadPoolExecutor(max_workers=len(jobs)) as ex:
        outs = list(ex.map(_run, jobs))
    if verbose:
        for o in outs:
            if o.strip():
                print(o)
    _run([nvcc, "-shared", ARCH, "-Xcompiler", "-fopenmp", "-o", LIB] + objs + ["-lcudart", "-lgomp", "-lpthread"])
    return LIB


if __name__ == "__main__":
    print(build(verbose="-v" in sys.argv))
