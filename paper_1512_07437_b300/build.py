"""Builds libqp.so in-tree for sm_103a (nvcc -gencode arch=compute_103a,code=sm_103a).

Every source is compiled to its own object in parallel (one nvcc process per
source, objects under _build/), then the objects are linked into libqp.so.

Usage: python -m paper_1512_07437_b300.build [--verbose]
"""
from __future__ import annotations

import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "csrc")
OBJ = os.path.join(HERE, "_build")
OUT = os.path.join(HERE, "libqp.so")
SOURCES = ["qp_f32_w1.cu", "qp_f32_w2.cu", "qp_kernels.cu", "qp_api.cpp", "qp_server.cpp", "qp_static.cu",
           "qp_tree.cu", "qp_budget.cu", "qp_consistency.cu", "qp_split.cpp"]
HEADERS = ["qp_internal.h", "qp_host.h", "qp_f32.cuh"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = [*ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    return "nvcc"


def needs_build() -> bool:
    if not os.path.exists(OUT):
        return True
    t = os.path.getmtime(OUT)
    deps = [os.path.join(SRC, f) for f in SOURCES + HEADERS]
    deps.append(os.path.join(os.path.dirname(HERE), "include", "qp.h"))
    return any(os.path.getmtime(d) > t for d in deps if os.path.exists(d))


def _compile(src: str, verbose: bool):
    obj = os.path.join(OBJ, os.path.splitext(src)[0] + ".o")
    cmd = [nvcc(), *FLAGS, "-c", "-o", obj]
    if verbose and src.endswith(".cu"):
        cmd += ["-Xptxas", "-v"]
    cmd.append(os.path.join(SRC, src))
    r = subprocess.run(cmd, capture_output=True, text=True)
    return obj, r


def build(verbose: bool = False, force: bool = False) -> str:
    if not force and not needs_build():
        return OUT
    os.makedirs(OBJ, exist_ok=True)
    jobs = min(len(SOURCES), os.cpu_count() or 1)
    with ThreadPoolExecutor(jobs) as ex:
        results = list(ex.map(lambda s: _compile(s, verbose), SOURCES))
    failed = False
    for (obj, r), src in zip(results, SOURCES):
        if verbose or r.returncode != 0:
            sys.stderr.write(r.stdout + r.stderr)
        if r.returncode != 0:
            sys.stderr.write(f"nvcc failed on {src}\n")
            failed = True
    if failed:
        raise RuntimeError("nvcc failed building libqp.so")
    tmp = OUT + f".tmp{os.getpid()}"
    cmd = [nvcc(), *ARCH, "-shared", "-o", tmp, *[obj for obj, _ in results], "-lcudart"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if verbose or r.returncode != 0:
        sys.stderr.write(r.stdout + r.stderr)
    if r.returncode != 0:
        raise RuntimeError("nvcc failed linking libqp.so")
    os.replace(tmp, OUT)
    return OUT


if __name__ == "__main__":
    build(verbose="--verbose" in sys.argv, force=True)
    print(OUT)
