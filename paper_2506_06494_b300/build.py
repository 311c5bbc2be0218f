"""Builds libjgs2.so in-tree for sm_103a with nvcc (no JIT cache; the .so ships with the tree).

    python -m paper_2506_06494_b300.build
"""
from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "libjgs2.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
SOURCES = ["jgs2_host.cu", "jgs2_precompute.cpp", "jgs2_static.cu", "jgs2_peaks.cu", "jgs2_gpu_solve.cu", "jgs2_cloth.cu"]


def sources():
    return [os.path.join(CSRC, s) for s in SOURCES]


def build(force: bool = False, verbose: bool = False) -> str:
    deps = sources() + [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".h", ".cuh"))]
    deps.append(os.path.join(HERE, "..", "include", "jgs2.h"))
    if not force and os.path.exists(OUT) and all(os.path.getmtime(OUT) >= os.path.getmtime(d) for d in deps):
        return OUT
    nvcc = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
    objs = []
    build_dir = os.path.join(HERE, "_build")
    os.makedirs(build_dir, exist_ok=True)
    for src in sources():
        obj = os.path.join(build_dir, os.path.basename(src) + ".o")
        if src.endswith(".cu"):
            cmd = [nvcc, *ARCH, "-lineinfo", "-O3", "-std=c++17", "-Xcompiler", "-fPIC,-fopenmp",
                   "-c", src, "-o", obj]
        else:
            cmd = ["g++", "-O3", "-march=x86-64-v4", "-std=c++17", "-fPIC", "-fopenmp",
                   "-I/usr/local/cuda/include", "-c", src, "-o", obj]
        if verbose:
            print(" ".join(cmd), file=sys.stderr)
        subprocess.run(cmd, check=True)
        objs.append(obj)
    tmp = OUT + ".tmp"
    cmd = [nvcc, *ARCH, "-shared", "-Xcompiler", "-fPIC", "-o", tmp, *objs, "-lgomp", "-lcudart"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, OUT)
    return OUT


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
