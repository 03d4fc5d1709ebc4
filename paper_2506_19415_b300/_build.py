"""Builds libvm3dgs.so in-tree: nvcc for the sm_103a kernels, g++ (OpenMP) for
the host page builder, linked against the shared CUDA runtime."""
from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "libvm3dgs.so")
BUILD = os.path.join(HERE, "_build")
CUDA = os.environ.get("CUDA_HOME", "/usr/local/cuda")
NVCC = os.path.join(CUDA, "bin", "nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]

# kernels whose discrete results are fp32 formulas evaluated exactly as written
EXACT = {"k_project.cu", "k_feedback.cu", "k_residency.cu", "k_prefetch.cu", "k_mesh.cu"}
CU = ["k_project.cu", "k_feedback.cu", "k_residency.cu", "k_stream.cu", "k_sort.cu", "k_blend.cu", "renderer.cu",
      "k_mlp.cu", "prefetcher.cu", "k_prefetch.cu",
      "sort_noalloc.cu", "batch.cu", "k_mesh.cu"]
CPP = ["build_pages.cpp", "scene.cpp", "mesh_proxy.cpp", "vq.cpp"]
HEADERS = ["renderer.cuh", "scene.h", "mlp.cuh", "prefetcher.cuh", "block_sel.cuh", "tma.cuh", "coverage.cuh", "mesh.h"]


def _newer(src_list, target):
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(s) > t for s in src_list)


def _run(cmd):
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        sys.stderr.write(" ".join(cmd) + "\n" + r.stdout + r.stderr)
        raise RuntimeError("compile failed: " + os.path.basename(cmd[-1]))
    return r.stdout + r.stderr


def build(force: bool = False, verbose: bool = False) -> str:
    os.makedirs(BUILD, exist_ok=True)
    hdrs = [os.path.join(CSRC, h) for h in HEADERS] + [os.path.join(HERE, "..", "include", "vm3dgs.h")]
    objs = []
    for f in CU:
        src = os.path.join(CSRC, f)
        obj = os.path.join(BUILD, f + ".o")
        objs.append(obj)
        if force or _newer([src] + hdrs + [__file__], obj):
            flags = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-fopenmp", "--expt-relaxed-constexpr"]
            if f in EXACT:
                flags += ["-fmad=false", "-prec-div=true", "-prec-sqrt=true", "-ftz=false"]
            if verbose:
                flags += ["-Xptxas", "-v"]
            out = _run([NVCC, *ARCH, *flags, "-c", "-o", obj, src])
            if verbose:
                sys.stderr.write(out)
    for f in CPP:
        src = os.path.join(CSRC, f)
        obj = os.path.join(BUILD, f + ".o")
        objs.append(obj)
        if force or _newer([src] + hdrs + [__file__], obj):
            _run(["g++", "-O3", "-std=c++17", "-fPIC", "-fopenmp", "-ffp-contract=off", "-fno-fast-math",
                  "-I" + os.path.join(CUDA, "include"), "-c", "-o", obj, src])
    if force or _newer(objs, OUT):
        tmp = OUT + ".tmp%d" % os.getpid()
        _run([NVCC, *ARCH, "-shared", "-cudart", "shared", "-o", tmp, *objs, "-Xcompiler", "-fopenmp", "-lgomp"])
        os.replace(tmp, OUT)
    return OUT


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose="-v" in sys.argv)
    print(OUT)
