"""Build the CUDA library libcola_gb300.so in-tree (sm_103a), compiling sources in parallel.

Usage: python -m paper_1301_0322_gb300.build [--force]
"""
import concurrent.futures
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libcola_gb300.so")
SOURCES = ["api.cu", "coeffs.cpp", "fft_kernels.cu", "pm_kernels.cu", "ic_kernels.cu", "power_kernels.cu",
           "power_noalloc.cu", "pm_fft_kernels.cu", "adjoint_kernels.cu", "ensemble.cu",
           "fof.cu"]
HEADERS = ["cola_internal.cuh", "fft.cuh", "pm_common.cuh", "profiler.cuh", "pm_bodies.cuh", "particle_bodies.cuh",
           "tma.cuh"]
NVCC = os.environ.get("NVCC", "nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-std=c++17", "-O3", "-lineinfo", "-Xcompiler", "-fPIC"] + ARCH


def _mtime(path):
    return os.path.getmtime(path) if os.path.exists(path) else -1.0


def _compile(src):
    obj = os.path.join(BUILD, src + ".o")
    deps = [os.path.join(CSRC, src)] + [os.path.join(CSRC, h) for h in HEADERS]
    deps.append(os.path.join(HERE, "..", "include", "cola.h"))
    if _mtime(obj) >= max(_mtime(d) for d in deps):
        return obj, None
    cmd = [NVCC] + FLAGS + ["-c", os.path.join(CSRC, src), "-o", obj]
    res = subprocess.run(cmd, capture_output=True, text=True)
    if res.returncode != 0:
        return obj, " ".join(cmd) + "\n" + res.stdout + res.stderr
    return obj, None


def build(force=False, verbose=True):
    """Compile every source for sm_103a and link the shared library; returns its path."""
    os.makedirs(BUILD, exist_ok=True)
    if force:
        for f in os.listdir(BUILD):
            os.remove(os.path.join(BUILD, f))
    with concurrent.futures.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        results = list(ex.map(_compile, SOURCES))
    errors = [e for _, e in results if e]
    if errors:
        raise RuntimeError("CUDA build failed:\n" + "\n".join(errors))
    objs = [o for o, _ in results]
    if force or _mtime(LIB) < max(_mtime(o) for o in objs):
        cmd = [NVCC] + ARCH + ["-shared", "-o", LIB] + objs
        res = subprocess.run(cmd, capture_output=True, text=True)
        if res.returncode != 0:
            raise RuntimeError("link failed:\n" + " ".join(cmd) + "\n" + res.stdout + res.stderr)
    if verbose:
        print("built", LIB)
    return LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv)
