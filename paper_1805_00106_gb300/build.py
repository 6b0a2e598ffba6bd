"""Build libsr.so in-tree: CUDA sources with nvcc for sm_103a only, host C++ with
g++, linked into paper_1805_00106_gb300/libsr.so (objects under _build/)."""
from __future__ import annotations

import os
import subprocess
import sys
import threading
from concurrent.futures import ThreadPoolExecutor

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(PKG, "libsr.so")
CUDA = os.environ.get("CUDA_HOME", "/usr/local/cuda")
NVCC = os.path.join(CUDA, "bin", "nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
CU_SRCS = ["sr_extend.cu", "sr_extend_m0.cu", "sr_extend_m1.cu", "sr_extend_m2.cu", "sr_kernels.cu", "sr_report.cu", "sr_cal.cu",
           "sr_traceback.cu", "sr_noalloc.cu"]
CPP_SRCS = ["sr_index.cpp", "sr_session.cpp", "sr_serve.cpp", "sr_sam.cpp", "sr_pool.cpp"]
_lock = threading.Lock()


def _deps():
    out = []
    for d in (CSRC, INCLUDE):
        for f in os.listdir(d):
            if f.endswith((".cu", ".cpp", ".h", ".cuh")):
                out.append(os.path.join(d, f))
    return out


def _stale(target, deps):
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def _run(cmd):
    r = subprocess.run(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)
    if r.returncode != 0:
        raise RuntimeError("build failed: " + " ".join(cmd) + "\n" + r.stdout)
    return r.stdout


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile every CUDA and host source of libsr and link the shared library."""
    with _lock:
        deps = _deps()
        if not force and not _stale(LIB, deps):
            return LIB
        os.makedirs(BUILD, exist_ok=True)
        jobs = []
        for f in CU_SRCS:
            src, obj = os.path.join(CSRC, f), os.path.join(BUILD, f + ".o")
            jobs.append([NVCC, *ARCH, "-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC",
                         "-Xptxas", "-v" if verbose else "-O3", "-I", INCLUDE, "-c", src, "-o", obj])
        for f in CPP_SRCS:
            src, obj = os.path.join(CSRC, f), os.path.join(BUILD, f + ".o")
            jobs.append(["g++", "-O2", "-std=c++17", "-fPIC", "-Wall", "-I", INCLUDE, "-I",
                         os.path.join(CUDA, "include"), "-c", src, "-o", obj])
        with ThreadPoolExecutor(max(1, min(len(jobs), os.cpu_count() or 1))) as ex:
            logs = list(ex.map(_run, jobs))
        if verbose:
            for lg in logs:
                sys.stdout.write(lg)
        objs = [os.path.join(BUILD, f + ".o") for f in CU_SRCS + CPP_SRCS]
        tmp = LIB + f".tmp{os.getpid()}"
        _run(["g++", "-shared", "-o", tmp, *objs, "-L", os.path.join(CUDA, "lib64"), "-lcudart",
              "-lpthread", "-Wl,-rpath," + os.path.join(CUDA, "lib64")])
        os.replace(tmp, LIB)
        return LIB


if __name__ == "__main__":
    t = __import__("time").time()
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
    print(f"built in {__import__('time').time() - t:.1f}s")
