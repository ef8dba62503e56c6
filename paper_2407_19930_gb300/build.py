"""Build librpa_gpu.so in-tree (paper_2407_19930_gb300/_build/) for sm_103a.

Every CUDA translation unit is compiled by nvcc in parallel with
``-gencode arch=compute_103a,code=sm_103a``; the host grid code by g++; the
result is linked into one shared library with the CUDA runtime linked
statically.  No cmake, no torch extension machinery.
"""
from __future__ import annotations

import concurrent.futures
import glob
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "csrc")
INC = os.path.join(os.path.dirname(HERE), "include")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "librpa_gpu.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _nvcc() -> str:
    for c in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build librpa_gpu")


def _sources():
    return sorted(glob.glob(os.path.join(SRC, "*.cu")) + glob.glob(os.path.join(SRC, "*.cpp")))


def _deps():
    return (_sources() + glob.glob(os.path.join(SRC, "*.h")) + glob.glob(os.path.join(INC, "*.h")) +
            [os.path.join(HERE, "probe", "peaks.cu")])


def up_to_date() -> bool:
    if not os.path.exists(LIB) or not os.path.exists(os.path.join(BUILD, "libpeaks.so")):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(p) <= t for p in _deps())


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and up_to_date():
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    nvcc = _nvcc()
    cuda_home = os.path.dirname(os.path.dirname(nvcc))

    def compile_one(src):
        obj = os.path.join(BUILD, os.path.basename(src) + ".o")
        if src.endswith(".cu"):
            cmd = [nvcc, *ARCH, "-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-I", INC,
                   "-c", src, "-o", obj]
        else:
            cmd = ["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-fPIC", "-I", INC, "-I", os.path.join(cuda_home, "include"),
                   "-c", src, "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("compile failed: %s\n%s%s" % (" ".join(cmd), r.stdout, r.stderr))
        if verbose and r.stderr:
            print(r.stderr)
        return obj

    with concurrent.futures.ThreadPoolExecutor(max_workers=max(2, os.cpu_count() or 2)) as ex:
        objs = list(ex.map(compile_one, _sources()))
    tmp = LIB + ".tmp%d" % os.getpid()
    cmd = [nvcc, *ARCH, "-shared", "-o", tmp, *objs]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed: %s\n%s%s" % (" ".join(cmd), r.stdout, r.stderr))
    os.replace(tmp, LIB)
    _build_probe(nvcc)
    return LIB


PROBE_SRC = os.path.join(HERE, "probe", "peaks.cu")
PROBE_LIB = os.path.join(BUILD, "libpeaks.so")


def _build_probe(nvcc: str) -> str:
    """The FP64 peak probes the benchmark measures its roofline against (a library of its own,
    outside the C ABI)."""
    cmd = [nvcc, *ARCH, "-O3", "-std=c++17", "-Xcompiler", "-fPIC", "-shared", PROBE_SRC, "-o", PROBE_LIB]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("compile failed: %s\n%s%s" % (" ".join(cmd), r.stdout, r.stderr))
    return PROBE_LIB


if __name__ == "__main__":
    print(build(force=True, verbose=True))
