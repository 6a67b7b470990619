"""Builds the CUDA library ``libgcmgpu.so`` in-tree with nvcc for sm_103a.

Only the C-ABI symbols (``gcm_*`` / ``gfc_*``) are exported; the statically
linked CUDA runtime stays private to the library so that it never binds to
another runtime loaded in the same process.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
LIB = os.path.join(PKG, "libgcmgpu.so")
PROBE_LIB = os.path.join(PKG, "libgcmprobe.so")  # microbenchmarks (probe_rates.cu), not the product
BUILD_DIR = os.path.join(PKG, "_build")

SOURCES = ["gcm_kernels.cu", "gcm_api.cu", "gcm_noalloc.cu", "gfc_fits.cu", "gcm_stream.cu", "gcm_batch.cu", "gcm_server.cu"]
PROBE_SOURCE = "probe_rates.cu"
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _nvcc() -> str:
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", shutil.which("nvcc")):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libgcmgpu.so")


def _inputs():
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f != PROBE_SOURCE]
    files += [os.path.join(INCLUDE, f) for f in os.listdir(INCLUDE)]
    files += [os.path.join(PKG, "exports.map"), os.path.abspath(__file__)]
    return files


def up_to_date() -> bool:
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(f) <= t for f in _inputs())


def build_probes(force: bool = False, verbose: bool = False) -> str:
    """libgcmprobe.so: the rate microbenchmarks (one translation unit)."""
    src = os.path.join(CSRC, PROBE_SOURCE)
    if not force and os.path.exists(PROBE_LIB) and os.path.getmtime(PROBE_LIB) >= max(
            os.path.getmtime(src), os.path.getmtime(os.path.abspath(__file__))):
        return PROBE_LIB
    tmp = PROBE_LIB + ".tmp.%d" % os.getpid()
    cmd = [_nvcc(), "-shared"] + ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-o", tmp, src,
                                         "-cudart", "static"]
    if verbose:
        print(" ".join(cmd), file=sys.stderr)
    subprocess.check_call(cmd)
    os.replace(tmp, PROBE_LIB)
    return PROBE_LIB


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and up_to_date():
        return LIB
    nvcc = _nvcc()
    os.makedirs(BUILD_DIR, exist_ok=True)
    common = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I", INCLUDE, "-I", CSRC]
    extra = os.environ.get("GCMGPU_NVCC_FLAGS", "").split()

    def compile_one(src: str) -> str:
        obj = os.path.join(BUILD_DIR, src.replace(".cu", ".o"))
        cmd = [nvcc, "-c", os.path.join(CSRC, src), "-o", obj] + common + extra
        if verbose:
            print(" ".join(cmd), file=sys.stderr)
        subprocess.check_call(cmd)
        return obj

    with ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(compile_one, SOURCES))
    tmp = LIB + ".tmp.%d" % os.getpid()
    cmd = [nvcc, "-shared"] + ARCH + ["-o", tmp] + objs + [
        "-Xlinker", "--version-script=" + os.path.join(PKG, "exports.map"), "-cudart", "static"]
    if verbose:
        print(" ".join(cmd), file=sys.stderr)
    subprocess.check_call(cmd)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
    print(build_probes(force="--force" in sys.argv, verbose=True))
