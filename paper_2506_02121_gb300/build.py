"""Build libccgpu.so (the CUDA library behind include/cc.h) in-tree for sm_103a.

Each translation unit is compiled by nvcc in parallel, then linked into
``paper_2506_02121_gb300/libccgpu.so`` against the shared CUDA runtime (the one PyTorch
also loads), so that streams and device pointers pass freely between the two.
"""
from __future__ import annotations

import concurrent.futures
import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(PKG, "csrc")
ROOT = os.path.dirname(PKG)
LIB = os.path.join(PKG, "libccgpu.so")
# FMA-rate probes for the roofline denominators (a measurement tool, not part of the method)
PROBE_LIB = os.path.join(PKG, "libccprobe.so")
PROBE_SRC = "probe_peaks.cu"
BUILD_DIR = os.path.join(ROOT, "_build")
SOURCES = ["cc_api.cu", "aberth.cu", "polish.cu", "raster.cu", "static_scratch.cu", "batch.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr"]
# The tracer inlines its per-root code once per thread slot, and the slot a root takes in a
# sweep follows the order of shared-memory atomics; with contraction of a*b + c into FMA left
# to the compiler, the copies could round differently and a root's result would depend on
# its slot.  Its fused operations are all written out (fmaf, packed fma), so contraction is
# off there and every copy computes the same value.
EXTRA = {"aberth.cu": ["-fmad=false"]}


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found (CUDA 13 toolkit required to build libccgpu)")


def _deps_mtime() -> float:
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f != PROBE_SRC] + [
        os.path.join(ROOT, "include", "cc.h"), os.path.abspath(__file__)]
    return max(os.path.getmtime(f) for f in files if os.path.isfile(f))


def build_probe(force: bool = False) -> str:
    src = os.path.join(CSRC, PROBE_SRC)
    if not force and os.path.exists(PROBE_LIB) and os.path.getmtime(PROBE_LIB) >= os.path.getmtime(src):
        return PROBE_LIB
    tmp = PROBE_LIB + f".tmp{os.getpid()}"
    r = subprocess.run([nvcc(), *ARCH, *FLAGS, "-shared", "-cudart", "shared", src, "-o", tmp],
                       capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for {PROBE_SRC}:\n{r.stderr}")
    os.replace(tmp, PROBE_LIB)
    return PROBE_LIB


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= _deps_mtime():
        build_probe(force)
        return LIB
    os.makedirs(BUILD_DIR, exist_ok=True)
    cc = nvcc()

    def compile_one(src: str) -> str:
        obj = os.path.join(BUILD_DIR, src.replace(".cu", ".o"))
        cmd = [cc, *ARCH, *FLAGS, *EXTRA.get(src, []), "-c", os.path.join(CSRC, src), "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src}:\n{r.stderr}")
        if verbose and r.stderr:
            sys.stderr.write(r.stderr)
        return obj

    with concurrent.futures.ThreadPoolExecutor(max_workers=len(SOURCES) + 1) as ex:
        probe = ex.submit(build_probe, force)
        objs = list(ex.map(compile_one, SOURCES))
        probe.result()
    tmp = LIB + f".tmp{os.getpid()}"
    r = subprocess.run([cc, *ARCH, "-shared", "-cudart", "shared", "-o", tmp, *objs], capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stderr}")
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
