"""Build the in-tree shared libraries with nvcc for sm_103a (no CMake, no setuptools).

``libpngf.so``       the C ABI of include/pngf.h (every CUDA kernel of the hot path)
``libpngf_peaks.so`` FP64 / FP32 FMA throughput probes used for the roofline

Translation units compile in parallel into ``_build/``; the link step puts the
libraries next to this file, where the binding loads them from.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(ROOT, "_build")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]

LIBS = {
    "libpngf.so": ["api.cu", "factor.cu", "sweep.cu", "sweep_mixed.cu", "batch.cu", "flush_tc.cu", "gradient.cu",
                   "general.cu", "pec.cu"],
    "libpngf_peaks.so": ["peaks.cu"],
}


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _flags():
    return ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I", INCLUDE, "-I", CSRC,
                   "--expt-relaxed-constexpr"]


def _compile(src: str, obj: str, extra) -> str:
    cmd = [nvcc(), "-c", src, "-o", obj] + _flags() + list(extra)
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for {os.path.basename(src)}:\n{r.stdout}\n{r.stderr}")
    return r.stderr


def _stale(target: str, deps) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def build(verbose: bool = False, force: bool = False, ptxas_info: bool = False) -> dict:
    """Compile every library; returns {name: path}."""
    os.makedirs(BUILD, exist_ok=True)
    headers = [os.path.join(CSRC, h) for h in os.listdir(CSRC) if h.endswith((".cuh", ".h"))]
    headers.append(os.path.join(INCLUDE, "pngf.h"))
    extra = ["-Xptxas", "-v"] if ptxas_info else []
    jobs = []
    for lib, srcs in LIBS.items():
        for s in srcs:
            src = os.path.join(CSRC, s)
            obj = os.path.join(BUILD, s.replace(".cu", ".o"))
            if force or _stale(obj, [src] + headers):
                jobs.append((src, obj))
    logs = {}
    if jobs:
        with cf.ThreadPoolExecutor(max_workers=min(8, len(jobs))) as ex:
            futs = {ex.submit(_compile, s, o, extra): s for s, o in jobs}
            for f in cf.as_completed(futs):
                logs[os.path.basename(futs[f])] = f.result()
    out = {}
    for lib, srcs in LIBS.items():
        objs = [os.path.join(BUILD, s.replace(".cu", ".o")) for s in srcs]
        target = os.path.join(PKG, lib)
        if force or _stale(target, objs):
            cmd = [nvcc(), "-shared", "-o", target] + objs + ARCH + ["-cudart", "shared"]
            r = subprocess.run(cmd, capture_output=True, text=True)
            if r.returncode != 0:
                raise RuntimeError(f"link failed for {lib}:\n{r.stdout}\n{r.stderr}")
        out[lib] = target
    if verbose:
        for k, v in logs.items():
            if v.strip():
                print(f"--- {k}\n{v}", file=sys.stderr)
    return out


if __name__ == "__main__":
    build(verbose=True, force="--force" in sys.argv, ptxas_info="--ptxas" in sys.argv)
    print("built:", ", ".join(LIBS))
