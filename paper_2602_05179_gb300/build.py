"""In-tree build of the CUDA libraries (sm_103a only).

    libsdp.so     the operators (csrc/*.cu), C ABI in include/sdp.h
    libsdpgen.so  the seeded device input generator (workloads/gen.cu)

Each translation unit is compiled by its own nvcc process in parallel, then
linked with the static CUDA runtime.  Rebuilds only what is out of date.
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(PKG, "_build")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
              "-Xcompiler", "-ffp-contract=off", "--fmad=false", "-I", INCLUDE]
LIBS = {
    "libsdp.so": sorted(glob.glob(os.path.join(PKG, "csrc", "*.cu"))),
    "libsdpgen.so": sorted(glob.glob(os.path.join(PKG, "workloads", "*.cu"))),
}


def _nvcc() -> str:
    for c in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found")


def _deps(src: str) -> list[str]:
    d = [src] + glob.glob(os.path.join(os.path.dirname(src), "*.cuh"))
    d += glob.glob(os.path.join(INCLUDE, "*.h"))
    return d


def _stale(target: str, deps: list[str]) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(x) > t for x in deps)


def _compile(src: str, extra: list[str]) -> str:
    obj = os.path.join(BUILD, os.path.basename(src) + ".o")
    if _stale(obj, _deps(src)):
        cmd = [_nvcc(), *ARCH, *NVCC_FLAGS, *extra, "-c", src, "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
    return obj


def build(verbose: bool = False) -> dict:
    os.makedirs(BUILD, exist_ok=True)
    out = {}
    jobs = []
    with cf.ThreadPoolExecutor(max_workers=max(2, os.cpu_count() or 2)) as ex:
        for lib, srcs in LIBS.items():
            extra: list[str] = []
            jobs.append((lib, [ex.submit(_compile, s, extra) for s in srcs]))
        for lib, futs in jobs:
            objs = [f.result() for f in futs]
            target = os.path.join(PKG, lib)
            if _stale(target, objs):
                tmp = target + f".tmp{os.getpid()}"
                cmd = [_nvcc(), *ARCH, "-shared", "-o", tmp, *objs]
                r = subprocess.run(cmd, capture_output=True, text=True)
                if r.returncode != 0:
                    raise RuntimeError(f"link failed for {lib}:\n{r.stdout}\n{r.stderr}")
                os.replace(tmp, target)
            out[lib] = target
            if verbose:
                print("built", target)
    return out


if __name__ == "__main__":
    build(verbose=True)
    sys.exit(0)
