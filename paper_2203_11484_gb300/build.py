"""Compiles libvpl.so in-tree with nvcc for sm_103a (GB300).

Each translation unit compiles in parallel; the shared library links the
CUDA runtime statically and exports only the C ABI of include/vpl.h.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor
from typing import List

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
LIBDIR = os.path.join(PKG, "_lib")
LIB = os.path.join(LIBDIR, "libvpl.so")
SOURCES = ["capi.cu", "build.cu", "generate.cu", "gather.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    for c in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libvpl")


def cflags(extra: List[str] = ()) -> List[str]:
    return (ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
                    "-Xcompiler", "-ffp-contract=off", "-Xcompiler", "-fvisibility=hidden",
                    "-I", INCLUDE, "-I", CSRC] + list(extra))


def _deps_mtime() -> float:
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    files.append(os.path.join(INCLUDE, "vpl.h"))
    files.append(os.path.abspath(__file__))
    return max(os.path.getmtime(f) for f in files)


def build_library(force: bool = False, verbose: bool = False, ptxas_info: bool = False) -> str:
    """VPL_NVCC_EXTRA (environment) adds nvcc flags, e.g. -DVPL_GATHER_MIN_BLOCKS=7;
    a change of those flags forces a rebuild."""
    os.makedirs(LIBDIR, exist_ok=True)
    tuning = os.environ.get("VPL_NVCC_EXTRA", "").split()
    stamp = os.path.join(LIBDIR, "flags.txt")
    old = open(stamp).read() if os.path.exists(stamp) else ""
    if (not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= _deps_mtime()
            and old == " ".join(tuning)):
        return LIB
    cc = nvcc()
    extra = (["-Xptxas", "-v"] if ptxas_info else []) + tuning

    def compile_one(src: str):
        obj = os.path.join(LIBDIR, src.replace(".cu", ".o"))
        cmd = [cc] + cflags(extra) + ["-c", os.path.join(CSRC, src), "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{r.stdout}\n{r.stderr}")
        return obj, r.stdout + r.stderr

    with ThreadPoolExecutor(max_workers=len(SOURCES)) as pool:
        results = list(pool.map(compile_one, SOURCES))
    if verbose or ptxas_info:
        for obj, log in results:
            if log.strip():
                sys.stderr.write(f"== {os.path.basename(obj)}\n{log}\n")
    tmp = LIB + ".tmp"
    cmd = [cc] + ARCH + ["-shared", "-o", tmp] + [o for o, _ in results]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB)
    with open(stamp, "w") as f:
        f.write(" ".join(tuning))
    return LIB


if __name__ == "__main__":
    print(build_library(force="--force" in sys.argv, verbose=True,
                        ptxas_info="--ptxas" in sys.argv))
