"""Build the CUDA library liblbve.so in-tree for sm_103a (nvcc, no cmake).

Each translation unit compiles in parallel; the FP64 parity unit is built with FMA
contraction off so its expressions round exactly as written.
"""
from __future__ import annotations

import concurrent.futures as cf
import fcntl
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "liblbve.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
COMMON = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-I", CSRC, "-I", INCLUDE]
UNITS = {
    "lbve_api.cu": [],
    "lbve_f64.cu": ["--fmad=false"],
    "lbve_f32.cu": [],
    "lbve_f16.cu": [],
    "lbve_bf16.cu": [],
    "lbve_noalloc.cu": [],
    "lbve2d.cu": ["--fmad=false"],  # the 2-D step; its FP64 mode evaluates as written
}


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build liblbve.so")


def _sources_mtime() -> float:
    paths = [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [os.path.join(INCLUDE, f) for f in os.listdir(INCLUDE)]
    paths.append(__file__)
    return max(os.path.getmtime(p) for p in paths)


def _fresh() -> bool:
    return os.path.exists(LIB) and os.path.getmtime(LIB) >= _sources_mtime()


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and _fresh():
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    # one builder at a time (parallel test workers may all ask for the library)
    with open(os.path.join(BUILD, ".lock"), "w") as lk:
        fcntl.flock(lk, fcntl.LOCK_EX)
        try:
            if not force and _fresh():
                return LIB
            return _build(verbose)
        finally:
            fcntl.flock(lk, fcntl.LOCK_UN)


def _build(verbose: bool) -> str:
    cc = nvcc()

    def compile_unit(name):
        obj = os.path.join(BUILD, name.replace(".cu", ".o"))
        cmd = [cc, *ARCH, *COMMON, *UNITS[name], "-c", os.path.join(CSRC, name), "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {name}:\n{r.stderr}")
        if verbose and r.stderr:
            sys.stderr.write(r.stderr)
        return obj

    with cf.ThreadPoolExecutor(max_workers=len(UNITS)) as ex:
        objs = list(ex.map(compile_unit, UNITS))
    tmp = LIB + f".tmp{os.getpid()}"
    r = subprocess.run([cc, *ARCH, "-shared", "-o", tmp, *objs], capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stderr}")
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
