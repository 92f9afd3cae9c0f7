"""Build libmp.so (CUDA, sm_103a) in-tree with nvcc.

Translation units, compiled in parallel:
  mp_api.cu    host side of the C ABI
  mp_fp64.cu   field records, release, FP64 tracking (-fmad=false: no FMA
               contraction, so FP64 results round exactly as written)
  mp_usg.cu    FP64 tracking on rectangular unstructured grids (-fmad=false)
  mp_mixed.cu  mixed-precision tracking (contraction allowed)
  mp_mixed_f64t.cu  the same with FP64 travel time and near-zero branch
  mp_noalloc.cu  the entry point that allocates no device memory
"""
from __future__ import annotations

import os
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(PKG, "libmp.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]

UNITS = {
    "mp_api.cu": [],
    "mp_fp64.cu": ["-fmad=false"],
    "mp_usg.cu": ["-fmad=false"],
    "mp_mixed.cu": [],
    "mp_mixed_f64t.cu": [],
    "mp_noalloc.cu": [],
}


def _nvcc() -> str:
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if c and (os.path.sep not in c or os.path.exists(c)):
            return c
    return "nvcc"


def _deps():
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [os.path.join(INCLUDE, "mp.h"), __file__]
    return max(os.path.getmtime(f) for f in files)


def build_lib(force: bool = False, verbose: bool = False) -> str:
    """Compile every CUDA unit for sm_103a and link libmp.so; returns its path."""
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= _deps():
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    nvcc = _nvcc()
    procs = []
    objs = []
    for src, extra in UNITS.items():
        obj = os.path.join(BUILD, src.replace(".cu", ".o"))
        objs.append(obj)
        cmd = [nvcc, "-O3", "-std=c++17", *ARCH, "-lineinfo", "-Xcompiler", "-fPIC", "-Xptxas", "-v",
               "-I", INCLUDE, "-I", CSRC, *extra, "-c", os.path.join(CSRC, src), "-o", obj]
        log = open(obj + ".log", "w")
        procs.append((src, subprocess.Popen(cmd, stdout=log, stderr=subprocess.STDOUT), log, obj + ".log"))
    failed = []
    for src, p, log, logpath in procs:
        rc = p.wait()
        log.close()
        if rc != 0:
            failed.append((src, open(logpath).read()))
    if failed:
        msg = "\n".join(f"--- {s}\n{t}" for s, t in failed)
        raise RuntimeError(f"nvcc failed:\n{msg}")
    tmp = LIB + f".tmp{os.getpid()}"
    subprocess.check_call([nvcc, "-shared", *ARCH, "-cudart", "shared", "-o", tmp, *objs,
                           "-Xlinker", "-rpath,/usr/local/cuda/lib64"])
    os.replace(tmp, LIB)
    if verbose:
        for src, _, _, logpath in procs:
            sys.stdout.write(open(logpath).read())
    return LIB


if __name__ == "__main__":
    print(build_lib(force="--force" in sys.argv, verbose=True))
