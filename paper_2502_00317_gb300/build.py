"""Builds libkc.so in-tree (paper_2502_00317_gb300/_build/) with nvcc for sm_103a.

The translation units compile in parallel, then link into one shared library
with the C ABI of include/kclique.h.  No cmake, one -gencode.
"""
from __future__ import annotations

import concurrent.futures as cf
import hashlib
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libkc.so")
SOURCES = ["kc_api.cu", "kc_prep.cu", "kc_enum.cu", "kc_serve.cu", "kc_tune.cu", "kc_enum_w1.cu", "kc_enum_w2.cu", "kc_enum_w4.cu",
           "kc_enum_w8.cu", "kc_enum_w16.cu", "kc_enum_w32.cu"]
PEAK_SOURCE = "kc_peak.cu"  # separate library: the benchmark's integer-pipe peak
PEAK_LIB = os.path.join(BUILD, "libkc_peak.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
# Register caps of the enumerator units.  The kernels of widths 1 and 2 are
# bounded to 64 registers, width 4 to about 85, wider ones to 128
# (kc_block_threads / kc_min_blocks); the searches of a width are also called
# out of line by the kernels of wider roots (their narrow subproblems), so
# each unit is capped at the smallest bound among its callers.
MAXRREG = {"kc_enum_w1.cu": 64, "kc_enum_w2.cu": 64, "kc_enum_w4.cu": 128, "kc_enum_w8.cu": 128,
           "kc_enum_w16.cu": 128, "kc_enum_w32.cu": 128}


def nvcc() -> str:
    for c in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found")


def _flags(extra=()):
    return [*ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I", INCLUDE, "-I", CSRC, *extra]


def _digest() -> str:
    h = hashlib.sha256()
    for name in sorted(set(os.listdir(CSRC)) - {PEAK_SOURCE}) + [os.path.join("..", "..", "include", "kclique.h")]:
        p = os.path.normpath(os.path.join(CSRC, name))
        if os.path.isfile(p):
            h.update(name.encode())
            h.update(open(p, "rb").read())
    h.update(" ".join(_flags() + ["-rdc=true"] + [f"{k}:{v}" for k, v in sorted(MAXRREG.items())]).encode())
    return h.hexdigest()


def build_peak(force: bool = False) -> str:
    """Compile libkc_peak.so (the integer-pipe peak microbenchmark) and return its path."""
    os.makedirs(BUILD, exist_ok=True)
    src = os.path.join(CSRC, PEAK_SOURCE)
    if force or not os.path.exists(PEAK_LIB) or os.path.getmtime(PEAK_LIB) < os.path.getmtime(src):
        tmp = PEAK_LIB + f".tmp{os.getpid()}"
        cmd = [nvcc(), *_flags(), "-shared", src, "-o", tmp, "-lcudart"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {PEAK_SOURCE}:\n{r.stdout}\n{r.stderr}")
        os.replace(tmp, PEAK_LIB)
    return PEAK_LIB


def build(force: bool = False, verbose: bool = False, extra_flags=()) -> str:
    """Compile (if sources changed) and return the path of libkc.so."""
    os.makedirs(BUILD, exist_ok=True)
    stamp = os.path.join(BUILD, "libkc.stamp")
    dig = _digest()
    if not force and os.path.exists(LIB) and os.path.exists(stamp) and open(stamp).read() == dig:
        return LIB
    cc = nvcc()

    def compile_one(src):
        obj = os.path.join(BUILD, src.replace(".cu", ".o"))
        # relocatable device code: each width's searches are compiled once, in
        # its own unit, and called from the kernels of every other width
        cap = [f"-maxrregcount={MAXRREG[src]}"] if src in MAXRREG else []
        cmd = [cc, *_flags(extra_flags), "-rdc=true", *cap, "-c", os.path.join(CSRC, src), "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
        if verbose and (r.stdout or r.stderr):
            print(r.stdout, r.stderr)
        return obj

    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(compile_one, SOURCES))
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = [cc, *ARCH, "-shared", "-rdc=true", "-o", tmp, *objs, "-lcudart"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB)
    with open(stamp, "w") as f:
        f.write(dig)
    return LIB


if __name__ == "__main__":
    import sys

    print(build(force="--force" in sys.argv, verbose=True,
                extra_flags=["-Xptxas", "-v"] if "--ptxas" in sys.argv else ()))
