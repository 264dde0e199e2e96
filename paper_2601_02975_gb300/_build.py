"""Build the CUDA library libccmg.so in-tree for sm_103a.

Host translation units are compiled with g++ and the device one with nvcc,
in parallel, then linked with nvcc into paper_2601_02975_gb300/libccmg.so.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libccmg.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _nvcc() -> str:
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", shutil.which("nvcc")):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _run(cmd):
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("build step failed:\n" + " ".join(cmd) + "\n" + r.stdout + r.stderr)
    return r.stdout + r.stderr


def sources():
    return sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC)
                  if f.endswith((".cpp", ".cu", ".cuh", ".h")))


def build(verbose: bool = False, force: bool = False) -> str:
    """Compile libccmg.so if any source is newer than it; return its path."""
    srcs = sources()
    if (not force and os.path.exists(LIB)
            and os.path.getmtime(LIB) >= max(os.path.getmtime(s) for s in srcs)
            and os.path.getmtime(LIB) >= os.path.getmtime(os.path.join(HERE, "..", "include", "ccmg.h"))):
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    nvcc = _nvcc()
    inc = ["-I", os.path.join(HERE, "..", "include"), "-I", CSRC]
    jobs = []
    objs = []
    for name in ("geom.cpp", "disc.cpp"):
        obj = os.path.join(BUILD, name + ".o")
        objs.append(obj)
        # no contraction of a * b + c into one rounding: the host setup then
        # gives the same bits on x86-64 and on aarch64 (where gcc fuses by default)
        jobs.append(["g++", "-std=c++17", "-O2", "-fPIC", "-ffp-contract=off", "-Wall",
                     "-Wno-unused-variable", "-c", os.path.join(CSRC, name), "-o", obj] + inc)
    obj = os.path.join(BUILD, "capi.cu.o")
    objs.append(obj)
    jobs.append([nvcc, "-std=c++17", "-O3", "-lineinfo", *ARCH, "-Xcompiler", "-fPIC",
                 "-Xcompiler", "-ffp-contract=off",
                 "-Xptxas", "-v" if verbose else "-O3",
                 "-c", os.path.join(CSRC, "capi.cu"), "-o", obj] + inc)
    # the device setup steps: no fused multiply-adds, so they round like the host
    obj = os.path.join(BUILD, "setup_dev.cu.o")
    objs.append(obj)
    jobs.append([nvcc, "-std=c++17", "-O3", "-lineinfo", *ARCH, "-Xcompiler", "-fPIC",
                 "-Xcompiler", "-ffp-contract=off", "--fmad=false",
                 "-Xptxas", "-v" if verbose else "-O3",
                 "-c", os.path.join(CSRC, "setup_dev.cu"), "-o", obj] + inc)
    with ThreadPoolExecutor(max_workers=len(jobs)) as ex:
        outs = list(ex.map(_run, jobs))
    if verbose:
        for o in outs:
            sys.stdout.write(o)
    tmp = LIB + ".tmp"
    _run([nvcc, "-shared", *ARCH, "-cudart", "static", "-o", tmp] + objs + ["-lpthread"])
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(verbose="-v" in sys.argv, force="-f" in sys.argv))
