"""Builds libdist.so in-tree: CUDA sources for sm_103a with nvcc, the host
planner with the same toolchain, compiled in parallel and linked into one
shared library next to this file.  ``python -m paper_2408_10743_gb300.build``.
"""
from __future__ import annotations

import hashlib
import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libdist.so")

CU_SOURCES = ["api.cu", "batch.cu", "enum.cu", "intpeak.cu", "iso.cu", "noalloc.cu"]
CPP_SOURCES = ["plan.cpp", "stab.cpp", "iso.cpp"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
# Warnings are errors: a host-only function called from a host-device
# function, for one, is only a warning, and the device code then calls
# nothing sensible.
NVCC_FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-Xptxas", "-v", "-Werror", "all-warnings",
              "-I", CSRC, "-I", INCLUDE]
CXX_FLAGS = ["-O2", "-std=c++17", "-fPIC", "-Wall", "-I", CSRC, "-I", INCLUDE]


def _nvcc() -> str:
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (os.path.sep not in cand or os.path.exists(cand)):
            return cand
    return "nvcc"


def _digest() -> str:
    h = hashlib.sha256()
    for d in (CSRC, INCLUDE):
        for name in sorted(os.listdir(d)):
            p = os.path.join(d, name)
            if os.path.isfile(p):
                h.update(name.encode())
                with open(p, "rb") as fh:
                    h.update(fh.read())
    h.update(" ".join(ARCH + NVCC_FLAGS + CXX_FLAGS).encode())
    h.update(os.uname().machine.encode())
    return h.hexdigest()


def build(force: bool = False, verbose: bool = False) -> str:
    """Compiles (if sources changed) and returns the path of libdist.so."""
    os.makedirs(BUILD, exist_ok=True)
    stamp = os.path.join(BUILD, "stamp")
    dig = _digest()
    if not force and os.path.exists(LIB) and os.path.exists(stamp):
        with open(stamp) as fh:
            if fh.read().strip() == dig:
                return LIB
    nvcc = _nvcc()
    jobs = []
    for s in CU_SOURCES:
        obj = os.path.join(BUILD, s + ".o")
        jobs.append(([nvcc] + ARCH + NVCC_FLAGS + ["-c", os.path.join(CSRC, s), "-o", obj], obj))
    for s in CPP_SOURCES:
        obj = os.path.join(BUILD, s + ".o")
        jobs.append((["g++"] + CXX_FLAGS + ["-c", os.path.join(CSRC, s), "-o", obj], obj))

    def run(job):
        cmd, _ = job
        return subprocess.run(cmd, capture_output=True, text=True)

    with ThreadPoolExecutor(max_workers=len(jobs)) as ex:
        results = list(ex.map(run, jobs))
    log = []
    for (cmd, _), res in zip(jobs, results):
        log.append("$ " + " ".join(cmd) + "\n" + res.stdout + res.stderr)
        if res.returncode != 0:
            sys.stderr.write("\n".join(log))
            raise RuntimeError("compilation failed: " + " ".join(cmd))
    with open(os.path.join(BUILD, "compile.log"), "w") as fh:
        fh.write("\n".join(log))
    tmp = LIB + ".tmp.%d" % os.getpid()
    link = [nvcc] + ARCH + ["-shared", "-o", tmp] + [o for _, o in jobs] + ["-lcudart"]
    res = subprocess.run(link, capture_output=True, text=True)
    if res.returncode != 0:
        sys.stderr.write(res.stdout + res.stderr)
        raise RuntimeError("link failed")
    os.replace(tmp, LIB)
    with open(stamp, "w") as fh:
        fh.write(dig)
    if verbose:
        print("\n".join(log))
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
