"""In-tree build of libfpt.so for sm_103a (nvcc, no cmake).

Compiles the translation units in parallel and links them into
``paper_2410_13683_gb300/libfpt.so``. Rebuilds only when a source is newer
than the library (or ``force``).
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(ROOT, "_build")
LIB = os.path.join(PKG, "libfpt.so")
# debug build with the device bounds checks (-DFPT_CHECKS); loaded when the
# environment sets FPT_CHECKS=1
LIB_CHECKS = os.path.join(PKG, "libfpt_checks.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
CUDA_SOURCES = ["fpt_kernels.cu", "fpt_abi.cu", "fpt_mlp.cu"]
CXX_SOURCES = ["fpt_tables.cpp"]


def _nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libfpt.so")


def _sources():
    srcs = [os.path.join(CSRC, s) for s in CUDA_SOURCES + CXX_SOURCES]
    return [s for s in srcs if os.path.exists(s)]


def _deps():
    out = _sources()
    out += [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".h", ".cuh"))]
    out.append(os.path.join(INCLUDE, "fpt.h"))
    return out


def needs_build(checks: bool = False) -> bool:
    lib = LIB_CHECKS if checks else LIB
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    return any(os.path.getmtime(d) > t for d in _deps())


def build(force: bool = False, verbose: bool = False, checks: bool = False) -> str:
    """Build libfpt.so, or with checks=True libfpt_checks.so (device bounds
    checks compiled in, -DFPT_CHECKS); returns the library's path."""
    lib = LIB_CHECKS if checks else LIB
    if not force and not needs_build(checks):
        return lib
    nvcc = _nvcc()
    bdir = os.path.join(BUILD, "checks") if checks else BUILD
    os.makedirs(bdir, exist_ok=True)
    common = ["-O3", "-std=c++17", "-Xcompiler", "-fPIC", "-I", INCLUDE, "-I", CSRC]
    if checks:
        common.append("-DFPT_CHECKS")
    procs, objs = [], []
    for src in _sources():
        obj = os.path.join(bdir, os.path.basename(src) + ".o")
        if src.endswith(".cu"):
            cmd = [nvcc] + ARCH + ["-lineinfo"] + common + ["-c", src, "-o", obj]
        else:
            cmd = [nvcc, "-x", "c++"] + common + ["-c", src, "-o", obj]
        if verbose:
            print(" ".join(cmd), file=sys.stderr)
        procs.append((src, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
        objs.append(obj)
    failed = []
    for src, p in procs:
        out, _ = p.communicate()
        if p.returncode != 0:
            failed.append((src, out.decode(errors="replace")))
        elif verbose and out:
            print(out.decode(errors="replace"), file=sys.stderr)
    if failed:
        raise RuntimeError("libfpt build failed:\n" + "\n".join(f"{s}:\n{o}" for s, o in failed))
    tmp = lib + f".tmp{os.getpid()}"
    cmd = [nvcc] + ARCH + ["-shared", "-o", tmp] + objs + ["-lcudart"]
    r = subprocess.run(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)
    if r.returncode != 0:
        raise RuntimeError("libfpt link failed:\n" + r.stdout.decode(errors="replace"))
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv, checks="--checks" in sys.argv))
