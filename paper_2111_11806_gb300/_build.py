"""Build libdfvrb.so (the C-ABI CUDA library) in-tree with nvcc for sm_103a.

The translation units (one per precision and dimension, plus the C ABI) are
compiled in parallel, then linked into paper_2111_11806_gb300/libdfvrb.so.
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
ROOT = os.path.dirname(HERE)
INCLUDE = os.path.join(ROOT, "include")
OBJDIR = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libdfvrb.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-std=c++17", "-O3", "-lineinfo", "-Xcompiler", "-fPIC", "-I" + INCLUDE]


def nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libdfvrb.so")


# dfv_inst_tu.cu holds one launcher table; it is compiled once per
# (precision, dimension, number of materials).
TU = os.path.join(CSRC, "dfv_inst_tu.cu")
TU_COMBOS = [(prec, dim, nmat) for prec in ("f32", "f64") for dim in (1, 2, 3) for nmat in (1, 2, 3)]


def sources():
    """(source, object name, extra defines, FP32 flags?) of every translation unit."""
    out = []
    for src in sorted(glob.glob(os.path.join(CSRC, "*.cu"))):
        if src == TU:
            continue
        base = os.path.basename(src).replace(".cu", "")
        out.append((src, base, [], "_f32_" in base))
    for prec, dim, nmat in TU_COMBOS:
        name = "ops_%s_d%d_n%d" % (prec, dim, nmat)
        defs = ["-DDFV_TU_REAL=%s" % ("float" if prec == "f32" else "double"), "-DDFV_TU_DIM=%d" % dim,
                "-DDFV_TU_NMAT=%d" % nmat, "-DDFV_TU_NAME=" + name]
        out.append((TU, "dfv_inst_" + name, defs, prec == "f32"))
    return out


def headers():
    return sorted(glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(CSRC, "*.h"))
                  + glob.glob(os.path.join(INCLUDE, "*.h")))


def _stale(target, deps):
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


# The FP32 translation units use the fast single-precision divide and square
# root and flush single-precision denormals to zero (double precision is
# unaffected): the approximate reciprocal and square root are then one
# instruction each, with no range fix-up.  The states' magnitudes and their
# non-zero differences stay many decades above the denormal range (1.2e-38);
# the FP32 form's accuracy target is a relative L1 of 1e-4 against the FP64
# solution.
FP32_FLAGS = ["-prec-div=false", "-prec-sqrt=false", "-ftz=true"]


def _compile(unit, extra):
    src, name, defs, fp32 = unit
    obj = os.path.join(OBJDIR, name + ".o")
    if _stale(obj, [src] + headers() + [os.path.abspath(__file__)]):
        flags = FP32_FLAGS if fp32 else []
        cmd = [nvcc()] + ARCH + FLAGS + flags + defs + list(extra) + ["-c", src, "-o", obj + ".tmp"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed on %s:\n%s\n%s" % (src, r.stdout, r.stderr))
        os.replace(obj + ".tmp", obj)
    return obj


def build(force: bool = False, extra=(), jobs: int = 0) -> str:
    """Compile and link; returns the library path.  Rebuilds only what is
    older than its sources or headers unless `force`."""
    os.makedirs(OBJDIR, exist_ok=True)
    srcs = sources()
    if force:
        for o in glob.glob(os.path.join(OBJDIR, "*.o")):
            os.remove(o)
    jobs = jobs or min(len(srcs), max(1, os.cpu_count() or 1))
    # the kernel tables first: they are the longest compilations
    srcs = sorted(srcs, key=lambda u: 0 if u[0] == TU else 1)
    with cf.ThreadPoolExecutor(max_workers=jobs) as ex:
        objs = list(ex.map(lambda s: _compile(s, extra), srcs))
    if force or _stale(LIB, objs):
        tmp = LIB + ".%d.tmp" % os.getpid()
        cmd = [nvcc()] + ARCH + ["-shared", "-o", tmp] + objs + ["-lcudart"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("link failed:\n%s\n%s" % (r.stdout, r.stderr))
        os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build())
