"""Build libcbct.so in-tree with nvcc for sm_103a (GB300).

Each translation unit under csrc/ is compiled in parallel to an object file,
then linked into ``paper_1001_0599_gb300/libcbct.so``. Objects live in
``paper_1001_0599_gb300/_build/`` (git-ignored). Rebuilds only what changed.
"""
from __future__ import annotations

import concurrent.futures
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libcbct.so")
# (source, object, extra nvcc flags): the transpose's template variants are
# split over six objects so they compile in parallel
SOURCES = [("api.cu", "api.o", ()), ("fp.cu", "fp.o", ())] + \
    [("bp.cu", f"bp{u}.o", (f"-DBP_MODE_UNIT={u}",)) for u in range(6)] + \
    [("bps.cu", f"bps{u}.o", (f"-DBS_UNIT={u}",)) for u in range(3)] + \
    [("tv.cu", "tv.o", ()), ("misc.cu", "misc.o", ()), ("noalloc.cu", "noalloc.o", ()), ("eq6.cu", "eq6.o", ()),
     ("gather.cu", "gather.o", ()), ("serve.cu", "serve.o", ())]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    exe = shutil.which("nvcc")
    if exe:
        return exe
    cand = "/usr/local/cuda/bin/nvcc"
    if os.path.exists(cand):
        return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libcbct")


def _flags(extra=()):
    return ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I", INCLUDE,
                   "--expt-relaxed-constexpr", *extra]


def _deps():
    hdrs = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cuh", ".h"))]
    hdrs.append(os.path.join(INCLUDE, "cbct.h"))
    return max(os.path.getmtime(h) for h in hdrs)


def _compile(unit, verbose: bool, extra) -> str:
    src, objname, defs = unit
    obj = os.path.join(BUILD, objname)
    path = os.path.join(CSRC, src)
    if os.path.exists(obj) and os.path.getmtime(obj) >= max(os.path.getmtime(path), _deps()):
        return obj
    tmp = obj + f".tmp{os.getpid()}"   # concurrent builds (one per rank) never share a temporary
    cmd = [nvcc(), *_flags(tuple(extra) + tuple(defs)), "-c", path, "-o", tmp]
    if verbose:
        cmd.insert(1, "-Xptxas=-v")
    res = subprocess.run(cmd, capture_output=True, text=True)
    if res.returncode != 0:
        raise RuntimeError(f"nvcc failed on {src}:\n{res.stdout}\n{res.stderr}")
    if verbose and res.stderr:
        sys.stderr.write(res.stderr)
    os.replace(tmp, obj)
    return obj


def build(force: bool = False, verbose: bool = False, extra=()) -> str:
    os.makedirs(BUILD, exist_ok=True)
    if force:
        for f in os.listdir(BUILD):
            os.remove(os.path.join(BUILD, f))
    with concurrent.futures.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(lambda s: _compile(s, verbose, extra), SOURCES))
    if os.path.exists(LIB) and os.path.getmtime(LIB) >= max(os.path.getmtime(o) for o in objs):
        return LIB
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = [nvcc(), *ARCH, "-shared", "-o", tmp, *objs, "-Xcompiler", "-fPIC", "-lpthread"]
    res = subprocess.run(cmd, capture_output=True, text=True)
    if res.returncode != 0:
        raise RuntimeError(f"link failed:\n{res.stdout}\n{res.stderr}")
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
