"""Build the CUDA library libdpg.so in-tree (nvcc, sm_103a only).

Usage: ``python -m paper_1711_00984_gb300.build [--force] [--debug]``.  Translation units
are compiled in parallel, then linked into ``paper_1711_00984_gb300/_build/libdpg.so``.
``--debug`` (``build(debug=True)``) builds the bounds-checked variant
``_build_debug/libdpg_debug.so`` (``-DDPG_DEBUG_BOUNDS``): every kernel checks its memory
indices against the extents it was given and reports DPG_ERR_BOUNDS through the status
word instead of making the access; load it with ``paper_1711_00984_gb300.load(path)``.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
SO = os.path.join(BUILD, "libdpg.so")
BUILD_DEBUG = os.path.join(HERE, "_build_debug")
SO_DEBUG = os.path.join(BUILD_DEBUG, "libdpg_debug.so")
SOURCES = ["dpg_setup.cu", "dpg_kernels.cu", "dpg_tc.cu", "dpg_tcc.cu", "dpg_capi.cu", "dpg_noalloc.cu",
           "dpg_condense.cu", "dpg_condense5.cu"]
HEADERS = ["dpg_internal.h", "dpg_setup.h", "dpg_kernels.h", "dpg_registry.h", "dpg_digits.cuh", "dpg_trace.h", "dpg_tcgen05.cuh"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _flags(debug: bool = False):
    return ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
                   "-I", os.path.join(ROOT, "include"), "--expt-relaxed-constexpr"] + (
                       ["-DDPG_DEBUG_BOUNDS"] if debug else [])


def _stale(target: str, deps) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False, debug: bool = False) -> str:
    bdir, so = (BUILD_DEBUG, SO_DEBUG) if debug else (BUILD, SO)
    os.makedirs(bdir, exist_ok=True)
    hdrs = [os.path.join(CSRC, h) for h in HEADERS] + [os.path.join(ROOT, "include", "dpg.h")]
    objs, jobs = [], []
    for src in SOURCES:
        s = os.path.join(CSRC, src)
        o = os.path.join(bdir, src.replace(".cu", ".o"))
        objs.append(o)
        if force or _stale(o, [s] + hdrs):
            jobs.append([nvcc()] + _flags(debug) + ["-c", s, "-o", o])

    def run(cmd):
        if verbose:
            print(" ".join(cmd), flush=True)
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed:\n{' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
        return r.stderr

    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        for msg in ex.map(run, jobs):
            if verbose and msg:
                print(msg)
    if force or jobs or _stale(so, objs):
        tmp = so + f".tmp{os.getpid()}"
        run([nvcc()] + ARCH + ["-shared", "-o", tmp] + objs + ["-lcudart_static", "-lrt", "-ldl", "-lpthread"])
        os.replace(tmp, so)
    return so


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True, debug="--debug" in sys.argv))
