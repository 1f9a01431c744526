"""Build libdgt.so (the C-ABI CUDA library) in-tree with nvcc for sm_103a.

Each translation unit is compiled in parallel, then linked into
``paper_1307_4569_gb300/lib/libdgt.so``.  Rebuilds only when a source or header is
newer than the library.  No CMake, no torch extension machinery.

``build(debug=True)`` compiles the same sources with ``-DDGT_DEBUG`` into
``lib/libdgt_debug.so`` (guard-zone bounds checking after every launch, include/dgt.h);
the binding loads it instead of the release library when ``DGT_DEBUG=1``.
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
LIBDIR = os.path.join(HERE, "lib")
OBJDIR = os.path.join(HERE, "lib", "obj")
LIB = os.path.join(LIBDIR, "libdgt.so")
LIB_DEBUG = os.path.join(LIBDIR, "libdgt_debug.so")
OBJDIR_DEBUG = os.path.join(HERE, "lib", "obj_debug")
SOURCES = ["engine_zak.cu", "engine_aux.cu", "plan.cu", "p2_cols_f32.cu", "p2_rows_f32.cu", "p2_cols_f64.cu",
           "p2_rows_f64.cu", "mr_f32.cu", "mr_f64.cu", "debug.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _deps() -> list[str]:
    out = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cu", ".cuh", ".h"))]
    out.append(os.path.join(ROOT, "include", "dgt.h"))
    return out


def up_to_date(debug: bool = False) -> bool:
    lib = LIB_DEBUG if debug else LIB
    if not os.path.exists(lib):
        return False
    t = os.path.getmtime(lib)
    return all(os.path.getmtime(p) <= t for p in _deps())


def build(force: bool = False, verbose: bool = False, extra_flags: list[str] | None = None,
          debug: bool = False) -> str:
    lib = LIB_DEBUG if debug else LIB
    objdir = OBJDIR_DEBUG if debug else OBJDIR
    if not force and up_to_date(debug):
        return lib
    os.makedirs(objdir, exist_ok=True)
    nvcc = _nvcc()
    flags = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr",
             "-I", os.path.join(ROOT, "include"), "-I", CSRC] + ARCH + (extra_flags or [])
    if debug:
        flags.append("-DDGT_DEBUG")

    def one(src):
        obj = os.path.join(objdir, src.replace(".cu", ".o"))
        cmd = [nvcc, "-c", os.path.join(CSRC, src), "-o", obj] + flags
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed for %s:\n%s\n%s" % (src, " ".join(cmd), r.stderr))
        if verbose and r.stderr:
            sys.stderr.write(r.stderr)
        return obj

    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(one, SOURCES))
    tmp = lib + ".tmp"
    cmd = [nvcc, "-shared", "-o", tmp] + objs + ARCH + ["-lcudart"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n%s\n%s" % (" ".join(cmd), r.stderr))
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv, debug="--debug" in sys.argv))
