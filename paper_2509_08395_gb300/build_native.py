"""Compiles the CUDA sources of this package into ``lib/libsindi.so`` (sm_103a only), and the same sources
with every bounds check of ``csrc/checks.cuh`` compiled in (``-DSINDI_CHECKS=1``) into
``lib/libsindi_checked.so``, which tests load through ``SINDI_LIBRARY``.

Each ``csrc/*.cu`` file is compiled to an object in parallel, then nvcc links
the shared library with the CUDA runtime linked statically, so the library
needs nothing but the NVIDIA driver at load time. Objects and the library are
build products (ignored by git).

    python -m paper_2509_08395_gb300.build_native [--force] [--ptxas-verbose]
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OBJ = os.path.join(HERE, "_build")
OBJ_CHECKED = os.path.join(HERE, "_build_checked")
LIBDIR = os.path.join(HERE, "lib")
LIB = os.path.join(LIBDIR, "libsindi.so")
LIB_CHECKED = os.path.join(LIBDIR, "libsindi_checked.so")
ROOT = os.path.dirname(HERE)

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++17", "--expt-relaxed-constexpr", "-Xcompiler", "-fPIC,-O2",
              "-I" + os.path.join(ROOT, "include")]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found (CUDA toolkit required to build the native library)")


def _sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _headers():
    return sorted(glob.glob(os.path.join(CSRC, "*.cuh"))) + [os.path.join(ROOT, "include", "sindi.h")]


def _stale(target: str, deps) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose_ptxas: bool = False, checked: bool = True) -> str:
    """Builds lib/libsindi.so (and, with `checked`, lib/libsindi_checked.so); objects compile in parallel."""
    os.makedirs(LIBDIR, exist_ok=True)
    cc = nvcc()
    heads = _headers()
    variants = [(OBJ, LIB, [])] + ([(OBJ_CHECKED, LIB_CHECKED, ["-DSINDI_CHECKS=1"])] if checked else [])
    jobs = []
    objs = {}
    for obj_dir, lib, defs in variants:
        os.makedirs(obj_dir, exist_ok=True)
        objs[lib] = []
        for src in _sources():
            obj = os.path.join(obj_dir, os.path.basename(src)[:-3] + ".o")
            objs[lib].append(obj)
            if force or _stale(obj, [src] + heads):
                cmd = [cc, *ARCH, *NVCC_FLAGS, *defs, "-c", src, "-o", obj]
                if verbose_ptxas and not defs:
                    cmd += ["-Xptxas", "-v"]
                jobs.append(cmd)

    def run(cmd):
        p = subprocess.run(cmd, capture_output=True, text=True)
        return cmd, p

    with cf.ThreadPoolExecutor(max_workers=max(1, min(len(jobs), os.cpu_count() or 4))) as ex:
        for cmd, p in ex.map(run, jobs):
            if p.returncode != 0 or verbose_ptxas:
                sys.stderr.write(p.stdout + p.stderr)
            if p.returncode != 0:
                raise RuntimeError("nvcc failed: " + " ".join(cmd))
    for _, lib, _ in variants:
        if force or jobs or _stale(lib, objs[lib]):
            tmp = lib + f".tmp{os.getpid()}"
            cmd = [cc, *ARCH, "-shared", "-cudart", "static", *objs[lib], "-o", tmp]
            p = subprocess.run(cmd, capture_output=True, text=True)
            if p.returncode != 0:
                sys.stderr.write(p.stdout + p.stderr)
                raise RuntimeError("link failed: " + " ".join(cmd))
            os.replace(tmp, lib)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose_ptxas="--ptxas-verbose" in sys.argv))
