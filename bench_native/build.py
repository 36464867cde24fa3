"""Builds the benchmark's native helpers into ``bench_native/lib/`` (git-ignored build products):

- ``libsindi_probe.so`` from ``scatter_peak.cu`` (nvcc, sm_103a): the shared-memory scatter-add probe
  whose measured rate is the scan's secondary roofline;
- ``libsindi_load.so`` from ``serve_load.c`` (gcc): the open-loop load generator of the serving leg.

Neither is part of the search library; ``bench.py`` loads them.

    python bench_native/build.py [--force]
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
LIBDIR = os.path.join(HERE, "lib")
PROBE_SRC = os.path.join(HERE, "scatter_peak.cu")
PROBE_LIB = os.path.join(LIBDIR, "libsindi_probe.so")
LOAD_SRC = os.path.join(HERE, "serve_load.c")
LOAD_LIB = os.path.join(LIBDIR, "libsindi_load.so")


def _stale(target: str, src: str) -> bool:
    return not os.path.exists(target) or os.path.getmtime(src) > os.path.getmtime(target)


def _run(cmd, target):
    tmp = target + f".tmp{os.getpid()}"
    p = subprocess.run(cmd + ["-o", tmp], capture_output=True, text=True)
    if p.returncode != 0:
        sys.stderr.write(p.stdout + p.stderr)
        raise RuntimeError("build failed: " + " ".join(cmd))
    os.replace(tmp, target)


def build(force: bool = False) -> None:
    os.makedirs(LIBDIR, exist_ok=True)
    if force or _stale(LOAD_LIB, LOAD_SRC):
        _run(["gcc", "-O2", "-std=c11", "-D_POSIX_C_SOURCE=200809L", "-fPIC", "-shared", "-pthread", LOAD_SRC,
              "-lm"], LOAD_LIB)
    if force or _stale(PROBE_LIB, PROBE_SRC):
        nvcc = os.environ.get("NVCC") or shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
        _run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-lineinfo", "-Xcompiler", "-fPIC",
              "-shared", "-cudart", "static", PROBE_SRC], PROBE_LIB)


if __name__ == "__main__":
    build(force="--force" in sys.argv)
    print(PROBE_LIB, LOAD_LIB)
