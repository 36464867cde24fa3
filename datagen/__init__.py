"""Seeded synthetic sparse inputs (CSR) shared by the oracle, the tests and the bench.

This package draws inputs only; it contains none of the search method's
arithmetic. The C source (``gen.c``) is compiled on first use with gcc into
``libsindigen.so`` beside it (``build()`` does it explicitly).

Workloads stand in for the paper's datasets (Table "Dataset Statistics",
Section 5.1: SPLADE-1M/FULL, AntSparse, NQ, RANDOM-5M), which are not
available: Zipf-distributed dims (a vocabulary with a heavy head), lognormal
values, and nnz per row drawn from the distributions listed in ``WORKLOADS``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass, field, replace

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gen.c")
_LIB = os.path.join(_HERE, "libsindigen.so")
_lock = threading.Lock()
_lib = None

NNZ_POISSON, NNZ_LOGNORMAL, NNZ_UNIFORM = 0, 1, 2
VAL_LOGNORMAL, VAL_UNIFORM = 0, 1


class _GenParams(ctypes.Structure):
    _fields_ = [
        ("n_rows", ctypes.c_int64),
        ("dim", ctypes.c_int32),
        ("nnz_kind", ctypes.c_int32),
        ("nnz_a", ctypes.c_double),
        ("nnz_b", ctypes.c_double),
        ("nnz_min", ctypes.c_int32),
        ("nnz_max", ctypes.c_int32),
        ("zipf_s", ctypes.c_double),
        ("val_kind", ctypes.c_int32),
        ("val_sigma", ctypes.c_double),
        ("seed", ctypes.c_uint64),
    ]


def build(force: bool = False) -> str:
    """Compile gen.c into libsindigen.so (gcc, OpenMP). Returns the path."""
    with _lock:
        if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
            tmp = _LIB + f".tmp{os.getpid()}"
            subprocess.check_call(
                ["gcc", "-O2", "-std=c11", "-fno-math-errno", "-ffp-contract=off", "-fPIC", "-shared", "-fopenmp", _SRC,
                 "-o", tmp, "-lm"]
            )
            os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        lib.gen_row_nnz.argtypes = [ctypes.POINTER(_GenParams), ctypes.c_void_p]
        lib.gen_row_nnz.restype = ctypes.c_int
        lib.gen_fill.argtypes = [ctypes.POINTER(_GenParams), ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
        lib.gen_fill.restype = ctypes.c_int
        _lib = lib
    return _lib


@dataclass(frozen=True)
class RowDist:
    """How one matrix (docs or queries) is drawn."""

    n_rows: int
    nnz_kind: int
    nnz_a: float
    nnz_b: float = 0.0
    nnz_min: int = 0
    nnz_max: int = 1 << 30
    val_kind: int = VAL_LOGNORMAL
    val_sigma: float = 1.0


@dataclass(frozen=True)
class Workload:
    """A synthetic search workload: docs, queries and the search knobs."""

    name: str
    dim: int
    zipf_s: float
    docs: RowDist
    queries: RowDist
    k: int
    gamma: int
    alpha: float
    window: int
    doc_seed: int
    query_seed: int
    value_dtype: str = "f32"
    notes: str = ""
    extra: dict = field(default_factory=dict)

    def scaled(self, n_docs: int | None = None, n_queries: int | None = None, **kw) -> "Workload":
        """Same distributions at another size (used for bounded samples and small tests)."""
        w = self
        if n_docs is not None:
            w = replace(w, docs=replace(w.docs, n_rows=int(n_docs)))
        if n_queries is not None:
            w = replace(w, queries=replace(w.queries, n_rows=int(n_queries)))
        if kw:
            w = replace(w, **kw)
        return w


# lognormal nnz uses sigma_ln = 0.5 and mu_ln = ln(mean) - sigma_ln^2 / 2
WORKLOADS: dict[str, Workload] = {
    # 10k docs x 1,024 dims; exact search, no pruning, no rerank
    "exact-10k": Workload(
        name="exact-10k", dim=1024, zipf_s=1.1,
        docs=RowDist(10_000, NNZ_POISSON, 32.0, val_sigma=1.0),
        queries=RowDist(100, NNZ_POISSON, 8.0, nnz_min=1, val_sigma=1.0),
        k=10, gamma=0, alpha=1.0, window=4096, doc_seed=1001, query_seed=2001,
    ),
    # 1M docs x 30,522 dims; mass-ratio pruning alpha = 0.5, rerank 500, top-50; window 16,384 (measured
    # best for both schedules on this size)
    "pruned-1m": Workload(
        name="pruned-1m", dim=30522, zipf_s=1.05,
        docs=RowDist(1_000_000, NNZ_LOGNORMAL, 120.0, 0.5, 10, 400, val_sigma=0.8),
        queries=RowDist(1_000, NNZ_LOGNORMAL, 45.0, 0.5, 5, 150, val_sigma=0.8),
        k=50, gamma=500, alpha=0.5, window=16384, doc_seed=1002, query_seed=2002,
    ),
    # 8.8M docs, 10k queries of uneven nnz U[5, 200]
    "batched-8.8m": Workload(
        name="batched-8.8m", dim=30522, zipf_s=1.05,
        docs=RowDist(8_800_000, NNZ_LOGNORMAL, 120.0, 0.5, 10, 400, val_sigma=0.8),
        queries=RowDist(10_000, NNZ_UNIFORM, 5, 200, 5, 200, val_sigma=0.8),
        k=50, gamma=500, alpha=0.5, window=8192, doc_seed=1003, query_seed=2003,
    ),
    # the 8.8M index with FP16 / FP8 postings; 10k queries nnz mean 45; rerank 1,000
    "lowprec-8.8m": Workload(
        name="lowprec-8.8m", dim=30522, zipf_s=1.05,
        docs=RowDist(8_800_000, NNZ_LOGNORMAL, 120.0, 0.5, 10, 400, val_sigma=0.8),
        queries=RowDist(10_000, NNZ_LOGNORMAL, 45.0, 0.5, 5, 150, val_sigma=0.8),
        k=50, gamma=1000, alpha=0.5, window=8192, doc_seed=1003, query_seed=2004,
        value_dtype="f16",
    ),
    # 25M docs x 250k dims, FP16 postings, Poisson arrivals
    "serve-25m": Workload(
        name="serve-25m", dim=250_000, zipf_s=1.0,
        docs=RowDist(25_000_000, NNZ_LOGNORMAL, 120.0, 0.5, 10, 400, val_sigma=0.8),
        queries=RowDist(10_000, NNZ_LOGNORMAL, 40.0, 0.5, 3, 300, val_sigma=0.8),
        k=50, gamma=500, alpha=0.5, window=8192, doc_seed=1005, query_seed=2005,
        value_dtype="f16",
    ),
}


# the sparsity sweep of Sec. 5 (RANDOM-1M): 1M documents of 120 entries, dims and values uniform at
# random, d from 10k to 100k; queries from the same generator
for _d in (10_000, 30_000, 50_000, 70_000, 100_000):
    _n = f"uniform-1m-d{_d // 1000}k"
    WORKLOADS[_n] = Workload(
        name=_n, dim=_d, zipf_s=0.0,
        docs=RowDist(1_000_000, NNZ_UNIFORM, 120, 120, 120, 120, val_kind=VAL_UNIFORM),
        queries=RowDist(1_000, NNZ_UNIFORM, 120, 120, 120, 120, val_kind=VAL_UNIFORM),
        k=50, gamma=500, alpha=0.5, window=8192, doc_seed=1006, query_seed=2006,
    )
del _d, _n


def generate(dist: RowDist, dim: int, zipf_s: float, seed: int):
    """Draw one CSR matrix. Returns (indptr int64[n+1], indices int32[nnz], values float32[nnz])."""
    lib = _load()
    p = _GenParams(
        n_rows=dist.n_rows, dim=dim, nnz_kind=dist.nnz_kind, nnz_a=float(dist.nnz_a),
        nnz_b=float(dist.nnz_b), nnz_min=int(dist.nnz_min), nnz_max=int(min(dist.nnz_max, 1 << 30)),
        zipf_s=float(zipf_s), val_kind=dist.val_kind, val_sigma=float(dist.val_sigma),
        seed=int(seed) & ((1 << 64) - 1),
    )
    nnz = np.empty(dist.n_rows, dtype=np.int64)
    if lib.gen_row_nnz(ctypes.byref(p), nnz.ctypes.data) != 0:
        raise RuntimeError("gen_row_nnz failed")
    indptr = np.zeros(dist.n_rows + 1, dtype=np.int64)
    np.cumsum(nnz, out=indptr[1:])
    total = int(indptr[-1])
    indices = np.empty(total, dtype=np.int32)
    values = np.empty(total, dtype=np.float32)
    rc = lib.gen_fill(ctypes.byref(p), indptr.ctypes.data, indices.ctypes.data, values.ctypes.data)
    if rc != 0:
        raise RuntimeError(f"gen_fill failed ({rc})")
    return indptr, indices, values


def docs(w: Workload):
    """Document CSR of a workload."""
    return generate(w.docs, w.dim, w.zipf_s, w.doc_seed)


def queries(w: Workload):
    """Query CSR of a workload."""
    return generate(w.queries, w.dim, w.zipf_s, w.query_seed)


def random_csr(n_rows: int, dim: int, mean_nnz: float, seed: int, zipf_s: float = 1.1,
               val_sigma: float = 1.0, nnz_min: int = 0, nnz_max: int = 1 << 30, uniform_values=False):
    """Small ad-hoc CSR (Poisson nnz) for edge-case tests."""
    d = RowDist(n_rows, NNZ_POISSON, float(mean_nnz), nnz_min=nnz_min, nnz_max=nnz_max,
                val_kind=VAL_UNIFORM if uniform_values else VAL_LOGNORMAL, val_sigma=val_sigma)
    return generate(d, dim, zipf_s, seed)
