"""Python face of the SINDI oracle (``oracle.c``): a plain single-threaded FP64 CPU reference.

TEST INFRASTRUCTURE ONLY: the test suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` are the only callers. The CUDA path never
imports this package, and this package never imports the CUDA path.

Every function cites the passage of arXiv 2509.08395 it follows; the C source
holds the arithmetic.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

F32, F16, E4M3 = 0, 1, 2
PRUNES = {"mass": 0, "vector_number": 1, "list": 2, "mass_list": 3}
_DTYPES = {"f32": F32, "f16": F16, "f8": E4M3, "e4m3": E4M3}

_i64p = ctypes.c_void_p


def compile_library(src: str, out: str) -> None:
    """gcc with no FMA contraction and no fast-math: every FP64 operation rounds as written."""
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math",
                           "-fPIC", "-shared", src, "-o", out, "-lm"])


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so beside it (when missing or older than the source)."""
    with _lock:
        if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
            tmp = _LIB + f".tmp{os.getpid()}"
            compile_library(_SRC, tmp)
            os.replace(tmp, _LIB)
    return _LIB


def _load():
    """Load liboracle.so, or the library ORACLE_LIBRARY names: another build of
    an oracle.c (the mutation tests load copies with planted mistakes)."""
    global _lib
    if _lib is not None:
        return _lib
    path = os.environ.get("ORACLE_LIBRARY") or build()
    L = ctypes.CDLL(path)
    vp, i64, i32, dbl = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_double
    L.orc_dataset_create.argtypes = [vp, vp, vp, i64, i32, ctypes.POINTER(ctypes.c_int)]
    L.orc_dataset_create.restype = vp
    L.orc_dataset_free.argtypes = [vp]
    L.orc_dataset_nnz.argtypes = [vp]
    L.orc_dataset_nnz.restype = i64
    L.orc_dataset_export.argtypes = [vp, vp, vp, vp]
    L.orc_inner_product.argtypes = [vp, i64, vp, i64]
    L.orc_inner_product.restype = dbl
    L.orc_brute_force.argtypes = [vp, vp, i64, i64, vp, vp]
    L.orc_brute_force.restype = i64
    L.orc_all_scores.argtypes = [vp, vp, i64, vp]
    L.orc_alpha_mass.argtypes = [vp, vp, i64, dbl, vp]
    L.orc_alpha_mass.restype = i64
    L.orc_build.argtypes = [vp, i64, dbl, i32, ctypes.POINTER(ctypes.c_int)]
    L.orc_build.restype = vp
    L.orc_build_ex.argtypes = [vp, i64, dbl, i32, i32, i64, ctypes.POINTER(ctypes.c_int)]
    L.orc_build_ex.restype = vp
    L.orc_index_free.argtypes = [vp]
    L.orc_index_sigma.argtypes = [vp]
    L.orc_index_sigma.restype = i64
    L.orc_index_postings.argtypes = [vp]
    L.orc_index_postings.restype = i64
    L.orc_index_export.argtypes = [vp, vp, vp, vp, vp, vp]
    L.orc_list_vmax.argtypes = [vp, vp]
    L.orc_search.argtypes = [vp, vp, i64, dbl, i64, i64, vp, vp, vp, vp, vp]
    L.orc_search.restype = i64
    L.orc_f16_encode.argtypes = [ctypes.c_float]
    L.orc_f16_encode.restype = ctypes.c_uint16
    L.orc_f16_decode.argtypes = [ctypes.c_uint16]
    L.orc_f16_decode.restype = ctypes.c_float
    L.orc_e4m3_encode.argtypes = [ctypes.c_float]
    L.orc_e4m3_encode.restype = ctypes.c_uint8
    L.orc_e4m3_decode.argtypes = [ctypes.c_uint8]
    L.orc_e4m3_decode.restype = ctypes.c_float
    _lib = L
    return L


def _c(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


class Dataset:
    """Canonical sparse dataset (Definition 1): rows sorted by dim, explicit zeros dropped, FP64 values.

    Raises ValueError for a malformed CSR (decreasing indptr, dim outside
    [0, d), duplicate dim in a row, non-finite value)."""

    def __init__(self, indptr, indices, values, dim: int):
        L = _load()
        self._keep = (_c(indptr, np.int64), _c(indices, np.int32), _c(values, np.float32))
        ip, ix, v = self._keep
        self.n = len(ip) - 1
        self.dim = int(dim)
        err = ctypes.c_int(0)
        self._h = L.orc_dataset_create(ip.ctypes.data, ix.ctypes.data, v.ctypes.data, self.n, self.dim,
                                       ctypes.byref(err))
        if not self._h:
            raise ValueError(f"oracle rejected the CSR (code {err.value})")

    def __del__(self):
        h = getattr(self, "_h", None)
        if h and _lib is not None:
            _lib.orc_dataset_free(h)
            self._h = None

    @property
    def nnz(self) -> int:
        return int(_load().orc_dataset_nnz(self._h))

    def export(self):
        """(indptr int64, dims int32, values float64) of the canonical rows."""
        ptr = np.empty(self.n + 1, np.int64)
        dims = np.empty(max(self.nnz, 1), np.int32)
        vals = np.empty(max(self.nnz, 1), np.float64)
        _load().orc_dataset_export(self._h, ptr.ctypes.data, dims.ctypes.data, vals.ctypes.data)
        return ptr, dims[: self.nnz], vals[: self.nnz]


def inner_product(D: Dataset, i: int, Q: Dataset, r: int) -> float:
    """delta(x_i, q_r), Definition 2, summed over Omega in ascending dim order (FP64)."""
    return float(_load().orc_inner_product(D._h, int(i), Q._h, int(r)))


def brute_force(D: Dataset, Q: Dataset, r: int, k: int):
    """Exact top-k MIPS for query r (Definition 3), order (score desc, id asc)."""
    kk = max(min(k, D.n), 0)
    ids = np.empty(max(kk, 1), np.int64)
    sc = np.empty(max(kk, 1), np.float64)
    n = _load().orc_brute_force(D._h, Q._h, int(r), int(k), ids.ctypes.data, sc.ctypes.data)
    if n < 0:
        raise MemoryError("oracle brute force failed")
    return ids[:n], sc[:n]


def all_scores(D: Dataset, Q: Dataset, r: int) -> np.ndarray:
    """delta(x_i, q_r) for every document i (Definition 2)."""
    out = np.empty(D.n, np.float64)
    _load().orc_all_scores(D._h, Q._h, int(r), out.ctypes.data)
    return out


def alpha_mass(dims, values, alpha: float) -> np.ndarray:
    """Positions (into the given row, in pi order) of the alpha-mass subvector.

    Definitions "Mass of a Vector" and "alpha-Mass Subvector" (Sec. 4.1): pi
    orders entries by |x| descending (ties: lower dim first); r is the
    smallest count whose prefix of |x| reaches alpha * mass (FP64)."""
    d = _c(dims, np.int32)
    v = _c(values, np.float32)
    out = np.empty(max(len(d), 1), np.int64)
    r = _load().orc_alpha_mass(d.ctypes.data, v.ctypes.data, len(d), float(alpha), out.ctypes.data)
    if r < 0:
        raise MemoryError
    return out[:r]


class Index:
    """Algorithm 3 (ApproximateSindiConstruction): alpha-mass every document, then Algorithm 1.

    Lists I_{j,w} (Sec. 3.3.1) hold (global id, value) in ascending id; the
    unpruned dataset stays attached for reordering (Algorithm 3 returns it)."""

    def __init__(self, D: Dataset, window: int, alpha: float = 1.0, dtype: str = "f32", prune: str = "mass",
                 prune_n: int = 0):
        """prune: "mass" (alpha-mass, Sec. 4.1), "vector_number" (prune_n entries per document),
        "list" (prune_n entries per list I_j) or "mass_list" (alpha-mass, then list pruning)."""
        L = _load()
        self.D = D
        self.window = int(window)
        self.alpha = float(alpha)
        self.dtype = dtype
        self.prune = prune
        self.prune_n = int(prune_n)
        err = ctypes.c_int(0)
        self._h = L.orc_build_ex(D._h, self.window, self.alpha, _DTYPES[dtype], PRUNES[prune], self.prune_n,
                                 ctypes.byref(err))
        if not self._h:
            raise ValueError(f"oracle build failed (code {err.value})")
        self.sigma = int(L.orc_index_sigma(self._h))
        self.postings = int(L.orc_index_postings(self._h))

    def __del__(self):
        h = getattr(self, "_h", None)
        if h and _lib is not None:
            _lib.orc_index_free(h)
            self._h = None

    def export(self):
        """Lists as arrays: seg[d*sigma+1] (list (j,w) = seg[j*sigma+w] .. seg[j*sigma+w+1]),
        pid[P] global ids, pval[P] stored values (FP64), scale[d], kept[n] (r_i per doc)."""
        S = self.D.dim * self.sigma
        seg = np.empty(S + 1, np.int64)
        pid = np.empty(max(self.postings, 1), np.int64)
        pval = np.empty(max(self.postings, 1), np.float64)
        scale = np.empty(self.D.dim, np.float32)
        kept = np.empty(max(self.D.n, 1), np.int64)
        _load().orc_index_export(self._h, seg.ctypes.data, pid.ctypes.data, pval.ctypes.data,
                                 scale.ctypes.data, kept.ctypes.data)
        return seg, pid[: self.postings], pval[: self.postings], scale, kept[: self.D.n]

    def list_vmax(self) -> np.ndarray:
        """The largest |stored value| of every list I_j over all its windows (FP64, [d]; cached)."""
        if getattr(self, "_vmax", None) is None:
            out = np.empty(max(self.D.dim, 1), np.float64)
            _load().orc_list_vmax(self._h, out.ctypes.data)
            self._vmax = out[: self.D.dim]
        return self._vmax

    def search(self, Q: Dataset, r: int, k: int, gamma: int = 0, beta: float = 1.0, want_coarse: bool = False):
        """Algorithm 4 for query r: beta-mass query, Algorithm 2 for gamma candidates, exact reorder.

        gamma == 0 skips the reorder (coarse top-k is the answer). Returns
        (ids, scores) best-first, plus (coarse_ids, coarse_scores) when asked."""
        n_docs = self.D.n
        kk = max(min(k, n_docs), 1)
        gg = max(min(gamma, n_docs), 1)
        ids = np.empty(kk, np.int64)
        sc = np.empty(kk, np.float64)
        cids = np.empty(gg, np.int64)
        csc = np.empty(gg, np.float64)
        nco = ctypes.c_int64(0)
        n = _load().orc_search(self._h, Q._h, int(r), float(beta), int(gamma), int(k), ids.ctypes.data,
                               sc.ctypes.data, cids.ctypes.data if want_coarse else None,
                               csc.ctypes.data if want_coarse else None, ctypes.byref(nco))
        if n < 0:
            raise ValueError(f"oracle search failed ({n})")
        if want_coarse:
            return ids[:n], sc[:n], cids[: nco.value], csc[: nco.value]
        return ids[:n], sc[:n]


def f16_encode(x: float) -> int:
    """IEEE binary16 bits of an FP32 value, round to nearest even."""
    return int(_load().orc_f16_encode(ctypes.c_float(x)))


def f16_decode(h: int) -> float:
    return float(_load().orc_f16_decode(ctypes.c_uint16(h)))


def e4m3_encode(x: float) -> int:
    """OCP FP8 E4M3 code of an FP32 value, round to nearest even, saturating at +-448."""
    return int(_load().orc_e4m3_encode(ctypes.c_float(x)))


def e4m3_decode(c: int) -> float:
    return float(_load().orc_e4m3_decode(ctypes.c_uint8(c)))


def recall(found, truth) -> float:
    """Recall = |R intersect R*| / |R*| (Sec. 5.1, performance metrics)."""
    truth = set(int(t) for t in truth)
    if not truth:
        return 1.0
    return len(truth.intersection(int(f) for f in found)) / len(truth)


def recall_tie_aware(found, truth, truth_scores, D: Dataset, Q: Dataset, r: int) -> float:
    """Recall that also counts a returned document whose exact score delta (Definition 2) reaches the exact
    k-th score of R* = truth (best-first, with its FP64 scores): documents tied with the k-th one are equally
    correct answers, whichever of them the tie rule put into R*. Capped at 1."""
    truth = [int(t) for t in truth]
    if not truth:
        return 1.0
    tset, kth = set(truth), float(truth_scores[len(truth) - 1])
    hits = sum(1 for f in dict.fromkeys(int(x) for x in found)
               if 0 <= f < D.n and (f in tset or inner_product(D, f, Q, r) >= kth))
    return min(hits, len(truth)) / len(truth)
