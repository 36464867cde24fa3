"""Python binding of the C ABI in include/sindi.h (ctypes; argument marshalling only).

Functions keep the C names (``sindi_build``, ``sindi_search``, ...) and take
torch tensors or numpy arrays; every step of the search runs in the CUDA
kernels of ``lib/libsindi.so``. There is no CPU fallback: if the library is
missing, loading raises.

``Index`` is a small convenience wrapper over the same calls.
"""
from __future__ import annotations

import ctypes
import os
import weakref

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "lib", "libsindi.so")

SINDI_OK, SINDI_ERR_INVALID_ARG, SINDI_ERR_INVALID_DATA, SINDI_ERR_OOM = 0, 1, 2, 3
SINDI_ERR_CUDA, SINDI_ERR_TIMEOUT, SINDI_ERR_UNSUPPORTED = 4, 5, 6
SINDI_F32, SINDI_F16, SINDI_F8E4M3 = 0, 1, 2
SINDI_MODE_PLAIN, SINDI_MODE_BATCHED = 0, 1
DTYPES = {"f32": SINDI_F32, "f16": SINDI_F16, "f8": SINDI_F8E4M3, "e4m3": SINDI_F8E4M3}
MODES = {"plain": SINDI_MODE_PLAIN, "batched": SINDI_MODE_BATCHED}
SINDI_PRUNE_MASS, SINDI_PRUNE_VECTOR_NUMBER, SINDI_PRUNE_LIST, SINDI_PRUNE_MASS_LIST = 0, 1, 2, 3
SINDI_SCAN_PIPELINED = 1  # block_threads value of the pipelined window scan
SINDI_ACCUM_AUTO, SINDI_ACCUM_F32, SINDI_ACCUM_FIXED32 = 0, 1, 2
ACCUMS = {"auto": SINDI_ACCUM_AUTO, "f32": SINDI_ACCUM_F32, "fixed32": SINDI_ACCUM_FIXED32}


def _accum(accum: str) -> int:
    """sindi_accumulator value of `accum` ("auto", "f32" or "fixed32")."""
    if accum not in ACCUMS:
        raise ValueError(f"accum must be one of {sorted(ACCUMS)}, not {accum!r}")
    return ACCUMS[accum]
PRUNES = {"mass": SINDI_PRUNE_MASS, "vector_number": SINDI_PRUNE_VECTOR_NUMBER, "list": SINDI_PRUNE_LIST,
          "mass_list": SINDI_PRUNE_MASS_LIST}
STATUS_NAMES = {0: "SINDI_OK", 1: "SINDI_ERR_INVALID_ARG", 2: "SINDI_ERR_INVALID_DATA", 3: "SINDI_ERR_OOM",
                4: "SINDI_ERR_CUDA", 5: "SINDI_ERR_TIMEOUT", 6: "SINDI_ERR_UNSUPPORTED"}


class SindiError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class sindi_build_params(ctypes.Structure):
    _fields_ = [("window", ctypes.c_uint32), ("value_dtype", ctypes.c_int32), ("alpha", ctypes.c_double),
                ("prune", ctypes.c_int32), ("prune_n", ctypes.c_uint32)]


class sindi_search_params(ctypes.Structure):
    _fields_ = [("k", ctypes.c_uint32), ("gamma", ctypes.c_uint32), ("beta", ctypes.c_double),
                ("mode", ctypes.c_uint32), ("block_threads", ctypes.c_uint32), ("group", ctypes.c_uint32),
                ("accumulator", ctypes.c_uint32)]


class sindi_index_info_t(ctypes.Structure):
    _fields_ = [("n_docs", ctypes.c_int64), ("dim", ctypes.c_int32), ("value_dtype", ctypes.c_int32),
                ("window", ctypes.c_uint32), ("n_windows", ctypes.c_uint32), ("postings", ctypes.c_int64),
                ("doc_nnz", ctypes.c_int64), ("index_bytes", ctypes.c_int64), ("doc_bytes", ctypes.c_int64),
                ("alpha", ctypes.c_double), ("prune", ctypes.c_int32), ("prune_n", ctypes.c_uint32)]


class sindi_stats_t(ctypes.Structure):
    _fields_ = [("launches", ctypes.c_uint64), ("scan_launches", ctypes.c_uint64), ("queries", ctypes.c_uint64),
                ("scan_ms", ctypes.c_double), ("scan_timed", ctypes.c_uint64)]


class sindi_server_params(ctypes.Structure):
    _fields_ = [("max_batch", ctypes.c_uint32), ("max_slots", ctypes.c_uint32), ("max_query_nnz", ctypes.c_uint32),
                ("max_wait_us", ctypes.c_uint32), ("memory_budget", ctypes.c_uint64),
                ("search", sindi_search_params)]


class sindi_server_stats_t(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_uint64), ("completed", ctypes.c_uint64), ("failed", ctypes.c_uint64),
                ("batches", ctypes.c_uint64), ("n_slots", ctypes.c_uint32), ("peak_in_flight", ctypes.c_uint32),
                ("slot_bytes", ctypes.c_uint64), ("mean_batch", ctypes.c_double), ("p50_ms", ctypes.c_double),
                ("p99_ms", ctypes.c_double), ("max_ms", ctypes.c_double)]


_lib = None

# name -> (restype, argtypes)
_SIGS = {
    "sindi_build": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32,
                                   ctypes.POINTER(sindi_build_params), ctypes.c_void_p,
                                   ctypes.POINTER(ctypes.c_void_p)]),
    "sindi_search": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                    ctypes.c_int64, ctypes.POINTER(sindi_search_params), ctypes.c_void_p,
                                    ctypes.c_void_p, ctypes.c_void_p]),
    "sindi_search_noalloc": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                            ctypes.c_int64, ctypes.POINTER(sindi_search_params), ctypes.c_void_p,
                                            ctypes.c_void_p, ctypes.c_void_p]),
    "sindi_check": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "sindi_index_info": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(sindi_index_info_t)]),
    "sindi_index_export": (ctypes.c_int, [ctypes.c_void_p] * 6),
    "sindi_merge_topk": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64,
                                        ctypes.c_uint32, ctypes.c_void_p, ctypes.c_uint32, ctypes.c_void_p,
                                        ctypes.c_void_p, ctypes.c_void_p]),
    "sindi_set_timing": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    "sindi_index_save": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_char_p]),
    "sindi_index_load": (ctypes.c_int, [ctypes.c_char_p, ctypes.c_void_p, ctypes.POINTER(ctypes.c_void_p)]),
    "sindi_get_stats": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(sindi_stats_t)]),
    "sindi_reset_stats": (ctypes.c_int, [ctypes.c_void_p]),
    "sindi_index_free": (None, [ctypes.c_void_p]),
    "sindi_plan_create": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                         ctypes.c_int64, ctypes.POINTER(sindi_search_params), ctypes.c_void_p,
                                         ctypes.c_void_p, ctypes.POINTER(ctypes.c_void_p)]),
    "sindi_plan_launch": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "sindi_plan_free": (None, [ctypes.c_void_p]),
    "sindi_server_create": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(sindi_server_params),
                                           ctypes.POINTER(ctypes.c_void_p)]),
    "sindi_server_submit": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32,
                                           ctypes.POINTER(ctypes.c_uint64)]),
    "sindi_server_poll": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_int32, ctypes.c_void_p,
                                         ctypes.c_void_p, ctypes.POINTER(ctypes.c_double)]),
    "sindi_server_stats": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(sindi_server_stats_t), ctypes.c_int]),
    "sindi_server_destroy": (None, [ctypes.c_void_p]),
    "sindi_last_error": (ctypes.c_char_p, []),
    "sindi_version": (ctypes.c_char_p, []),
}


def load(path: str | None = None) -> ctypes.CDLL:
    """Load lib/libsindi.so, or the library SINDI_LIBRARY names (e.g. lib/libsindi_checked.so, the build with
    every bounds check compiled in); raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or os.environ.get("SINDI_LIBRARY") or LIB_PATH
    if not os.path.exists(path):
        raise RuntimeError(f"native library missing: {path} (build it with __graft_entry__.build() or "
                           "python -m paper_2509_08395_gb300.build_native)")
    lib = ctypes.CDLL(path)
    for name, (res, args) in _SIGS.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def _check(status: int, what: str):
    if status != SINDI_OK:
        raise SindiError(status, f"{what}: {load().sindi_last_error().decode(errors='replace')}")


def _ptr(a, dtype):
    """Data pointer of a contiguous torch tensor or numpy array of the given numpy dtype."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        if a.dtype != dtype or not a.flags.c_contiguous:
            raise TypeError(f"expected a contiguous {np.dtype(dtype).name} array")
        return a.ctypes.data
    import torch
    tmap = {np.int64: torch.int64, np.int32: torch.int32, np.float32: torch.float32,
            np.uint32: torch.uint32 if hasattr(torch, "uint32") else torch.int32}
    if a.dtype != tmap[dtype] and not (dtype == np.uint32 and a.dtype == torch.int32):
        raise TypeError(f"expected a {tmap[dtype]} tensor, got {a.dtype}")
    if not a.is_contiguous():
        raise TypeError("expected a contiguous tensor")
    return a.data_ptr()


def _numel(a) -> int:
    return int(a.size) if isinstance(a, np.ndarray) else int(a.numel())


def _require(a, n: int, what: str):
    """The C calls get bare pointers and cannot see buffer sizes: check them here, before the call."""
    if a is not None and _numel(a) < n:
        raise ValueError(f"{what} holds {_numel(a)} elements, the call needs {n}")


def _stream(stream, *tensors):
    """A raw cudaStream_t: the given one (an int or a torch.cuda.Stream), else the current stream of the first
    device tensor, else None (the legacy default stream)."""
    if stream is not None:
        return getattr(stream, "cuda_stream", stream)
    for t in tensors:
        if t is not None and not isinstance(t, np.ndarray) and t.is_cuda:
            import torch
            return torch.cuda.current_stream(t.device).cuda_stream
    return None


def _require_search(q_indptr, out_ids, out_scores, n_queries: int, k: int):
    _require(q_indptr, int(n_queries) + 1, "q_indptr")
    _require(out_ids, int(n_queries) * int(k), "out_ids")
    _require(out_scores, int(n_queries) * int(k), "out_scores")


# ---- the C entry points, same names -------------------------------------------------
def sindi_build(indptr, indices, values, n_docs: int, dim: int, window: int = 0, alpha: float = 1.0,
                value_dtype: str = "f32", stream=None, prune: str = "mass", prune_n: int = 0) -> int:
    """Algorithm 3 on the device; returns the opaque index handle (int)."""
    lib = load()
    prm = sindi_build_params(window=int(window), value_dtype=DTYPES[value_dtype], alpha=float(alpha),
                             prune=PRUNES[prune], prune_n=int(prune_n))
    _require(indptr, int(n_docs) + 1, "indptr")
    out = ctypes.c_void_p()
    st = lib.sindi_build(_ptr(indptr, np.int64), _ptr(indices, np.int32), _ptr(values, np.float32), int(n_docs),
                         int(dim), ctypes.byref(prm), _stream(stream, indptr), ctypes.byref(out))
    _check(st, "sindi_build")
    return out.value


def sindi_search(index: int, q_indptr, q_indices, q_values, n_queries: int, out_ids, out_scores, k: int,
                 gamma: int = 0, beta: float = 1.0, mode: str = "plain", stream=None, block: int = 0,
                 group: int = 0, accum: str = "auto") -> None:
    """Algorithm 4 for every query row; writes out_ids (uint32/int32) and out_scores (float32), [n_queries, k].
    accum: the coarse scan's score window, "auto", "f32" or "fixed32" (sindi_accumulator)."""
    lib = load()
    prm = sindi_search_params(k=int(k), gamma=int(gamma), beta=float(beta), mode=MODES[mode], block_threads=int(block),
                              group=int(group), accumulator=_accum(accum))
    _require_search(q_indptr, out_ids, out_scores, n_queries, k)
    st = lib.sindi_search(ctypes.c_void_p(index), _ptr(q_indptr, np.int64), _ptr(q_indices, np.int32),
                          _ptr(q_values, np.float32), int(n_queries), ctypes.byref(prm), _ptr(out_ids, np.uint32),
                          _ptr(out_scores, np.float32), _stream(stream, q_indptr, out_ids))
    _check(st, "sindi_search")


def sindi_search_noalloc(index: int, q_indptr, q_indices, q_values, n_queries: int, out_ids, out_scores, k: int,
                         gamma: int = 0, beta: float = 1.0, mode: str = "plain", stream=None,
                         block: int = 0, group: int = 0, accum: str = "auto") -> None:
    """sindi_search for callers that cannot allocate device memory: all working memory comes from the library's
    static 8 MiB device array. Device tensors only; calls that overlap on the GPU race on that array."""
    lib = load()
    prm = sindi_search_params(k=int(k), gamma=int(gamma), beta=float(beta), mode=MODES[mode], block_threads=int(block),
                              group=int(group), accumulator=_accum(accum))
    _require_search(q_indptr, out_ids, out_scores, n_queries, k)
    st = lib.sindi_search_noalloc(ctypes.c_void_p(index), _ptr(q_indptr, np.int64), _ptr(q_indices, np.int32),
                                  _ptr(q_values, np.float32), int(n_queries), ctypes.byref(prm),
                                  _ptr(out_ids, np.uint32), _ptr(out_scores, np.float32),
                                  _stream(stream, q_indptr, out_ids))
    _check(st, "sindi_search_noalloc")


def sindi_check(index: int, stream=None) -> None:
    _check(load().sindi_check(ctypes.c_void_p(index), _stream(stream)), "sindi_check")


def sindi_index_info(index: int) -> dict:
    info = sindi_index_info_t()
    _check(load().sindi_index_info(ctypes.c_void_p(index), ctypes.byref(info)), "sindi_index_info")
    return {f: getattr(info, f) for f, _ in sindi_index_info_t._fields_}


def sindi_index_export(index: int, parts=("seg", "ids", "vals", "scale", "kept")) -> dict:
    """Copy the lists to host numpy arrays: seg, ids, vals, scale, kept (only the named parts)."""
    info = sindi_index_info(index)
    S = info["dim"] * info["n_windows"]
    P = info["postings"]
    vdt = {SINDI_F32: np.float32, SINDI_F16: np.uint16, SINDI_F8E4M3: np.uint8}[info["value_dtype"]]
    arrs = {
        "seg": lambda: np.empty(S + 1, np.uint32),
        "ids": lambda: np.empty(max(P, 1), np.uint16),
        "vals": lambda: np.empty(max(P, 1), vdt),
        "scale": lambda: np.empty(info["dim"], np.float32),
        "kept": lambda: np.empty(max(info["n_docs"], 1), np.uint32),
    }
    out = {name: arrs[name]() for name in parts}
    ptr = {name: (out[name].ctypes.data if name in out else None) for name in arrs}
    _check(load().sindi_index_export(ctypes.c_void_p(index), ptr["seg"], ptr["ids"], ptr["vals"], ptr["scale"],
                                     ptr["kept"]), "sindi_index_export")
    for name, n in (("ids", P), ("vals", P), ("kept", info["n_docs"])):
        if name in out:
            out[name] = out[name][:n]
    out["info"] = info
    return out


def sindi_index_save(index: int, path: str) -> None:
    _check(load().sindi_index_save(ctypes.c_void_p(index), os.fsencode(path)), "sindi_index_save")


def sindi_index_load(path: str, stream=None) -> int:
    """Rebuild an index written by sindi_index_save; returns the handle."""
    out = ctypes.c_void_p()
    s = _stream(stream)
    _check(load().sindi_index_load(os.fsencode(path), ctypes.c_void_p(int(s or 0)), ctypes.byref(out)),
           "sindi_index_load")
    return out.value


def sindi_set_timing(index: int, enable: bool) -> None:
    _check(load().sindi_set_timing(ctypes.c_void_p(index), 1 if enable else 0), "sindi_set_timing")


def sindi_get_stats(index: int) -> dict:
    s = sindi_stats_t()
    _check(load().sindi_get_stats(ctypes.c_void_p(index), ctypes.byref(s)), "sindi_get_stats")
    return {f: getattr(s, f) for f, _ in sindi_stats_t._fields_}


def sindi_reset_stats(index: int) -> None:
    _check(load().sindi_reset_stats(ctypes.c_void_p(index)), "sindi_reset_stats")


def sindi_index_free(index: int) -> None:
    if index:
        load().sindi_index_free(ctypes.c_void_p(index))


def sindi_version() -> str:
    return load().sindi_version().decode()


# ---- convenience wrapper ------------------------------------------------------------
def sindi_merge_topk(ids, scores, id_offsets, k: int, out=None, stream=None):
    """Top-k over document shards: ids/scores are device tensors [n_shards, n_queries, k_in] of per-shard rows
    (local ids), id_offsets the global id of each shard's first document. Returns (ids, scores) [n_queries, k]."""
    import torch

    S, nq, k_in = ids.shape
    off = np.ascontiguousarray(np.asarray(id_offsets, dtype=np.int64))
    if off.shape != (S,):
        raise ValueError("one id offset per shard")
    if out is None:
        out = (torch.empty((nq, k), dtype=torch.int32, device=ids.device),
               torch.empty((nq, k), dtype=torch.float32, device=ids.device))
    ids = ids.contiguous()
    scores = scores.contiguous()
    _check(load().sindi_merge_topk(_ptr(ids, np.uint32), _ptr(scores, np.float32), int(S), int(nq), int(k_in),
                                   off.ctypes.data, int(k), _ptr(out[0], np.uint32), _ptr(out[1], np.float32),
                                   _stream(stream, ids, out[0])), "sindi_merge_topk")
    return out


class Index:
    """A device-resident SINDI index (owns the C handle)."""

    def __init__(self, indptr, indices, values, dim: int, window: int = 0, alpha: float = 1.0,
                 value_dtype: str = "f32", stream=None, prune: str = "mass", prune_n: int = 0):
        n_docs = (indptr.shape[0] if hasattr(indptr, "shape") else len(indptr)) - 1
        self._dependents = weakref.WeakSet()  # plans and servers over this index
        self.handle = sindi_build(indptr, indices, values, n_docs, dim, window, alpha, value_dtype, stream, prune,
                                  prune_n)
        self.info = sindi_index_info(self.handle)

    def search(self, q_indptr, q_indices, q_values, k: int, gamma: int = 0, beta: float = 1.0,
               mode: str = "plain", out=None, stream=None, block: int = 0, group: int = 0, accum: str = "auto"):
        """Returns (ids, scores) of shape [n_queries, k]; device tensors for device queries."""
        n_q = (q_indptr.shape[0] if hasattr(q_indptr, "shape") else len(q_indptr)) - 1
        if out is None:
            if isinstance(q_indptr, np.ndarray):
                out = (np.empty((n_q, k), np.uint32), np.empty((n_q, k), np.float32))
            else:
                import torch
                dev = q_indptr.device
                out = (torch.empty((n_q, k), dtype=torch.int32, device=dev),
                       torch.empty((n_q, k), dtype=torch.float32, device=dev))
        sindi_search(self.handle, q_indptr, q_indices, q_values, n_q, out[0], out[1], k, gamma, beta, mode, stream,
                     block, group, accum)
        return out

    def save(self, path: str) -> None:
        """Write the index to `path` (sindi_index_save)."""
        sindi_index_save(self.handle, path)

    @classmethod
    def load(cls, path: str, stream=None) -> "Index":
        """An index read back from `path` (sindi_index_load)."""
        obj = cls.__new__(cls)
        obj._dependents = weakref.WeakSet()
        obj.handle = sindi_index_load(path, stream)
        obj.info = sindi_index_info(obj.handle)
        return obj

    def check(self, stream=None):
        sindi_check(self.handle, stream)

    def export(self, parts=("seg", "ids", "vals", "scale", "kept")) -> dict:
        return sindi_index_export(self.handle, parts)

    def close(self):
        """Free the index; plans and servers still open over it are closed first (they must not outlive it)."""
        for dep in list(getattr(self, "_dependents", ())):
            dep.close()
        if getattr(self, "handle", None):
            sindi_index_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


# ---- graph-captured batched search -------------------------------------------------
def sindi_plan_create(index: int, q_indptr, q_indices, q_values, n_queries: int, out_ids, out_scores, k: int,
                      gamma: int = 0, beta: float = 1.0, block: int = 0, group: int = 0, accum: str = "auto") -> int:
    prm = sindi_search_params(k=int(k), gamma=int(gamma), beta=float(beta), mode=SINDI_MODE_BATCHED, block_threads=int(block),
                              group=int(group), accumulator=_accum(accum))
    _require_search(q_indptr, out_ids, out_scores, n_queries, k)
    out = ctypes.c_void_p()
    _check(load().sindi_plan_create(ctypes.c_void_p(index), _ptr(q_indptr, np.int64), _ptr(q_indices, np.int32),
                                    _ptr(q_values, np.float32), int(n_queries), ctypes.byref(prm),
                                    _ptr(out_ids, np.uint32), _ptr(out_scores, np.float32), ctypes.byref(out)),
           "sindi_plan_create")
    return out.value


def sindi_plan_launch(plan: int, stream=None) -> None:
    if stream is None:
        import torch
        stream = torch.cuda.current_stream().cuda_stream
    stream = _stream(stream)
    _check(load().sindi_plan_launch(ctypes.c_void_p(plan), stream), "sindi_plan_launch")


def sindi_plan_free(plan: int) -> None:
    if plan:
        load().sindi_plan_free(ctypes.c_void_p(plan))


class Plan:
    """A batched search of fixed device buffers, captured once as a CUDA graph."""

    def __init__(self, index: "Index", q_indptr, q_indices, q_values, k: int, gamma: int = 0, out=None,
                 block: int = 0, group: int = 0, accum: str = "auto"):
        import torch
        self.index = index
        n_q = q_indptr.shape[0] - 1
        self.inputs = (q_indptr, q_indices, q_values)
        if out is None:
            out = (torch.empty((n_q, k), dtype=torch.int32, device=q_indptr.device),
                   torch.empty((n_q, k), dtype=torch.float32, device=q_indptr.device))
        self.out = out
        self.handle = sindi_plan_create(index.handle, q_indptr, q_indices, q_values, n_q, out[0], out[1], k, gamma,
                                        block=block, group=group, accum=accum)
        index._dependents.add(self)

    def launch(self, stream=None):
        sindi_plan_launch(self.handle, stream)
        return self.out

    def close(self):
        if getattr(self, "handle", None):
            sindi_plan_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


# ---- serving (continuous batching) -----------------------------------------------
def sindi_server_create(index: int, k: int, gamma: int = 0, beta: float = 1.0, max_batch: int = 0,
                        max_slots: int = 0, max_query_nnz: int = 0, max_wait_us: int = 0,
                        memory_budget: int = 0, accum: str = "auto") -> int:
    prm = sindi_server_params(max_batch=max_batch, max_slots=max_slots, max_query_nnz=max_query_nnz,
                              max_wait_us=max_wait_us, memory_budget=memory_budget,
                              search=sindi_search_params(k=k, gamma=gamma, beta=beta, mode=SINDI_MODE_BATCHED,
                                                         block_threads=0, accumulator=_accum(accum)))
    out = ctypes.c_void_p()
    _check(load().sindi_server_create(ctypes.c_void_p(index), ctypes.byref(prm), ctypes.byref(out)),
           "sindi_server_create")
    return out.value


def sindi_server_submit(server: int, q_indices, q_values) -> int:
    qi = np.ascontiguousarray(q_indices, dtype=np.int32)
    qv = np.ascontiguousarray(q_values, dtype=np.float32)
    t = ctypes.c_uint64()
    _check(load().sindi_server_submit(ctypes.c_void_p(server), qi.ctypes.data, qv.ctypes.data, len(qi),
                                      ctypes.byref(t)), "sindi_server_submit")
    return t.value


def sindi_server_poll(server: int, ticket: int, k: int, wait_ms: int = -1):
    """(ids, scores, latency_ms) once the request is done; None while it is still running."""
    ids = np.empty(k, np.uint32)
    sc = np.empty(k, np.float32)
    lat = ctypes.c_double()
    st = load().sindi_server_poll(ctypes.c_void_p(server), ctypes.c_uint64(ticket), int(wait_ms), ids.ctypes.data,
                                  sc.ctypes.data, ctypes.byref(lat))
    if st == SINDI_ERR_TIMEOUT:
        return None
    _check(st, "sindi_server_poll")
    return ids, sc, lat.value


def sindi_server_stats(server: int, reset: bool = False) -> dict:
    s = sindi_server_stats_t()
    _check(load().sindi_server_stats(ctypes.c_void_p(server), ctypes.byref(s), 1 if reset else 0),
           "sindi_server_stats")
    return {f: getattr(s, f) for f, _ in sindi_server_stats_t._fields_}


def sindi_server_destroy(server: int) -> None:
    if server:
        load().sindi_server_destroy(ctypes.c_void_p(server))


class Server:
    """Continuous-batching request loop over an Index (owns the C handle)."""

    def __init__(self, index: "Index", k: int, gamma: int = 0, **kw):
        self.index = index  # keeps the index alive
        self.k = k
        self.handle = sindi_server_create(index.handle, k, gamma, **kw)
        index._dependents.add(self)

    def submit(self, q_indices, q_values) -> int:
        return sindi_server_submit(self.handle, q_indices, q_values)

    def poll(self, ticket: int, wait_ms: int = -1):
        return sindi_server_poll(self.handle, ticket, self.k, wait_ms)

    def stats(self, reset: bool = False) -> dict:
        return sindi_server_stats(self.handle, reset)

    def close(self):
        if getattr(self, "handle", None):
            sindi_server_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
