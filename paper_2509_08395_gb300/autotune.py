"""Self-tuning of the search: window size (lambda), scan block shape and reorder pool (gamma).

The paper tunes lambda with a CPU cache model (Sec. 3.4) and gamma by grid
search (App. E). On the GPU neither cache model carries over, so everything is
measured on the device:

  1. exact reference: an unpruned index (alpha = 1) searched without
     reordering returns the exact top-k (FP32 accumulation of the same
     products), the yardstick for Recall@k;
  2. for every candidate window, the pruned index is built and the smallest
     gamma of the grid that reaches the recall target is found;
  3. at that gamma every (schedule, block shape) pair is timed with CUDA
     events on the sample queries; the fastest configuration that meets the
     target wins.

Windows default to the powers of two the shared-memory window allows, plus
the windows that give one or two windows per SM (sigma a multiple of the SM
count). Results can be cached in a JSON file keyed by the workload shape and
the GPU.
"""
from __future__ import annotations

import json
import os
import time

import numpy as np

from . import sindi


def _recall(found: np.ndarray, truth: np.ndarray) -> float:
    hits = 0
    for f, t in zip(found, truth):
        hits += len(set(f.tolist()) & set(t.tolist()))
    return hits / max(1, truth.size)


def _time_search(idx, q, k, gamma, mode, block, repeats):
    import torch

    ids, sc = idx.search(*q, k=k, gamma=gamma, mode=mode, block=block)  # warm
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    best = float("inf")
    for _ in range(repeats):
        e0.record()
        idx.search(*q, k=k, gamma=gamma, mode=mode, block=block, out=(ids, sc))
        e1.record()
        torch.cuda.synchronize()
        best = min(best, e0.elapsed_time(e1))
    n_q = q[0].shape[0] - 1
    return n_q / (best / 1000.0), ids


def default_windows(n_docs: int, sm_count: int):
    ws = {w for w in (2048, 4096, 8192, 16384, 32768) if w <= max(2048, n_docs)}
    for per_sm in (1, 2):
        w = -(-n_docs // (sm_count * per_sm))
        w = ((w + 31) // 32) * 32
        if 256 <= w <= 32768:
            ws.add(w)
    return sorted(ws)


def autotune(indptr, indices, values, dim: int, q_indptr, q_indices, q_values, k: int, alpha: float,
             recall_target: float = 0.99, windows=None, gammas=(100, 200, 300, 500, 750, 1000, 1500, 2000, 4000),
             blocks=(0, 1, 256, 512, 1024), modes=("plain", "batched"), value_dtype: str = "f32", repeats: int = 3,
             cache: str | None = None, alphas=None) -> dict:
    """Tune (window, gamma, schedule, block) on device tensors of documents and sample queries; with
    `alphas`, the pruning ratio too (each alpha is tried at every window).

    Returns the chosen configuration and the table of every measurement."""
    alphas = [float(alpha)] if alphas is None else [float(a) for a in alphas]
    import torch

    dev = q_indptr.device
    props = torch.cuda.get_device_properties(dev)
    n_docs = int(indptr.shape[0] - 1)
    key = json.dumps([n_docs, int(dim), int(indices.shape[0]), alphas, int(k), float(recall_target),
                      value_dtype, props.name, int(q_indptr.shape[0] - 1)])
    if cache and os.path.exists(cache):
        with open(cache) as f:
            book = json.load(f)
        if key in book:
            return book[key]
    if windows is None:
        windows = default_windows(n_docs, props.multi_processor_count)
    q = (q_indptr, q_indices, q_values)
    t0 = time.perf_counter()
    with sindi.Index(indptr, indices, values, dim, window=max(windows), alpha=1.0) as exact:
        truth, _ = exact.search(*q, k=k, gamma=0, mode="batched")
        truth = truth.cpu().numpy().view(np.uint32)
    table = []
    best = None
    for a in alphas:
        for w in windows:
            with sindi.Index(indptr, indices, values, dim, window=w, alpha=a, value_dtype=value_dtype) as idx:
                chosen = None
                for g in gammas:
                    if g < k:
                        continue
                    ids, _ = idx.search(*q, k=k, gamma=g, mode="batched")
                    r = _recall(ids.cpu().numpy().view(np.uint32), truth)
                    table.append({"alpha": a, "window": w, "gamma": g, "recall": r})
                    if r >= recall_target:
                        chosen = (g, r)
                        break
                if chosen is None:
                    continue
                g, r = chosen
                for mode in modes:
                    for b in blocks:
                        qps, _ = _time_search(idx, q, k, g, mode, b, repeats)
                        row = {"alpha": a, "window": w, "gamma": g, "recall": r, "mode": mode, "block": b,
                               "qps": qps}
                        table.append(row)
                        if best is None or qps > best["qps"]:
                            best = dict(row)
    result = {"choice": best, "recall_target": recall_target, "table": table,
              "seconds": time.perf_counter() - t0, "gpu": props.name}
    if cache:
        book = {}
        if os.path.exists(cache):
            with open(cache) as f:
                book = json.load(f)
        book[key] = result
        with open(cache, "w") as f:
            json.dump(book, f, indent=1)
    return result
