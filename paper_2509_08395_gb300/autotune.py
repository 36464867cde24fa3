"""Self-tuning of the search: window size (lambda), scan block shape, queries per scan block and reorder
pool (gamma).

The paper tunes lambda with a cache model (Sec. 3.4: a double power law in
lambda, one term for the random accesses to the score array that grow with
the window, one for the list switches that shrink with it) and gamma by grid
search (App. E). The CPU cache behind that model does not carry over, but its
shape does: per query, a GPU pays a fixed cost per window (offsets, term
table, the window's cut) and a per-slot and per-posting cost that grows with
the window (fewer blocks fit an SM). So the same double power law, fitted to
measured times at a few anchor windows, serves as a prior that narrows the
windows worth measuring (`window_model`). Everything else is measured on the
device:

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
count); with `window_prior` only those nearest the fitted optimum are
measured. Results can be cached in a JSON file keyed by the workload shape and
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


def _time_search(idx, q, k, gamma, mode, block, repeats, group=1):
    import torch

    ids, sc = idx.search(*q, k=k, gamma=gamma, mode=mode, block=block, group=group)  # warm
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    best = float("inf")
    for _ in range(repeats):
        e0.record()
        idx.search(*q, k=k, gamma=gamma, mode=mode, block=block, out=(ids, sc), group=group)
        e1.record()
        torch.cuda.synchronize()
        best = min(best, e0.elapsed_time(e1))
    n_q = q[0].shape[0] - 1
    return n_q / (best / 1000.0), ids


def fit_window_model(lams, times, exps=np.linspace(0.05, 2.0, 40)):
    """Least-squares fit of T(lambda) = c_rand lambda^a + c_evict lambda^-b + c0 (Sec. 3.4) to measured times.

    The exponents (a, b) are searched on a grid; for each pair the coefficients solve a non-negative linear
    least-squares problem (every term a cost). Returns the fit and lambda* = (c_evict b / (c_rand a))^(1/(a+b)),
    the minimum of the fitted curve (None when one of the two terms vanishes)."""
    from scipy.optimize import nnls

    lam = np.asarray(lams, np.float64)
    t = np.asarray(times, np.float64)
    best = None
    for a in exps:
        for b in exps:
            M = np.stack([lam ** a, lam ** -b, np.ones_like(lam)], axis=1)
            coef, res = nnls(M, t)
            if best is None or res < best[0]:
                best = (res, a, b, coef)
    res, a, b, (c_rand, c_evict, c0) = best
    lam_star = None
    if c_rand > 0 and c_evict > 0:
        lam_star = float((c_evict * b / (c_rand * a)) ** (1.0 / (a + b)))
    return {"a": float(a), "b": float(b), "c_rand": float(c_rand), "c_evict": float(c_evict), "c0": float(c0),
            "residual": float(res), "lambda_star": lam_star}


def windows_near(lam_star, candidates, n: int = 3):
    """The n candidate windows closest to lambda* on a log scale (all of them when there is no optimum)."""
    if lam_star is None:
        return sorted(candidates)
    return sorted(sorted(candidates, key=lambda w: abs(np.log(w / lam_star)))[:n])


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
             cache: str | None = None, alphas=None, groups=(1, 2, 4), window_prior: bool = False,
             prior_anchors=(2048, 4096, 8192, 16384, 32768)) -> dict:
    """Tune (window, gamma, schedule, block, queries per batched scan block) on device tensors of documents and
    sample queries; with `alphas`, the pruning ratio too (each alpha is tried at every window). With
    `window_prior`, the batched search's time at the anchor windows is fitted with the double power law of
    Sec. 3.4 and only the windows nearest its optimum are tuned.

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
    model = None
    if window_prior:
        anchors = [w for w in prior_anchors if w <= max(2048, n_docs)]
        times = []
        for w in anchors:
            with sindi.Index(indptr, indices, values, dim, window=w, alpha=alphas[0], value_dtype=value_dtype) as idx:
                qps, _ = _time_search(idx, q, k, min(max(k, 500), max(gammas)), "batched", 0, repeats)
                times.append(1.0 / qps)
        model = fit_window_model(anchors, times)
        model["anchors"] = anchors
        model["seconds_per_query"] = times
        windows = windows_near(model["lambda_star"], windows)
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
                        for grp in (groups if mode == "batched" and b in (0, 512, 1024) else (1,)):
                            qps, _ = _time_search(idx, q, k, g, mode, b, repeats, grp)
                            row = {"alpha": a, "window": w, "gamma": g, "recall": r, "mode": mode, "block": b,
                                   "group": grp, "qps": qps}
                            table.append(row)
                            if best is None or qps > best["qps"]:
                                best = dict(row)
    result = {"choice": best, "recall_target": recall_target, "table": table, "window_model": model,
              "recall_vs": "GPU exact search (alpha = 1, gamma = 0)",
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
