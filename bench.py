"""Benchmark of the SINDI search hot path on GB300.

One step = one pass of the search over the workload's query batch (every query:
window scan + window top-gamma, cross-window merge, exact rerank), with the
index and the queries resident in HBM. The index build runs once before the
timed region and is reported separately (build_ms).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gb300|reference]
                    [--workload pruned-1m] [--mode plain|batched]

Under torchrun (N > 1) every rank searches its own share of queries against a
replica of the index (queries are independent: weak scaling, no collective on
the data path); the barrier and the max over ranks use torch.distributed.
"""
from __future__ import annotations

import argparse
import ctypes
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import datagen  # noqa: E402

L2_BYTES = 129 * 1024 * 1024
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
FALLBACK_HBM_GBS = 6800.0
NOMINAL_HBM_GBS = 8000.0


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=5)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", choices=["gb300", "reference"], default="gb300")
    p.add_argument("--workload", default="pruned-1m")
    p.add_argument("--mode", choices=["plain", "batched"], default="plain")
    p.add_argument("--window", type=int, default=0, help="0 = the workload's window")
    p.add_argument("--block", type=int, default=0, help="scan block shape (sindi_search_params.block_threads)")
    p.add_argument("--group", type=int, default=0, help="batched schedule: queries per scan block")
    p.add_argument("--accum", choices=["auto", "f32", "fixed32"], default="auto",
                   help="score window of the coarse scan (sindi_search_params.accumulator)")
    p.add_argument("--queries", type=int, default=0, help="0 = the workload's query count")
    p.add_argument("--cpu-seconds", type=float, default=12.0, help="bound of the oracle sample")
    p.add_argument("--value-dtype", choices=["f32", "f16", "f8"], default=None,
                   help="posting value type of the main index (default: the workload's)")
    p.add_argument("--no-forms", action="store_true", help="skip the batched / low-precision / serving side lines")
    p.add_argument("--ablation", action="store_true",
                   help="add the pruning-method ablation (mass / vector-number / list / mass+list) of the workload")
    p.add_argument("--sparsity-sweep", action="store_true",
                   help="add the uniform-random sparsity sweep (1M docs x d in 10k..100k), autotuned to recall 0.99")
    p.add_argument("--serve-seconds", type=float, default=2.0, help="length of each offered load's schedule")
    p.add_argument("--no-scale", action="store_true",
                   help="skip the full-size side legs of configs 3-5 (8.8M and 25M documents)")
    p.add_argument("--scale-steps", type=int, default=3, help="timed graph launches per full-size leg")
    p.add_argument("--scale-queries", type=int, default=0, help="0 = every query of configs 3-5 (10,000)")
    p.add_argument("--scale-serve-sweep", default="0.25,0.5,0.75,0.9,1.1",
                   help="offered loads of the serve-25m serving leg (fractions of its batched capacity)")
    p.add_argument("--serve-sweep", default=None,
                   help="comma-separated offered loads (fractions of batched QPS) for the serving leg "
                        "(default 0.25,0.5,0.75,0.9,1.1)")
    return p.parse_args()


# ---------------------------------------------------------------------------
def dist_setup(n):
    import torch

    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch.distributed as dist

        backend = "nccl" if torch.cuda.is_available() else "gloo"
        if torch.cuda.is_available():
            torch.cuda.set_device(local)
        dist.init_process_group(backend)
    elif torch.cuda.is_available():
        torch.cuda.set_device(0)
    return rank, ws, local


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist

        dist.barrier()


def rank_queries(w, rank, ws):
    """Weak scaling: the global query set holds the workload's queries once per rank, and every rank
    searches its contiguous share as CSR (rank 0's share is the workload's own query set)."""
    from paper_2509_08395_gb300.shard import shard_range

    per_rank = w.queries.n_rows
    gqp, gqx, gqv = datagen.queries(w.scaled(n_queries=per_rank * ws))
    q_lo, q_hi = shard_range(per_rank * ws, rank, ws)
    qp = gqp[q_lo: q_hi + 1] - gqp[q_lo]
    qx = np.ascontiguousarray(gqx[gqp[q_lo]: gqp[q_hi]])
    qv = np.ascontiguousarray(gqv[gqp[q_lo]: gqp[q_hi]])
    return qp, qx, qv


def max_over_ranks(x, ws):
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist

    t = torch.tensor([x], dtype=torch.float64, device="cuda" if torch.cuda.is_available() else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


class Clocks:
    """Samples SM clocks and throttle reasons with nvidia-smi while running."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = str(gpu_index)
        try:
            import torch

            u = getattr(torch.cuda.get_device_properties(gpu_index), "uuid", None)
            if u is not None:
                self.gpu = "GPU-" + str(u)
        except Exception:
            pass
        self.proc = None
        self.path = os.path.join("/tmp", f"sindi_clocks_{os.getpid()}.csv")

    def __enter__(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"], stdout=self.f,
                                         stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            time.sleep(0.2)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.f.close()

    def summary(self):
        if self.proc is None or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        rows = []
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append((float(parts[1]), float(parts[2]), parts[4:9]))
            except ValueError:
                continue
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for _, _, flags in rows:
            for n, f in zip(names, flags[1:]):
                if f.lower() in ("active", "0x1", "1"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(r[0] for r in rows), "sm_max_mhz": max(r[1] for r in rows),
                "samples": len(rows), "reasons": sorted(reasons)}


def measured_hbm_peak():
    try:
        with open(PEAKS_FILE) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return FALLBACK_HBM_GBS, "fallback"


def profile_traffic(kernel_src_sha):
    """Per-launch DRAM bytes of the scan kernel from the committed ncu summary, if it was taken on this source."""
    path = os.path.join(ROOT, "profiles", "scan_window_pruned-1m.md")
    try:
        text = open(path).read()
    except OSError:
        return None
    m = re.search(r"source_sha256:\s*([0-9a-f]{64})", text)
    t = re.search(r"dram_bytes_per_launch:\s*([0-9.eE+]+)", text)
    if m and t and m.group(1) == kernel_src_sha:
        return float(t.group(1))
    return None


def bench_native_lib(name):
    """Path of a bench helper library (bench_native/build.py builds them), or None if it cannot be built."""
    import importlib.util

    try:
        spec = importlib.util.spec_from_file_location("sindi_bench_native_build",
                                                      os.path.join(ROOT, "bench_native", "build.py"))
        mod = importlib.util.module_from_spec(spec)
        spec.loader.exec_module(mod)
        mod.build()
    except Exception as e:  # noqa: BLE001 - the leg that needs it reports None
        print(f"bench: bench_native build failed: {e!r}", file=sys.stderr, flush=True)
    path = os.path.join(ROOT, "bench_native", "lib", name)
    return path if os.path.exists(path) else None


def scatter_peak(window: int, block: int = 512):
    """Measured FP32 shared-memory atomicAdd rate (adds/s) of this GPU: the probe library fills every SM with
    `block`-thread blocks that each add at random slots of a `window`-float shared array, as the scan does."""
    path = bench_native_lib("libsindi_probe.so")
    if path is None:
        return None
    lib = ctypes.CDLL(path)
    f = lib.sindi_probe_scatter_peak
    f.restype = ctypes.c_int
    f.argtypes = [ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32, ctypes.POINTER(ctypes.c_double),
                  ctypes.POINTER(ctypes.c_double)]
    rate, ms = ctypes.c_double(0.0), ctypes.c_double(0.0)
    rc = f(window, block, 256, ctypes.byref(rate), ctypes.byref(ms))
    return rate.value if rc == 0 else None


def scatter_forms(window: int, block: int = 512):
    """adds/s of five forms of the shared-memory scatter (bench_native/scatter_peak.cu): the scan's FP32
    atomicAdd at random slots and with the 32 lanes on 32 banks, a plain load-add-store by the warp that owns
    the slots (random, and on 32 banks), and a uint32 atomicAdd. None if the probe is unavailable."""
    path = bench_native_lib("libsindi_probe.so")
    if path is None:
        return None
    lib = ctypes.CDLL(path)
    f = lib.sindi_probe_scatter_mode
    f.restype = ctypes.c_int
    f.argtypes = [ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32, ctypes.POINTER(ctypes.c_double)]
    w = 1 << (max(32 * (block // 32), int(window)) - 1).bit_length()   # a power of two the probe accepts
    w = min(w, 32768)
    out = {"window": w, "block": block, "unit": "adds/s"}
    for mode, name in enumerate(("f32_atomic_random", "f32_atomic_banks", "owner_rmw_random", "owner_rmw_banks",
                                 "u32_atomic_random")):
        rate = ctypes.c_double(0.0)
        out[name] = rate.value if f(mode, w, block, 256, ctypes.byref(rate)) == 0 and f(
            mode, w, block, 256, ctypes.byref(rate)) == 0 else None
    return out


def _timed_qps(torch, fn, nq, reps, flush, stream):
    for _ in range(3):  # warm: a repeated plain call is recorded as a graph on its second run
        fn()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    tot = 0.0
    for _ in range(reps):
        flush.zero_()
        e0.record(stream)
        fn()
        e1.record(stream)
        torch.cuda.synchronize()
        tot += e0.elapsed_time(e1)
    return nq * reps / (tot / 1000.0)


def _recall_rows(ids, truth):
    return float(np.mean([len(set(a.tolist()) & set(b.tolist())) / max(1, len(b)) for a, b in zip(ids, truth)]))


def fp64_truth_sample(ip, ix, v, qp, qx, qv, dim, k, n=40):
    """FP64 exact top-k (the oracle's brute force, Definition 3) of n query rows spread over the batch, for
    Recall@k against FP64 exact. Returns (D, Q, {row: (ids, scores)})."""
    import oracle

    D = oracle.Dataset(ip, ix, v, dim)
    Q = oracle.Dataset(qp, qx, qv, dim)
    rows = list(range(0, Q.n, max(1, Q.n // n)))[:n]
    return D, Q, _fp64_truth(D, Q, rows, k)


def _choice_ids(sindi, dd, qd, dim, k, choice):
    """Result ids of the autotuner's chosen configuration on the given queries."""
    with sindi.Index(*dd, dim, window=choice["window"], alpha=choice["alpha"]) as idx:
        ids, _ = idx.search(*qd, k=k, gamma=choice["gamma"], mode=choice["mode"], block=choice["block"],
                            group=choice.get("group", 1))
        idx.check()
        return ids.cpu().numpy().view(np.uint32)


def pruning_ablation(sindi, torch, dev, w, ip, ix, v, q_dev, nq, steps, flush, stream, fp64=None):
    """The pruning methods of Sec. 4.1 on the workload (ablation of Sec. 5): postings kept, Recall@k with the
    workload's reorder depth against FP64 exact on sampled queries (`fp64` = (D, Q, truth)) and, on every
    query, against the exact GPU search (alpha = 1, no reorder; a proxy), and plain-schedule QPS."""
    grid = ([("mass", 0, a) for a in (0.4, 0.5, 0.6)] + [("vector_number", n, 1.0) for n in (15, 25, 40)] +
            [("list", n, 1.0) for n in (2000, 5000, 10000)] + [("mass_list", n, w.alpha) for n in (2000, 5000)])
    dip, dix, dv = (torch.from_numpy(a).to(dev) for a in (ip, ix, v))
    with sindi.Index(dip, dix, dv, w.dim, window=w.window, alpha=1.0) as exact:
        truth, _ = exact.search(*q_dev, k=w.k, gamma=0, mode="batched")
        truth = truth.cpu().numpy().view(np.uint32)
    rows = []
    for prune, n, a in grid:
        with sindi.Index(dip, dix, dv, w.dim, window=w.window, alpha=a, prune=prune, prune_n=n) as idx:
            ids = torch.empty((nq, w.k), dtype=torch.int32, device=dev)
            sc = torch.empty((nq, w.k), dtype=torch.float32, device=dev)
            qps = _timed_qps(torch, lambda: idx.search(*q_dev, k=w.k, gamma=w.gamma, mode="plain", out=(ids, sc)),
                             nq, steps, flush, stream)
            idx.check()
            hids = ids.cpu().numpy().view(np.uint32)
            row = {"prune": prune, "prune_n": n, "alpha": a, "postings": idx.info["postings"],
                   "recall_at_k_proxy": _recall_rows(hids, truth), "qps": qps, "gamma": w.gamma}
            if fp64 is not None:
                row["recall_at_k_vs_fp64"], row["recall_at_k_tie_aware_vs_fp64"] = _recall_vs_fp64(hids, fp64[2],
                                                                                                  fp64[0], fp64[1])
            rows.append(row)
    return {"rows": rows, "recall_vs": "FP64 oracle brute force on sampled queries (recall_at_k_vs_fp64); the "
                                       "proxy is the exact GPU search (alpha = 1, gamma = 0) on every query",
            "schedule": "plain"}


def sparsity_sweep(sindi, torch, dev, steps, flush, stream, dims=(10, 30, 50, 70, 100)):
    """Sec. 5's uniform-random sparsity sweep: for each d, the autotuned (alpha, window, gamma, schedule) with
    the highest QPS at Recall@50 >= 0.99 against the exact GPU search (the tuner's proxy), that choice's
    Recall@50 against FP64 exact on sampled queries, and the exact search's own QPS."""
    import datagen
    from paper_2509_08395_gb300 import autotune

    out = []
    for d in dims:
        w = datagen.WORKLOADS[f"uniform-1m-d{d}k"]
        ip, ix, v = datagen.docs(w)
        qp, qx, qv = datagen.queries(w)
        dd = [torch.from_numpy(a).to(dev) for a in (ip, ix, v)]
        qd = [torch.from_numpy(a).to(dev) for a in (qp, qx, qv)]
        nq = len(qp) - 1
        t0 = time.perf_counter()
        tuned = autotune.autotune(*dd, w.dim, *qd, k=w.k, alpha=w.alpha, alphas=(0.3, 0.5, 0.7, 0.9),
                                  recall_target=0.99, blocks=(512,), groups=(1,), window_prior=True)
        with sindi.Index(*dd, w.dim, window=w.window, alpha=1.0) as exact:
            exact_qps = _timed_qps(torch, lambda: exact.search(*qd, k=w.k, gamma=0, mode="batched"), nq, steps,
                                   flush, stream)
            postings_exact = exact.info["postings"]
        row = {"workload": w.name, "dim": w.dim, "choice": tuned["choice"], "exact_batched_qps": exact_qps,
               "postings_unpruned": postings_exact, "window_model": tuned["window_model"],
               "seconds": time.perf_counter() - t0}
        if tuned["choice"]:
            D, Q, truth = fp64_truth_sample(ip, ix, v, qp, qx, qv, w.dim, w.k, n=20)
            row["recall_at_k_vs_fp64"], row["recall_at_k_tie_aware_vs_fp64"] = _recall_vs_fp64(
                _choice_ids(sindi, dd, qd, w.dim, w.k, tuned["choice"]), truth, D, Q)
            row["recall_sample"] = f"{len(truth)} queries, FP64 oracle brute force"
        out.append(row)
        del dd, qd
    return out


def source_sha():
    """sha256 of the scan's sources without their comments and blank lines (a comment edit does not change
    the kernel an ncu capture measured)."""
    h = hashlib.sha256()
    for f in ("search.cu", "primitives.cuh", "common.cuh"):
        with open(os.path.join(ROOT, "paper_2509_08395_gb300", "csrc", f), encoding="utf-8") as fh:
            text = fh.read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        text = re.sub(r"//[^\n]*", "", text)
        lines = [ln.rstrip() for ln in text.splitlines() if ln.strip()]
        h.update("\n".join(lines).encode())
    return h.hexdigest()


def postings_touched(seg, sigma, dim, qp, qx):
    """Per query: sum over its terms of |I_j| (all windows) = postings the scan reads."""
    j = np.arange(dim, dtype=np.int64)
    lens = seg[(j + 1) * sigma].astype(np.int64) - seg[j * sigma].astype(np.int64)
    out = np.empty(len(qp) - 1, np.int64)
    for r in range(len(qp) - 1):
        out[r] = lens[qx[qp[r]:qp[r + 1]]].sum()
    return out


# ---------------------------------------------------------------------------
class _LoadResult(ctypes.Structure):
    _fields_ = [("offered_qps", ctypes.c_double), ("achieved_qps", ctypes.c_double), ("seconds", ctypes.c_double),
                ("requests", ctypes.c_int64), ("failed", ctypes.c_int64), ("p50_ms", ctypes.c_double),
                ("p99_ms", ctypes.c_double), ("max_ms", ctypes.c_double), ("mean_ms", ctypes.c_double),
                ("server_p50_ms", ctypes.c_double), ("server_p99_ms", ctypes.c_double),
                ("lag_p99_ms", ctypes.c_double), ("lag_max_ms", ctypes.c_double)]


def serve_open_loop(sindi, idx, qp, qx, qv, k, gamma, offered_qps, seconds, seed=7, max_batch=128, slots=8):
    """Open-loop Poisson arrivals into the continuous-batching server, driven by the native load generator
    (bench_native/serve_load.c: a submitting thread on the schedule and a polling thread, no GIL). Latency runs
    from each request's scheduled arrival to its results on the host."""
    path = bench_native_lib("libsindi_load.so")
    if path is None:
        raise RuntimeError("bench_native/lib/libsindi_load.so could not be built")
    gen = ctypes.CDLL(path)
    gen.sindi_load_open_loop.restype = ctypes.c_int
    gen.sindi_load_open_loop.argtypes = [ctypes.c_void_p] * 6 + [ctypes.c_int64, ctypes.c_uint32, ctypes.c_double,
                                                                 ctypes.c_double, ctypes.c_uint64,
                                                                 ctypes.POINTER(_LoadResult)]
    lib = sindi.load()
    submit = ctypes.cast(lib.sindi_server_submit, ctypes.c_void_p)
    poll = ctypes.cast(lib.sindi_server_poll, ctypes.c_void_p)
    qp = np.ascontiguousarray(qp, np.int64)
    qx = np.ascontiguousarray(qx, np.int32)
    qv = np.ascontiguousarray(qv, np.float32)
    res = _LoadResult()
    with sindi.Server(idx, k=k, gamma=gamma, max_batch=max_batch, max_slots=slots, max_wait_us=200,
                      max_query_nnz=int(np.diff(qp).max())) as srv:
        rc = gen.sindi_load_open_loop(ctypes.c_void_p(srv.handle), submit, poll, qp.ctypes.data, qx.ctypes.data,
                                      qv.ctypes.data, len(qp) - 1, k, float(offered_qps), float(seconds), seed,
                                      ctypes.byref(res))
        st = srv.stats()
    if rc != 0:
        raise RuntimeError("sindi_load_open_loop refused its arguments")
    out = {f: getattr(res, f) for f, _ in _LoadResult._fields_}
    out.update({"mean_batch": st["mean_batch"], "slots": st["n_slots"], "peak_in_flight": st["peak_in_flight"],
                "max_batch": max_batch, "latency_from": "scheduled arrival (open loop)"})
    return out


def serve_sweep(sindi, idx, qp, qx, qv, k, gamma, capacity_qps, fractions, seconds):
    """Offered loads as fractions of the batched schedule's measured capacity, up to and past saturation."""
    return [serve_open_loop(sindi, idx, qp, qx, qv, k, gamma, f * capacity_qps, seconds, seed=7 + i)
            for i, f in enumerate(fractions)]


# ---------------------------------------------------------------------------
# Configs 3-5 of the workload list at full size (side legs of the default run)
def _fp64_truth(D, Q, rows, k):
    """FP64 exact top-k (Definition 3) of the sampled query rows, one row per host thread (the oracle's C calls
    release the GIL)."""
    import concurrent.futures

    import oracle

    with concurrent.futures.ThreadPoolExecutor(max_workers=os.cpu_count() or 1) as ex:
        res = list(ex.map(lambda r: oracle.brute_force(D, Q, r, k), rows))
    return dict(zip(rows, res))


def _recall_vs_fp64(ids, truth, D, Q):
    import oracle

    plain = [oracle.recall(ids[r], t[0]) for r, t in truth.items()]
    tie = [oracle.recall_tie_aware(ids[r], t[0], t[1], D, Q, r) for r, t in truth.items()]
    return float(np.mean(plain)), float(np.mean(tie))


def _score_errors(idx, torch, dev, w, ip, ix, v, qp, qx, qv, D, Q, rows, final_ids, final_sc):
    """Max relative score error against FP64 on sampled rows: coarse (the GPU's gamma = 0 scores, quantised
    postings, against the FP64 dot product of the same document's alpha-mass subvector with the query), in
    the FP32 window (the default at gamma = 0) and in the fixed-point window (the default when the search
    reorders), and final (the reordered FP32 scores against exact delta)."""
    import oracle

    sub = [torch.from_numpy(a).to(dev) for a in (np.concatenate([[0], np.cumsum([qp[r + 1] - qp[r] for r in rows])]),
                                                  np.concatenate([qx[qp[r]:qp[r + 1]] for r in rows]),
                                                  np.concatenate([qv[qp[r]:qp[r + 1]] for r in rows]))]
    coarse = {}
    for accum in ("f32", "fixed32"):
        cids, csc = idx.search(*sub, k=w.k, gamma=0, mode="batched", accum=accum)
        coarse[accum] = (cids.cpu().numpy().view(np.uint32), csc.cpu().numpy())
    ce = {"f32": 0.0, "fixed32": 0.0}
    fe = 0.0
    for n, r in enumerate(rows):
        qd = dict(zip(qx[qp[r]:qp[r + 1]].tolist(), qv[qp[r]:qp[r + 1]].astype(np.float64).tolist()))
        for accum, (cids, csc) in coarse.items():
            for i, sc in zip(cids[n], csc[n]):
                a, b = ip[i], ip[i + 1]
                pos = oracle.alpha_mass(ix[a:b], v[a:b], w.alpha)
                ref = sum(qd.get(int(j), 0.0) * float(x) for j, x in zip(ix[a:b][pos], v[a:b][pos]))
                if ref != 0.0:
                    ce[accum] = max(ce[accum], abs(float(sc) - ref) / abs(ref))
        for i, sc in zip(final_ids[r], final_sc[r]):
            ex = oracle.inner_product(D, int(i), Q, r)
            if ex != 0.0:
                fe = max(fe, abs(float(sc) - ex) / abs(ex))
    return {"coarse_max_rel_err_vs_fp64": ce["f32"], "coarse_fixed_window_max_rel_err_vs_fp64": ce["fixed32"],
            "final_max_rel_err_vs_fp64": fe, "score_error_queries": len(rows)}


def plan_leg(sindi, torch, dev, w, dd, qp, qx, qv, dtype, steps, warmup, flush, stream, D, Q, truth, host_docs):
    """One config at full size: build, then every query of the batch in one graph launch (sindi_plan), timed with
    CUDA events on the launching stream; recall@k against FP64 on the sampled rows of `truth`."""
    ip, ix, v = host_docs
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    idx = sindi.Index(*dd, w.dim, window=w.window, alpha=w.alpha, value_dtype=dtype)
    torch.cuda.synchronize()
    build_ms = 1000 * (time.perf_counter() - t0)
    try:
        q_dev = [torch.from_numpy(a).to(dev) for a in (qp, qx, qv)]
        nq = len(qp) - 1
        with sindi.Plan(idx, *q_dev, k=w.k, gamma=w.gamma) as plan:
            for _ in range(warmup):
                plan.launch(stream.cuda_stream)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            ms = []
            for _ in range(steps):
                flush.zero_()
                e0.record(stream)
                plan.launch(stream.cuda_stream)
                e1.record(stream)
                torch.cuda.synchronize()
                ms.append(e0.elapsed_time(e1))
            idx.check()
            ids = plan.out[0].cpu().numpy().view(np.uint32)
            sc = plan.out[1].cpu().numpy()
        step_ms = float(np.mean(ms))
        info = idx.info
        seg = idx.export(parts=("seg",))["seg"]
        touched = postings_touched(seg, info["n_windows"], w.dim, qp, qx)
        vbytes = {0: 4, 1: 2, 2: 1}[info["value_dtype"]]
        scan_bytes = float(touched.sum() * (2 + vbytes) + np.diff(qp).sum() * (info["n_windows"] * 8 + 8))
        recall, recall_tie = _recall_vs_fp64(ids, truth, D, Q)
        errs = _score_errors(idx, torch, dev, w, ip, ix, v, qp, qx, qv, D, Q, sorted(truth)[:4], ids, sc)
        out = {"workload": w.name, "posting_dtype": dtype, "n_docs": w.docs.n_rows, "dim": w.dim, "queries": nq,
               "k": w.k, "gamma": w.gamma, "alpha": w.alpha, "window": info["window"],
               "n_windows": info["n_windows"], "postings": info["postings"], "build_ms": build_ms,
               "qps": nq / (step_ms / 1000.0), "ms_per_step": step_ms, "steps": steps,
               "schedule": "batched, one graph launch per step (sindi_plan)",
               "recall_at_k_vs_fp64": recall, "recall_at_k_tie_aware_vs_fp64": recall_tie,
               "recall_sample": f"{len(truth)} queries evenly spread, FP64 oracle brute force",
               "postings_per_query": float(touched.mean()),
               "scan_bytes_per_s": scan_bytes / (step_ms / 1000.0),
               "scan_bytes_basis": "posting bytes (id + value) of every query's lists plus offsets, per step "
                                   "time (lists shared by queries are read once from HBM and served from L2)",
               "adds_per_s": float(touched.sum()) / (step_ms / 1000.0)}
        out.update(errs)
        return out, idx
    except Exception:
        idx.close()
        raise


def scale_legs(sindi, torch, dev, args, flush, stream, base_qps_fn=None):
    """Configs 3 (batched, 8.8M docs, 10k uneven queries), 4 (FP16 / FP8 postings on that index, gamma 1,000)
    and 5 (25M docs x 250k dims, FP16, open-loop serving) at full size."""
    import oracle

    out = {}
    n_truth = 16
    # configs 3 and 4 share their 8.8M documents
    w3, w4 = datagen.WORKLOADS["batched-8.8m"], datagen.WORKLOADS["lowprec-8.8m"]
    t0 = time.perf_counter()
    ip, ix, v = datagen.docs(w3)
    gen_s = time.perf_counter() - t0
    dd = [torch.from_numpy(a).to(dev) for a in (ip, ix, v)]
    D = oracle.Dataset(ip, ix, v, w3.dim)
    # the lowprec-8.8m queries also on FP32 postings: the reduced-precision legs' baseline in the same schedule
    for w, dtypes in ((w3, ("f32",)), (w4, ("f32", "f16", "f8"))):
        qp, qx, qv = datagen.queries(w)
        if args.scale_queries:
            n = min(args.scale_queries, len(qp) - 1)
            qp, qx, qv = qp[: n + 1], qx[: qp[n]], qv[: qp[n]]
        Q = oracle.Dataset(qp, qx, qv, w.dim)
        rows = list(range(0, Q.n, max(1, Q.n // n_truth)))[:n_truth]
        truth = _fp64_truth(D, Q, rows, w.k)
        for dt in dtypes:
            leg, idx = plan_leg(sindi, torch, dev, w, dd, qp, qx, qv, dt, args.scale_steps, 1, flush, stream, D, Q,
                                truth, (ip, ix, v))
            idx.close()
            leg["docs_generated_s"] = gen_s
            out[f"{w.name}/{dt}"] = leg
    del dd, D
    torch.cuda.empty_cache()
    # serve-25m: 25M documents, FP16 postings; batched capacity, then open-loop serving up to saturation
    w5 = datagen.WORKLOADS["serve-25m"]
    t0 = time.perf_counter()
    ip, ix, v = datagen.docs(w5)
    gen_s = time.perf_counter() - t0
    dd = [torch.from_numpy(a).to(dev) for a in (ip, ix, v)]
    D = oracle.Dataset(ip, ix, v, w5.dim)
    qp, qx, qv = datagen.queries(w5)
    if args.scale_queries:
        n = min(args.scale_queries, len(qp) - 1)
        qp, qx, qv = qp[: n + 1], qx[: qp[n]], qv[: qp[n]]
    Q = oracle.Dataset(qp, qx, qv, w5.dim)
    rows = list(range(0, Q.n, max(1, Q.n // 8)))[:8]
    truth = _fp64_truth(D, Q, rows, w5.k)
    leg, idx = plan_leg(sindi, torch, dev, w5, dd, qp, qx, qv, w5.value_dtype, args.scale_steps, 1, flush, stream,
                        D, Q, truth, (ip, ix, v))
    del dd
    try:
        leg["docs_generated_s"] = gen_s
        fractions = [float(f) for f in args.scale_serve_sweep.split(",")]
        leg["serving"] = {"capacity_qps": leg["qps"], "capacity_from": "the batched plan leg above",
                          "points": serve_sweep(sindi, idx, qp, qx, qv, w5.k, w5.gamma, leg["qps"], fractions,
                                                args.serve_seconds)}
    finally:
        idx.close()
    out[f"{w5.name}/{w5.value_dtype}"] = leg
    return out


def cpu_oracle_sample(w, ip, ix, v, qp, qx, qv, budget_s, gpu_ids=None, k=None):
    """The oracle as it stands, single-threaded, on a bounded sample of the workload's queries.

    Returns (qps, n_sampled, recall list vs FP64 brute force for the GPU ids if given, the all-cores
    baseline, tie-aware recall list)."""
    import oracle

    D = oracle.Dataset(ip, ix, v, w.dim)
    Q = oracle.Dataset(qp, qx, qv, w.dim)
    I = oracle.Index(D, window=w.window, alpha=w.alpha)
    done, t0 = 0, time.perf_counter()
    elapsed = 0.0
    while done < Q.n and elapsed < budget_s:
        I.search(Q, done, k=w.k, gamma=w.gamma)
        done += 1
        elapsed = time.perf_counter() - t0
    qps = done / elapsed if elapsed > 0 else 0.0
    # the same oracle on every host core: one query per thread at a time (the oracle's C search holds no
    # shared state and ctypes releases the GIL during it), on the next queries, for about half the budget
    import concurrent.futures
    import threading

    cores = os.cpu_count() or 1
    lock = threading.Lock()
    nxt = [done % max(1, Q.n)]
    stop_at = time.perf_counter() + budget_s / 2

    def worker(_):
        n = 0
        while n == 0 or time.perf_counter() < stop_at:
            with lock:
                r = nxt[0] % Q.n  # the queries in turn, from where the single-thread pass stopped
                nxt[0] += 1
            I.search(Q, r, k=w.k, gamma=w.gamma)
            n += 1
        return n

    t_all = time.perf_counter()
    with concurrent.futures.ThreadPoolExecutor(max_workers=cores) as ex:
        n_all = sum(ex.map(worker, range(cores)))
    el_all = time.perf_counter() - t_all
    all_cores = {"value": n_all / el_all if el_all > 0 else 0.0, "unit": "queries/s", "cores": cores,
                 "kind": "oracle", "sample": f"{n_all} queries of {w.name} on {cores} threads, one query per thread "
                                             f"at a time (about {el_all:.0f} s)"}
    recalls, recalls_tie = [], []
    if gpu_ids is not None:
        # FP64 exact ground truth on an evenly spread sample of the same queries
        t1 = time.perf_counter()
        step = max(1, Q.n // 40)
        for r in range(0, Q.n, step):
            truth, tsc = oracle.brute_force(D, Q, r, k)
            recalls.append(oracle.recall(gpu_ids[r], truth))
            recalls_tie.append(oracle.recall_tie_aware(gpu_ids[r], truth, tsc, D, Q, r))
            if time.perf_counter() - t1 > budget_s:
                break
    return qps, done, recalls, all_cores, recalls_tie


def run_reference(args):
    """--impl reference: the FP64 oracle on the host cores, bounded samples of the workload per step."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle

    w = datagen.WORKLOADS[args.workload]
    if args.window:
        w = w.scaled(window=args.window)
    ip, ix, v = datagen.docs(w)
    qp, qx, qv = datagen.queries(w)
    D = oracle.Dataset(ip, ix, v, w.dim)
    Q = oracle.Dataset(qp, qx, qv, w.dim)
    I = oracle.Index(D, window=w.window, alpha=w.alpha)
    per_step = 4
    nxt = 0
    for _ in range(args.warmup):
        for _ in range(per_step):
            I.search(Q, nxt % Q.n, k=w.k, gamma=w.gamma)
            nxt += 1
    t0 = time.perf_counter()
    for _ in range(args.steps):
        for _ in range(per_step):
            I.search(Q, nxt % Q.n, k=w.k, gamma=w.gamma)
            nxt += 1
    el = time.perf_counter() - t0
    qps = args.steps * per_step / el
    line = {
        "impl": "reference", "metric": "QPS at Recall@50>=0.99 (sparse MIPS, top-50)", "value": qps,
        "unit": "queries/s", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1000 * el / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic",
        "config": {"workload": w.name, "n_docs": w.docs.n_rows, "dim": w.dim, "k": w.k, "gamma": w.gamma,
                   "alpha": w.alpha, "window": w.window, "queries_per_step": per_step},
        "cpu_baseline": {"value": qps, "unit": "queries/s", "cores": 1, "kind": "oracle",
                         "sample": f"{args.steps * per_step} queries of {w.name}, single-threaded FP64 oracle"},
        "e2e": {"value": qps, "unit": "queries/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
        return
    import torch

    import paper_2509_08395_gb300 as sindi

    rank, ws, local = dist_setup(args.gpus)
    dev = torch.device("cuda", local)
    w = datagen.WORKLOADS[args.workload]
    if args.window:
        w = w.scaled(window=args.window)
    if args.queries:
        w = w.scaled(n_queries=args.queries)
    ip, ix, v = datagen.docs(w)
    qp, qx, qv = rank_queries(w, rank, ws)
    nq = len(qp) - 1

    t_b0 = time.perf_counter()
    dip, dix, dv = (torch.from_numpy(a).to(dev) for a in (ip, ix, v))
    torch.cuda.synchronize()
    t_b1 = time.perf_counter()
    main_dtype = args.value_dtype or w.value_dtype
    idx = sindi.Index(dip, dix, dv, w.dim, window=w.window, alpha=w.alpha, value_dtype=main_dtype)
    torch.cuda.synchronize()
    build_ms = 1000 * (time.perf_counter() - t_b1)
    h2d_docs_ms = 1000 * (t_b1 - t_b0)
    del dip, dix, dv
    info = idx.info

    q_dev = [torch.from_numpy(a).to(dev) for a in (qp, qx, qv)]
    out_ids = torch.empty((nq, w.k), dtype=torch.int32, device=dev)
    out_sc = torch.empty((nq, w.k), dtype=torch.float32, device=dev)
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)

    def step(mode, accum=None):
        idx.search(*q_dev, k=w.k, gamma=w.gamma, mode=mode, out=(out_ids, out_sc), block=args.block,
                   group=args.group if mode == "batched" else 0, accum=accum or args.accum)

    for _ in range(args.warmup):
        step(args.mode)
    idx.check()
    torch.cuda.synchronize()

    # ---- timed region: device time of K steps, L2 flushed between steps
    sindi.sindi_reset_stats(idx.handle)
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    barrier(ws)
    torch.cuda.synchronize()
    with Clocks(local) as clk:
        for e0, e1 in evs:
            flush.zero_()
            e0.record(stream)
            step(args.mode)
            e1.record(stream)
        torch.cuda.synchronize()
    barrier(ws)
    stats = sindi.sindi_get_stats(idx.handle)
    dev_ms = sum(e0.elapsed_time(e1) for e0, e1 in evs)
    dev_ms_max = max_over_ranks(dev_ms, ws)
    idx.check()
    value = ws * nq * args.steps / (dev_ms_max / 1000.0)
    launches = int(stats["launches"])

    # ---- roofline pass: CUDA events around every scan launch (same steps again)
    sindi.sindi_reset_stats(idx.handle)
    sindi.sindi_set_timing(idx.handle, True)
    for _ in range(args.steps):
        flush.zero_()
        step(args.mode)
    torch.cuda.synchronize()
    sindi.sindi_set_timing(idx.handle, False)
    st2 = sindi.sindi_get_stats(idx.handle)
    scan_ms_per_launch = st2["scan_ms"] / max(1, st2["scan_timed"])
    ex = idx.export()
    sigma = info["n_windows"]
    touched = postings_touched(ex["seg"], sigma, w.dim, qp, qx)
    vbytes = {0: 4, 1: 2, 2: 1}[info["value_dtype"]]
    nterms = np.diff(qp)
    # algorithmic bytes of one scan launch: postings (uint16 id + value) + the two offsets of every
    # (term, window) + the query's terms; a plain launch covers one query, a batched launch all of them
    per_query_bytes = touched * (2 + vbytes) + nterms * sigma * 8 + nterms * 8
    scan_launches_per_step = max(1, st2["scan_timed"] // max(1, args.steps))
    if args.mode == "plain":
        # one query per launch: its lists are the bytes the launch must read
        alg_bytes_per_launch = float(per_query_bytes.mean())
    else:
        # a launch group reads each list it touches from HBM at least once (queries holding the same term
        # share it through L2): the union of the group's lists, plus the per-query offsets and terms
        group = -(-nq // scan_launches_per_step)
        j = np.arange(w.dim, dtype=np.int64)
        list_bytes = (ex["seg"][(j + 1) * sigma].astype(np.int64) - ex["seg"][j * sigma].astype(np.int64)) * (2 + vbytes)
        per_group = []
        for g0 in range(0, nq, group):
            terms = np.unique(qx[qp[g0]:qp[min(nq, g0 + group)]])
            per_group.append(float(list_bytes[terms].sum()) +
                             float((nterms[g0:g0 + group] * (sigma * 8 + 8)).sum()))
        alg_bytes_per_launch = float(np.mean(per_group))
    achieved_gbs = alg_bytes_per_launch / (scan_ms_per_launch / 1000.0) / 1e9
    # the same bytes for every scan of the timed region over the region's time (the plain schedule runs
    # many queries' scans at once; merge and rerank share the region, so this is a lower bound)
    achieved_step_gbs = alg_bytes_per_launch * scan_launches_per_step * args.steps / (dev_ms_max / 1000.0) / 1e9
    # scatter-adds (one shared-memory atomicAdd per posting and query): the scan kernel's own rate
    # (timed pass), the whole step's rate, and the probe's measured rate of that operation on this GPU
    adds_per_s = float(touched.sum()) * args.steps / (st2["scan_ms"] / 1000.0)
    adds_per_s_step = float(touched.sum()) * args.steps / (dev_ms_max / 1000.0)
    adds_forms = scatter_forms(int(info["window"])) if rank == 0 else None
    fixed_sums = args.accum == "fixed32" or (args.accum == "auto" and w.gamma > 0)
    if fixed_sums:
        # the fixed-point window adds with a native integer atomic: its probe form is the op's peak
        adds_peak = (adds_forms or {}).get("u32_atomic_random")
        adds_peak_from = ("measured: uint32 shared-memory atomicAdd probe at random slots of a window-sized "
                          "array, every SM full (libsindi_probe), the fixed-point window's add")
    else:
        adds_peak = scatter_peak(int(info["window"]))
        adds_peak_from = ("measured: FP32 shared-memory atomicAdd probe at random slots of a window-sized array, "
                          "every SM full (libsindi_probe)")
    peak, peak_kind = measured_hbm_peak()
    sha = source_sha()

    # ---- e2e through the public C ABI with pinned host buffers (copies inside the timed region)
    h_ip = torch.from_numpy(qp).pin_memory()
    h_ix = torch.from_numpy(qx).pin_memory()
    h_v = torch.from_numpy(qv).pin_memory()
    h_ids = torch.empty((nq, w.k), dtype=torch.int32).pin_memory()
    h_sc = torch.empty((nq, w.k), dtype=torch.float32).pin_memory()
    for _ in range(max(1, args.warmup)):
        idx.search(h_ip, h_ix, h_v, k=w.k, gamma=w.gamma, mode=args.mode, out=(h_ids, h_sc), stream=stream.cuda_stream,
                   block=args.block, group=args.group if args.mode == "batched" else 0, accum=args.accum)
    barrier(ws)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        idx.search(h_ip, h_ix, h_v, k=w.k, gamma=w.gamma, mode=args.mode, out=(h_ids, h_sc), stream=stream.cuda_stream,
                   block=args.block, group=args.group if args.mode == "batched" else 0, accum=args.accum)
    torch.cuda.synchronize()
    e2e_s = max_over_ranks(time.perf_counter() - t0, ws)
    barrier(ws)
    e2e = ws * nq * args.steps / e2e_s
    h2d = int(h_ip.numel() * 8 + h_ix.numel() * 4 + h_v.numel() * 4)
    d2h = int(h_ids.numel() * 4 + h_sc.numel() * 4)
    gpu_ids = out_ids.cpu().numpy().view(np.uint32)
    assert np.array_equal(gpu_ids, h_ids.numpy().view(np.uint32)), "host-buffer results differ from device results"

    # ---- side forms on the same queries (batched schedule; FP16 / FP8 postings). The optional legs run
    # after the headline measurement; a leg that fails is reported in side_errors and the line still prints.
    side_errors = []

    def side_failed(leg, e):
        side_errors.append(f"{leg}: {type(e).__name__}: {e}")
        print(f"bench: {leg} failed: {e!r}", file=sys.stderr, flush=True)

    forms = {}
    if not args.no_forms:
        try:
            def timed(fn, reps):
                for _ in range(3):  # warm: a repeated plain call is recorded as a graph on its second run
                    fn()
                torch.cuda.synchronize()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                tot = 0.0
                for _ in range(reps):
                    flush.zero_()
                    e0.record(stream)
                    fn()
                    e1.record(stream)
                    torch.cuda.synchronize()
                    tot += e0.elapsed_time(e1)
                return nq * reps / (tot / 1000.0)

            other = "batched" if args.mode == "plain" else "plain"
            forms[other] = {"qps": timed(lambda: step(other), args.steps)}
            forms[other]["ids_equal_to_main"] = float(np.mean(out_ids.cpu().numpy().view(np.uint32)
                                                              == gpu_ids))
            if args.accum != "f32":
                # Alg. 2's FP32 score window in both schedules, for comparison with the fixed-point window
                for m in (args.mode, other):
                    forms["f32_window_" + m] = {"qps": timed(lambda: step(m, "f32"), args.steps)}
                    forms["f32_window_" + m]["ids_equal_to_main"] = float(np.mean(
                        out_ids.cpu().numpy().view(np.uint32) == gpu_ids))
            if nq <= 65535:
                # the batched search captured once as a CUDA graph: one graph launch per step
                with sindi.Plan(idx, *q_dev, k=w.k, gamma=w.gamma, accum=args.accum) as plan:
                    forms["batched_graph"] = {"qps": timed(lambda: plan.launch(stream.cuda_stream), args.steps)}
                    gids = plan.out[0].cpu().numpy().view(np.uint32)
                    forms["batched_graph"]["ids_equal_to_main"] = float(np.mean(gids == gpu_ids))
            # the autotuner on the same documents and queries
            from paper_2509_08395_gb300 import autotune

            dip, dix, dv = (torch.from_numpy(a).to(dev) for a in (ip, ix, v))
            tuned = autotune.autotune(dip, dix, dv, w.dim, *q_dev, k=w.k, alpha=w.alpha, recall_target=0.99,
                                      window_prior=True)
            forms["autotuned"] = dict(tuned["choice"] or {}, seconds=tuned["seconds"],
                                      recall_proxy_vs="GPU exact search (alpha = 1, gamma = 0), every query",
                                      window_model=tuned["window_model"])
            if tuned["choice"]:
                # re-scored below against FP64 exact on the sampled queries
                forms["autotuned"]["_ids_only"] = _choice_ids(sindi, (dip, dix, dv), q_dev, w.dim, w.k,
                                                              tuned["choice"])
            else:
                forms["autotuned"]["table"] = tuned["table"]
            del dip, dix, dv
            for dt in ("f16", "f8"):
                dip, dix, dv = (torch.from_numpy(a).to(dev) for a in (ip, ix, v))
                with sindi.Index(dip, dix, dv, w.dim, window=w.window, alpha=w.alpha, value_dtype=dt) as lp:
                    del dip, dix, dv
                    oi = torch.empty_like(out_ids)
                    os_ = torch.empty_like(out_sc)
                    # the other schedule too: reduced precision is a posting format, either schedule reads it
                    oth = "batched" if args.mode == "plain" else "plain"
                    forms[dt + "_" + oth] = {"qps": timed(lambda: lp.search(*q_dev, k=w.k, gamma=w.gamma, mode=oth,
                                                                            out=(oi, os_)), args.steps)}
                    qps = timed(lambda: lp.search(*q_dev, k=w.k, gamma=w.gamma, mode=args.mode, out=(oi, os_)),
                                args.steps)
                    lp.check()
                    # coarse scores alone (gamma = 0) of the first queries, for the quantisation error
                    n_err = min(8, nq)
                    cq = [torch.from_numpy(a).to(dev) for a in (qp[: n_err + 1], qx[: qp[n_err]], qv[: qp[n_err]])]
                    _, csc = lp.search(*cq, k=w.k, gamma=0)
                    forms[dt + "_" + args.mode] = {"qps": qps, "_ids": oi.cpu().numpy().view(np.uint32),
                                                   "_sc": os_.cpu().numpy(), "_coarse": csc.cpu().numpy()}
        except Exception as e:  # noqa: BLE001 - reported in the line
            side_failed("forms", e)
            forms = {name: f for name, f in forms.items() if "_ids" not in f and "_ids_only" not in f}

    ablation = None
    if args.ablation and rank == 0:
        try:
            ablation = pruning_ablation(sindi, torch, dev, w, ip, ix, v, q_dev, nq, args.steps, flush, stream,
                                        fp64_truth_sample(ip, ix, v, qp, qx, qv, w.dim, w.k))
        except Exception as e:  # noqa: BLE001 - reported in the line
            side_failed("pruning_ablation", e)
    sweep = None
    if rank == 0 and (args.sparsity_sweep or not args.no_scale):
        try:
            # the whole sweep when asked for; otherwise its d = 30k point as a side leg of the default run
            sweep = sparsity_sweep(sindi, torch, dev, args.steps, flush, stream,
                                   dims=(10, 30, 50, 70, 100) if args.sparsity_sweep else (30,))
        except Exception as e:  # noqa: BLE001 - reported in the line
            side_failed("sparsity_sweep", e)

    serving = None
    if rank == 0 and (args.serve_sweep or not args.no_forms):
        base = value if args.mode == "batched" else forms.get("batched", {}).get("qps", value)
        fractions = [float(f) for f in (args.serve_sweep or "0.25,0.5,0.75,0.9,1.1").split(",")]
        try:
            serving = {"capacity_qps": base, "capacity_from": "batched schedule of the main leg",
                       "points": serve_sweep(sindi, idx, qp, qx, qv, w.k, w.gamma, base, fractions,
                                             args.serve_seconds)}
        except Exception as e:  # noqa: BLE001 - reported in the line
            side_failed("serving", e)

    # ---- configs 3-5 at full size (rank 0; one GPU holds each index)
    scale = None
    if rank == 0 and not args.no_scale:
        try:
            scale = scale_legs(sindi, torch, dev, args, flush, stream)
        except Exception as e:  # noqa: BLE001 - reported in the line
            side_failed("scale", e)

    # ---- CPU baseline (oracle) + recall against FP64 exact, rank 0 only
    cpu = None
    recall = recall_tie = None
    score_error = None
    if rank == 0:
        qps_cpu, n_cpu, recalls, cpu_all, recalls_tie = cpu_oracle_sample(w, ip, ix, v, qp, qx, qv, args.cpu_seconds,
                                                                          gpu_ids, w.k)
        if main_dtype != "f32":
            # score error of the reduced-precision main index against FP64 (coarse and final)
            import oracle

            D = oracle.Dataset(ip, ix, v, w.dim)
            Q = oracle.Dataset(qp, qx, qv, w.dim)
            I32 = oracle.Index(D, window=w.window, alpha=w.alpha)
            n_err = min(8, nq)
            cq = [torch.from_numpy(a).to(dev) for a in (qp[: n_err + 1], qx[: qp[n_err]], qv[: qp[n_err]])]
            _, csc = idx.search(*cq, k=w.k, gamma=0)
            csc = csc.cpu().numpy()
            fsc = out_sc.cpu().numpy()
            ce = fe = 0.0
            for r in range(n_err):
                _, osc = I32.search(Q, r, k=w.k, gamma=0)
                ce = max(ce, float(np.max(np.abs(csc[r, : len(osc)] - osc) / np.abs(osc))))
                for i, sc in zip(gpu_ids[r], fsc[r]):
                    ex = oracle.inner_product(D, int(i), Q, r)
                    fe = max(fe, abs(float(sc) - ex) / abs(ex))
            score_error = {"coarse_max_rel_err_vs_fp64": ce, "final_max_rel_err_vs_fp64": fe, "queries": n_err}
        recall = float(np.mean(recalls)) if recalls else None
        recall_tie = float(np.mean(recalls_tie)) if recalls_tie else None
        cpu = {"value": qps_cpu, "unit": "queries/s", "cores": 1, "kind": "oracle",
               "sample": f"first {n_cpu} of {nq} queries of {w.name} (Algorithm 4, FP64, single thread, "
                         f"about {args.cpu_seconds:.0f} s)"}
        if forms:
            import oracle

            D = oracle.Dataset(ip, ix, v, w.dim)
            Q = oracle.Dataset(qp, qx, qv, w.dim)
            step_r = max(1, nq // 40)
            truth = {r: oracle.brute_force(D, Q, r, w.k)[0] for r in range(0, nq, step_r)}
            I32 = oracle.Index(D, window=w.window, alpha=w.alpha)
            for name, f in forms.items():
                if "_ids_only" in f:
                    f["recall_at_k_vs_fp64"] = float(np.mean([oracle.recall(f["_ids_only"][r], t)
                                                              for r, t in truth.items()]))
                    f["recall_sample"] = f"{len(truth)} queries, FP64 oracle brute force"
                    del f["_ids_only"]
                if "_ids" in f:
                    f["recall_at_k"] = float(np.mean([oracle.recall(f["_ids"][r], t) for r, t in truth.items()]))
                    # score error against FP64: coarse (quantised postings vs unquantised FP64 Algorithm 2,
                    # rank by rank) and final (FP32 reorder vs exact FP64 delta of the same document)
                    ce, fe = 0.0, 0.0
                    for r in range(f["_coarse"].shape[0]):
                        _, osc = I32.search(Q, r, k=w.k, gamma=0)
                        n = len(osc)
                        ce = max(ce, float(np.max(np.abs(f["_coarse"][r, :n] - osc) / np.abs(osc))))
                        for i, sc in zip(f["_ids"][r], f["_sc"][r]):
                            ex = oracle.inner_product(D, int(i), Q, r)
                            fe = max(fe, abs(float(sc) - ex) / abs(ex))
                    f["coarse_max_rel_err_vs_fp64"] = ce
                    f["final_max_rel_err_vs_fp64"] = fe
                    for key in ("_ids", "_sc", "_coarse"):
                        del f[key]
    if rank != 0:
        return
    clocks = clk.summary()
    line = {
        "metric": "QPS at Recall@50>=0.99 (sparse MIPS, top-50)",
        "value": value,
        "unit": "queries/s",
        "n_gpus": ws,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": dev_ms_max / args.steps,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32",
        "posting_dtype": main_dtype,
        "data": "synthetic",
        "config": {"workload": w.name, "n_docs": w.docs.n_rows, "dim": w.dim, "queries_per_rank": nq,
                   "k": w.k, "gamma": w.gamma, "alpha": w.alpha, "window": info["window"],
                   "n_windows": sigma, "postings": info["postings"], "mode": args.mode,
                   "block": args.block, "group": args.group if args.mode == "batched" else 0,
                   "accumulator": args.accum,
                   "window_sums": "fixed32" if fixed_sums else "f32",
                   "batch": 1 if args.mode == "plain" else nq,
                   "l2": "flushed between steps (256 MiB write)"},
        "recall_at_k": recall,
        "recall_at_k_tie_aware": recall_tie,
        "score_error": score_error,
        "build_ms": build_ms,
        "h2d_docs_ms": h2d_docs_ms,
        "gpu_launches": launches,
        "e2e": {"value": e2e, "unit": "queries/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "roofline": {"bound": "hbm", "achieved": achieved_step_gbs, "peak": peak, "unit": "GB/s",
                     "frac": achieved_step_gbs / peak, "peak_kind": peak_kind,
                     "frac_of_nominal_8tbs": achieved_step_gbs / NOMINAL_HBM_GBS,
                     "achieved_basis": "algorithmic bytes of every scan launch of the timed region / the region's "
                                       "CUDA-event time: scans of different queries overlap on their streams, so "
                                       "a launch's average duration is the region's time over its launches "
                                       "(merge and rerank share that time, so this is a lower bound)",
                     "achieved_one_chain": achieved_gbs, "frac_one_chain": achieved_gbs / peak,
                     "ms_per_launch_one_chain": scan_ms_per_launch,
                     "traffic": profile_traffic(sha), "kernel": "scan_window_kernel",
                     "alg_bytes_per_launch": alg_bytes_per_launch, "launches_per_step": scan_launches_per_step,
                     "ms_per_launch": dev_ms_max / args.steps / scan_launches_per_step,
                     "postings_per_query": float(touched.mean()),
                     "scatter_adds": {"per_s": adds_per_s_step, "per_s_one_chain": adds_per_s, "peak": adds_peak,
                                      "frac": adds_per_s_step / adds_peak if adds_peak else None,
                                      "frac_one_chain": adds_per_s / adds_peak if adds_peak else None,
                                      "unit": "posting updates/s",
                                      "peak_from": adds_peak_from,
                                      "forms": adds_forms}},
        "cpu_baseline": cpu,
        "cpu_baseline_all_cores": cpu_all,
        "clocks": clocks,
        "forms": forms,
        "pruning_ablation": ablation,
        "sparsity_sweep": sweep,
        "serving": serving,
        "scale": scale,
        "scan_source_sha256": sha,
        "side_errors": side_errors,
    }
    print(json.dumps(line), flush=True)
    idx.close()
    if ws > 1:
        import torch.distributed as dist

        dist.destroy_process_group()


if __name__ == "__main__":
    main()
