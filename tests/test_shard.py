"""Multi-rank paths on CPU ranks (gloo, world size 2): query shards and document shards + top-k merge.

The per-shard searches here are the FP64 oracle's brute force on each rank's
documents; what is under test is the sharding and the all-gather merge.
"""
import os
import socket

import numpy as np
import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

import datagen
import oracle
from paper_2509_08395_gb300.shard import PAD_ID, merge_topk, shard_range


def test_shard_ranges_cover_everything_once():
    for n in (0, 1, 7, 1000, 1_000_003):
        for world in (1, 2, 3, 8):
            for align in (1, 4096):
                parts = [shard_range(n, r, world, align) for r in range(world)]
                assert parts[0][0] == 0 and parts[-1][1] == n
                for (a, b), (c, d) in zip(parts, parts[1:]):
                    assert b == c and a <= b
                assert all(lo % align == 0 for lo, _ in parts if lo < n)


def test_merge_topk_order_and_padding():
    ids = np.array([[[5, 1, PAD_ID]], [[9, 2, 3]]], np.uint32)
    sc = np.array([[[3.0, 2.0, -np.inf]], [[3.0, 2.0, 1.0]]], np.float32)
    mi, ms = merge_topk(ids, sc, 4)
    assert mi.tolist() == [[5, 9, 1, 2]] and ms.tolist() == [[3.0, 3.0, 2.0, 2.0]]
    mi, ms = merge_topk(ids[:1], sc[:1], 4)
    assert mi.tolist() == [[5, 1, PAD_ID, PAD_ID]] and np.isneginf(ms[0, 2:]).all()


def test_merge_topk_matches_a_per_row_sort():
    """The vectorised host merge against a plain per-row sort by (score desc, id asc), with tied scores,
    padding in every shard and rows with fewer than k entries."""
    rng = np.random.default_rng(4)
    S, nq, ks, k = 3, 50, 7, 10
    ids = rng.permutation(10_000)[: S * nq * ks].reshape(S, nq, ks).astype(np.uint32)
    sc = rng.integers(0, 5, (S, nq, ks)).astype(np.float32)   # many ties
    pad = rng.random((S, nq, ks)) < 0.3
    ids[pad] = PAD_ID
    sc[pad] = -np.inf
    mi, ms = merge_topk(ids, sc, k)
    for q in range(nq):
        items = [(-float(sc[s, q, j]), int(ids[s, q, j])) for s in range(S) for j in range(ks) if ids[s, q, j] != PAD_ID]
        items.sort()
        want_ids = [i for _, i in items[:k]] + [PAD_ID] * max(0, k - len(items))
        assert mi[q].tolist() == want_ids
        np.testing.assert_array_equal(ms[q][: len(items[:k])], [-x for x, _ in items[:k]])
        assert np.isneginf(ms[q][len(items[:k]):]).all()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, result_path):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_2509_08395_gb300.shard import gather_merge

    ip, ix, v = datagen.random_csr(3001, 200, 15.0, seed=5, zipf_s=1.0)
    qp, qx, qv = datagen.random_csr(12, 200, 10.0, seed=6, zipf_s=1.0, nnz_min=1)
    k = 20
    # document shard of this rank (window-aligned ranges)
    lo, hi = shard_range(3001, rank, world, align=256)
    sip = ip[lo: hi + 1] - ip[lo]
    D = oracle.Dataset(sip, ix[ip[lo]: ip[hi]], v[ip[lo]: ip[hi]], 200)
    Q = oracle.Dataset(qp, qx, qv, 200)
    ids = np.full((Q.n, k), PAD_ID, np.uint32)
    sc = np.full((Q.n, k), -np.inf, np.float32)
    for r in range(Q.n):
        a, b = oracle.brute_force(D, Q, r, k)
        ids[r, : len(a)] = a
        sc[r, : len(a)] = b.astype(np.float32)
    mi, ms = gather_merge(ids, sc, lo, k)
    # query shard of this rank, gathered back
    qlo, qhi = shard_range(Q.n, rank, world)
    import torch
    mine = torch.tensor([qlo, qhi], dtype=torch.int64)
    allq = [torch.empty_like(mine) for _ in range(world)]
    dist.all_gather(allq, mine)
    if rank == 0:
        np.savez(result_path, ids=mi, sc=ms, qranges=np.stack([a.numpy() for a in allq]))
    dist.barrier()
    dist.destroy_process_group()


def test_document_shards_merge_to_the_global_topk(tmp_path):
    path = str(tmp_path / "merged.npz")
    mp.spawn(_worker, args=(2, _free_port(), path), nprocs=2, join=True)
    out = np.load(path)
    ip, ix, v = datagen.random_csr(3001, 200, 15.0, seed=5, zipf_s=1.0)
    qp, qx, qv = datagen.random_csr(12, 200, 10.0, seed=6, zipf_s=1.0, nnz_min=1)
    D, Q = oracle.Dataset(ip, ix, v, 200), oracle.Dataset(qp, qx, qv, 200)
    for r in range(Q.n):
        a, b = oracle.brute_force(D, Q, r, 20)
        assert out["ids"][r].tolist() == a.tolist()
        np.testing.assert_array_equal(out["sc"][r], b.astype(np.float32))
    qr = out["qranges"]
    assert qr[0][0] == 0 and qr[-1][1] == Q.n and qr[0][1] == qr[1][0]


def _bench_worker(rank, world, port, result_path):
    """bench.py's multi-rank pieces on gloo ranks: the query share of each rank, the barrier and the
    max over ranks that the timed region's duration goes through."""
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench

    w = datagen.WORKLOADS["exact-10k"].scaled(n_queries=37)
    qp, qx, qv = bench.rank_queries(w, rank, world)
    bench.barrier(world)
    slowest = bench.max_over_ranks(10.0 + rank, world)
    np.savez(f"{result_path}.{rank}.npz", qp=qp, qx=qx, qv=qv, slowest=slowest)
    bench.barrier(world)
    dist.destroy_process_group()


def test_bench_ranks_split_the_weak_scaling_query_set(tmp_path):
    """Every rank searches its own share of the global query set (the workload's queries once per rank),
    the shares together are that set in order, rank 0's share is the workload's own query set, and every
    rank reports the slowest rank's time."""
    world = 2
    path = str(tmp_path / "bench")
    mp.spawn(_bench_worker, args=(world, _free_port(), path), nprocs=world, join=True)
    parts = [np.load(f"{path}.{r}.npz") for r in range(world)]
    assert all(float(p["slowest"]) == 10.0 + world - 1 for p in parts)
    w = datagen.WORKLOADS["exact-10k"].scaled(n_queries=37)
    gqp, gqx, gqv = datagen.queries(w.scaled(n_queries=37 * world))
    assert [len(p["qp"]) - 1 for p in parts] == [37] * world
    np.testing.assert_array_equal(np.concatenate([p["qx"] for p in parts]), gqx)
    np.testing.assert_array_equal(np.concatenate([p["qv"] for p in parts]), gqv)
    starts = np.concatenate([[0], np.cumsum([len(p["qx"]) for p in parts])])
    for r, p in enumerate(parts):
        np.testing.assert_array_equal(p["qp"] + starts[r], gqp[37 * r: 37 * (r + 1) + 1])
    own = datagen.queries(w)
    for a, b in zip((parts[0]["qp"], parts[0]["qx"], parts[0]["qv"]), own):
        np.testing.assert_array_equal(a, b)
