"""Splitting the search across GPUs (one process per GPU, torch.distributed).

Queries are independent and windows are independent, so the work splits two
ways, neither of which changes any result:

* query sharding: every rank holds a replica of the index and searches a
  contiguous share of the queries. No collective touches the data path
  (bench.py --gpus N; weak scaling).
* document sharding: rank r holds the documents of a contiguous id range
  (aligned to the window, so no window straddles two ranks) and searches it
  for every query; each rank's top-k lists are all-gathered and merged with
  the search's own order (score descending, then lower id), so the merged
  list is the top-k over all documents.
"""
from __future__ import annotations

import numpy as np

PAD_ID = 0xFFFFFFFF


def shard_range(n: int, rank: int, world: int, align: int = 1) -> tuple[int, int]:
    """[lo, hi) of rank's contiguous share of n units, boundaries on multiples of `align`."""
    if world <= 0 or not 0 <= rank < world:
        raise ValueError("bad rank / world")
    blocks = -(-n // align)
    lo = (blocks * rank // world) * align
    hi = (blocks * (rank + 1) // world) * align
    return min(lo, n), min(hi, n)


def merge_topk(ids, scores, k: int):
    """Merge per-shard result rows. ids/scores: [shards, queries, k_shard] (ids already global).

    Returns ([queries, k] uint32 ids, [queries, k] float32 scores), best first, padded like a search row."""
    ids = np.asarray(ids).astype(np.int64) & 0xFFFFFFFF
    scores = np.asarray(scores, dtype=np.float32)
    s, nq, ks = ids.shape
    flat_ids = ids.transpose(1, 0, 2).reshape(nq, s * ks)
    flat_sc = scores.transpose(1, 0, 2).reshape(nq, s * ks)
    out_ids = np.full((nq, k), PAD_ID, np.uint32)
    out_sc = np.full((nq, k), -np.inf, np.float32)
    for q in range(nq):
        keep = flat_ids[q] != PAD_ID
        qi, qs = flat_ids[q][keep], flat_sc[q][keep]
        order = np.lexsort((qi, -qs.astype(np.float64)))[:k]
        out_ids[q, : len(order)] = qi[order]
        out_sc[q, : len(order)] = qs[order]
    return out_ids, out_sc


def gather_merge(local_ids, local_scores, id_offset: int, k: int, group=None):
    """All-gather every rank's [queries, k] rows (local ids shifted by id_offset) and merge them."""
    import torch
    import torch.distributed as dist

    ids = np.asarray(local_ids).astype(np.int64) & 0xFFFFFFFF
    glob = np.where(ids == PAD_ID, PAD_ID, ids + id_offset)
    t_ids = torch.from_numpy(glob)
    t_sc = torch.from_numpy(np.asarray(local_scores, dtype=np.float32))
    world = dist.get_world_size(group)
    all_ids = [torch.empty_like(t_ids) for _ in range(world)]
    all_sc = [torch.empty_like(t_sc) for _ in range(world)]
    dist.all_gather(all_ids, t_ids, group=group)
    dist.all_gather(all_sc, t_sc, group=group)
    return merge_topk(np.stack([a.numpy() for a in all_ids]), np.stack([a.numpy() for a in all_sc]), k)


class DocShardedIndex:
    """This rank's part of a document-sharded index (the documents of its id range)."""

    def __init__(self, indptr, indices, values, dim: int, rank: int, world: int, window: int = 0,
                 alpha: float = 1.0, value_dtype: str = "f32", device=None):
        import torch

        from .sindi import Index

        n = len(indptr) - 1
        self.window = window or 8192
        self.lo, self.hi = shard_range(n, rank, world, align=self.window)
        ip = np.asarray(indptr[self.lo: self.hi + 1], dtype=np.int64)
        seg_ix = np.asarray(indices[ip[0]: ip[-1]], dtype=np.int32)
        seg_v = np.asarray(values[ip[0]: ip[-1]], dtype=np.float32)
        ip = ip - ip[0]
        dev = device or torch.device("cuda", torch.cuda.current_device())
        to = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
        self.index = Index(to(ip), to(seg_ix), to(seg_v), dim, window=self.window, alpha=alpha,
                           value_dtype=value_dtype)

    def search(self, q_indptr, q_indices, q_values, k: int, gamma: int = 0, mode: str = "batched", group=None):
        ids, sc = self.index.search(q_indptr, q_indices, q_values, k=k, gamma=gamma, mode=mode)
        return gather_merge(ids.cpu().numpy().view(np.uint32), sc.cpu().numpy(), self.lo, k, group)
