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
    """Merge per-shard result rows on the host. ids/scores: [shards, queries, k_shard] (ids already global).

    Returns ([queries, k] uint32 ids, [queries, k] float32 scores), best first (score desc, id asc), padded
    like a search row. One sort over all rows (the row is the leading key)."""
    ids = np.asarray(ids).astype(np.int64) & 0xFFFFFFFF
    scores = np.asarray(scores, dtype=np.float32)
    s, nq, ks = ids.shape
    m = s * ks
    flat_ids = ids.transpose(1, 0, 2).reshape(nq, m)
    flat_sc = scores.transpose(1, 0, 2).reshape(nq, m)
    valid = flat_ids != PAD_ID
    sc_key = np.where(valid, -flat_sc.astype(np.float64), np.inf)   # padding sorts last
    id_key = np.where(valid, flat_ids, PAD_ID)
    rows = np.repeat(np.arange(nq, dtype=np.int64), m)
    order = np.lexsort((id_key.ravel(), sc_key.ravel(), rows)).reshape(nq, m) - (np.arange(nq) * m)[:, None]
    take = order[:, : min(k, m)]
    out_ids = np.full((nq, k), PAD_ID, np.uint32)
    out_sc = np.full((nq, k), -np.inf, np.float32)
    ok = np.take_along_axis(valid, take, axis=1)
    out_ids[:, : take.shape[1]] = np.where(ok, np.take_along_axis(flat_ids, take, axis=1), PAD_ID)
    out_sc[:, : take.shape[1]] = np.where(ok, np.take_along_axis(flat_sc, take, axis=1), -np.inf)
    return out_ids, out_sc


def gather_merge(local_ids, local_scores, id_offset: int, k: int, group=None):
    """All-gather every rank's [queries, k_local] rows (local ids; this rank's documents start at global id
    `id_offset`) and merge them into the global top-k.

    Device tensors stay on the device: under NCCL they are gathered as they are (under another backend
    through host memory) and merged by the library's sindi_merge_topk. Host arrays are gathered and merged
    on the host (merge_topk)."""
    import torch
    import torch.distributed as dist

    world = dist.get_world_size(group)
    if isinstance(local_ids, torch.Tensor) and local_ids.is_cuda:
        from .sindi import sindi_merge_topk

        dev = local_ids.device
        t_ids = local_ids.contiguous().view(torch.int32)
        t_sc = local_scores.contiguous()
        t_off = torch.tensor([int(id_offset)], dtype=torch.int64)
        on_device = dist.get_backend(group) == "nccl"
        if on_device:
            t_off = t_off.to(dev)
        else:
            t_ids, t_sc = t_ids.cpu(), t_sc.cpu()
        all_ids = [torch.empty_like(t_ids) for _ in range(world)]
        all_sc = [torch.empty_like(t_sc) for _ in range(world)]
        all_off = [torch.empty_like(t_off) for _ in range(world)]
        dist.all_gather(all_ids, t_ids, group=group)
        dist.all_gather(all_sc, t_sc, group=group)
        dist.all_gather(all_off, t_off, group=group)
        ids = torch.stack(all_ids).to(dev)
        sc = torch.stack(all_sc).to(dev)
        offsets = [int(o.item()) for o in all_off]
        return sindi_merge_topk(ids, sc, offsets, k)
    ids = np.asarray(local_ids).astype(np.int64) & 0xFFFFFFFF
    t_ids = torch.from_numpy(np.where(ids == PAD_ID, PAD_ID, ids + int(id_offset)))
    t_sc = torch.from_numpy(np.asarray(local_scores, dtype=np.float32))
    all_ids = [torch.empty_like(t_ids) for _ in range(world)]
    all_sc = [torch.empty_like(t_sc) for _ in range(world)]
    dist.all_gather(all_ids, t_ids, group=group)
    dist.all_gather(all_sc, t_sc, group=group)
    return merge_topk(np.stack([a.numpy() for a in all_ids]), np.stack([a.numpy() for a in all_sc]), k)


class DocShardedIndex:
    """This rank's part of a document-sharded index (the documents of its id range, aligned to the window)."""

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

    def local_search(self, q_indptr, q_indices, q_values, k: int, gamma: int = 0, mode: str = "batched"):
        """This shard's rows (device tensors, local ids); the shard's documents start at global id self.lo."""
        return self.index.search(q_indptr, q_indices, q_values, k=k, gamma=gamma, mode=mode)

    def search(self, q_indptr, q_indices, q_values, k: int, gamma: int = 0, mode: str = "batched", group=None):
        """The global top-k: this shard's rows, all-gathered from every rank and merged on the device."""
        ids, sc = self.local_search(q_indptr, q_indices, q_values, k, gamma, mode)
        return gather_merge(ids, sc, self.lo, k, group)

    def close(self):
        self.index.close()
