"""Document sharding on the device: shards built as indexes of their own, their rows merged by
sindi_merge_topk, against the FP64 oracle over all documents (needs a GB300)."""
import os
import socket

import numpy as np
import pytest

import datagen
import oracle
from parity import check_ranked, check_reranked

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # collected on CPU machines, never run there
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_2509_08395_gb300 as sindi  # noqa: E402
from paper_2509_08395_gb300.shard import DocShardedIndex, PAD_ID, merge_topk  # noqa: E402

DEV = torch.device("cuda:0")


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


@pytest.fixture(scope="module")
def data():
    w = datagen.WORKLOADS["pruned-1m"].scaled(n_docs=30_001, n_queries=24)
    ip, ix, v = datagen.docs(w)
    qp, qx, qv = datagen.queries(w)
    return w, (ip, ix, v), (qp, qx, qv), oracle.Dataset(ip, ix, v, w.dim), oracle.Dataset(qp, qx, qv, w.dim)


@pytest.mark.parametrize("world", [2, 3])
def test_document_shards_merge_on_the_device_to_the_global_topk(data, world):
    """Exact search (alpha = 1, no reorder) on each window-aligned document shard, merged on the device: the
    global top-k of the FP64 brute force over all documents."""
    w, (ip, ix, v), (qp, qx, qv), D, Q = data
    shards = [DocShardedIndex(ip, ix, v, w.dim, r, world, window=4096, alpha=1.0) for r in range(world)]
    try:
        q = [dev(a) for a in (qp, qx, qv)]
        rows = [s.local_search(*q, k=50, gamma=0) for s in shards]
        ids = torch.stack([r[0] for r in rows])
        sc = torch.stack([r[1] for r in rows])
        mi, ms = sindi.sindi_merge_topk(ids, sc, [s.lo for s in shards], 40)
        torch.cuda.synchronize()
        mi, ms = mi.cpu().numpy().view(np.uint32).astype(np.int64), ms.cpu().numpy()
        # the host merge of the same rows agrees
        gids = ids.cpu().numpy().view(np.uint32).astype(np.int64)
        for n, s in enumerate(shards):
            gids[n] = np.where(gids[n] == PAD_ID, PAD_ID, gids[n] + s.lo)
        hi, hs = merge_topk(gids, sc.cpu().numpy(), 40)
        np.testing.assert_array_equal(hi.astype(np.int64), mi)
        np.testing.assert_array_equal(hs, ms)
    finally:
        for s in shards:
            s.close()
    for r in range(Q.n):
        oi, os_ = oracle.brute_force(D, Q, r, 104)
        check_ranked(mi[r], ms[r], oi, os_, 40, D.n, what=f"world {world} query {r}")


def test_document_shards_with_pruning_and_reorder(data):
    """alpha = 0.5 with a reorder pool of 300 per shard: every shard's candidates include its part of the global
    top-300, so the merged answer is the exact top-k of an admissible candidate set."""
    w, (ip, ix, v), (qp, qx, qv), D, Q = data
    I = oracle.Index(D, window=4096, alpha=0.5)
    shards = [DocShardedIndex(ip, ix, v, w.dim, r, 2, window=4096, alpha=0.5) for r in range(2)]
    try:
        q = [dev(a) for a in (qp, qx, qv)]
        rows = [s.local_search(*q, k=20, gamma=300) for s in shards]
        mi, ms = sindi.sindi_merge_topk(torch.stack([r[0] for r in rows]), torch.stack([r[1] for r in rows]),
                                        [s.lo for s in shards], 20)
        torch.cuda.synchronize()
    finally:
        for s in shards:
            s.close()
    mi, ms = mi.cpu().numpy().view(np.uint32).astype(np.int64), ms.cpu().numpy()
    for r in range(Q.n):
        truth, _ = oracle.brute_force(D, Q, r, 20)
        assert len(set(truth.tolist()) & set(mi[r].tolist())) >= 19, r
        for rank in range(20):
            exact = oracle.inner_product(D, int(mi[r, rank]), Q, r)
            assert abs(ms[r, rank] - exact) <= 1e-5 * abs(exact)
        assert np.all(np.diff(ms[r]) <= 0)


def test_merge_refuses_bad_arguments(data):
    ids = torch.zeros((2, 3, 4), dtype=torch.int32, device=DEV)
    sc = torch.zeros((2, 3, 4), dtype=torch.float32, device=DEV)
    with pytest.raises(sindi.SindiError, match="INVALID_ARG"):
        sindi.sindi_merge_topk(ids, sc, [0, 10], 2000)            # k above 1024
    with pytest.raises(sindi.SindiError, match="INVALID_ARG"):
        sindi.sindi_merge_topk(ids.cpu(), sc.cpu(), [0, 10], 4)  # host memory
    with pytest.raises(sindi.SindiError, match="INVALID_ARG"):
        sindi.sindi_merge_topk(ids, sc, [-1, 10], 4)             # negative offset
    big = torch.zeros((3, 1, 4000), dtype=torch.int32, device=DEV)
    with pytest.raises(sindi.SindiError, match="INVALID_ARG"):
        sindi.sindi_merge_topk(big, big.float(), [0, 1, 2], 10)  # 12,000 entries per query


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_gather_merge_keeps_device_rows_on_the_device(data):
    """gather_merge with device tensors in a one-rank process group: the rows are gathered, merged by the
    library on the device, and come back as device tensors equal to the shard's own top-k."""
    import torch.distributed as dist

    from paper_2509_08395_gb300.shard import gather_merge

    w, (ip, ix, v), (qp, qx, qv), D, Q = data
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(_free_port()))
    dist.init_process_group("gloo", rank=0, world_size=1)
    try:
        with sindi.Index(dev(ip), dev(ix), dev(v), w.dim, window=4096, alpha=1.0) as idx:
            ids, sc = idx.search(dev(qp), dev(qx), dev(qv), k=30, gamma=0)
            mi, ms = gather_merge(ids, sc, 0, 30)
            assert mi.is_cuda and ms.is_cuda
            np.testing.assert_array_equal(mi.cpu().numpy(), ids.cpu().numpy())
            np.testing.assert_array_equal(ms.cpu().numpy(), sc.cpu().numpy())
    finally:
        dist.destroy_process_group()
