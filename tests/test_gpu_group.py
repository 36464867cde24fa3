"""Query-group window scan of the batched schedule (one block per window and group of queries, each posting
loaded once for every query of the group holding its term) vs the FP64 oracle, through the C ABI."""
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

DEV = torch.device("cuda:0")


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def search(idx, qp, qx, qv, k, gamma, group, block=0):
    ids, sc = idx.search(dev(qp), dev(qx), dev(qv), k=k, gamma=gamma, mode="batched", group=group, block=block)
    idx.check()
    return ids.cpu().numpy().view(np.uint32).astype(np.int64), sc.cpu().numpy()


@pytest.fixture(scope="module")
def small():
    # 40,000 docs of the pruned-1m distribution; 41 queries, so that groups of 2, 3, 4, 5 and 8 end ragged
    w = datagen.WORKLOADS["pruned-1m"].scaled(n_docs=40_000, n_queries=41)
    ip, ix, v = datagen.docs(w)
    qp, qx, qv = datagen.queries(w)
    return w, (ip, ix, v), (qp, qx, qv), oracle.Dataset(ip, ix, v, w.dim), oracle.Dataset(qp, qx, qv, w.dim)


@pytest.mark.parametrize("window,group,block,dtype", [
    (4096, 0, 0, "f32"),      # the default: one query per block
    (4096, 3, 1024, "f32"),
    (1024, 8, 512, "f32"),
    (8192, 5, 1024, "f16"),
    (300, 8, 512, "f32"),     # a window that is not a multiple of 4 slots
    (16384, 2, 512, "f8"),
    (16384, 4, 0, "f32"),     # more than shared memory holds: reduced to 3
    (2048, 1, 512, "f32"),    # one block per (query, window)
])
def test_group_scan_coarse_parity(small, window, group, block, dtype):
    """Coarse top-100 (gamma = 0) of every query, whatever its group, equals the oracle's Algorithm 2 on the
    same (dequantised) postings within the FP32 rule."""
    w, (ip, ix, v), (qp, qx, qv), D, Q = small
    I = oracle.Index(D, window=window, alpha=0.5, dtype=dtype)
    with sindi.Index(dev(ip), dev(ix), dev(v), w.dim, window=window, alpha=0.5, value_dtype=dtype) as idx:
        ids, sc = search(idx, qp, qx, qv, k=100, gamma=0, group=group, block=block)
    for r in range(Q.n):
        oi, os_ = I.search(Q, r, k=164, gamma=0)
        check_ranked(ids[r], sc[r], oi, os_, 100, D.n, what=f"group {group} query {r}")


@pytest.mark.parametrize("window,group,gamma,k", [(4096, 4, 300, 20), (8192, 3, 500, 50), (1024, 8, 1000, 100)])
def test_group_scan_rerank_parity(small, window, group, gamma, k):
    """Algorithm 4 through the group scan: the reordered top-k is the exact top-k of an admissible candidate
    set."""
    w, (ip, ix, v), (qp, qx, qv), D, Q = small
    I = oracle.Index(D, window=window, alpha=0.5)
    with sindi.Index(dev(ip), dev(ix), dev(v), w.dim, window=window, alpha=0.5) as idx:
        ids, sc = search(idx, qp, qx, qv, k=k, gamma=gamma, group=group)
    touched = 0
    for r in range(Q.n):
        touched += check_reranked(ids[r], sc[r], D, Q, r, I, k, gamma, what=f"group {group} query {r}")
    assert touched <= 2


@pytest.mark.parametrize("group", [4, 8])
def test_group_scan_long_queries_take_several_passes(small, group):
    """Queries of 300 to 700 terms: a group holds more entries than one pass of the union hash takes (512), so
    a dim may reach two passes and is added as two terms; every (query, term) pair still counts once."""
    w, (ip, ix, v), _, D, _ = small
    qp, qx, qv = datagen.generate(datagen.RowDist(11, datagen.NNZ_UNIFORM, 300, 700, 300, 700, val_sigma=0.8),
                                  w.dim, w.zipf_s, 93)
    Q = oracle.Dataset(qp, qx, qv, w.dim)
    I = oracle.Index(D, window=2048, alpha=0.5)
    with sindi.Index(dev(ip), dev(ix), dev(v), w.dim, window=2048, alpha=0.5) as idx:
        ids, sc = search(idx, qp, qx, qv, k=50, gamma=0, group=group)
        rids, rsc = search(idx, qp, qx, qv, k=20, gamma=400, group=group)
    for r in range(Q.n):
        oi, os_ = I.search(Q, r, k=114, gamma=0)
        check_ranked(ids[r], sc[r], oi, os_, 50, D.n, what=f"coarse query {r}")
        check_reranked(rids[r], rsc[r], D, Q, r, I, 20, 400, what=f"rerank query {r}")


def test_group_scan_shared_and_degenerate_queries(small):
    """A batch whose groups hold the same query twice (every term shared), an empty query, a query of explicit
    zeros, one-term queries and a query whose terms no document holds: each row equals the oracle's."""
    w, (ip, ix, v), (qp, qx, qv), D, _ = small
    rows = []
    q0 = list(zip(qx[qp[0]:qp[1]].tolist(), qv[qp[0]:qp[1]].tolist()))
    q1 = list(zip(qx[qp[1]:qp[2]].tolist(), qv[qp[1]:qp[2]].tolist()))
    held = set(ix.tolist())
    unheld = [j for j in range(w.dim - 1, 0, -1) if j not in held][:3]
    rows += [q0, q0, [], [(int(qx[0]), 0.0), (int(qx[1]), 0.0)], [(0, 1.5)], [(1, 0.25)], q1,
             [(j, 1.0) for j in unheld], q1, q0]
    qp2 = np.zeros(len(rows) + 1, np.int64)
    qp2[1:] = np.cumsum([len(r) for r in rows])
    qx2 = np.array([j for r in rows for j, _ in r], np.int32)
    qv2 = np.array([x for r in rows for _, x in r], np.float32)
    Q = oracle.Dataset(qp2, qx2, qv2, w.dim)
    I = oracle.Index(D, window=4096, alpha=0.5)
    with sindi.Index(dev(ip), dev(ix), dev(v), w.dim, window=4096, alpha=0.5) as idx:
        for group in (2, 4, 8):
            ids, sc = search(idx, qp2, qx2, qv2, k=30, gamma=0, group=group)
            for r in range(Q.n):
                # the whole ranking: rows without a positive score are one tie group over every document
                oi, os_ = I.search(Q, r, k=D.n, gamma=0)
                check_ranked(ids[r], sc[r], oi, os_, 30, D.n, what=f"group {group} row {r}")


def test_group_scan_in_a_plan(small):
    """The graph-captured batched search (sindi_plan_*) with query groups: two launches, the queries' values
    changed in place between them, both equal the oracle's."""
    w, (ip, ix, v), (qp, qx, qv), D, Q = small
    I = oracle.Index(D, window=4096, alpha=0.5)
    with sindi.Index(dev(ip), dev(ix), dev(v), w.dim, window=4096, alpha=0.5) as idx:
        dq = [dev(qp), dev(qx), dev(qv)]
        with sindi.Plan(idx, *dq, k=20, gamma=300, group=4) as plan:
            for rep in range(2):
                if rep == 1:
                    dq[2].mul_(2.0)  # scores double, ranks stay
                plan.launch(torch.cuda.current_stream().cuda_stream)
                torch.cuda.synchronize()
                idx.check()
                ids = plan.out[0].cpu().numpy().view(np.uint32).astype(np.int64)
                sc = plan.out[1].cpu().numpy() / (2.0 if rep == 1 else 1.0)
                for r in range(Q.n):
                    check_reranked(ids[r], sc[r], D, Q, r, I, 20, 300, what=f"plan launch {rep} query {r}")
