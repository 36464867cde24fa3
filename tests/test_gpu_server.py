"""Serving form: continuous batching through sindi_server_* (needs a GB300)."""
import numpy as np
import pytest

import datagen
import oracle
from parity import REL_TOL, check_reranked, tie_groups

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_2509_08395_gb300 as sindi  # noqa: E402

DEV = torch.device("cuda:0")


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


@pytest.fixture(scope="module")
def setup():
    w = datagen.WORKLOADS["pruned-1m"].scaled(n_docs=30_000, n_queries=64)
    ip, ix, v = datagen.docs(w)
    qp, qx, qv = datagen.queries(w)
    idx = sindi.Index(_dev(ip), _dev(ix), _dev(v), w.dim, window=4096, alpha=0.5)
    yield w, idx, (ip, ix, v), (qp, qx, qv)
    idx.close()


def _rows(q):
    qp, qx, qv = q
    return [(qx[qp[r]:qp[r + 1]], qv[qp[r]:qp[r + 1]]) for r in range(len(qp) - 1)]


def _same(a_ids, a_sc, b_ids, b_sc, what):
    np.testing.assert_allclose(a_sc, b_sc, rtol=REL_TOL, atol=0, err_msg=what)
    for a, b in tie_groups(b_sc.astype(np.float64)):
        if b < len(b_ids):
            assert set(a_ids[a:b].tolist()) == set(b_ids[a:b].tolist()), (what, a, b)


def test_each_result_is_the_same_alone_and_in_the_mix(setup):
    """A request served alone equals the same request served among 63 others (tolerance of the parity tests),
    and both equal sindi_search; the answers also pass the oracle's Algorithm 4 check."""
    w, idx, (ip, ix, v), q = setup
    rows = _rows(q)
    k, gamma = 50, 500
    ref_ids, ref_sc = idx.search(*[_dev(a) for a in q], k=k, gamma=gamma)
    ref_ids = ref_ids.cpu().numpy().view(np.uint32)
    ref_sc = ref_sc.cpu().numpy()
    with sindi.Server(idx, k=k, gamma=gamma, max_batch=8, max_slots=4) as srv:
        alone = []
        for qi, qv in rows:
            t = srv.submit(qi, qv)
            alone.append(srv.poll(t, wait_ms=-1))
        tickets = [srv.submit(qi, qv) for qi, qv in rows]
        mix = [srv.poll(t, wait_ms=-1) for t in tickets]
        st = srv.stats()
    assert st["completed"] == 2 * len(rows) and st["failed"] == 0
    assert st["batches"] < 2 * len(rows)  # the mix was batched
    D = oracle.Dataset(ip, ix, v, w.dim)
    Q = oracle.Dataset(*q, w.dim)
    I = oracle.Index(D, window=4096, alpha=0.5)
    for r in range(len(rows)):
        _same(mix[r][0], mix[r][1], alone[r][0], alone[r][1], f"mix vs alone, query {r}")
        _same(alone[r][0], alone[r][1], ref_ids[r], ref_sc[r], f"alone vs sindi_search, query {r}")
        if r % 8 == 0:
            check_reranked(mix[r][0], mix[r][1], D, Q, r, I, k, gamma, what=f"served query {r}")


def test_batches_overlap_on_the_device(setup):
    w, idx, _, q = setup
    rows = _rows(q) * 4
    with sindi.Server(idx, k=10, gamma=100, max_batch=4, max_slots=8) as srv:
        tickets = [srv.submit(qi, qv) for qi, qv in rows]
        for t in tickets:
            assert srv.poll(t, wait_ms=-1) is not None
        st = srv.stats()
    assert st["n_slots"] == 8
    assert st["peak_in_flight"] >= 2, st
    assert st["p99_ms"] >= st["p50_ms"] > 0


def test_memory_admission(setup):
    w, idx, _, q = setup
    with sindi.Server(idx, k=10, gamma=100, max_batch=16, max_slots=8) as srv:
        slot = srv.stats()["slot_bytes"]
    with pytest.raises(sindi.SindiError, match="OOM"):
        sindi.Server(idx, k=10, gamma=100, max_batch=16, max_slots=8, memory_budget=slot - 1)
    with sindi.Server(idx, k=10, gamma=100, max_batch=16, max_slots=8, memory_budget=2 * slot + 1) as srv:
        assert srv.stats()["n_slots"] == 2
        qi, qv = _rows(q)[0]
        assert srv.poll(srv.submit(qi, qv), wait_ms=-1) is not None


def test_rejections_and_shutdown_with_work_in_flight(setup):
    w, idx, _, q = setup
    srv = sindi.Server(idx, k=10, gamma=0, max_batch=4, max_slots=2, max_query_nnz=256)
    with pytest.raises(sindi.SindiError, match="INVALID_ARG"):
        srv.submit(np.arange(257, dtype=np.int32), np.ones(257, np.float32))
    with pytest.raises(sindi.SindiError, match="INVALID_ARG"):
        srv.poll(123456789)
    pending = [srv.submit(qi, qv) for qi, qv in _rows(q)]
    first = srv.poll(pending[0], wait_ms=-1)
    assert first is not None
    srv.close()  # finishes queued and running requests, then frees the slots
    assert srv.handle is None
