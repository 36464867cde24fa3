"""Batched form: graph-captured plans, scan block shapes and the autotuner (needs a GB300)."""
import numpy as np
import pytest

import datagen
import oracle
from parity import REL_TOL, tie_groups

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_2509_08395_gb300 as sindi  # noqa: E402
from paper_2509_08395_gb300 import autotune  # noqa: E402

DEV = torch.device("cuda:0")


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def _same(a_ids, a_sc, b_ids, b_sc, what):
    a_ids = np.asarray(a_ids).view(np.uint32)
    b_ids = np.asarray(b_ids).view(np.uint32)
    np.testing.assert_allclose(a_sc, b_sc, rtol=REL_TOL, atol=0, err_msg=what)
    for r in range(b_ids.shape[0]):
        for a, b in tie_groups(b_sc[r].astype(np.float64)):
            if b < b_ids.shape[1]:
                assert set(a_ids[r, a:b].tolist()) == set(b_ids[r, a:b].tolist()), (what, r, a, b)


@pytest.fixture(scope="module")
def setup():
    w = datagen.WORKLOADS["pruned-1m"].scaled(n_docs=40_000, n_queries=96)
    ip, ix, v = datagen.docs(w)
    qp, qx, qv = datagen.queries(w)
    idx = sindi.Index(_dev(ip), _dev(ix), _dev(v), w.dim, window=4096, alpha=0.5)
    yield w, idx, (ip, ix, v), (qp, qx, qv)
    idx.close()


def test_plan_replays_the_batched_search(setup):
    """One graph launch = the batched search; contents of the query buffers may change between launches."""
    w, idx, _, (qp, qx, qv) = setup
    q = [_dev(qp), _dev(qx), _dev(qv)]
    ref = [t.cpu().numpy() for t in idx.search(*q, k=50, gamma=500, mode="batched")]
    with sindi.Plan(idx, *q, k=50, gamma=500) as plan:
        for _ in range(2):
            ids, sc = plan.launch()
            torch.cuda.synchronize()
            idx.check()
            _same(ids.cpu().numpy(), sc.cpu().numpy(), ref[0], ref[1], "plan vs search")
        q[2].mul_(2.0)  # new query weights in the same buffers
        ref2 = [t.cpu().numpy() for t in idx.search(*q, k=50, gamma=500, mode="batched")]
        ids, sc = plan.launch()
        torch.cuda.synchronize()
        _same(ids.cpu().numpy(), sc.cpu().numpy(), ref2[0], ref2[1], "plan after new contents")
        np.testing.assert_allclose(ref2[1], 2 * ref[1], rtol=1e-6)


@pytest.mark.parametrize("mode", ["plain", "batched"])
def test_block_shapes_give_the_same_results(setup, mode):
    w, idx, _, (qp, qx, qv) = setup
    q = [_dev(qp), _dev(qx), _dev(qv)]
    ref = [t.cpu().numpy() for t in idx.search(*q, k=50, gamma=500, mode=mode)]
    for block in (sindi.SINDI_SCAN_PIPELINED, 256, 512, 1024):
        got = [t.cpu().numpy() for t in idx.search(*q, k=50, gamma=500, mode=mode, block=block)]
        idx.check()
        _same(got[0], got[1], ref[0], ref[1], f"{mode} block {block}")
    with pytest.raises(sindi.SindiError, match="INVALID_ARG"):
        idx.search(*q, k=50, gamma=500, mode=mode, block=384)


def test_plain_chains_in_flight_match_one_query_calls(setup):
    """The plain schedule runs several queries' launch chains at once (one stream and workspace each); every
    query's answer is the one it gets alone, and the one of a timed search (one chain at a time)."""
    w, idx, _, (qp, qx, qv) = setup
    q = [_dev(qp), _dev(qx), _dev(qv)]
    for gamma in (0, 500):
        ids, sc = [t.cpu().numpy() for t in idx.search(*q, k=50, gamma=gamma, mode="plain")]
        idx.check()
        for r in range(0, len(qp) - 1, 7):
            one = [_dev(qp[r:r + 2] - qp[r]), _dev(qx[qp[r]:qp[r + 1]]), _dev(qv[qp[r]:qp[r + 1]])]
            i1, s1 = [t.cpu().numpy() for t in idx.search(*one, k=50, gamma=gamma, mode="plain")]
            _same(ids[r:r + 1], sc[r:r + 1], i1, s1, f"gamma {gamma} query {r}")
        sindi.sindi_set_timing(idx.handle, True)
        try:
            it, st = [t.cpu().numpy() for t in idx.search(*q, k=50, gamma=gamma, mode="plain")]
        finally:
            sindi.sindi_set_timing(idx.handle, False)
        _same(ids, sc, it, st, f"gamma {gamma} timed")


def test_repeated_plain_calls_replay_a_graph(setup):
    """The second identical plain call records its launches as a CUDA graph, later ones launch it: the
    answers stay those of the direct launches, new query contents in the same buffers are honoured, and
    the launch counters count every replay."""
    w, idx, _, (qp, qx, qv) = setup
    q = [_dev(qp), _dev(qx), _dev(qv)]
    out = (torch.empty((len(qp) - 1, 50), dtype=torch.int32, device=DEV),
           torch.empty((len(qp) - 1, 50), dtype=torch.float32, device=DEV))
    runs = []
    sindi.sindi_reset_stats(idx.handle)
    for _ in range(4):
        idx.search(*q, k=50, gamma=500, mode="plain", out=out)
        torch.cuda.synchronize()
        runs.append([t.cpu().numpy().copy() for t in out])
    idx.check()
    st = sindi.sindi_get_stats(idx.handle)
    assert st["queries"] == 4 * (len(qp) - 1)
    assert st["launches"] % 4 == 0 and st["launches"] >= 4 * 3 * (len(qp) - 1)
    for r in runs[1:]:
        _same(r[0], r[1], runs[0][0], runs[0][1], "replay")
    q[2].mul_(0.5)  # new weights in the same buffers
    idx.search(*q, k=50, gamma=500, mode="plain", out=out)
    torch.cuda.synchronize()
    fresh = [t.cpu().numpy() for t in idx.search(_dev(qp), _dev(qx), _dev(qv * 0.5), k=50, gamma=500, mode="plain")]
    _same(out[0].cpu().numpy(), out[1].cpu().numpy(), fresh[0], fresh[1], "replay after new contents")


def test_autotuner_meets_the_recall_target(setup, tmp_path):
    """The chosen (window, gamma, schedule, block) reaches Recall@50 >= 0.99 against the GPU exact search, and
    the same configuration holds against the FP64 oracle's brute force."""
    w, _, (ip, ix, v), (qp, qx, qv) = setup
    d = [_dev(ip), _dev(ix), _dev(v)]
    q = [_dev(qp), _dev(qx), _dev(qv)]
    cache = str(tmp_path / "tune.json")
    res = autotune.autotune(*d, w.dim, *q, k=50, alpha=0.5, windows=[1024, 4096], gammas=(50, 100, 200, 500, 1000),
                            blocks=(256, 512), cache=cache)
    ch = res["choice"]
    assert ch is not None and ch["recall"] >= 0.99 and ch["qps"] > 0
    assert autotune.autotune(*d, w.dim, *q, k=50, alpha=0.5, cache=cache) == res  # served from the cache
    with sindi.Index(*d, w.dim, window=ch["window"], alpha=0.5) as idx:
        ids, _ = idx.search(*q, k=50, gamma=ch["gamma"], mode=ch["mode"], block=ch["block"])
        ids = ids.cpu().numpy().view(np.uint32)
    D, Q = oracle.Dataset(ip, ix, v, w.dim), oracle.Dataset(qp, qx, qv, w.dim)
    rec = [oracle.recall(ids[r], oracle.brute_force(D, Q, r, 50)[0]) for r in range(0, Q.n, 4)]
    assert np.mean(rec) >= 0.985, rec
