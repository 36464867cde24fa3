"""sindi_search_noalloc: the search for callers that cannot allocate device memory.

Some callers fix their device memory at start-up, or hand every allocation to
a framework that owns the GPU, or run a latency-critical loop where the
implicit synchronisation of an allocation is not allowed. For them the library
offers one entry point that takes all working memory from a static 8 MiB
device array. This file checks, through the C ABI, that it returns what
sindi_search returns (same tolerance as the parity tests) on two calls in a
row, since the array keeps the previous call's contents, and that it refuses
work that does not fit. It is collected last on purpose.
"""
import numpy as np
import pytest

import datagen
from parity import REL_TOL, tie_groups

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_2509_08395_gb300 as sindi  # noqa: E402

DEV = torch.device("cuda:0")


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def _same_results(ids, sc, ref_ids, ref_sc, what):
    """Equal within the parity tolerance: scores close; ids equal across every gap wider than it."""
    np.testing.assert_allclose(sc, ref_sc, rtol=REL_TOL, atol=0, err_msg=what)
    for r in range(ref_ids.shape[0]):
        for a, b in tie_groups(ref_sc[r].astype(np.float64)):
            if b < ref_ids.shape[1]:
                assert set(ids[r, a:b].tolist()) == set(ref_ids[r, a:b].tolist()), (what, r, a, b)
            else:
                # the group that straddles rank k may be cut differently
                assert len(set(ids[r, a:b].tolist())) == b - a, (what, r)


@pytest.fixture(scope="module")
def index_and_queries():
    w = datagen.WORKLOADS["pruned-1m"].scaled(n_docs=30_000, n_queries=24)
    ip, ix, v = datagen.docs(w)
    qp, qx, qv = datagen.queries(w)
    idx = sindi.Index(_dev(ip), _dev(ix), _dev(v), w.dim, window=4096, alpha=0.5)
    yield idx, (_dev(qp), _dev(qx), _dev(qv)), len(qp) - 1
    idx.close()


@pytest.mark.parametrize("k,gamma,mode", [(50, 500, "plain"), (10, 0, "plain"), (50, 500, "batched"),
                                          (100, 1000, "batched")])
def test_noalloc_matches_search_on_two_calls_in_a_row(index_and_queries, k, gamma, mode):
    idx, q, nq = index_and_queries
    ref_ids, ref_sc = idx.search(*q, k=k, gamma=gamma, mode=mode)
    idx.check()
    ref_ids = ref_ids.cpu().numpy().view(np.uint32)
    ref_sc = ref_sc.cpu().numpy()
    for call in range(2):
        ids = torch.full((nq, k), -7, dtype=torch.int32, device=DEV)
        sc = torch.full((nq, k), 123.0, dtype=torch.float32, device=DEV)
        sindi.sindi_search_noalloc(idx.handle, *q, nq, ids, sc, k=k, gamma=gamma, mode=mode)
        idx.check()
        _same_results(ids.cpu().numpy().view(np.uint32), sc.cpu().numpy(), ref_ids, ref_sc,
                      f"call {call}, k={k}, gamma={gamma}, {mode}")


def test_noalloc_refuses_what_does_not_fit_and_host_buffers():
    # 1.2M one-entry documents, window 1,024, gamma 8,192: one query's candidate buffer alone is
    # 1,172 windows x 2 x 1,024 x 8 B = 19.2 MB, more than the 8 MiB array
    n, dim = 1_200_000, 100
    rng = np.random.default_rng(1)
    ip = np.arange(n + 1, dtype=np.int64)
    ix = rng.integers(0, dim, n).astype(np.int32)
    v = np.ones(n, np.float32)
    with sindi.Index(_dev(ip), _dev(ix), _dev(v), dim, window=1024) as idx:
        qp, qx, qv = _dev(np.array([0, 2], np.int64)), _dev(np.array([3, 5], np.int32)), _dev(np.ones(2, np.float32))
        ids = torch.empty((1, 10), dtype=torch.int32, device=DEV)
        sc = torch.empty((1, 10), dtype=torch.float32, device=DEV)
        with pytest.raises(sindi.SindiError, match="UNSUPPORTED.*static scratch"):
            sindi.sindi_search_noalloc(idx.handle, qp, qx, qv, 1, ids, sc, k=10, gamma=8192)
        # what fits still works on the same index afterwards
        sindi.sindi_search_noalloc(idx.handle, qp, qx, qv, 1, ids, sc, k=10, gamma=0)
        idx.check()
        ref_ids, ref_sc = idx.search(qp, qx, qv, k=10, gamma=0)
        np.testing.assert_array_equal(ids.cpu().numpy(), ref_ids.cpu().numpy())
        with pytest.raises(sindi.SindiError, match="INVALID_ARG"):
            sindi.sindi_search_noalloc(idx.handle, qp.cpu().numpy(), qx.cpu().numpy(), qv.cpu().numpy(), 1,
                                       ids, sc, k=10)
