"""The fixed-point score window (sindi_accumulator FIXED32) against the FP64 oracle (needs a GB300).

The window holds 32-bit integers in units of 2^-e per (query, window); a coarse score of m products is within
the FP32 dot-product bound of its products plus m * 2^-(e+1) <= m * B * 2^-30 of the exact score (parity.
fixed_extra). These tests check that bound on every returned score, the answer's ids against it, the
independence of the sums from the order of the adds, and the unit's adaptation to the data's magnitude."""
import ctypes

import numpy as np
import pytest

import datagen
import oracle
from parity import check_ranked_conditioned, check_reranked, fixed_extra, signed_copy

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # collected on CPU machines, never run there
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_2509_08395_gb300 as sindi  # noqa: E402
import paper_2509_08395_gb300.sindi as native  # noqa: E402

DEV = torch.device("cuda:0")


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def search(idx, q, k, gamma=0, mode="plain", accum="fixed32", block=0):
    ids, sc = idx.search(*(dev(a) for a in q), k=k, gamma=gamma, mode=mode, accum=accum, block=block)
    idx.check()
    return ids.cpu().numpy().view(np.uint32).astype(np.int64), sc.cpu().numpy()


def exact_scores(I, Ia, Q, Qa, n, r):
    """Exact FP64 coarse score of every document and its sum of |products| (the oracle over |x| and |q|)."""
    s, a = np.empty(n), np.empty(n)
    oi, os_ = I.search(Q, r, k=n, gamma=0)
    s[oi] = os_
    oi, os_ = Ia.search(Qa, r, k=n, gamma=0)
    a[oi] = os_
    return s, a


def _workload(n_docs, n_queries, signed, scale=1.0):
    w = datagen.WORKLOADS["pruned-1m"].scaled(n_docs=n_docs, n_queries=n_queries)
    ip, ix, v = datagen.docs(w)
    qp, qx, qv = datagen.queries(w)
    if signed:
        v, qv = signed_copy(v, 3), signed_copy(qv, 5)
    v = (v * np.float32(scale)).astype(np.float32)
    qv = (qv * np.float32(scale)).astype(np.float32)
    return w, (ip, ix, v), (qp, qx, qv)


@pytest.mark.parametrize("mode,signed,window", [("plain", False, 4096), ("batched", False, 2048),
                                                ("plain", True, 4096), ("batched", True, 8192)])
def test_fixed_window_coarse_parity(mode, signed, window):
    """gamma = 0 with the fixed-point window: every returned score within its bound of the exact FP64 score,
    scores descending, and no document left out that certainly beats a returned one."""
    w, (ip, ix, v), (qp, qx, qv) = _workload(40_000, 24, signed)
    D, Q = oracle.Dataset(ip, ix, v, w.dim), oracle.Dataset(qp, qx, qv, w.dim)
    Da, Qa = oracle.Dataset(ip, ix, np.abs(v), w.dim), oracle.Dataset(qp, qx, np.abs(qv), w.dim)
    I = oracle.Index(D, window=window, alpha=0.5)
    Ia = oracle.Index(Da, window=window, alpha=0.5)   # alpha-mass ranks |x|: the same kept entries
    with sindi.Index(dev(ip), dev(ix), dev(v), w.dim, window=window, alpha=0.5) as idx:
        ids, sc = search(idx, (qp, qx, qv), k=100, mode=mode)
    for r in range(Q.n):
        s, a = exact_scores(I, Ia, Q, Qa, D.n, r)
        check_ranked_conditioned(ids[r], sc[r], s, a, int(qp[r + 1] - qp[r]), 100, what=f"query {r}",
                                 extra=fixed_extra(I, Q, r))


@pytest.mark.parametrize("scale", [1e-12, 1e12])
def test_fixed_window_unit_follows_the_data(scale):
    """Values 10^12 times smaller or larger: the window's unit 2^-e moves with B, so the same bound holds (a
    fixed unit would round every product to zero, or overflow)."""
    w, (ip, ix, v), (qp, qx, qv) = _workload(20_000, 12, False, scale)
    D, Q = oracle.Dataset(ip, ix, v, w.dim), oracle.Dataset(qp, qx, qv, w.dim)
    I = oracle.Index(D, window=4096, alpha=0.5)
    with sindi.Index(dev(ip), dev(ix), dev(v), w.dim, window=4096, alpha=0.5) as idx:
        ids, sc = search(idx, (qp, qx, qv), k=50, mode="batched")
        rids, rsc = search(idx, (qp, qx, qv), k=20, gamma=300, mode="plain", accum="auto")
    for r in range(Q.n):
        s, a = exact_scores(I, I, Q, Q, D.n, r)   # non-negative data: a = s
        check_ranked_conditioned(ids[r], sc[r], s, a, int(qp[r + 1] - qp[r]), 50, what=f"query {r}",
                                 extra=fixed_extra(I, Q, r))
        check_reranked(rids[r], rsc[r], D, Q, r, I, 20, 300, what=f"rerank query {r}")


def test_fixed_window_sums_do_not_depend_on_the_order_of_the_adds():
    """Integer sums are exact: the same search twice, and the plain and batched schedules (different blocks
    and different orders of the atomic adds, the same 512-thread block shape and so the same unit), give
    bit-identical scores and ids, with and without the reorder."""
    w, (ip, ix, v), (qp, qx, qv) = _workload(40_000, 40, False)
    with sindi.Index(dev(ip), dev(ix), dev(v), w.dim, window=4096, alpha=0.5) as idx:
        for gamma, accum in ((0, "fixed32"), (300, "auto")):
            a = search(idx, (qp, qx, qv), k=50, gamma=gamma, mode="plain", accum=accum)
            b = search(idx, (qp, qx, qv), k=50, gamma=gamma, mode="plain", accum=accum)
            c = search(idx, (qp, qx, qv), k=50, gamma=gamma, mode="batched", accum=accum)
            for x in (b, c):
                np.testing.assert_array_equal(a[0], x[0])
                np.testing.assert_array_equal(a[1].view(np.uint32), x[1].view(np.uint32))


@pytest.mark.parametrize("mode", ["plain", "batched"])
def test_fixed_window_queries_longer_than_one_term_table(mode):
    """Queries of 700 distinct terms, more than one 512-term table holds: the window's unit comes from a pass
    of its own over all the query's terms before the first table's adds. Coarse scores within the bound of
    the exact FP64 scores, descending, and no left-out document certainly beats a returned one."""
    w, (ip, ix, v), _ = _workload(40_000, 2, False)
    rng = np.random.default_rng(21)
    nq, nt = 6, 700
    qx = np.concatenate([np.sort(rng.choice(w.dim, nt, replace=False)) for _ in range(nq)]).astype(np.int32)
    qv = rng.lognormal(0.0, 0.8, nq * nt).astype(np.float32)
    qp = np.arange(0, nq * nt + 1, nt, dtype=np.int64)
    D, Q = oracle.Dataset(ip, ix, v, w.dim), oracle.Dataset(qp, qx, qv, w.dim)
    I = oracle.Index(D, window=4096, alpha=0.5)
    with sindi.Index(dev(ip), dev(ix), dev(v), w.dim, window=4096, alpha=0.5) as idx:
        ids, sc = search(idx, (qp, qx, qv), k=50, mode=mode)
    for r in range(Q.n):
        s, a = exact_scores(I, I, Q, Q, D.n, r)
        check_ranked_conditioned(ids[r], sc[r], s, a, nt, 50, what=f"query {r}", extra=fixed_extra(I, Q, r))


@pytest.mark.parametrize("mode", ["plain", "batched"])
def test_fixed_window_falls_back_to_the_full_cut_on_crowded_bounds(mode):
    """40,000 documents of one score (exact ties) but 20 higher ones: every bounded fixed-point window holds far
    more slots at the bound than it may emit, so it converts its sums to FP32 and falls back on the full cut.
    The answer's scores must be the exact ones (a cut that kept reading FP32 bits as fixed-point sums would
    return scores thousands of times too large), descending, and no document left out may certainly beat a
    returned one."""
    n, dim = 40_000, 16
    rows = [[(1, 1.0), (2, 0.5), (3, 0.25)] for _ in range(n)]
    rng = np.random.default_rng(11)
    for i in rng.choice(n, 20, replace=False):
        rows[i] = [(1, 1.5), (2, 0.5), (3, 0.25)]
    ip = np.array([0] + [3 * (i + 1) for i in range(n)], np.int64)
    ix = np.array([j for r in rows for j, _ in r], np.int32)
    v = np.array([x for r in rows for _, x in r], np.float32)
    qp = np.array([0, 3, 5], np.int64)
    qx = np.array([1, 2, 3, 1, 3], np.int32)
    qv = np.array([1.0, 1.0, 1.0, 2.0, 0.5], np.float32)
    D, Q = oracle.Dataset(ip, ix, v, dim), oracle.Dataset(qp, qx, qv, dim)
    I = oracle.Index(D, window=4096, alpha=1.0)
    with sindi.Index(dev(ip), dev(ix), dev(v), dim, window=4096, alpha=1.0) as idx:
        ids, sc = search(idx, (qp, qx, qv), k=50, mode=mode)
    for r in range(Q.n):
        s, a = exact_scores(I, I, Q, Q, D.n, r)
        check_ranked_conditioned(ids[r], sc[r], s, a, int(qp[r + 1] - qp[r]), 50, what=f"query {r}",
                                 extra=fixed_extra(I, Q, r))


def test_plain_lanes_reuse_workspaces_across_queries():
    """The plain schedule runs a lane's queries one after another on one workspace, which each query's merge
    leaves at zero for the next. With gamma 2,000 most queries' candidates exceed one merge block's filter
    buffer, so both merge blocks read the query's histogram before the workspace is reset. 200 queries (about
    8 per lane): three plain calls and the batched schedule give bit-identical answers, and sampled rows
    reorder to the oracle's answer."""
    w, (ip, ix, v), (qp, qx, qv) = _workload(40_000, 200, False)
    D, Q = oracle.Dataset(ip, ix, v, w.dim), oracle.Dataset(qp, qx, qv, w.dim)
    I = oracle.Index(D, window=4096, alpha=0.5)
    with sindi.Index(dev(ip), dev(ix), dev(v), w.dim, window=4096, alpha=0.5) as idx:
        runs = [search(idx, (qp, qx, qv), k=20, gamma=2000, mode="plain", accum="auto") for _ in range(3)]
        runs.append(search(idx, (qp, qx, qv), k=20, gamma=2000, mode="batched", accum="auto"))
    for x in runs[1:]:
        np.testing.assert_array_equal(runs[0][0], x[0])
        np.testing.assert_array_equal(runs[0][1].view(np.uint32), x[1].view(np.uint32))
    for r in range(0, Q.n, 13):
        check_reranked(runs[0][0][r], runs[0][1][r], D, Q, r, I, 20, 2000, what=f"query {r}")


@pytest.mark.parametrize("mode", ["plain", "batched"])
def test_both_windows_reorder_to_the_oracle_answer(mode):
    """gamma > 0 with either window (FP32 atomics, or the default fixed point): each answer is the oracle's
    Algorithm 4 answer under the rounding of its own window."""
    w, (ip, ix, v), (qp, qx, qv) = _workload(40_000, 30, False)
    D, Q = oracle.Dataset(ip, ix, v, w.dim), oracle.Dataset(qp, qx, qv, w.dim)
    I = oracle.Index(D, window=4096, alpha=0.5)
    with sindi.Index(dev(ip), dev(ix), dev(v), w.dim, window=4096, alpha=0.5) as idx:
        fx = search(idx, (qp, qx, qv), k=20, gamma=400, mode=mode, accum="auto")
        f32 = search(idx, (qp, qx, qv), k=20, gamma=400, mode=mode, accum="f32")
    for r in range(Q.n):
        check_reranked(fx[0][r], fx[1][r], D, Q, r, I, 20, 400, what=f"fixed query {r}")
        check_reranked(f32[0][r], f32[1][r], D, Q, r, I, 20, 400, what=f"f32 query {r}", fixed=False)


@pytest.mark.parametrize("dtype", ["f16", "f8"])
def test_fixed_window_reduced_precision_postings(dtype):
    """FP16 / E4M3 postings (the E4M3 list scale folded into the term weight) with the fixed-point window:
    coarse scores within the bound of the oracle's scores on the same dequantised values."""
    w, (ip, ix, v), (qp, qx, qv) = _workload(30_000, 16, False)
    D, Q = oracle.Dataset(ip, ix, v, w.dim), oracle.Dataset(qp, qx, qv, w.dim)
    I = oracle.Index(D, window=4096, alpha=0.5, dtype=dtype)
    with sindi.Index(dev(ip), dev(ix), dev(v), w.dim, window=4096, alpha=0.5, value_dtype=dtype) as idx:
        ids, sc = search(idx, (qp, qx, qv), k=50, mode="plain")
    for r in range(Q.n):
        s, a = exact_scores(I, I, Q, Q, D.n, r)
        check_ranked_conditioned(ids[r], sc[r], s, a, int(qp[r + 1] - qp[r]), 50, what=f"{dtype} query {r}",
                                 extra=fixed_extra(I, Q, r))


def test_accumulator_outside_the_enum_is_rejected():
    w, (ip, ix, v), (qp, qx, qv) = _workload(2_000, 2, False)
    with sindi.Index(dev(ip), dev(ix), dev(v), w.dim, window=1024, alpha=0.5) as idx:
        q = [dev(a) for a in (qp, qx, qv)]
        ids = torch.empty((2, 10), dtype=torch.int32, device=DEV)
        sc = torch.empty((2, 10), dtype=torch.float32, device=DEV)
        prm = native.sindi_search_params(k=10, gamma=0, beta=1.0, mode=0, block_threads=0, group=0, accumulator=3)
        st = native.load().sindi_search(ctypes.c_void_p(idx.handle), ctypes.c_void_p(q[0].data_ptr()),
                                        ctypes.c_void_p(q[1].data_ptr()), ctypes.c_void_p(q[2].data_ptr()), 2,
                                        ctypes.byref(prm), ctypes.c_void_p(ids.data_ptr()),
                                        ctypes.c_void_p(sc.data_ptr()),
                                        ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
        assert st == native.SINDI_ERR_INVALID_ARG
        assert b"accumulator" in native.load().sindi_last_error()
