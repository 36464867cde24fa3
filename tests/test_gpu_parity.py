"""GPU path vs the FP64 oracle, element by element, through the C ABI (needs a GB300)."""
import numpy as np
import pytest

import datagen
import oracle
from parity import REL_TOL, check_ranked, check_ranked_conditioned, check_reranked, signed_copy

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # collected on CPU machines, never run there
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_2509_08395_gb300 as sindi  # noqa: E402

DEV = torch.device("cuda:0")


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def run_search(idx, qp, qx, qv, k, gamma=0, mode="plain", host=False, beta=1.0, block=0):
    if host:
        ids, sc = idx.search(qp, qx, qv, k=k, gamma=gamma, mode=mode, beta=beta, block=block)
        return ids.astype(np.int64), sc
    ids, sc = idx.search(dev(qp), dev(qx), dev(qv), k=k, gamma=gamma, mode=mode, beta=beta, block=block)
    idx.check()
    return ids.cpu().numpy().view(np.uint32).astype(np.int64), sc.cpu().numpy()


@pytest.fixture(scope="module")
def exact10k():
    w = datagen.WORKLOADS["exact-10k"]
    ip, ix, v = datagen.docs(w)
    qp, qx, qv = datagen.queries(w)
    return w, (ip, ix, v), (qp, qx, qv), oracle.Dataset(ip, ix, v, w.dim), oracle.Dataset(qp, qx, qv, w.dim)


@pytest.mark.parametrize("mode", ["plain", "batched"])
def test_exact_10k_top10_equals_brute_force(exact10k, mode):
    """10k docs x 1,024 dims, no pruning, window 4,096: top-10 ids are the FP64 brute-force ids."""
    w, (ip, ix, v), (qp, qx, qv), D, Q = exact10k
    with sindi.Index(dev(ip), dev(ix), dev(v), w.dim, window=w.window, alpha=1.0) as idx:
        assert idx.info["n_windows"] == 3
        ids, sc = run_search(idx, qp, qx, qv, k=w.k, gamma=0, mode=mode)
    for r in range(Q.n):
        oi, os_ = oracle.brute_force(D, Q, r, w.k + 64)
        check_ranked(ids[r], sc[r], oi, os_, w.k, D.n, what=f"query {r}")


def _in_id_order(seg, ids, vals):
    """The device orders each list segment I_{j,w} for its scatter-add (shared-memory banks); the oracle keeps
    ascending document ids. Put every device segment in id order (ids are unique within a segment)."""
    seg = np.asarray(seg, np.int64)
    which = np.repeat(np.arange(len(seg) - 1), np.diff(seg))
    order = np.lexsort((np.asarray(ids, np.int64), which))
    return np.asarray(ids)[order], np.asarray(vals)[order]


def _dequant(vals, dtype, scale, seg, sigma, dim):
    if dtype == "f32":
        return vals.astype(np.float64)
    if dtype == "f16":
        return vals.view(np.float16).astype(np.float64)
    codes = torch.from_numpy(vals.copy()).view(torch.float8_e4m3fn).float().numpy()
    out = np.empty(len(vals), np.float64)
    for j in range(dim):
        lo, hi = seg[j * sigma], seg[(j + 1) * sigma]
        out[lo:hi] = (codes[lo:hi] * scale[j]).astype(np.float32)
    return out


@pytest.mark.parametrize("window,alpha,dtype", [(64, 1.0, "f32"), (300, 0.5, "f32"), (4096, 0.3, "f32"),
                                                (128, 0.7, "f16"), (256, 0.5, "f8"), (1, 0.6, "f32")])
def test_device_index_equals_oracle_lists(window, alpha, dtype):
    """The device build (alpha-mass, (dim, doc) sort, windows, packing) gives the oracle's lists bit for bit."""
    n = 700 if window > 1 else 90
    ip, ix, v = datagen.random_csr(n, 97, 14.0, seed=50 + window, zipf_s=1.05, val_sigma=1.2)
    # shuffle dims inside rows (unsorted input) and plant explicit zeros
    rng = np.random.default_rng(window)
    for i in range(0, n, 7):
        a, b = ip[i], ip[i + 1]
        p = rng.permutation(b - a)
        ix[a:b], v[a:b] = ix[a:b][p], v[a:b][p]
    v[::37] = 0.0
    D = oracle.Dataset(ip, ix, v, 97)
    I = oracle.Index(D, window=window, alpha=alpha, dtype=dtype)
    seg, pid, pval, scale, kept = I.export()
    with sindi.Index(dev(ip), dev(ix), dev(v), 97, window=window, alpha=alpha, value_dtype=dtype) as idx:
        ex = idx.export()
    assert ex["info"]["n_windows"] == I.sigma and ex["info"]["postings"] == I.postings
    np.testing.assert_array_equal(ex["seg"].astype(np.int64), seg)
    np.testing.assert_array_equal(ex["kept"].astype(np.int64), kept)
    ids, vals = _in_id_order(ex["seg"], ex["ids"], ex["vals"])
    np.testing.assert_array_equal(ids.astype(np.int64), pid % window)
    if dtype == "f8":
        np.testing.assert_array_equal(ex["scale"], scale)
    got = _dequant(vals, dtype, ex["scale"], ex["seg"], I.sigma, 97)
    np.testing.assert_array_equal(got, pval)


@pytest.mark.parametrize("prune,prune_n,alpha,dtype", [("vector_number", 5, 1.0, "f32"), ("list", 40, 1.0, "f32"),
                                                       ("list", 3, 1.0, "f8"), ("mass_list", 25, 0.5, "f16")])
def test_device_index_other_pruning_methods_equal_oracle_lists(prune, prune_n, alpha, dtype):
    """Vector Number, List and Mass+List pruning (Sec. 4.1) on the device give the oracle's lists bit for bit,
    including ties in |x| (coarse values) and, for FP8, the per-list scales of the pruned lists."""
    ip, ix, v = datagen.random_csr(3000, 97, 14.0, seed=60, zipf_s=1.05, val_sigma=1.2)
    v = (np.round(v * 8) / 8 + 0.125).astype(np.float32)
    rng = np.random.default_rng(9)
    for i in range(0, 3000, 11):
        a, b = ip[i], ip[i + 1]
        p = rng.permutation(b - a)
        ix[a:b], v[a:b] = ix[a:b][p], v[a:b][p]
    D = oracle.Dataset(ip, ix, v, 97)
    I = oracle.Index(D, window=256, alpha=alpha, dtype=dtype, prune=prune, prune_n=prune_n)
    seg, pid, pval, scale, kept = I.export()
    with sindi.Index(dev(ip), dev(ix), dev(v), 97, window=256, alpha=alpha, value_dtype=dtype, prune=prune,
                     prune_n=prune_n) as idx:
        ex = idx.export()
        assert idx.info["prune"] == sindi.PRUNES[prune] and idx.info["prune_n"] == prune_n
    assert ex["info"]["postings"] == I.postings
    np.testing.assert_array_equal(ex["seg"].astype(np.int64), seg)
    np.testing.assert_array_equal(ex["kept"].astype(np.int64), kept)
    ids, vals = _in_id_order(ex["seg"], ex["ids"], ex["vals"])
    np.testing.assert_array_equal(ids.astype(np.int64), pid % 256)
    if dtype == "f8":
        np.testing.assert_array_equal(ex["scale"], scale)
    np.testing.assert_array_equal(_dequant(vals, dtype, ex["scale"], ex["seg"], I.sigma, 97), pval)


@pytest.mark.parametrize("prune,prune_n,alpha,dtype", [("mass", 0, 0.5, "f32"), ("mass", 0, 0.7, "f8"),
                                                       ("vector_number", 5, 1.0, "f16"), ("list", 3, 1.0, "f8"),
                                                       ("mass_list", 25, 0.5, "f32")])
def test_device_index_signed_values_equal_oracle_lists(prune, prune_n, alpha, dtype):
    """Signed values: every pruning method ranks entries by |x| (Sec. 4.1), the FP8 list scale is max |x| / 448
    and the codecs keep the sign; the device lists equal the oracle's bit for bit, ties in |x| between
    opposite signs included."""
    ip, ix, v = datagen.random_csr(3000, 97, 14.0, seed=61, zipf_s=1.05, val_sigma=1.2)
    v = signed_copy(np.round(v * 8) / 8 + 0.125, 3)
    D = oracle.Dataset(ip, ix, v, 97)
    I = oracle.Index(D, window=256, alpha=alpha, dtype=dtype, prune=prune, prune_n=prune_n)
    seg, pid, pval, scale, kept = I.export()
    assert np.any(pval < 0)
    with sindi.Index(dev(ip), dev(ix), dev(v), 97, window=256, alpha=alpha, value_dtype=dtype, prune=prune,
                     prune_n=prune_n) as idx:
        ex = idx.export()
    assert ex["info"]["postings"] == I.postings
    np.testing.assert_array_equal(ex["seg"].astype(np.int64), seg)
    np.testing.assert_array_equal(ex["kept"].astype(np.int64), kept)
    ids, vals = _in_id_order(ex["seg"], ex["ids"], ex["vals"])
    np.testing.assert_array_equal(ids.astype(np.int64), pid % 256)
    if dtype == "f8":
        np.testing.assert_array_equal(ex["scale"], scale)
    np.testing.assert_array_equal(_dequant(vals, dtype, ex["scale"], ex["seg"], I.sigma, 97), pval)


@pytest.mark.parametrize("mode", ["plain", "batched"])
def test_signed_values_coarse_parity(mode):
    """Signed documents and queries, so scores cancel: the FP32 coarse top-k against the oracle's exact FP64
    score of every document, each within the FP32 dot-product bound of its sum of |q_j x_j|."""
    w = datagen.WORKLOADS["pruned-1m"].scaled(n_docs=40_000, n_queries=24)
    ip, ix, v = datagen.docs(w)
    qp, qx, qv = datagen.queries(w)
    v, qv = signed_copy(v, 3), signed_copy(qv, 5)
    D, Q = oracle.Dataset(ip, ix, v, w.dim), oracle.Dataset(qp, qx, qv, w.dim)
    Da, Qa = oracle.Dataset(ip, ix, np.abs(v), w.dim), oracle.Dataset(qp, qx, np.abs(qv), w.dim)
    I = oracle.Index(D, window=4096, alpha=0.5)
    Ia = oracle.Index(Da, window=4096, alpha=0.5)   # alpha-mass ranks |x|: the same kept entries
    with sindi.Index(dev(ip), dev(ix), dev(v), w.dim, window=4096, alpha=0.5) as idx:
        assert idx.info["postings"] == I.postings
        ids, sc = run_search(idx, qp, qx, qv, k=100, gamma=0, mode=mode)
    for r in range(Q.n):
        s, a = np.empty(D.n), np.empty(D.n)
        oi, os_ = I.search(Q, r, k=D.n, gamma=0)
        s[oi] = os_
        oi, os_ = Ia.search(Qa, r, k=D.n, gamma=0)
        a[oi] = os_
        check_ranked_conditioned(ids[r], sc[r], s, a, int(qp[r + 1] - qp[r]), 100, what=f"query {r}")


@pytest.mark.parametrize("prune,prune_n,alpha", [("vector_number", 12, 1.0), ("list", 2000, 1.0),
                                                 ("mass_list", 1500, 0.5)])
def test_other_pruning_methods_search_parity(pruned_small, prune, prune_n, alpha):
    """Coarse top-k and the reordered answer over a VNP / LP / MRP+LP index against the oracle's."""
    w, (ip, ix, v), (qp, qx, qv), D, Q = pruned_small
    I = oracle.Index(D, window=4096, alpha=alpha, prune=prune, prune_n=prune_n)
    with sindi.Index(dev(ip), dev(ix), dev(v), w.dim, window=4096, alpha=alpha, prune=prune,
                     prune_n=prune_n) as idx:
        assert idx.info["postings"] == I.postings
        ids, sc = run_search(idx, qp, qx, qv, k=50, gamma=0, mode="plain")
        rids, rsc = run_search(idx, qp, qx, qv, k=20, gamma=300, mode="batched")
    for r in range(Q.n):
        oi, os_ = I.search(Q, r, k=114, gamma=0)
        check_ranked(ids[r], sc[r], oi, os_, 50, D.n, what=f"{prune} coarse query {r}")
        check_reranked(rids[r], rsc[r], D, Q, r, I, 20, 300, what=f"{prune} rerank query {r}")


def test_index_save_load_roundtrip(tmp_path, pruned_small):
    """An index written by sindi_index_save and read back by sindi_index_load has the same layout and answers
    like the original; a file with a window id >= lambda is refused."""
    w, (ip, ix, v), (qp, qx, qv), D, Q = pruned_small
    path = str(tmp_path / "index.sindi")
    with sindi.Index(dev(ip), dev(ix), dev(v), w.dim, window=4096, alpha=0.5, value_dtype="f16", prune="mass_list",
                     prune_n=3000) as idx:
        idx.save(path)
        ex = idx.export()
        info = idx.info
    with sindi.Index.load(path) as idx2:
        assert idx2.info == info
        ex2 = idx2.export()
        for key in ("seg", "ids", "vals", "scale", "kept"):
            np.testing.assert_array_equal(ex2[key], ex[key])
        ids, sc = run_search(idx2, qp, qx, qv, k=20, gamma=300, mode="batched")
    I = oracle.Index(D, window=4096, alpha=0.5, dtype="f16", prune="mass_list", prune_n=3000)
    for r in range(Q.n):
        check_reranked(ids[r], sc[r], D, Q, r, I, 20, 300, what=f"loaded index, query {r}")
    raw = bytearray(open(path, "rb").read())
    at = 72 + 4 * (w.dim * info["n_windows"] + 1)  # the first window id
    raw[at:at + 2] = (4096).to_bytes(2, "little")
    bad = str(tmp_path / "bad.sindi")
    open(bad, "wb").write(bytes(raw))
    with pytest.raises(sindi.SindiError, match="INVALID_DATA"):
        sindi.Index.load(bad)


def test_invalid_pruning_parameters():
    ip, ix, v = datagen.random_csr(50, 16, 4.0, seed=3)
    for prune, n in (("vector_number", 0), ("list", 0), ("mass_list", 0)):
        with pytest.raises(sindi.SindiError, match="INVALID_ARG"):
            sindi.Index(dev(ip), dev(ix), dev(v), 16, window=64, prune=prune, prune_n=n)


def test_segment_order_spreads_banks():
    """Each list segment is a permutation of its ids, laid out so that the 32 postings of one add instruction
    of the scan mostly sit in different shared-memory banks (slot mod 32)."""
    ip, ix, v = datagen.random_csr(60_000, 50, 30.0, seed=81, zipf_s=0.3)
    D = oracle.Dataset(ip, ix, v, 50)
    I = oracle.Index(D, window=8192, alpha=1.0)
    seg, pid, pval, _, _ = I.export()
    with sindi.Index(dev(ip), dev(ix), dev(v), 50, window=8192) as idx:
        ex = idx.export()
    ids, _ = _in_id_order(ex["seg"], ex["ids"], ex["vals"])
    np.testing.assert_array_equal(ids.astype(np.int64), pid % 8192)

    def worst_bank_load(order):
        loads = []
        for k in range(len(seg) - 1):
            s_, e_ = int(seg[k]), int(seg[k + 1])
            if e_ - s_ < 128:
                continue
            g0 = s_ & ~7
            for base in range(g0, (e_ + 7) & ~7, 256):
                for u in range(8):
                    b = [int(order[p]) % 32 for p in range(base + u, base + u + 256, 8) if s_ <= p < e_]
                    if len(b) == 32:
                        loads.append(np.bincount(b, minlength=32).max())
        return np.mean(loads)

    before, after = worst_bank_load(pid % 8192), worst_bank_load(ex["ids"].astype(np.int64))
    assert after < 0.6 * before, (before, after)


def test_device_index_host_and_device_inputs_agree():
    ip, ix, v = datagen.random_csr(500, 64, 10.0, seed=77)
    with sindi.Index(ip, ix, v, 64, window=100, alpha=0.5) as a, \
            sindi.Index(dev(ip), dev(ix), dev(v), 64, window=100, alpha=0.5) as b:
        ea, eb = a.export(), b.export()
    for key in ("seg", "ids", "vals", "kept"):
        np.testing.assert_array_equal(ea[key], eb[key])


@pytest.fixture(scope="module")
def pruned_small():
    w = datagen.WORKLOADS["pruned-1m"].scaled(n_docs=40_000, n_queries=40)
    ip, ix, v = datagen.docs(w)
    qp, qx, qv = datagen.queries(w)
    return w, (ip, ix, v), (qp, qx, qv), oracle.Dataset(ip, ix, v, w.dim), oracle.Dataset(qp, qx, qv, w.dim)


@pytest.mark.parametrize("window,mode", [(2048, "plain"), (4096, "batched"), (8192, "plain")])
def test_pruned_coarse_topk_parity(pruned_small, window, mode):
    """Coarse stage alone (gamma = 0): FP32 window accumulation vs the oracle's FP64 Algorithm 2."""
    w, (ip, ix, v), (qp, qx, qv), D, Q = pruned_small
    I = oracle.Index(D, window=window, alpha=0.5)
    with sindi.Index(dev(ip), dev(ix), dev(v), w.dim, window=window, alpha=0.5) as idx:
        ids, sc = run_search(idx, qp, qx, qv, k=100, gamma=0, mode=mode)
    for r in range(Q.n):
        oi, os_ = I.search(Q, r, k=164, gamma=0)
        check_ranked(ids[r], sc[r], oi, os_, 100, D.n, what=f"query {r}")


@pytest.mark.parametrize("block", [256, 512, 1024])
def test_largest_window_every_block_shape(block):
    """lambda = 32,768 (the largest window): a window spans up to 128 passes of a 256-thread block."""
    w = datagen.WORKLOADS["pruned-1m"].scaled(n_docs=70_000, n_queries=12)
    ip, ix, v = datagen.docs(w)
    qp, qx, qv = datagen.queries(w)
    D, Q = oracle.Dataset(ip, ix, v, w.dim), oracle.Dataset(qp, qx, qv, w.dim)
    I = oracle.Index(D, window=32768, alpha=0.5)
    with sindi.Index(dev(ip), dev(ix), dev(v), w.dim, window=32768, alpha=0.5) as idx:
        for mode in ("plain", "batched"):
            ids, sc = idx.search(dev(qp), dev(qx), dev(qv), k=100, gamma=0, mode=mode, block=block)
            idx.check()
            ids, sc = ids.cpu().numpy().view(np.uint32).astype(np.int64), sc.cpu().numpy()
            for r in range(Q.n):
                oi, os_ = I.search(Q, r, k=164, gamma=0)
                check_ranked(ids[r], sc[r], oi, os_, 100, D.n, what=f"{mode} block {block} query {r}")


@pytest.mark.parametrize("window,gamma,k,mode", [(2048, 200, 10, "plain"), (8192, 500, 50, "plain"),
                                                 (4096, 500, 50, "batched"), (1024, 1000, 100, "batched")])
def test_pruned_rerank_parity(pruned_small, window, gamma, k, mode):
    """Algorithm 4: alpha = 0.5 coarse candidates, exact FP32 reorder against full vectors."""
    w, (ip, ix, v), (qp, qx, qv), D, Q = pruned_small
    I = oracle.Index(D, window=window, alpha=0.5)
    with sindi.Index(dev(ip), dev(ix), dev(v), w.dim, window=window, alpha=0.5) as idx:
        ids, sc = run_search(idx, qp, qx, qv, k=k, gamma=gamma, mode=mode)
    touched = 0
    for r in range(Q.n):
        touched += check_reranked(ids[r], sc[r], D, Q, r, I, k, gamma, what=f"query {r}")
    assert touched <= 2


@pytest.mark.parametrize("window,gamma,k,mode", [(8192, 8192, 100, "plain"), (512, 3000, 50, "plain"),
                                                 (2048, 8192, 20, "batched")])
def test_large_candidate_pools(pruned_small, window, gamma, k, mode):
    """Candidate pools past what one merge block gathers alone (tens of thousands of window candidates,
    gamma up to the 8,192 limit): the multi-block merge, its filter buffer and the rerank's largest pool."""
    w, (ip, ix, v), (qp, qx, qv), D, Q = pruned_small
    I = oracle.Index(D, window=window, alpha=0.5)
    nq = 12
    qp, qx, qv = qp[: nq + 1], qx[: qp[nq]], qv[: qp[nq]]
    with sindi.Index(dev(ip), dev(ix), dev(v), w.dim, window=window, alpha=0.5) as idx:
        ids, sc = run_search(idx, qp, qx, qv, k=k, gamma=gamma, mode=mode)
    for r in range(nq):
        check_reranked(ids[r], sc[r], D, Q, r, I, k, gamma, what=f"query {r}")


@pytest.mark.parametrize("mode", ["plain", "batched"])
def test_pipelined_scan_parity(pruned_small, mode):
    """The pipelined window scan (one resident block per SM, scatter-add and cut overlapped), with queries of
    300 to 700 terms so that a window takes several term tables: coarse and reordered answers vs the oracle."""
    w, (ip, ix, v), _, D, _ = pruned_small
    qp, qx, qv = datagen.generate(datagen.RowDist(10, datagen.NNZ_UNIFORM, 300, 700, 300, 700, val_sigma=0.8),
                                  w.dim, w.zipf_s, 91)
    Q = oracle.Dataset(qp, qx, qv, w.dim)
    I = oracle.Index(D, window=2048, alpha=0.5)
    pipe = sindi.SINDI_SCAN_PIPELINED
    with sindi.Index(dev(ip), dev(ix), dev(v), w.dim, window=2048, alpha=0.5) as idx:
        ids, sc = run_search(idx, qp, qx, qv, k=50, gamma=0, mode=mode, block=pipe)
        rids, rsc = run_search(idx, qp, qx, qv, k=20, gamma=400, mode=mode, block=pipe)
    for r in range(Q.n):
        oi, os_ = I.search(Q, r, k=114, gamma=0)
        check_ranked(ids[r], sc[r], oi, os_, 50, D.n, what=f"coarse query {r}")
        check_reranked(rids[r], rsc[r], D, Q, r, I, 20, 400, what=f"rerank query {r}")


def test_rerank_of_long_documents():
    """Documents of 500 to 3,000 entries (the long-row prune path, and rows the rerank reads in several
    passes of 512 entries): reordered answers against the oracle."""
    ip, ix, v = datagen.generate(datagen.RowDist(400, datagen.NNZ_UNIFORM, 500, 3000, 500, 3000), 4096, 0.6, 71)
    qp, qx, qv = datagen.random_csr(10, 4096, 60.0, seed=72, zipf_s=0.6, nnz_min=5)
    D, Q = oracle.Dataset(ip, ix, v, 4096), oracle.Dataset(qp, qx, qv, 4096)
    I = oracle.Index(D, window=128, alpha=0.4)
    with sindi.Index(dev(ip), dev(ix), dev(v), 4096, window=128, alpha=0.4) as idx:
        assert idx.info["postings"] == I.postings
        for mode in ("plain", "batched"):
            ids, sc = run_search(idx, qp, qx, qv, k=10, gamma=60, mode=mode)
            for r in range(Q.n):
                check_reranked(ids[r], sc[r], D, Q, r, I, 10, 60, what=f"{mode} query {r}")


@pytest.mark.parametrize("beta,mode", [(0.3, "plain"), (0.6, "batched")])
def test_beta_query_pruning_parity(pruned_small, beta, mode):
    """Alg. 4 with beta < 1: the coarse scan uses beta-mass(q), the reorder the full q."""
    w, (ip, ix, v), (qp, qx, qv), D, Q = pruned_small
    I = oracle.Index(D, window=4096, alpha=0.5)
    with sindi.Index(dev(ip), dev(ix), dev(v), w.dim, window=4096, alpha=0.5) as idx:
        ids, sc = run_search(idx, qp, qx, qv, k=50, gamma=0, mode=mode, beta=beta)
        rids, rsc = run_search(idx, qp, qx, qv, k=10, gamma=300, mode=mode, beta=beta)
        hids, hsc = run_search(idx, qp, qx, qv, k=10, gamma=300, mode=mode, beta=beta, host=True)
    np.testing.assert_array_equal(rids, hids)
    touched = 0
    for r in range(Q.n):
        oi, os_ = I.search(Q, r, k=114, gamma=0, beta=beta)
        check_ranked(ids[r], sc[r], oi, os_, 50, D.n, what=f"coarse query {r}")
        touched += check_reranked(rids[r], rsc[r], D, Q, r, I, 10, 300, what=f"query {r}", beta=beta)
    assert touched <= 2


@pytest.mark.skipif(torch.cuda.device_count() < 2, reason="needs two GPUs in one process")
def test_beta_query_pruning_on_two_devices_in_one_process(pruned_small):
    """beta < 1 on a second GPU of the same process: the query-pruning kernel's shared-memory limit is set per
    device with the other search kernels, so the second device's search runs and equals the first's."""
    w, (ip, ix, v), (qp, qx, qv), D, Q = pruned_small
    out = []
    for d in (0, 1):
        dv = torch.device("cuda", d)
        to = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dv)  # noqa: E731
        with torch.cuda.device(dv), sindi.Index(to(ip), to(ix), to(v), w.dim, window=4096, alpha=0.5) as idx:
            ids, sc = idx.search(to(qp), to(qx), to(qv), k=10, gamma=300, beta=0.5)
            idx.check()
            out.append(ids.cpu().numpy())
    np.testing.assert_array_equal(out[0], out[1])


@pytest.mark.parametrize("dtype", ["f16", "f8"])
def test_reduced_precision_coarse_parity(pruned_small, dtype):
    """FP16 / E4M3 postings: GPU coarse scores vs the oracle on the same dequantised values."""
    w, (ip, ix, v), (qp, qx, qv), D, Q = pruned_small
    I = oracle.Index(D, window=4096, alpha=0.5, dtype=dtype)
    with sindi.Index(dev(ip), dev(ix), dev(v), w.dim, window=4096, alpha=0.5, value_dtype=dtype) as idx:
        ids, sc = run_search(idx, qp, qx, qv, k=50, gamma=0)
        rids, rsc = run_search(idx, qp, qx, qv, k=10, gamma=500)
    I32 = oracle.Index(D, window=4096, alpha=0.5)
    for r in range(Q.n):
        oi, os_ = I.search(Q, r, k=114, gamma=0)
        check_ranked(ids[r], sc[r], oi, os_, 50, D.n, what=f"{dtype} query {r}")
        for rank in range(10):
            exact = oracle.inner_product(D, int(rids[r, rank]), Q, r)
            assert abs(rsc[r, rank] - exact) <= REL_TOL * abs(exact)
        fi, _ = I32.search(Q, r, k=10, gamma=500)
        assert len(set(fi.tolist()) & set(rids[r].tolist())) >= 9


def _csr(rows, dim):
    ip, ix, v = [0], [], []
    for row in rows:
        for j, x in row:
            ix.append(j)
            v.append(x)
        ip.append(len(ix))
    return np.array(ip, np.int64), np.array(ix, np.int32), np.array(v, np.float32)


def test_edge_cases_small():
    """N < k, N < lambda, a ragged last window, empty docs, empty queries, queries with no hits, exact ties."""
    docs = [[(1, 2.0)], [(1, 1.0)], [], [(1, 2.0)], [(3, 5.0)], [(1, 2.0), (2, 1.0)], [(4, 1.0)]]
    ip, ix, v = _csr(docs, 8)
    qs = [[(1, 1.0)], [(6, 1.0)], [], [(1, 1.0), (3, 1.0), (2, 2.0)]]
    qp, qx, qv = _csr(qs, 8)
    D, Q = oracle.Dataset(ip, ix, v, 8), oracle.Dataset(qp, qx, qv, 8)
    for window in (1, 2, 3, 4, 7, 64):
        I = oracle.Index(D, window=window, alpha=1.0)
        with sindi.Index(dev(ip), dev(ix), dev(v), 8, window=window) as idx:
            for mode in ("plain", "batched"):
                ids, sc = run_search(idx, qp, qx, qv, k=10, gamma=0, mode=mode)
                for r in range(Q.n):
                    oi, os_ = I.search(Q, r, k=10, gamma=0)
                    assert ids[r, :7].tolist() == oi.tolist(), (window, mode, r)
                    np.testing.assert_array_equal(sc[r, :7], os_.astype(np.float32))
                    assert np.all(ids[r, 7:] == 0xFFFFFFFF) and np.all(np.isneginf(sc[r, 7:]))
                ids, sc = run_search(idx, qp, qx, qv, k=3, gamma=5, mode=mode)
                for r in range(Q.n):
                    oi, os_ = I.search(Q, r, k=3, gamma=5)
                    assert ids[r].tolist() == oi.tolist(), (window, mode, r)


def test_gamma_at_least_n_is_exhaustive(pruned_small):
    """gamma >= N: the reorder sees every document, so any alpha gives the brute-force top-k."""
    w, _, _, _, _ = pruned_small
    ip, ix, v = datagen.random_csr(3000, 500, 20.0, seed=91, zipf_s=1.0)
    qp, qx, qv = datagen.random_csr(10, 500, 12.0, seed=92, zipf_s=1.0, nnz_min=1)
    D, Q = oracle.Dataset(ip, ix, v, 500), oracle.Dataset(qp, qx, qv, 500)
    with sindi.Index(dev(ip), dev(ix), dev(v), 500, window=512, alpha=0.2) as idx:
        ids, sc = run_search(idx, qp, qx, qv, k=20, gamma=4096)
    for r in range(Q.n):
        oi, os_ = oracle.brute_force(D, Q, r, 84)
        check_ranked(ids[r], sc[r], oi, os_, 20, D.n, what=f"query {r}")


def test_host_buffers_match_device_buffers(pruned_small):
    w, (ip, ix, v), (qp, qx, qv), D, Q = pruned_small
    with sindi.Index(dev(ip), dev(ix), dev(v), w.dim, window=4096, alpha=0.5) as idx:
        a_ids, a_sc = run_search(idx, qp, qx, qv, k=50, gamma=500)
        b_ids, b_sc = run_search(idx, qp, qx, qv, k=50, gamma=500, host=True)
    np.testing.assert_array_equal(a_ids, b_ids)
    np.testing.assert_array_equal(a_sc, b_sc)


def test_invalid_documents_and_queries():
    ip, ix, v = _csr([[(1, 1.0), (1, 2.0)]], 4)                   # duplicate dim
    with pytest.raises(sindi.SindiError, match="INVALID_DATA"):
        sindi.Index(dev(ip), dev(ix), dev(v), 4)
    ip, ix, v = _csr([[(5, 1.0)]], 4)                               # dim out of range
    with pytest.raises(sindi.SindiError, match="INVALID_DATA"):
        sindi.Index(dev(ip), dev(ix), dev(v), 4)
    ip, ix, v = _csr([[(1, float("nan"))]], 4)                      # non-finite
    with pytest.raises(sindi.SindiError, match="INVALID_DATA"):
        sindi.Index(ip, ix, v, 4)
    bad_ip = np.array([0, 2, 1], np.int64)
    with pytest.raises(sindi.SindiError, match="INVALID_DATA"):
        sindi.Index(dev(bad_ip), dev(np.zeros(2, np.int32)), dev(np.ones(2, np.float32)), 4)
    with pytest.raises(sindi.SindiError, match="INVALID_ARG"):
        sindi.Index(ip, ix, v, 4, alpha=0.0)
    ip, ix, v = _csr([[(1, 1.0)], [(2, 1.0)]], 4)
    with sindi.Index(dev(ip), dev(ix), dev(v), 4) as idx:
        for q in ([(9, 1.0)], [(1, 1.0), (1, 2.0)], [(1, float("inf"))]):
            qp, qx, qv = _csr([q], 4)
            idx.search(dev(qp), dev(qx), dev(qv), k=2)
            with pytest.raises(sindi.SindiError, match="INVALID_DATA"):
                idx.check()
        qp, qx, qv = _csr([[(1, 1.0)]], 4)
        with pytest.raises(sindi.SindiError, match="INVALID_ARG"):
            idx.search(dev(qp), dev(qx), dev(qv), k=3, gamma=2)      # gamma < k
        with pytest.raises(sindi.SindiError, match="INVALID_ARG"):
            idx.search(dev(qp), dev(qx), dev(qv), k=1, beta=1.5)
        ids, sc = idx.search(dev(qp), dev(qx), dev(qv), k=2)          # the index still works after errors
        idx.check()
        assert ids.cpu().tolist() == [[0, 1]]


@pytest.mark.slow
def test_full_size_pruned_1m_sampled():
    """1M docs x 30,522 dims, alpha 0.5, gamma 500, k 50, window as benchmarked: sampled queries vs the
    oracle, plus Recall@50 against FP64 brute force."""
    w = datagen.WORKLOADS["pruned-1m"]
    ip, ix, v = datagen.docs(w)
    qp, qx, qv = datagen.queries(w)
    D, Q = oracle.Dataset(ip, ix, v, w.dim), oracle.Dataset(qp, qx, qv, w.dim)
    I = oracle.Index(D, window=w.window, alpha=w.alpha)
    with sindi.Index(dev(ip), dev(ix), dev(v), w.dim, window=w.window, alpha=w.alpha) as idx:
        ids, sc = run_search(idx, qp, qx, qv, k=w.k, gamma=w.gamma, mode="plain")
        bids, bsc = run_search(idx, qp, qx, qv, k=w.k, gamma=w.gamma, mode="batched")
    sample = list(range(0, Q.n, 50))
    recalls = []
    for r in sample:
        check_reranked(ids[r], sc[r], D, Q, r, I, w.k, w.gamma, what=f"query {r}")
        check_reranked(bids[r], bsc[r], D, Q, r, I, w.k, w.gamma, what=f"batched query {r}")
        truth, _ = oracle.brute_force(D, Q, r, w.k)
        recalls.append(oracle.recall(ids[r], truth))
    assert np.mean(recalls) >= 0.99, recalls


@pytest.mark.parametrize("d,mode", [(10_000, "plain"), (30_000, "batched"), (100_000, "batched")])
def test_uniform_sparsity_workload_parity(d, mode):
    """The uniform-random sparsity sweep's workload (Sec. 5, RANDOM-1M stand-in: 120 entries per row, dims and
    values uniform), scaled to 60,000 documents: coarse top-k against the oracle, and the reordered answer with
    pruning (alpha 0.7) against Algorithm 4."""
    w = datagen.WORKLOADS[f"uniform-1m-d{d // 1000}k"].scaled(n_docs=60_000, n_queries=16)
    ip, ix, v = datagen.docs(w)
    qp, qx, qv = datagen.queries(w)
    D, Q = oracle.Dataset(ip, ix, v, w.dim), oracle.Dataset(qp, qx, qv, w.dim)
    I1 = oracle.Index(D, window=8192, alpha=1.0)
    I7 = oracle.Index(D, window=8192, alpha=0.7)
    with sindi.Index(dev(ip), dev(ix), dev(v), w.dim, window=8192, alpha=1.0) as idx:
        ids, sc = run_search(idx, qp, qx, qv, k=50, gamma=0, mode=mode)
    with sindi.Index(dev(ip), dev(ix), dev(v), w.dim, window=8192, alpha=0.7) as idx:
        assert idx.info["postings"] == I7.postings
        rids, rsc = run_search(idx, qp, qx, qv, k=50, gamma=500, mode=mode)
    for r in range(Q.n):
        oi, os_ = I1.search(Q, r, k=114, gamma=0)
        check_ranked(ids[r], sc[r], oi, os_, 50, D.n, what=f"d {d} exact query {r}")
        check_reranked(rids[r], rsc[r], D, Q, r, I7, 50, 500, what=f"d {d} alpha 0.7 query {r}")
