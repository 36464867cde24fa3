"""Pins of the FP64 oracle against facts fixed outside the oracle itself.

Each test names what it pins and where that fact comes from: the paper's
worked examples (tests/golden, with citations), closed forms, library
routines (scipy.sparse products and transposes, numpy float16, torch
float8_e4m3fn), invariants the paper states, and brute force on tiny inputs.
"""
import itertools
import json
import os
from fractions import Fraction

import numpy as np
import pytest
import scipy.sparse as sp

import datagen
import oracle


def _csr_from_dicts(rows):
    indptr, idx, val = [0], [], []
    for r in rows:
        for j in sorted(int(k) for k in r):
            idx.append(j)
            val.append(r[str(j)] if str(j) in r else r[j])
        indptr.append(len(idx))
    return np.array(indptr, np.int64), np.array(idx, np.int32), np.array(val, np.float32)


def _scipy(ip, ix, v, dim):
    return sp.csr_matrix((v.astype(np.float64), ix, ip), shape=(len(ip) - 1, dim))


# --------------------------------------------------------------------------
# Worked example of Sec. 3.2 (figure "An Example of SINDI and Query Process")
# --------------------------------------------------------------------------
@pytest.fixture(scope="module")
def worked(golden_dir):
    with open(os.path.join(golden_dir, "worked_example.json")) as f:
        g = json.load(f)
    ip, ix, v = _csr_from_dicts(g["docs"])
    D = oracle.Dataset(ip, ix, v, g["dim"])
    return g, D


def _query(g, dims):
    q = {str(j): g["query"][str(j)] for j in dims}
    ip, ix, v = _csr_from_dicts([q])
    return oracle.Dataset(ip, ix, v, g["dim"])


def test_worked_example_accumulation_steps(worked):
    """A[4] after I_1 is 17.0, after I_5 is 31.0, final 36.1 = delta(x_4, q) (Sec. 3.2 example)."""
    g, D = worked
    facts = g["paper_facts"]
    assert D.n == facts["n_docs"]
    assert g["query"]["1"] * g["docs"][4]["1"] == pytest.approx(facts["after_I1_A4"], rel=1e-6)
    # one window spanning all 9 docs: the distance array of size 9 in the example
    I = oracle.Index(D, window=9, alpha=1.0)
    for dims, expect in [([1], facts["after_I1_A4"]), ([1, 5], facts["after_I5_A4"]),
                         ([1, 5, 8], facts["final_A4"])]:
        Q = _query(g, dims)
        ids, sc = I.search(Q, 0, k=9, gamma=0)
        s4 = dict(zip(ids.tolist(), sc.tolist()))[4]
        assert s4 == pytest.approx(expect, rel=1e-6)
    Q = _query(g, [1, 5, 8])
    ids, sc = I.search(Q, 0, k=9, gamma=0)
    assert ids[0] == facts["argmax"]
    assert sc[0] == pytest.approx(oracle.inner_product(D, 4, Q, 0), rel=0, abs=0)
    scored = sorted(int(i) for i, s in zip(ids, sc) if s != 0.0)
    assert scored == facts["scored_docs"]
    # x_4's entry in dim 2 is outside Omega(x_4, q) and must not contribute
    assert g["docs"][4].get(str(facts["x4_has_dim_outside_query"])) is not None
    assert oracle.inner_product(D, 4, Q, 0) == pytest.approx(6.8 * 2.5 + 7.0 * 2.0 + 3.4 * 1.5, rel=1e-6)


def test_worked_example_window_invariance(worked):
    """Window Switch changes only the visit order (Sec. 3.3.1): every lambda gives identical FP64 scores."""
    g, D = worked
    Q = _query(g, [1, 5, 8])
    ref = oracle.Index(D, window=9).search(Q, 0, k=9, gamma=0)
    for lam in (1, 2, 3, 4, 5, 8, 16):
        got = oracle.Index(D, window=lam).search(Q, 0, k=9, gamma=0)
        assert np.array_equal(got[0], ref[0]) and np.array_equal(got[1], ref[1])


def test_worked_example_brute_force(worked):
    g, D = worked
    Q = _query(g, [1, 5, 8])
    ids, sc = oracle.brute_force(D, Q, 0, 3)
    assert ids[0] == 4
    assert sc[0] == pytest.approx(36.1, rel=1e-6)


# --------------------------------------------------------------------------
# alpha-mass (Definitions "Mass of a Vector", "alpha-Mass Subvector")
# --------------------------------------------------------------------------
def test_alpha_mass_paper_vector(golden_dir):
    with open(os.path.join(golden_dir, "alpha_mass_example.json")) as f:
        g = json.load(f)
    dims, vals = g["vector"]["dims"], g["vector"]["values"]
    assert len(dims) == g["paper_facts"]["nnz"]
    for case in g["hand_derived"]:
        pos = oracle.alpha_mass(dims, vals, case["alpha"])
        assert len(pos) == case["r"], case
        assert [dims[p] for p in pos] == case["kept_dims"], case
    # the alpha = 0.7 case also holds in pure FP64 (no FP32 widening)
    s = 0.0
    for v in (0.8, 0.6):
        s += v
    assert s >= 0.7 * (0.8 + 0.6 + 0.4 + 0.2) and 0.8 < 0.7 * 2.0


def test_alpha_mass_dyadic_boundary(golden_dir):
    with open(os.path.join(golden_dir, "alpha_mass_example.json")) as f:
        g = json.load(f)["dyadic_boundary"]
    for case in g["cases"]:
        pos = oracle.alpha_mass(g["dims"], g["values"], case["alpha"])
        assert [g["dims"][p] for p in pos] == case["kept_dims"], case


def test_alpha_mass_brute_force_subsets():
    """r = the minimum size of ANY subset whose |x| sum reaches alpha * mass (exact rational
    arithmetic over all subsets), and the kept entries are the largest |x| (ties: lower dim)."""
    rng = np.random.default_rng(7)
    checked = 0
    for trial in range(300):
        n = int(rng.integers(1, 9))
        dims = sorted(rng.choice(50, size=n, replace=False).tolist())
        vals = rng.lognormal(0, 1, size=n).astype(np.float32)
        if trial % 5 == 0:                           # force ties in |x|
            vals[: n // 2] = vals[0]
        if trial % 7 == 0:
            vals = -vals                             # negative entries: |x| drives the order
        alpha = float(rng.choice([0.1, 0.3, 0.5, 0.7, 0.9, 0.999, 1.0]))
        mags = [Fraction(abs(float(v))) for v in vals]
        target = Fraction(alpha) * sum(mags, Fraction(0))
        best = None
        for size in range(1, n + 1):
            if any(sum((mags[i] for i in c), Fraction(0)) >= target for c in itertools.combinations(range(n), size)):
                best = size
                break
        pos = oracle.alpha_mass(dims, vals, alpha)
        if alpha < 1.0:
            # FP64 rounding may move r only when the threshold sits within rounding of a prefix
            srt = sorted(mags, reverse=True)
            prefix = [sum(srt[: t + 1], Fraction(0)) for t in range(n)]
            near = any(abs(float(p - target)) <= 1e-12 * float(target) for p in prefix)
            if near:
                continue
            assert len(pos) == best, (dims, vals, alpha)
        else:
            assert len(pos) == n
        kept = set(int(p) for p in pos)
        order = sorted(range(n), key=lambda i: (-abs(float(vals[i])), dims[i]))
        assert [int(p) for p in pos] == order[: len(pos)]
        assert all(abs(vals[a]) >= abs(vals[b]) for a in kept for b in range(n) if b not in kept)
        checked += 1
    assert checked > 250


def test_alpha_one_keeps_entries_below_fp64_resolution():
    """alpha = 1: with every entry non-zero, no proper prefix reaches the whole mass in exact arithmetic, so
    r = nnz, also when the tail lies below the FP64 resolution of the mass (an FP64 prefix sum would
    reach the mass after the first entry)."""
    dims = [0, 3, 7]
    vals = np.array([1.0, 2.0 ** -60, 2.0 ** -70], np.float32)
    mags = [Fraction(float(x)) for x in vals]
    assert sum(mags[:2], Fraction(0)) < sum(mags, Fraction(0))
    assert 1.0 + 2.0 ** -60 + 2.0 ** -70 == 1.0             # the FP64 sum loses the tail
    assert sorted(int(p) for p in oracle.alpha_mass(dims, vals, 1.0)) == [0, 1, 2]
    D = oracle.Dataset(np.array([0, 3], np.int64), np.array(dims, np.int32), vals, 8)
    _, kept = _entries(oracle.Index(D, window=4, alpha=1.0))
    assert kept.tolist() == [3]


# --------------------------------------------------------------------------
# Definition 2 / 3 against library routines and hand-computed values
# --------------------------------------------------------------------------
def test_inner_product_hand_values():
    # x = {0: 1.5, 2: -2.0, 7: 0.25}, q = {2: 4.0, 5: 9.0, 7: 8.0}: Omega = {2, 7}
    ip, ix, v = _csr_from_dicts([{"0": 1.5, "2": -2.0, "7": 0.25}])
    qp, qx, qv = _csr_from_dicts([{"2": 4.0, "5": 9.0, "7": 8.0}])
    D = oracle.Dataset(ip, ix, v, 8)
    Q = oracle.Dataset(qp, qx, qv, 8)
    assert oracle.inner_product(D, 0, Q, 0) == -2.0 * 4.0 + 0.25 * 8.0 == -6.0
    # disjoint supports give exactly 0
    qp2, qx2, qv2 = _csr_from_dicts([{"1": 3.0, "3": 1.0}])
    assert oracle.inner_product(D, 0, oracle.Dataset(qp2, qx2, qv2, 8), 0) == 0.0


def test_brute_force_matches_scipy_product():
    """All scores = X @ q from scipy.sparse (a library SpMV), and the top-k is its ordering."""
    ip, ix, v = datagen.random_csr(400, 64, 9.0, seed=11)
    qp, qx, qv = datagen.random_csr(20, 64, 5.0, seed=12, nnz_min=1)
    D, Q = oracle.Dataset(ip, ix, v, 64), oracle.Dataset(qp, qx, qv, 64)
    X = _scipy(ip, ix, v, 64)
    Qm = _scipy(qp, qx, qv, 64)
    S = (X @ Qm.T).toarray()
    for r in range(20):
        got = oracle.all_scores(D, Q, r)
        np.testing.assert_allclose(got, S[:, r], rtol=1e-13, atol=1e-13)
        ids, sc = oracle.brute_force(D, Q, r, 17)
        order = np.lexsort((np.arange(400), -got))[:17]
        assert np.array_equal(ids, order)


def test_brute_force_ties_and_small_n():
    # duplicated documents tie exactly: the lower id comes first
    ip, ix, v = _csr_from_dicts([{"1": 2.0}, {"1": 1.0}, {"1": 2.0}, {"3": 5.0}, {"1": 2.0}])
    qp, qx, qv = _csr_from_dicts([{"1": 1.0}])
    D, Q = oracle.Dataset(ip, ix, v, 4), oracle.Dataset(qp, qx, qv, 4)
    ids, sc = oracle.brute_force(D, Q, 0, 10)          # k > N returns N results
    assert ids.tolist() == [0, 2, 4, 1, 3] and sc.tolist() == [2.0, 2.0, 2.0, 1.0, 0.0]
    # an empty query scores every document 0: lowest ids win
    ep = np.array([0, 0], np.int64)
    E = oracle.Dataset(ep, np.zeros(0, np.int32), np.zeros(0, np.float32), 4)
    ids, sc = oracle.brute_force(D, E, 0, 3)
    assert ids.tolist() == [0, 1, 2] and sc.tolist() == [0.0, 0.0, 0.0]


def test_dataset_rejects_malformed_and_drops_zeros():
    bad = [
        (np.array([0, 2, 1], np.int64), np.array([0, 1], np.int32), np.ones(2, np.float32)),   # decreasing
        (np.array([0, 2], np.int64), np.array([0, 9], np.int32), np.ones(2, np.float32)),      # dim >= d
        (np.array([0, 1], np.int64), np.array([4], np.int32), np.ones(1, np.float32)),         # dim == d
        (np.array([0, 1], np.int64), np.array([2], np.int32), np.array([np.inf], np.float32)),  # infinity
        (np.array([0, 2], np.int64), np.array([3, 3], np.int32), np.ones(2, np.float32)),      # duplicate
        (np.array([0, 1], np.int64), np.array([1], np.int32), np.array([np.nan], np.float32)),  # NaN
        (np.array([0, 1], np.int64), np.array([-1], np.int32), np.ones(1, np.float32)),        # negative dim
    ]
    for ip, ix, v in bad:
        with pytest.raises(ValueError):
            oracle.Dataset(ip, ix, v, 4)
    D = oracle.Dataset(np.array([0, 3], np.int64), np.array([2, 0, 1], np.int32),
                       np.array([1.0, 0.0, 3.0], np.float32), 4)
    ptr, dims, vals = D.export()
    assert ptr.tolist() == [0, 2] and dims.tolist() == [1, 2] and vals.tolist() == [3.0, 1.0]


# --------------------------------------------------------------------------
# Algorithms 1 and 3: the lists
# --------------------------------------------------------------------------
def test_unpruned_lists_are_the_transpose():
    """alpha = 1: the concatenated windows of I_j are column j of D (scipy tocsc, a library transpose)."""
    ip, ix, v = datagen.random_csr(300, 40, 7.0, seed=21)
    D = oracle.Dataset(ip, ix, v, 40)
    for lam in (1, 7, 64, 300, 1000):
        I = oracle.Index(D, window=lam, alpha=1.0)
        seg, pid, pval, scale, kept = I.export()
        assert I.sigma == -(-300 // lam)
        C = _scipy(ip, ix, v, 40).tocsc()
        C.sort_indices()
        for j in range(40):
            lo, hi = seg[j * I.sigma], seg[(j + 1) * I.sigma]
            assert np.array_equal(pid[lo:hi], C.indices[C.indptr[j]:C.indptr[j + 1]])
            assert np.array_equal(pval[lo:hi], C.data[C.indptr[j]:C.indptr[j + 1]])
            for w in range(I.sigma):
                a, b = seg[j * I.sigma + w], seg[j * I.sigma + w + 1]
                assert np.all(pid[a:b] // lam == w)
        assert kept.tolist() == np.diff(ip).tolist()


def test_list_vmax_is_the_column_maximum():
    """orc_list_vmax over an unpruned index (signed values) is max |column j| of D, and over a List-Pruning
    index (which keeps each list's largest |x|) the same maximum: scipy's column maxima, a library routine."""
    ip, ix, v = datagen.random_csr(300, 40, 7.0, seed=23)
    v = np.where(np.arange(len(v)) % 3 == 1, -v, v).astype(np.float32)
    D = oracle.Dataset(ip, ix, v, 40)
    C = abs(_scipy(ip, ix, v, 40)).tocsc()
    col_max = np.asarray(C.max(axis=0).todense()).ravel()
    for I in (oracle.Index(D, window=64, alpha=1.0), oracle.Index(D, window=7, alpha=1.0, prune="list", prune_n=3)):
        np.testing.assert_array_equal(I.list_vmax(), col_max)
    empty = oracle.Index(oracle.Dataset(np.zeros(4, np.int64), np.zeros(0, np.int32), np.zeros(0, np.float32), 5),
                         window=2)
    np.testing.assert_array_equal(empty.list_vmax(), np.zeros(5))


def test_pruned_lists_hold_exactly_the_alpha_mass_entries():
    ip, ix, v = datagen.random_csr(200, 50, 12.0, seed=31)
    D = oracle.Dataset(ip, ix, v, 50)
    I = oracle.Index(D, window=16, alpha=0.5)
    seg, pid, pval, scale, kept = I.export()
    want = set()
    for i in range(200):
        row = slice(ip[i], ip[i + 1])
        pos = oracle.alpha_mass(ix[row], v[row], 0.5)
        assert kept[i] == len(pos)
        for p in pos:
            want.add((i, int(ix[row][p]), float(v[row][p])))
    got = set()
    for j in range(50):
        for w in range(I.sigma):
            for t in range(seg[j * I.sigma + w], seg[j * I.sigma + w + 1]):
                got.add((int(pid[t]), j, float(pval[t])))
    assert got == want and I.postings == sum(kept)


def _entries(I):
    """(doc, dim, stored value) of every posting of an oracle index, and its kept counts."""
    seg, pid, pval, scale, kept = I.export()
    out = set()
    for j in range(I.D.dim):
        for t in range(seg[j * I.sigma], seg[(j + 1) * I.sigma]):
            out.add((int(pid[t]), j, float(pval[t])))
    return out, kept


def _doc_rows(ip, ix, v):
    return [{(i, int(ix[t]), float(v[t])) for t in range(ip[i], ip[i + 1])} for i in range(len(ip) - 1)]


def test_pruning_methods_hand_example():
    """Vector Number, List and Mass+List pruning (Sec. 4.1, ablation of Sec. 5) on a 3 x 4 example worked
    by hand: doc0 = {0: .5, 1: 2, 3: 1}, doc1 = {1: 3, 2: .25}, doc2 = {0: 4, 1: 2, 2: 2}."""
    ip = np.array([0, 3, 5, 8], np.int64)
    ix = np.array([0, 1, 3, 1, 2, 0, 1, 2], np.int32)
    v = np.array([.5, 2, 1, 3, .25, 4, 2, 2], np.float32)
    D = oracle.Dataset(ip, ix, v, 4)
    cases = {
        # two largest |x| per doc; doc2's tie at |x| = 2 goes to the lower dim (1)
        ("vector_number", 2, 1.0): ({(0, 1, 2.0), (0, 3, 1.0), (1, 1, 3.0), (1, 2, .25), (2, 0, 4.0), (2, 1, 2.0)},
                                    [2, 2, 2]),
        # largest |x| per list: dim0 doc2, dim1 doc1, dim2 doc2, dim3 doc0
        ("list", 1, 1.0): ({(2, 0, 4.0), (1, 1, 3.0), (2, 2, 2.0), (0, 3, 1.0)}, [1, 1, 2]),
        # two per list: dim1 keeps doc1 (3) and, of the tie at 2 between doc0 and doc2, doc0
        ("list", 2, 1.0): ({(0, 0, .5), (2, 0, 4.0), (1, 1, 3.0), (0, 1, 2.0), (1, 2, .25), (2, 2, 2.0),
                            (0, 3, 1.0)}, [3, 2, 2]),
        # alpha 0.5 keeps {1: 2}, {1: 3}, {0: 4} (4 >= 0.5 * 8 exactly); then dim1 keeps doc1 only
        ("mass_list", 1, 0.5): ({(1, 1, 3.0), (2, 0, 4.0)}, [0, 1, 1]),
    }
    for (prune, n, alpha), (want, want_kept) in cases.items():
        I = oracle.Index(D, window=2, alpha=alpha, prune=prune, prune_n=n)
        got, kept = _entries(I)
        assert got == want, (prune, n, sorted(got))
        assert kept.tolist() == want_kept, (prune, n)
        assert I.postings == len(want)


def test_vector_number_pruning_invariants():
    """Every document keeps min(vn, nnz) entries, none smaller in |x| than one it drops (equal |x|: the lower
    dim stays); vn >= every nnz leaves the unpruned index."""
    ip, ix, v = datagen.random_csr(400, 60, 10.0, seed=41)
    v = np.round(v * 4) / 4 + 0.25  # coarse values: many equal |x| within a row
    v = np.where(np.arange(len(v)) % 3 == 1, -v, v).astype(np.float32)   # |x| ranks, not x
    D = oracle.Dataset(ip, ix, v, 60)
    rows = _doc_rows(ip, ix, v)
    full, _ = _entries(oracle.Index(D, window=32, alpha=1.0))
    for vn in (1, 3, 7, 1000):
        got, kept = _entries(oracle.Index(D, window=32, prune="vector_number", prune_n=vn))
        for i, row in enumerate(rows):
            mine = {e for e in got if e[0] == i}
            assert mine <= row and len(mine) == min(vn, len(row)) == kept[i]
            for (_, jk, xk) in mine:
                for (_, jd, xd) in row - mine:
                    assert abs(xk) > abs(xd) or (abs(xk) == abs(xd) and jk < jd)
        if vn == 1000:
            assert got == full


def test_list_pruning_invariants():
    """Every list I_j keeps min(l', |I_j|) entries, none smaller in |x| than one it drops (equal |x|: the
    lower doc stays); the kept counts per document add up; l' >= every list length leaves the unpruned
    index; alpha-mass followed by list pruning is list pruning of the alpha-mass lists."""
    ip, ix, v = datagen.random_csr(500, 30, 9.0, seed=43)
    v = np.round(v * 4) / 4 + 0.25
    v = np.where(np.arange(len(v)) % 3 == 1, -v, v).astype(np.float32)   # |x| ranks, not x
    D = oracle.Dataset(ip, ix, v, 30)
    full, _ = _entries(oracle.Index(D, window=64, alpha=1.0))
    mass, _ = _entries(oracle.Index(D, window=64, alpha=0.6))
    for base, prune, alpha in ((full, "list", 1.0), (mass, "mass_list", 0.6)):
        for lp in (1, 4, 25, 10**6):
            got, kept = _entries(oracle.Index(D, window=64, alpha=alpha, prune=prune, prune_n=lp))
            assert got <= base
            for j in range(30):
                lst = {e for e in base if e[1] == j}
                mine = {e for e in got if e[1] == j}
                assert len(mine) == min(lp, len(lst))
                for (ik, _, xk) in mine:
                    for (idr, _, xd) in lst - mine:
                        assert abs(xk) > abs(xd) or (abs(xk) == abs(xd) and ik < idr)
            for i in range(500):
                assert kept[i] == sum(1 for e in got if e[0] == i)
            if lp == 10**6:
                assert got == base


# --------------------------------------------------------------------------
# Algorithms 2 and 4: search
# --------------------------------------------------------------------------
@pytest.fixture(scope="module")
def small():
    w = datagen.WORKLOADS["exact-10k"].scaled(n_docs=1500, n_queries=25)
    ip, ix, v = datagen.docs(w)
    qp, qx, qv = datagen.queries(w)
    return w, (ip, ix, v), (qp, qx, qv), oracle.Dataset(ip, ix, v, w.dim), oracle.Dataset(qp, qx, qv, w.dim)


def test_unpruned_search_equals_brute_force_exactly(small):
    """alpha = 1 (no pruning): the window-accumulation top-k IS the brute-force top-k, bit for bit."""
    w, _, _, D, Q = small
    for lam in (64, 500, 4096):
        I = oracle.Index(D, window=lam, alpha=1.0)
        for r in range(Q.n):
            a = I.search(Q, r, k=10, gamma=0)
            b = oracle.brute_force(D, Q, r, 10)
            assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


def test_coarse_scores_match_scipy_on_pruned_docs(small):
    """Coarse scores = (pruned X) @ q via scipy for every document (k = N covers all)."""
    w, (ip, ix, v), (qp, qx, qv), D, Q = small
    I = oracle.Index(D, window=256, alpha=0.6)
    rows, cols, vals = [], [], []
    for i in range(D.n):
        row = slice(ip[i], ip[i + 1])
        for p in oracle.alpha_mass(ix[row], v[row], 0.6):
            rows.append(i); cols.append(int(ix[row][p])); vals.append(float(v[row][p]))
    Xp = sp.csr_matrix((vals, (rows, cols)), shape=(D.n, w.dim))
    Qm = _scipy(qp, qx, qv, w.dim)
    S = (Xp @ Qm.T).toarray()
    for r in range(0, Q.n, 3):
        ids, sc = I.search(Q, r, k=D.n, gamma=0)
        assert len(ids) == D.n
        np.testing.assert_allclose(sc, S[ids, r], rtol=1e-13, atol=1e-13)
        order = np.lexsort((np.arange(D.n), -S[:, r]))
        # orders agree wherever neighbouring library scores are not within rounding
        gap = np.abs(np.diff(S[order, r])) > 1e-12 * np.maximum(1.0, np.abs(S[order[:-1], r]))
        assert np.array_equal(ids[:-1][gap], order[:-1][gap])


def test_exhaustive_rerank_equals_brute_force(small):
    """gamma >= N makes the reorder exhaustive: any alpha returns the exact top-k (Alg. 4 with H = D)."""
    w, _, _, D, Q = small
    for alpha in (0.2, 0.5, 0.9):
        I = oracle.Index(D, window=300, alpha=alpha)
        for r in range(0, Q.n, 2):
            a = I.search(Q, r, k=10, gamma=D.n + 5)
            b = oracle.brute_force(D, Q, r, 10)
            assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


def test_rerank_scores_are_exact_and_candidates_are_coarse_topgamma(small):
    w, _, _, D, Q = small
    I = oracle.Index(D, window=128, alpha=0.4)
    for r in range(0, Q.n, 4):
        ids, sc, cids, csc = I.search(Q, r, k=10, gamma=40, want_coarse=True)
        c2 = I.search(Q, r, k=40, gamma=0)
        assert np.array_equal(cids, c2[0]) and np.array_equal(csc, c2[1])
        assert set(ids.tolist()) <= set(cids.tolist())
        for i, s in zip(ids, sc):
            assert s == oracle.inner_product(D, int(i), Q, r)
        exact = sorted(((oracle.inner_product(D, int(c), Q, r), -int(c)) for c in cids), reverse=True)[:10]
        assert [-e[1] for e in exact] == ids.tolist()


def test_search_edge_cases():
    # N < k, N < lambda, a query with no hits, an empty query, and a last window that is not full
    ip, ix, v = _csr_from_dicts([{"1": 1.0}, {"2": 2.0}, {}, {"1": 3.0, "2": 1.0}, {"3": 0.5}])
    D = oracle.Dataset(ip, ix, v, 6)
    I = oracle.Index(D, window=2, alpha=1.0)       # sigma = 3, last window holds one doc
    assert I.sigma == 3
    qp, qx, qv = _csr_from_dicts([{"1": 1.0, "2": 1.0}, {"5": 1.0}, {}])
    Q = oracle.Dataset(qp, qx, qv, 6)
    ids, sc = I.search(Q, 0, k=10, gamma=0)
    assert ids.tolist() == [3, 1, 0, 2, 4] and sc.tolist() == [4.0, 2.0, 1.0, 0.0, 0.0]
    for r in (1, 2):                               # no hits / empty: zero scores, lowest ids
        ids, sc = I.search(Q, r, k=3, gamma=0)
        assert ids.tolist() == [0, 1, 2] and sc.tolist() == [0.0] * 3
    ids, sc = I.search(Q, 0, k=2, gamma=3)
    assert ids.tolist() == [3, 1]


def test_beta_mass_query_pruning(small):
    """beta < 1 scans only the beta-mass entries of q; the reorder still uses the full q."""
    w, _, (qp, qx, qv), D, Q = small
    I = oracle.Index(D, window=256, alpha=1.0)
    for r in range(0, Q.n, 5):
        row = slice(qp[r], qp[r + 1])
        pos = oracle.alpha_mass(qx[row], qv[row], 0.5)
        sub = {str(int(qx[row][p])): float(qv[row][p]) for p in pos}
        sp_, sx, sv = _csr_from_dicts([sub])
        Qs = oracle.Dataset(sp_, sx, sv, w.dim)
        a = I.search(Q, r, k=10, gamma=0, beta=0.5)
        b = oracle.brute_force(D, Qs, 0, 10)
        assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
        full = I.search(Q, r, k=5, gamma=D.n, beta=0.5)
        assert np.array_equal(full[0], oracle.brute_force(D, Q, r, 5)[0])


# --------------------------------------------------------------------------
# Reduced-precision values (no counterpart in the paper; IEEE / OCP definitions)
# --------------------------------------------------------------------------
def test_f16_codec_matches_numpy():
    rng = np.random.default_rng(3)
    xs = np.concatenate([
        rng.lognormal(0, 3, 4000).astype(np.float32),
        -rng.lognormal(0, 3, 500).astype(np.float32),
        np.array([0.0, 65504.0, 65519.0, 65520.0, 6e-8, 3e-8, 2.98e-8, 1e-10, 1.0 + 2**-11, 1.0 + 3 * 2**-11],
                 np.float32),
    ])
    # exact halfway points between neighbouring float16 values
    h = np.arange(0x0400, 0x7BFF, 97, dtype=np.uint16).view(np.float16).astype(np.float64)
    h2 = np.nextafter(h.astype(np.float16), np.float16(np.inf)).astype(np.float64)
    xs = np.concatenate([xs, ((h + h2) / 2).astype(np.float32)])
    for x in xs:
        assert oracle.f16_encode(float(x)) == int(np.float32(x).astype(np.float16).view(np.uint16)), x
    for code in range(0, 0x7C00, 7):
        assert oracle.f16_decode(code) == float(np.uint16(code).view(np.float16))


def test_e4m3_codec_matches_torch():
    torch = pytest.importorskip("torch")
    codes = torch.arange(256, dtype=torch.uint8)
    ref = codes.view(torch.float8_e4m3fn).float().tolist()
    for c in range(256):
        got = oracle.e4m3_decode(c)
        if np.isnan(ref[c]):
            assert np.isnan(got)
        else:
            assert got == ref[c]
    rng = np.random.default_rng(5)
    xs = np.concatenate([rng.uniform(-448, 448, 3000), rng.lognormal(-3, 2, 2000)]).astype(np.float32)
    xs = xs[np.abs(xs) <= 448]
    finite = np.array([v for v in ref if not np.isnan(v)])
    finite = np.unique(finite)
    mids = ((finite[:-1] + finite[1:]) / 2).astype(np.float32)          # ties: round to even
    xs = np.concatenate([xs, mids])
    t = torch.from_numpy(xs).to(torch.float8_e4m3fn).view(torch.uint8).numpy()
    for x, c in zip(xs, t):
        assert oracle.e4m3_encode(float(x)) == int(c), x
    assert oracle.e4m3_encode(1e6) == 0x7E and oracle.e4m3_encode(-1e6) == 0xFE


def test_quantised_lists_store_dequantised_values():
    ip, ix, v = datagen.random_csr(200, 30, 8.0, seed=41, val_sigma=1.5)
    D = oracle.Dataset(ip, ix, v, 30)
    base = oracle.Index(D, window=64, alpha=1.0).export()
    f16 = oracle.Index(D, window=64, alpha=1.0, dtype="f16").export()
    assert np.array_equal(base[1], f16[1])
    np.testing.assert_array_equal(f16[2], base[2].astype(np.float32).astype(np.float16).astype(np.float64))
    f8 = oracle.Index(D, window=64, alpha=1.0, dtype="f8").export()
    seg, sigma = base[0], -(-200 // 64)
    for j in range(30):
        lo, hi = seg[j * sigma], seg[(j + 1) * sigma]
        if hi == lo:
            continue
        amax = np.float32(np.max(np.abs(base[2][lo:hi]).astype(np.float32)))
        sc = np.float32(amax / np.float32(448.0))
        assert f8[3][j] == sc
        import torch
        ratio = torch.from_numpy((base[2][lo:hi].astype(np.float32) / sc).astype(np.float32))
        deq = ratio.to(torch.float8_e4m3fn).float().numpy() * sc
        np.testing.assert_array_equal(f8[2][lo:hi], deq.astype(np.float64))
        # relative error of E4M3 is at most 2^-4 of the value for normal codes
        rel = np.abs(f8[2][lo:hi] - base[2][lo:hi]) / np.abs(base[2][lo:hi])
        assert np.all((rel <= 2.0 ** -4) | (np.abs(base[2][lo:hi]) < 2.0 ** -6 * sc))


def test_recall_definition():
    assert oracle.recall([1, 2, 3], [3, 2, 9, 8]) == 0.5
    assert oracle.recall([], [1]) == 0.0


def test_tie_aware_recall_hand_example():
    """Docs 1 and 3 are the same vector, so they tie at the k-th score. R* (k = 2) takes doc 1, the lower id.
    Returning doc 3 instead is a miss for plain recall and a hit for the tie-aware one. A doc below the k-th
    score, a repeated id and an id outside the dataset count for nothing."""
    ip, ix, v = _csr_from_dicts([{"0": 4.0}, {"0": 1.0, "1": 1.0}, {"1": 0.5}, {"0": 1.0, "1": 1.0}])
    D = oracle.Dataset(ip, ix, v, 2)
    qp, qx, qv = _csr_from_dicts([{"0": 1.0, "1": 1.0}])
    Q = oracle.Dataset(qp, qx, qv, 2)
    truth, ts = oracle.brute_force(D, Q, 0, 2)
    assert truth.tolist() == [0, 1] and ts.tolist() == [4.0, 2.0]      # scores 4, 2, 0.5, 2
    assert oracle.recall([0, 3], truth) == 0.5
    assert oracle.recall_tie_aware([0, 3], truth, ts, D, Q, 0) == 1.0
    assert oracle.recall_tie_aware([3, 2], truth, ts, D, Q, 0) == 0.5
    assert oracle.recall_tie_aware([3, 3], truth, ts, D, Q, 0) == 0.5
    assert oracle.recall_tie_aware([1, 3, 0], truth, ts, D, Q, 0) == 1.0   # capped at 1
    assert oracle.recall_tie_aware([0, 0xFFFFFFFF], truth, ts, D, Q, 0) == 0.5
