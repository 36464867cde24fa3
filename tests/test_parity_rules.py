"""The comparison rules of tests/parity.py, checked on the CPU against an FP32 emulation of the scan.

The GPU tests trust these rules, so they are tested here first. Each rule must accept every correct FP32
evaluation, whatever the order of its additions. It must also reject a planted error: an id swapped for a
worse one, a score off by more than its bound, or a repeated id.
"""
import numpy as np
import pytest

import datagen
import oracle
from parity import check_ranked_conditioned, fp32_sum_bound, signed_copy


def _fp32_scan(seg, pid, pval, sigma, n, qd, qv, rng):
    """Score every document in FP32 from the lists, one term after another in a random order (each
    addition rounded to FP32, as the shared-memory scatter-add does)."""
    A = np.zeros(n, np.float32)
    for t in rng.permutation(len(qd)):
        j = int(qd[t])
        lo, hi = seg[j * sigma], seg[(j + 1) * sigma]
        prod = np.float32(qv[t]) * pval[lo:hi].astype(np.float32)   # FP32 product, rounded once
        A[pid[lo:hi]] += prod                                         # ids unique within I_j
    return A


@pytest.fixture(scope="module")
def signed_case():
    w = datagen.WORKLOADS["pruned-1m"].scaled(n_docs=3000, n_queries=8)
    ip, ix, v = datagen.docs(w)
    qp, qx, qv = datagen.queries(w)
    v, qv = signed_copy(v, 3), signed_copy(qv, 5)
    D, Q = oracle.Dataset(ip, ix, v, w.dim), oracle.Dataset(qp, qx, qv, w.dim)
    Da = oracle.Dataset(ip, ix, np.abs(v), w.dim)
    Qa = oracle.Dataset(qp, qx, np.abs(qv), w.dim)
    I = oracle.Index(D, window=1024, alpha=0.5)
    Ia = oracle.Index(Da, window=1024, alpha=0.5)     # alpha-mass ranks |x|: the same kept entries
    return w, (qp, qx, qv), D, Q, I, Qa, Ia


def _exact(I, Q, r, n):
    ids, sc = I.search(Q, r, k=n, gamma=0)
    s = np.empty(n)
    s[ids] = sc
    return s


def test_conditioned_rule_accepts_fp32_and_rejects_planted_errors(signed_case):
    w, (qp, qx, qv), D, Q, I, Qa, Ia = signed_case
    seg, pid, pval, _, _ = I.export()
    k, n = 50, D.n
    rng = np.random.default_rng(11)
    cancelled = 0
    for r in range(Q.n):
        s, a = _exact(I, Q, r, n), _exact(Ia, Qa, r, n)
        assert np.all(np.abs(s) <= a * (1 + 1e-12))
        cancelled += int(np.sum((a > 0) & (np.abs(s) < 0.5 * a)))
        m = int(qp[r + 1] - qp[r])
        qd, qvv = qx[qp[r]:qp[r + 1]], qv[qp[r]:qp[r + 1]]
        for _ in range(3):                                            # three orders of the additions
            A = _fp32_scan(seg, pid, pval, I.sigma, n, qd, qvv, rng)
            order = np.lexsort((np.arange(n), -A.astype(np.float64)))
            gids, gsc = order[:k], A[order[:k]]
            check_ranked_conditioned(gids, gsc, s, a, m, k, what=f"query {r}")
        # planted: the k-th id replaced by a much worse document (its own score keeps the order)
        bad_ids, bad_sc = gids.copy(), gsc.astype(np.float64).copy()
        bad_ids[-1], bad_sc[-1] = order[k + 300], A[order[k + 300]]
        with pytest.raises(AssertionError):
            check_ranked_conditioned(bad_ids, bad_sc, s, a, m, k)
        # planted: the best score off by 1e-3 of its value (far above the bound)
        bad_sc = gsc.astype(np.float64).copy()
        bad_sc[0] *= 1 + 1e-3
        with pytest.raises(AssertionError):
            check_ranked_conditioned(gids, bad_sc, s, a, m, k)
        # planted: a repeated id
        bad_ids = gids.copy()
        bad_ids[1] = bad_ids[0]
        with pytest.raises(AssertionError):
            check_ranked_conditioned(bad_ids, gsc, s, a, m, k)
    assert cancelled > 100          # the data really has cancelling scores


def test_fp32_bound_is_tight_enough_to_order_documents(signed_case):
    """The per-document bound stays near m * 2^-24 of the absolute sum, far below the score gaps that decide
    the top-k (so the rule still pins the ids)."""
    w, (qp, qx, qv), D, Q, I, Qa, Ia = signed_case
    s, a = _exact(I, Q, 0, D.n), _exact(Ia, Qa, 0, D.n)
    m = int(qp[1] - qp[0])
    b = fp32_sum_bound(a, m)
    assert np.all(b <= (m + 2) * 2.0 ** -24 * a + 1e-300)
    top = np.sort(s)[::-1][:60]
    gaps = -np.diff(top)
    assert np.median(gaps) > 100 * np.max(b[np.argsort(-s)[:60]])


def _fp32_dot(row_d, row_v, qd, qv, rng):
    """delta(x, q) in FP32: each common term's product rounded, then added in a random order."""
    common, xi, qi = np.intersect1d(row_d, qd, return_indices=True)
    prods = (row_v[xi].astype(np.float32) * qv[qi].astype(np.float32)).astype(np.float32)
    acc = np.float32(0.0)
    for p in prods[rng.permutation(len(prods))]:
        acc = np.float32(acc + p)
    return acc


def test_conditioned_reorder_rule_accepts_fp32_and_rejects_planted_errors(signed_case):
    from parity import check_reranked_conditioned

    w, (qp, qx, qv), D, Q, I, Qa, Ia = signed_case
    ip, ix, v = D.export()
    Da = oracle.Dataset(ip, ix, np.abs(v).astype(np.float32), D.dim)
    seg, pid, pval, _, _ = I.export()
    k, gamma, n = 10, 200, D.n
    rng = np.random.default_rng(5)
    for r in range(Q.n):
        qd, qvv = qx[qp[r]:qp[r + 1]], qv[qp[r]:qp[r + 1]]
        m = len(qd)
        sc, ac = _exact(I, Q, r, n), _exact(Ia, Qa, r, n)
        sf, af = oracle.all_scores(D, Q, r), oracle.all_scores(Da, Qa, r)
        A = _fp32_scan(seg, pid, pval, I.sigma, n, qd, qvv, rng)
        cand = np.lexsort((np.arange(n), -A.astype(np.float64)))[:gamma]
        fin = np.array([_fp32_dot(ix[ip[i]:ip[i + 1]], v[ip[i]:ip[i + 1]], qd, qvv, rng) for i in cand], np.float32)
        order = np.lexsort((cand, -fin.astype(np.float64)))[:k]
        gids, gsc = cand[order], fin[order]
        check_reranked_conditioned(gids, gsc, sc, ac, m, sf, af, m, k, gamma, what=f"query {r}")
        # planted: a returned id replaced by a document far below the coarse pool
        far = int(np.lexsort((np.arange(n), -sc))[gamma + 400])
        bad = gids.copy()
        bad[-1] = far
        with pytest.raises(AssertionError, match="cannot be a coarse candidate"):
            check_reranked_conditioned(bad, gsc, sc, ac, m, sf, af, m, k, gamma)
        # planted: the best reordered document dropped for the candidate ranked k + 20 by its FP32 score
        full = np.lexsort((cand, -fin.astype(np.float64)))
        worse_ids = np.concatenate([gids[1:], cand[full[k + 20:k + 21]]])
        worse_sc = np.concatenate([gsc[1:], fin[full[k + 20:k + 21]]])
        with pytest.raises(AssertionError, match="certainly beats"):
            check_reranked_conditioned(worse_ids, worse_sc, sc, ac, m, sf, af, m, k, gamma)
        # planted: a score off by 1e-3 of its value
        off = gsc.astype(np.float64).copy()
        off[0] *= 1 + 1e-3
        with pytest.raises(AssertionError, match="bound"):
            check_reranked_conditioned(gids, off, sc, ac, m, sf, af, m, k, gamma)


def test_beat_counts_hand_example():
    """Scores 3, 0, 0, 1, 0 known to +-0.1 except the three exact zeros (no common term), which tie exactly
    and rank by id: counts of documents that certainly / might beat each one, worked by hand."""
    from parity import _beat_counts

    s = np.array([3.0, 0.0, 0.0, 1.0, 0.0])
    b = np.array([0.1, 1e-300, 1e-300, 0.1, 1e-300])
    certain, might = _beat_counts(s, b, s == 0)
    assert certain.tolist() == [0, 2, 3, 1, 4]
    assert might.tolist() == [0, 2, 3, 1, 4]
    # no longer exact: the zeros might beat one another but certainly beat none of each other
    certain, might = _beat_counts(s, np.full(5, 0.1), np.zeros(5, bool))
    assert certain.tolist() == [0, 2, 2, 1, 2] and might.tolist() == [0, 4, 4, 1, 4]


@pytest.fixture(scope="module")
def plain_case():
    w = datagen.WORKLOADS["pruned-1m"].scaled(n_docs=3000, n_queries=8)
    ip, ix, v = datagen.docs(w)
    qp, qx, qv = datagen.queries(w)
    D, Q = oracle.Dataset(ip, ix, v, w.dim), oracle.Dataset(qp, qx, qv, w.dim)
    I = oracle.Index(D, window=1024, alpha=0.5)
    return w, (ip, ix, v), (qp, qx, qv), D, Q, I


def test_ranked_rule_accepts_fp32_and_rejects_planted_errors(plain_case):
    """check_ranked (the coarse rule of the GPU tests, non-negative data) against FP32 scans of the oracle's
    own lists in random addition orders, and against answers with one planted error each."""
    from parity import PAD_ID, check_ranked

    w, _, (qp, qx, qv), D, Q, I = plain_case
    seg, pid, pval, _, _ = I.export()
    k, n = 50, D.n
    rng = np.random.default_rng(21)
    for r in range(Q.n):
        oi, os_ = I.search(Q, r, k=k + 64, gamma=0)
        A = _fp32_scan(seg, pid, pval, I.sigma, n, qx[qp[r]:qp[r + 1]], qv[qp[r]:qp[r + 1]], rng)
        order = np.lexsort((np.arange(n), -A.astype(np.float64)))[:k]
        gids, gsc = order.astype(np.int64), A[order]
        check_ranked(gids, gsc, oi, os_, k, n, what=f"query {r}")
        bad = gids.copy()
        bad[0] = oi[k + 40]                                  # a document far outside the top-k
        with pytest.raises(AssertionError):
            check_ranked(bad, gsc, oi, os_, k, n)
        off = gsc.astype(np.float64).copy()
        off[k // 2] *= 1 + 1e-4                              # ten times the tolerance
        with pytest.raises(AssertionError):
            check_ranked(gids, off, oi, os_, k, n)
        with pytest.raises(AssertionError):                  # padding where a document belongs
            check_ranked(np.concatenate([gids[:-1], [PAD_ID]]), np.concatenate([gsc[:-1], [-np.inf]]),
                         oi, os_, k, n)


def test_reranked_rule_accepts_fp32_and_rejects_planted_errors(plain_case):
    """check_reranked (the reorder rule of the GPU tests) against an FP32 emulation of Algorithm 4 (coarse
    top-gamma of an FP32 scan, FP32 exact scores of the candidates, top-k), and against planted errors."""
    from parity import check_reranked

    w, (ip, ix, v), (qp, qx, qv), D, Q, I = plain_case
    seg, pid, pval, _, _ = I.export()
    k, gamma, n = 10, 200, D.n
    rng = np.random.default_rng(22)
    for r in range(Q.n):
        qd, qvv = qx[qp[r]:qp[r + 1]], qv[qp[r]:qp[r + 1]]
        A = _fp32_scan(seg, pid, pval, I.sigma, n, qd, qvv, rng)
        cand = np.lexsort((np.arange(n), -A.astype(np.float64)))[:gamma]
        fin = np.array([_fp32_dot(ix[ip[i]:ip[i + 1]], v[ip[i]:ip[i + 1]], qd, qvv, rng) for i in cand], np.float32)
        order = np.lexsort((cand, -fin.astype(np.float64)))
        gids, gsc = cand[order[:k]], fin[order[:k]]
        check_reranked(gids, gsc, D, Q, r, I, k, gamma, what=f"query {r}")
        outside = np.setdiff1d(np.arange(n), cand)
        far = int(outside[np.argmin(A[outside])])           # the worst coarse score: never a candidate
        bad = gids.copy()
        bad[-1] = far
        with pytest.raises(AssertionError, match="not a coarse candidate"):
            check_reranked(bad, gsc, D, Q, r, I, k, gamma)
        off = gsc.astype(np.float64).copy()
        off[0] *= 1 + 1e-4
        with pytest.raises(AssertionError, match="score of"):
            check_reranked(gids, off, D, Q, r, I, k, gamma)
        worse = np.concatenate([gids[1:], cand[order[k + 30:k + 31]]])
        worse_sc = np.concatenate([gsc[1:], fin[order[k + 30:k + 31]]])
        with pytest.raises(AssertionError):
            check_reranked(worse, worse_sc, D, Q, r, I, k, gamma)
