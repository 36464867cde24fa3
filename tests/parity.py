"""Comparison rules between the GPU results and the FP64 oracle.

Tolerance: scores within REL_TOL = 1e-5 relative (FP32 accumulation of at
most a few hundred positive products stays below that). IDs must be
bit-identical wherever the oracle's scores separate them by more than the
tolerance; inside a group of near-equal oracle scores any order is valid,
and the lower id wins only among exact ties, which FP32 cannot guarantee to
reproduce.
"""
from __future__ import annotations

import numpy as np

import oracle

REL_TOL = 1e-5
PAD_ID = 0xFFFFFFFF


def _close(a, b, tol=REL_TOL):
    return abs(float(a) - float(b)) <= tol * max(abs(float(a)), abs(float(b)), 1e-30)


def tie_groups(scores, tol=REL_TOL):
    """Split a best-first score list into runs whose neighbours are within tol."""
    groups, start = [], 0
    for i in range(1, len(scores) + 1):
        if i == len(scores) or not _close(scores[i - 1], scores[i], tol):
            groups.append((start, i))
            start = i
    return groups


def check_ranked(gids, gsc, oids, osc, k, n_docs, tol=REL_TOL, what=""):
    """GPU top-k (gids, gsc) against the oracle's best-first list (oids, osc).

    The oracle list must extend past rank k far enough to close the tie group
    that straddles rank k (callers ask for k + 64 results)."""
    n = min(k, n_docs)
    gids = np.asarray(gids).astype(np.int64) & 0xFFFFFFFF
    gsc = np.asarray(gsc, np.float64)
    assert np.all(gids[n:] == PAD_ID) and np.all(np.isneginf(gsc[n:])), f"{what}: padding"
    for r in range(n):
        assert _close(gsc[r], osc[r], tol), f"{what}: score at rank {r}: gpu {gsc[r]!r} oracle {osc[r]!r}"
    groups = tie_groups(osc, tol)
    for a, b in groups:
        if a >= n:
            break
        want = set(int(x) for x in oids[a:b])
        got = set(int(x) for x in gids[a:min(b, n)])
        if b <= n:
            assert got == want, f"{what}: ranks [{a},{b}) gpu {sorted(got)} oracle {sorted(want)}"
        else:
            assert b < len(osc) or len(osc) >= n_docs, f"{what}: oracle list too short to close the last tie group"
            assert got <= want, f"{what}: boundary ranks [{a},{n}) gpu {sorted(got)} not in oracle group"


FIXED_UNIT = 2.0 ** -30


def _rows(Q):
    if getattr(Q, "_rows", None) is None:
        Q._rows = Q.export()
    return Q._rows


def fixed_extra(I, Q, r):
    """What a fixed-point window score (sindi_accumulator FIXED32) may add to the FP32 dot-product bound of
    its products: half a unit 2^-e per product, with 2^-(e+1) <= B * 2^-30 for B = the sum over the window's
    terms of |q_j| * vmax_j (vmax_j = the largest |stored value| of list I_j). Taken over all the query's
    terms (a B at least the window's) and m = the query's term count (at least the products of any
    document); a small allowance covers the FP32 evaluation of B on the device. The FP32 part, 2^-23 * a for
    a = the sum of |products|, is within fp32_sum_bound(a, m) for m >= 1."""
    ptr, dims, vals = _rows(Q)
    a, b = int(ptr[r]), int(ptr[r + 1])
    B = float(np.sum(np.abs(vals[a:b]) * I.list_vmax()[dims[a:b]]))
    return (b - a) * B * FIXED_UNIT * (1 + 1e-3)


def check_reranked(gids, gsc, D, Q, r, I, k, gamma, tol=REL_TOL, what="", beta=1.0, fixed=True):
    """GPU results of Algorithm 4 (pruned coarse stage + exact reorder of gamma candidates).

    The GPU's coarse scores are rounded (FP32 sums, or with `fixed` the fixed-point window that a search
    with gamma > 0 uses by default), so its candidate set may differ from the oracle's only by documents
    whose coarse score is within tol, or within twice the fixed-point allowance (fixed_extra), of the
    oracle's gamma-th coarse score ("ambiguous"). The GPU answer must be the exact top-k of some candidate
    set C with robust <= C <= robust + ambiguous. Returns the number of ambiguous documents that touched
    the answer."""
    n = min(k, D.n)
    g = min(gamma, D.n)
    cids, csc = I.search(Q, r, k=min(g + 256, D.n), gamma=0, beta=beta)
    s_g = csc[g - 1]
    atol = 2.0 * fixed_extra(I, Q, r) if fixed else 0.0

    def near(s):
        return _close(s, s_g, tol) or abs(s - s_g) <= atol

    if s_g == 0.0:
        # fewer than gamma documents score above zero: zero scores are exact on both sides (no product) and
        # both fill the pool with the lowest ids. A positive score within the fixed-point allowance may
        # round to zero, and lower-id zeros past the oracle's pool then take its place.
        amb = set(int(c) for c, s in zip(cids, csc) if 0.0 < s <= atol)
        if amb:
            amb |= set(int(c) for c, s in zip(cids[g:], csc[g:]) if s == 0.0)
        robust = set(int(c) for c in cids[:g]) - amb
    else:
        amb = set(int(c) for c, s in zip(cids, csc) if near(s))
        robust = set(int(c) for c in cids[:g]) - amb
        if len(cids) > g and near(csc[-1]) and len(cids) < D.n:
            raise AssertionError(f"{what}: coarse tie group at rank gamma longer than the probe")
    gids = np.asarray(gids).astype(np.int64) & 0xFFFFFFFF
    gsc = np.asarray(gsc, np.float64)
    assert np.all(gids[n:] == PAD_ID), f"{what}: padding"
    exact = {}

    def ex(i):
        if i not in exact:
            exact[i] = oracle.inner_product(D, i, Q, r)
        return exact[i]

    got = [int(x) for x in gids[:n]]
    assert len(set(got)) == n, f"{what}: duplicate ids {got}"
    for rank, i in enumerate(got):
        assert i in robust or i in amb, f"{what}: id {i} at rank {rank} was not a coarse candidate"
        assert _close(gsc[rank], ex(i), tol), f"{what}: score of {i}: gpu {gsc[rank]} exact {ex(i)}"
        if rank:
            assert ex(got[rank - 1]) >= ex(i) * (1 - tol) - 1e-30, f"{what}: order at rank {rank}"
    kth = ex(got[-1])
    gotset = set(got)
    for c in robust:
        if ex(c) > kth * (1 + tol) + 1e-30:
            assert c in gotset, f"{what}: robust candidate {c} (exact {ex(c)}) beats the k-th {kth} but is missing"
    touched = len(amb & gotset)
    oi, osc = I.search(Q, r, k=k, gamma=gamma, beta=beta)
    if not (amb & (gotset | set(int(x) for x in oi))):
        # no ambiguity reached the answer: the tie-group rule against the oracle itself
        full = sorted(((ex(c) if c in exact else oracle.inner_product(D, c, Q, r), c) for c in
                       set(int(x) for x in cids[:g])), key=lambda t: (-t[0], t[1]))
        check_ranked(gids, gsc, np.array([c for _, c in full]), np.array([s for s, _ in full]), k, D.n, tol, what)
    return touched


U32 = 2.0 ** -24   # unit roundoff of FP32


def fp32_sum_bound(a, m):
    """Largest error of an FP32 evaluation of a sum of at most m products, in any order and with each
    product rounded at most twice: gamma_{m+1} * a, where a = sum of |products| (exact) and
    gamma_n = n u / (1 - n u) (the dot-product bound of Higham, Accuracy and Stability of Numerical
    Algorithms, 2nd ed., Sec. 3.1). A small FP64 allowance covers the rounding of the exact side."""
    g = (m + 1) * U32 / (1 - (m + 1) * U32)
    return g * np.asarray(a, np.float64) * (1 + 1e-9) + 1e-300


def check_ranked_conditioned(gids, gsc, s, a, m, k, what="", extra=0.0):
    """GPU top-k over signed data against the exact FP64 scores s[i] of every document i.

    With signed values a score can cancel to near zero, so no relative tolerance holds. Each document gets
    its own bound b[i] = fp32_sum_bound(a[i], m), a[i] = sum of |q_j x_j| over its products. The GPU's
    scores must be within b of the exact ones and non-increasing, its ids distinct, and no document it
    left out may certainly beat one it returned: max over the rest of (s - b) <= min over the answer of
    (s + b). `extra` widens every bound (a fixed-point window: fixed_extra)."""
    s = np.asarray(s, np.float64)
    b = fp32_sum_bound(a, m) + extra
    n = min(k, len(s))
    gids = np.asarray(gids).astype(np.int64)[:n] & 0xFFFFFFFF
    gsc = np.asarray(gsc, np.float64)[:n]
    assert np.all(gids < len(s)), f"{what}: id out of range"
    assert len(set(gids.tolist())) == n, f"{what}: duplicate ids"
    err = np.abs(gsc - s[gids])
    bad = np.nonzero(err > b[gids])[0]
    assert len(bad) == 0, (f"{what}: rank {bad[0]} id {gids[bad[0]]}: gpu {gsc[bad[0]]!r} exact "
                           f"{s[gids[bad[0]]]!r} bound {b[gids[bad[0]]]!r}")
    assert np.all(np.diff(gsc) <= 0), f"{what}: scores not in descending order"
    rest = np.ones(len(s), bool)
    rest[gids] = False
    if rest.any():
        hi_out = np.max((s - b)[rest])
        lo_in = np.min((s + b)[gids])
        assert hi_out <= lo_in, f"{what}: a left-out document ({hi_out!r}) certainly beats a returned one ({lo_in!r})"


def signed_copy(values, every=3):
    """The same values with every `every`-th one negated (signed test data; no method arithmetic)."""
    v = np.array(values, np.float32, copy=True)
    v[1::every] = -v[1::every]
    return v


def _beat_counts(s, b, exact0):
    """For every document i: how many others certainly beat it (certain[i]) and how many might (might[i]),
    for scores known to within +-b. Documents with no common term (exact0) score exactly 0 on both sides, so
    between two of them the lower id wins, as the search's order rule says."""
    s = np.asarray(s, np.float64)
    lo, hi = s - b, s + b
    n = len(s)
    los, his = np.sort(lo), np.sort(hi)
    certain = n - np.searchsorted(los, hi, side="right")            # #{j : lo_j > hi_i}
    might = n - np.searchsorted(his, lo, side="left") - 1            # #{j != i : hi_j >= lo_i}
    z = np.nonzero(exact0)[0]                                        # ascending ids
    rank = np.arange(len(z))
    certain[z] += rank                                               # lower-id exact zeros beat i
    might[z] -= len(z) - 1 - rank                                    # higher-id exact zeros cannot
    return certain, might


def check_reranked_conditioned(gids, gsc, sc, ac, mc, sf, af, mf, k, gamma, what="", coarse_extra=0.0):
    """GPU results of Algorithm 4 over signed data, for one query.

    sc, ac: the exact coarse score of every document (pruned document, pruned query) and its sum of
    |products|; mc: the coarse query's term count. sf, af, mf: the same for the exact reorder score (full
    document, full query). The GPU takes the exact best gamma of its FP32 coarse scores, then the exact
    best k of their FP32 reorder scores. So: every returned id must be a possible candidate (fewer than
    gamma documents certainly beat it on the coarse score); its score must lie within the FP32 bound of
    sf; the scores must descend; and no certain candidate (fewer than gamma documents might beat it) that
    was left out may certainly beat a returned one on sf. `coarse_extra` widens the coarse bounds (a
    fixed-point window: fixed_extra)."""
    sc, sf = np.asarray(sc, np.float64), np.asarray(sf, np.float64)
    n_docs = len(sc)
    g, n = min(gamma, n_docs), min(k, n_docs)
    bc, bf = fp32_sum_bound(ac, mc) + coarse_extra, fp32_sum_bound(af, mf)
    certain_c, might_c = _beat_counts(sc, bc, np.asarray(ac) == 0)
    possible, certain = certain_c < g, might_c < g
    gids = np.asarray(gids).astype(np.int64)[:n] & 0xFFFFFFFF
    gsc = np.asarray(gsc, np.float64)[:n]
    assert np.all(gids < n_docs), f"{what}: id out of range"
    assert len(set(gids.tolist())) == n, f"{what}: duplicate ids"
    bad = np.nonzero(~possible[gids])[0]
    assert len(bad) == 0, f"{what}: id {gids[bad[0]]} at rank {bad[0]} cannot be a coarse candidate"
    err = np.abs(gsc - sf[gids])
    bad = np.nonzero(err > bf[gids])[0]
    assert len(bad) == 0, (f"{what}: rank {bad[0]} id {gids[bad[0]]}: gpu {gsc[bad[0]]!r} exact "
                           f"{sf[gids[bad[0]]]!r} bound {bf[gids[bad[0]]]!r}")
    assert np.all(np.diff(gsc) <= 0), f"{what}: scores not in descending order"
    left = certain.copy()
    left[gids] = False
    if left.any():
        hi_out = np.max((sf - bf)[left])
        lo_in = np.min((sf + bf)[gids])
        assert hi_out <= lo_in, (f"{what}: a certain candidate left out ({hi_out!r}) certainly beats a returned "
                                 f"document ({lo_in!r})")
        z_in = [int(i) for i in gids if af[i] == 0]
        z_out = np.nonzero(left & (np.asarray(af) == 0))[0]
        if z_in and len(z_out):
            assert z_out.min() > max(z_in), f"{what}: exact-zero ties must go to the lower ids"
