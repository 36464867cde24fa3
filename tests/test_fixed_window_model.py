"""A host model of the fixed-point score window (sindi_accumulator FIXED32), checked against exact sums.

The device's rule for one (query, window): B = the FP32 sum of |w_j| * vmax_j over the window's terms (w_j the
term weight, vmax_j the largest |stored value| of list j), e = 30 - x with 2^(x-1) <= B < 2^x, clamped so that
every |w_j| * 2^e < 2^127 and to [-126, 126] (0 when B = 0). Each product is the FP32 product of the weight
times 2^e (exact) and the stored value, rounded to the nearest integer (ties to even); the integer sums are
exact; the score is the FP32 conversion of the sum times 2^-e.

The model follows that rule in numpy and checks what the design depends on: no window sum reaches 2^31 even
when every product of a document sits at its bound with one sign and B is summed in any order, and a score of
m products is within 2^-23 * a + m * 2^-(e+1) <= 2^-23 * a + m * B * 2^-30 of the exact score. A mistake
planted in the model's B (one term's bound instead of the sum) must overflow on the adversarial case."""
import numpy as np
import pytest

F32 = np.float32


def exponent_bound(f):
    """x with 2^(x-1) <= f < 2^x for finite f > 0 (from the exponent field); subnormal: -126; inf: 140."""
    E = int((np.array(f, F32).view(np.uint32) >> 23) & 0xFF)
    return 140 if E == 0xFF else (-126 if E == 0 else E - 126)


def pow2f(e):
    return np.array((e + 127) << 23, np.uint32).view(F32)[()]


def window_exponent(wq, vmax, order=None):
    """The device's e for term weights wq and list bounds vmax (FP32), B summed in `order`."""
    idx = np.arange(len(wq)) if order is None else order
    B, M = F32(0), F32(0)
    for t in idx:
        B = F32(B + F32(abs(wq[t])) * F32(vmax[t]))
        M = max(M, F32(abs(wq[t])))
    if not B > 0:
        return 0
    e = 30 - exponent_bound(B)
    if M > 0:
        e = min(e, 127 - exponent_bound(M))
    return max(-126, min(126, e))


def fixed_score(wq, vals, e):
    """(integer sum, FP32 score) of the products wq[t] * vals[t] in the fixed-point window with unit 2^-e."""
    s = pow2f(e)
    units = [np.rint(F32(F32(w) * s) * F32(x)) for w, x in zip(wq, vals)]
    total = int(sum(int(u) for u in units))
    return total, F32(F32(total) * pow2f(-e))


def _terms(rng, n, lo, hi):
    wq = (10.0 ** rng.uniform(lo, hi, n)).astype(F32)
    vmax = (10.0 ** rng.uniform(lo, hi, n)).astype(F32)
    return wq, vmax


@pytest.mark.parametrize("n,lo,hi", [(1, 0, 0), (47, -1, 1), (400, -3, 3), (4096, -2, 2), (60, -30, -20),
                                     (60, 15, 18), (200, -8, 8)])
def test_no_window_sum_reaches_2_31(n, lo, hi):
    """Every product at its bound, all of one sign, B summed in three orders: |sum| < 2^31."""
    rng = np.random.default_rng(n * 7 + lo)
    wq, vmax = _terms(rng, n, lo, hi)
    for order in (None, np.argsort(wq * vmax), np.argsort(-(wq * vmax))):
        e = window_exponent(wq, vmax, order)
        for sign in (1, -1):
            total, _ = fixed_score(wq * F32(sign), vmax, e)
            assert abs(total) < 2 ** 31


@pytest.mark.parametrize("seed", range(6))
def test_score_error_within_the_bound(seed):
    """Random documents over random terms (signed, some cancelling): |score - exact| <= 2^-23 a + m 2^-(e+1)
    and m 2^-(e+1) <= m B 2^-30, with the exact sum taken in FP64 from the FP32 inputs."""
    rng = np.random.default_rng(100 + seed)
    n = int(rng.integers(1, 300))
    wq, vmax = _terms(rng, n, -2, 2)
    wq = wq * np.where(rng.random(n) < 0.3, F32(-1), F32(1)).astype(F32)
    e = window_exponent(wq, vmax)
    B = float(np.sum(np.abs(wq.astype(np.float64)) * vmax))
    for _ in range(50):
        m = int(rng.integers(1, n + 1))
        terms = rng.choice(n, m, replace=False)
        vals = (vmax[terms] * rng.uniform(0, 1, m)).astype(F32)
        exact = float(np.sum(wq[terms].astype(np.float64) * vals.astype(np.float64)))
        a = float(np.sum(np.abs(wq[terms].astype(np.float64) * vals.astype(np.float64))))
        _, score = fixed_score(wq[terms], vals, e)
        half_units = m * 2.0 ** (-(e + 1))
        assert half_units <= m * B * 2.0 ** -30 * (1 + 1e-6)
        assert abs(float(score) - exact) <= 2.0 ** -23 * a * (1 + 1e-6) + half_units * (1 + 1e-6)


def test_unit_clamps():
    """A weight so large that |w| * 2^e would pass 2^127 lowers e; tiny data stops at e = 126."""
    wq, vmax = np.array([F32(1e30)], F32), np.array([F32(1e-35)], F32)
    e = window_exponent(wq, vmax)
    assert abs(float(wq[0]) * 2.0 ** e) < 2.0 ** 127 and np.isfinite(F32(wq[0] * pow2f(e)))
    assert window_exponent(np.array([F32(1e-20)], F32), np.array([F32(1e-20)], F32)) == 126
    assert window_exponent(np.zeros(3, F32), np.ones(3, F32)) == 0


def test_a_planted_max_for_sum_overflows():
    """The rule with B taken as the largest |w_j| * vmax_j instead of their sum (a plausible slip: one term's
    bound for the window's) lets the adversarial sum of a 47-term query reach 2^31; the overflow test above
    would catch it."""
    rng = np.random.default_rng(5)
    wq, vmax = _terms(rng, 47, -1, 1)
    i = int(np.argmax(wq.astype(np.float64) * vmax))
    e = window_exponent(wq[i:i + 1], vmax[i:i + 1])
    total, _ = fixed_score(wq, vmax, e)
    assert abs(total) >= 2 ** 31


def test_emulated_window_on_oracle_lists_is_within_the_test_allowance():
    """The fixed-point window emulated on the oracle's own lists (an alpha-mass index of a small synthetic
    workload, signed values, window 256): every document's coarse score lies within the FP32 dot-product bound
    plus parity.fixed_extra of the exact FP64 score, and the GPU tests' comparison rule accepts the emulated
    top-k. So a GPU test that fails under that allowance points at the GPU, not at the allowance."""
    import datagen
    import oracle
    from parity import check_ranked_conditioned, fixed_extra, fp32_sum_bound, signed_copy

    w = datagen.WORKLOADS["pruned-1m"].scaled(n_docs=3000, n_queries=6)
    ip, ix, v = datagen.docs(w)
    qp, qx, qv = datagen.queries(w)
    v, qv = signed_copy(v, 3), signed_copy(qv, 5)
    D, Q = oracle.Dataset(ip, ix, v, w.dim), oracle.Dataset(qp, qx, qv, w.dim)
    Da, Qa = oracle.Dataset(ip, ix, np.abs(v), w.dim), oracle.Dataset(qp, qx, np.abs(qv), w.dim)
    lam = 256
    I = oracle.Index(D, window=lam, alpha=0.5)
    Ia = oracle.Index(Da, window=lam, alpha=0.5)
    seg, pid, pval, _, _ = I.export()
    sig = I.sigma
    vmax = I.list_vmax().astype(F32)
    qptr, qdims, qvals = Q.export()
    for r in range(Q.n):
        terms = qdims[qptr[r]:qptr[r + 1]]
        weights = qvals[qptr[r]:qptr[r + 1]].astype(F32)
        score = np.zeros(D.n, F32)
        for win in range(sig):
            lens = np.array([seg[j * sig + win + 1] - seg[j * sig + win] for j in terms])
            live = lens > 0
            e = window_exponent(weights[live], vmax[terms[live]]) if live.any() else 0
            acc = {}
            for j, wq in zip(terms[live], weights[live]):
                ws = F32(F32(wq) * pow2f(e))
                for p in range(seg[j * sig + win], seg[j * sig + win + 1]):
                    acc[int(pid[p])] = acc.get(int(pid[p]), 0) + int(np.rint(F32(ws * F32(pval[p]))))
            for doc, total in acc.items():
                assert abs(total) < 2 ** 31
                score[doc] = F32(F32(total) * pow2f(-e))
        s, a = np.empty(D.n), np.empty(D.n)
        oi, os_ = I.search(Q, r, k=D.n, gamma=0)
        s[oi] = os_
        oi, os_ = Ia.search(Qa, r, k=D.n, gamma=0)
        a[oi] = os_
        m = len(terms)
        extra = fixed_extra(I, Q, r)
        assert np.all(np.abs(score.astype(np.float64) - s) <= fp32_sum_bound(a, m) + extra), f"query {r}"
        order = sorted(range(D.n), key=lambda i: (-float(score[i]), i))[:50]
        check_ranked_conditioned(np.array(order), score[order], s, a, m, 50, what=f"query {r}", extra=extra)


def _fp32_bits_read_as_sums(keys, e=18):
    """A fault the scan once had: after a bounded fixed-point window converted its sums to FP32 for the full cut,
    the cut kept reading slots as integer sums, so each emitted score became (FP32 bits as an integer) * 2^-e."""
    from test_selection_model import keys_of
    ob = (keys >> np.uint64(32)).astype(np.uint64)
    u = np.where(ob & np.uint64(0x80000000), ob & np.uint64(0x7FFFFFFF), (~ob) & np.uint64(0xFFFFFFFF)).astype(np.uint32)
    as_sum = u.view(np.float32).view(np.int32).astype(np.float32)
    ids = np.uint64(0xFFFFFFFF) - (keys & np.uint64(0xFFFFFFFF))
    return keys_of((as_sum * F32(2.0 ** -e)).astype(F32), ids)


@pytest.mark.parametrize("schedule", ["plain_split", "batched"])
def test_a_bounded_window_that_falls_back_keeps_fp32_keys(schedule):
    """Windows whose slots at the bound outnumber what one window may emit (here: many equal scores) fall back
    on the full cut after converting their sums to FP32. The model of the device returns exactly the best g.
    With the fault planted (the cut still reading slots as fixed-point sums) the answer is taken over by a
    window that fell back, the symptom the GPU determinism test once showed: every returned id from one
    window."""
    from test_selection_model import search_model, truth
    lam, g = 512, 50
    rng = np.random.default_rng(3)
    scores = np.ones(8 * lam, F32)                      # massive ties: every slot of every window at the bound
    scores[rng.choice(2 * lam, 20, replace=False)] = F32(1.5)
    want = truth(scores, g)
    for seed in range(6):
        got = search_model(scores, lam, g, schedule, np.random.default_rng(seed))
        assert np.array_equal(got, want), seed
    planted = search_model(scores, lam, g, schedule, np.random.default_rng(0),
                           fallthrough_keys=_fp32_bits_read_as_sums)
    assert not np.array_equal(planted, want)
    ids = (np.uint64(0xFFFFFFFF) - (planted & np.uint64(0xFFFFFFFF))).astype(np.int64)
    assert len(set((ids // lam).tolist())) == 1         # one window's slots fill the answer
