"""The device's candidate selection returns exactly the best g, on adversarial scores.

A window of the coarse stage does not keep a heap (Alg. 2): each window emits
the slots that can still be among the query's best g, using 12-bit bins of
the 64-bit order key (score bits, inverted id), an 8-bit second level inside
the cut bin, an exact select when ties crowd the cut, and a running bound
taken from the query's histogram H of what earlier windows emitted. The merge
then keeps the candidates at or above the bin of the g-th emitted one and
selects. This file models those rules, as the scan and merge kernels apply
them, and checks on the CPU that, for any order in which windows finish and
any snapshot of H a window may see, the result is exactly the top g by
(score desc, id asc). Score patterns are chosen to stress the rules:
massive exact ties, all-zero windows, values crowded into one bin, signed
values, N below g, g above the window size.
"""
import zlib

import numpy as np
import pytest

HIST_BITS, SUB_BITS = 12, 8
KEY_BIN_SHIFT = 64 - HIST_BITS


def order_bits(x32):
    """FP32 -> uint32 whose unsigned order is the float order (negative: all bits flipped)."""
    u = np.asarray(x32, np.float32).view(np.uint32).astype(np.uint64)
    return np.where(u & 0x80000000, (~u) & 0xFFFFFFFF, u | 0x80000000)


def keys_of(scores32, ids):
    return (order_bits(scores32) << np.uint64(32)) | (np.uint64(0xFFFFFFFF) - ids.astype(np.uint64))


def bins_of(keys):
    return (keys >> np.uint64(KEY_BIN_SHIFT)).astype(np.int64)


def find_bin(hist, g):
    """(bin holding the g-th largest counting from the top, count above it, its count, total); bin 0 and
    count above = total when the total is below g (the kernels' convention)."""
    total = int(hist.sum())
    if total < g:
        return 0, total, 0, total
    above = 0
    for b in range(len(hist) - 1, -1, -1):
        c = int(hist[b])
        if above < g <= above + c:
            return b, above, c, total
        above += c
    raise AssertionError("unreachable")


ZERO_KEY_BITS = np.uint64(0x80000000)                 # order bits of +0.0


def window_emit(K, g_w, win_cap, bounded, pbin, skip_zero=False, fallthrough_keys=None, slack=0):
    """The keys one window emits (its n_eff slots' keys K). skip_zero: slots whose score is exactly 0 cannot
    count (every score >= 0 and the earlier windows hold at least g slots); a bounded window then emits only
    positive slots at or above the bound. fallthrough_keys: what a bounded window with more slots at the bound
    than it may emit does to the keys of the full cut it falls back on (None: nothing, as the device does).
    slack: a bounded window also emits the slots of this many bins below the bound (the fixed-point window's
    integer bound may emit a few slots just under it)."""
    b = bins_of(K)
    if bounded:
        ok = b >= pbin - slack
        if skip_zero:
            ok &= (K >> np.uint64(32)) > ZERO_KEY_BITS     # score > 0
        hi = K[ok]
        if len(hi) <= win_cap:
            return hi
        if fallthrough_keys is not None:
            out = window_emit(K, g_w, win_cap, False, 0)
            return fallthrough_keys(out)
    bw, above_bw, _, _ = find_bin(np.bincount(b, minlength=1 << HIST_BITS), g_w)
    lo = max(bw, pbin) if bounded else bw
    thr = np.uint64(lo) << np.uint64(KEY_BIN_SHIFT)
    if lo == bw:
        sub = ((K[b == bw] >> np.uint64(KEY_BIN_SHIFT - SUB_BITS)) & np.uint64((1 << SUB_BITS) - 1)).astype(np.int64)
        bw2, a2, o2, _ = find_bin(np.bincount(sub, minlength=1 << SUB_BITS), g_w - above_bw)
        c_cut = above_bw + a2 + o2
        thr = np.uint64((bw << SUB_BITS) | bw2) << np.uint64(KEY_BIN_SHIFT - SUB_BITS)
        if c_cut > win_cap:
            thr = np.sort(K)[-g_w]                      # exact: the window's g_w-th best key
    return K[K >= thr]


def search_model(scores32, lam, g, schedule, rng, zero_rule="device", fallthrough_keys=None, slack=0):
    """Candidates of every window under `schedule`, then the merge; returns the selected keys, best first.
    zero_rule: "device" skips zero-score slots of window w when no score is negative and w * lam >= g;
    "off" never skips; "always" skips them whenever no score is negative (a planted mistake)."""
    n = len(scores32)
    nonneg = bool(np.all(np.asarray(scores32) >= 0))
    sigma = -(-n // lam)
    keys = keys_of(scores32, np.arange(n))
    win_cap = 2 * min(g, lam)
    H = np.zeros(1 << HIST_BITS, np.int64)
    emitted = []
    history = [H.copy()]                                # H after each finished window, in finishing order

    def run(w, snapshot):
        K = keys[w * lam: min(n, (w + 1) * lam)]
        g_w = min(g, len(K))
        bounded, pbin = False, 0
        if snapshot is not None:
            pbin, _, _, total = find_bin(snapshot, g)
            bounded = total >= g
        skip = nonneg and ((zero_rule == "device" and w * lam >= g) or (zero_rule == "always" and w > 0))
        out = window_emit(K, g_w, win_cap, bounded, pbin, skip, fallthrough_keys, slack)
        assert len(out) <= max(win_cap, g_w)
        emitted.append(out)
        np.add.at(H, bins_of(out), 1)
        history.append(H.copy())

    order = [int(w) for w in rng.permutation(sigma)]
    if schedule == "none":                              # every window cut on its own
        for w in order:
            run(w, None)
    elif schedule == "batched":                         # a snapshot of H from any earlier moment
        for w in order:
            run(w, history[int(rng.integers(0, len(history)))])
    elif schedule == "plain_split":                     # the first windows alone, then the rest with the bound
        first = max(2, -(-sigma // 8)) if sigma >= 8 else sigma
        for w in rng.permutation(first):
            run(int(w), None)
        done_a = len(history) - 1
        for w in rng.permutation(np.arange(first, sigma)):
            run(int(w), history[int(rng.integers(done_a, len(history)))])
    C = np.concatenate(emitted) if emitted else np.zeros(0, np.uint64)
    g_m = min(g, len(C))
    bstar, _, _, _ = find_bin(H, g_m)
    survivors = C[bins_of(C) >= bstar]
    return np.sort(survivors)[::-1][:g_m]


def truth(scores32, g):
    keys = keys_of(scores32, np.arange(len(scores32)))
    return np.sort(keys)[::-1][: min(g, len(keys))]


def score_pattern(kind, n, rng):
    if kind == "sparse":                                # most slots untouched (zero), lognormal hits
        s = np.zeros(n, np.float32)
        hit = rng.random(n) < 0.05
        s[hit] = rng.lognormal(0, 1, hit.sum())
    elif kind == "ties":                                # a handful of distinct values, massive exact ties
        s = rng.choice(np.array([0.0, 0.5, 1.0, 2.0], np.float32), n, p=[0.7, 0.2, 0.08, 0.02])
    elif kind == "zeros":
        s = np.zeros(n, np.float32)
    elif kind == "one_bin":                             # all in one 12-bit bin, split by the lower bits
        s = (1.0 + rng.random(n) * 1e-3).astype(np.float32)
    elif kind == "one_subbin":                          # all in one 20-bit prefix: only the exact select separates
        s = (1.0 + rng.integers(0, 8, n) * np.float32(2.0 ** -23)).astype(np.float32)
    elif kind == "signed":
        s = (rng.normal(0, 1, n) * (rng.random(n) < 0.3)).astype(np.float32)
    else:
        raise ValueError(kind)
    return np.asarray(s, np.float32)


@pytest.mark.parametrize("schedule", ["none", "batched", "plain_split"])
@pytest.mark.parametrize("kind", ["sparse", "ties", "zeros", "one_bin", "one_subbin", "signed"])
def test_selection_returns_exactly_the_best_g(kind, schedule):
    rng = np.random.default_rng(zlib.crc32(f"{kind}/{schedule}".encode()))
    for trial in range(12):
        lam = int(rng.choice([64, 256, 1000]))
        n = int(rng.choice([1, 7, lam - 1, lam, 3 * lam + 5, 9 * lam + 1, 17 * lam]))
        g = int(rng.choice([1, 10, 50, 300, 2000]))
        s = score_pattern(kind, n, rng)
        got = search_model(s, lam, g, schedule, rng)
        want = truth(s, g)
        assert np.array_equal(got, want), (kind, schedule, lam, n, g)


@pytest.mark.parametrize("schedule", ["batched", "plain_split"])
@pytest.mark.parametrize("kind", ["sparse", "ties", "one_bin", "signed"])
def test_bounded_windows_may_emit_slots_under_the_bound(kind, schedule):
    """The fixed-point window compares a bounded window's sums with an integer bound that may sit a little
    under the FP32 bound, so a few slots below it are emitted too. Emitting the whole bin below the bound (a
    wider superset) still gives exactly the best g: the merge drops the extra slots."""
    rng = np.random.default_rng(zlib.crc32(f"slack/{kind}/{schedule}".encode()))
    for trial in range(10):
        lam = int(rng.choice([64, 256, 1000]))
        n = int(rng.choice([lam - 1, 3 * lam + 5, 9 * lam + 1, 17 * lam]))
        g = int(rng.choice([1, 10, 50, 300]))
        s = score_pattern(kind, n, rng)
        got = search_model(s, lam, g, schedule, rng, slack=1)
        assert np.array_equal(got, truth(s, g)), (kind, schedule, lam, n, g)


def test_model_keys_order_like_the_search():
    """The model's keys rank like (score desc, id asc), so its selection is that order."""
    s = np.array([1.0, 2.0, 2.0, -1.0, 0.0, 0.0], np.float32)
    order = np.argsort(keys_of(s, np.arange(6)))[::-1]
    assert order.tolist() == [1, 2, 0, 4, 5, 3]


def test_zero_skip_rule_needs_the_earlier_windows_to_hold_g_slots():
    """The zero-score rule of the window cut: without its condition (the earlier windows hold at least g slots)
    it drops zero-score documents that belong to the answer (fewer than g positive scores, windows smaller
    than g); with it the selection stays exact (the parametrised test above runs the device rule)."""
    rng = np.random.default_rng(5)
    failed = False
    for trial in range(40):
        lam, g = 64, 300
        n = 9 * lam + 1
        s = score_pattern("sparse", n, rng)
        want = truth(s, g)
        assert np.array_equal(search_model(s, lam, g, "batched", rng, zero_rule="device"), want)
        failed |= not np.array_equal(search_model(s, lam, g, "batched", rng, zero_rule="always"), want)
    assert failed
