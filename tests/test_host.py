"""Host-side logic that needs no GPU: workload generators, autotuner window candidates, bench accounting."""
import hashlib
import os
import sys

import numpy as np

import datagen

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_uniform_sparsity_workloads():
    """Sec. 5's sparsity sweep stand-in: 120 entries per row, dims unique and uniform over [0, d), values
    uniform in (0, 1]."""
    for d in (10, 30, 100):
        w = datagen.WORKLOADS[f"uniform-1m-d{d}k"].scaled(n_docs=3000, n_queries=20)
        ip, ix, v = datagen.docs(w)
        assert np.all(np.diff(ip) == 120)
        assert ix.min() >= 0 and ix.max() < w.dim
        for i in range(0, 3000, 97):
            row = ix[ip[i]:ip[i + 1]]
            assert len(np.unique(row)) == 120
        assert v.min() > 0 and v.max() <= 1
        # dims spread over the whole range (uniform, not Zipf): every decile gets about a tenth
        counts = np.histogram(ix, bins=10, range=(0, w.dim))[0]
        assert counts.min() > 0.8 * counts.mean()


def test_autotuner_window_candidates():
    from paper_2509_08395_gb300 import autotune

    for n_docs in (5_000, 1_000_000, 8_800_000):
        ws = autotune.default_windows(n_docs, 152)
        assert ws and all(256 <= w <= 32768 and w % 32 == 0 for w in ws)
        assert ws == sorted(set(ws))


def test_bench_postings_accounting():
    """bench.postings_touched sums |I_j| over a query's terms (all windows) from the offsets table."""
    import bench

    dim, sigma = 5, 3
    lens = np.arange(dim * sigma, dtype=np.int64) % 4  # |I_{j,w}|
    seg = np.zeros(dim * sigma + 1, np.int64)
    np.cumsum(lens, out=seg[1:])
    qp = np.array([0, 2, 5], np.int64)
    qx = np.array([0, 3, 1, 2, 4], np.int32)
    got = bench.postings_touched(seg, sigma, dim, qp, qx)
    per_dim = lens.reshape(dim, sigma).sum(axis=1)
    assert got.tolist() == [per_dim[0] + per_dim[3], per_dim[1] + per_dim[2] + per_dim[4]]


def test_bench_traffic_only_for_the_profiled_source():
    import bench

    assert bench.profile_traffic("0" * 64) is None
    h = hashlib.sha256()
    for f in ("search.cu", "primitives.cuh", "common.cuh"):
        with open(os.path.join(ROOT, "paper_2509_08395_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    t = bench.profile_traffic(h.hexdigest())
    assert t is None or t > 0


def test_cpu_oracle_sample_reports_recall_and_tie_aware_recall():
    """bench.py's CPU leg: the oracle timed on a bounded sample, and both recalls of GPU-shaped answers
    against FP64 brute force (exact answers score 1; answers taken from ranks k..2k-1 score below 1)."""
    import bench
    import oracle

    w = datagen.WORKLOADS["exact-10k"].scaled(n_docs=2000, n_queries=30)
    ip, ix, v = datagen.docs(w)
    qp, qx, qv = datagen.queries(w)
    D, Q = oracle.Dataset(ip, ix, v, w.dim), oracle.Dataset(qp, qx, qv, w.dim)
    top = [oracle.brute_force(D, Q, r, 2 * w.k)[0] for r in range(Q.n)]
    exact = np.stack([t[: w.k] for t in top]).astype(np.uint32)
    qps, done, recalls, all_cores, tie = bench.cpu_oracle_sample(w, ip, ix, v, qp, qx, qv, 0.5, exact, w.k)
    assert qps > 0 and done >= 1 and all_cores["cores"] >= 1 and all_cores["value"] > 0
    assert recalls and len(tie) == len(recalls)
    assert all(r == 1.0 for r in recalls) and all(t == 1.0 for t in tie)
    worse = np.stack([t[w.k: 2 * w.k] for t in top]).astype(np.uint32)
    _, _, recalls, _, tie = bench.cpu_oracle_sample(w, ip, ix, v, qp, qx, qv, 0.2, worse, w.k)
    assert np.mean(recalls) < 0.5 and all(t >= r for r, t in zip(recalls, tie))


def test_bench_command_line():
    """bench.py parses its command line without a GPU: the driver's flags and the documented extras."""
    import subprocess
    import sys

    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--help"], capture_output=True, text=True,
                       timeout=120)
    assert r.returncode == 0, r.stderr
    for flag in ("--gpus", "--steps", "--warmup", "--impl", "--mode", "--workload", "--ablation",
                 "--sparsity-sweep", "--no-forms", "--cpu-seconds"):
        assert flag in r.stdout, flag


def test_pruned_1m_inputs_follow_their_recipe():
    """The pruned-1m stand-in draws what its recipe states (a 200k-document sample): document nnz
    lognormal with mean 120 and sigma_ln 0.5 in [10, 400], query nnz mean 45 in [5, 150], values
    lognormal(0, 0.8), dims unique within a row and Zipf(1.05) over ranks (slope of the mid ranks'
    frequencies on a log-log scale), and the same rows for the same seed."""
    w = datagen.WORKLOADS["pruned-1m"].scaled(n_docs=200_000)
    ip, ix, v = datagen.docs(w)
    nnz = np.diff(ip)
    assert nnz.min() >= 10 and nnz.max() <= 400
    assert abs(nnz.mean() - 120) < 1.5
    assert abs(np.log(nnz).std() - 0.5) < 0.02
    qp, qx, qv = datagen.queries(w)
    qn = np.diff(qp)
    assert qn.min() >= 5 and qn.max() <= 150 and abs(qn.mean() - 45) < 3
    lv = np.log(v.astype(np.float64))
    assert np.all(v > 0) and abs(lv.mean()) < 0.01 and abs(lv.std() - 0.8) < 0.01
    assert ix.min() >= 0 and ix.max() < w.dim
    rows = np.repeat(np.arange(len(nnz)), nnz)
    assert np.all(np.diff(np.sort(rows.astype(np.int64) * w.dim + ix)) > 0)   # unique dims per row
    freq = np.bincount(ix, minlength=w.dim).astype(np.float64)
    r = np.arange(1000, 10000)                                                 # dim = rank - 1
    slope = np.polyfit(np.log(r + 1.0), np.log(freq[r]), 1)[0]
    assert abs(slope + 1.05) < 0.1, slope
    ip2, ix2, v2 = datagen.docs(w)
    assert np.array_equal(ip, ip2) and np.array_equal(ix, ix2) and np.array_equal(v, v2)
    ip3, _, _ = datagen.generate(w.docs, w.dim, w.zipf_s, w.doc_seed + 1)
    assert not np.array_equal(ip, ip3)


class _FakeTensor:
    """Just enough of a tensor for the autotuner's host logic (shape, device, .cpu().numpy())."""

    def __init__(self, a):
        self.a = np.asarray(a)
        self.shape = self.a.shape
        self.device = "fake"

    def cpu(self):
        return self

    def numpy(self):
        return self.a


def test_autotuner_choice_logic(monkeypatch, tmp_path):
    """The tuner's selection, with a fake index and timer: per window the smallest gamma of the grid that
    reaches the recall target, then the fastest (mode, block) at that gamma; the cache serves a repeated
    call; an unreachable target leaves no choice and reports the table."""
    import types

    import torch

    from paper_2509_08395_gb300 import autotune

    n_q, k = 20, 10
    truth = np.arange(n_q * k, dtype=np.uint32).reshape(n_q, k)
    # recall of a (window, gamma): a window of 4096 reaches 0.99 at gamma 300, 8192 already at 200
    need = {4096: 300, 8192: 200}

    class FakeIndex:
        def __init__(self, ip, ix, v, dim, window, alpha, value_dtype="f32"):
            self.window, self.alpha = window, alpha

        def __enter__(self):
            return self

        def __exit__(self, *exc):
            return False

        def search(self, *q, k, gamma, mode="batched", block=0, out=None, group=1):
            if self.alpha == 1.0 and gamma == 0:          # the exact reference
                return _FakeTensor(truth.view(np.int32)), None
            ids = truth.copy()
            if gamma < need[self.window]:
                ids[:, -1] += 10_000                      # one miss per query: recall 0.9
            return _FakeTensor(ids.view(np.int32)), None

    speed = {("plain", 0): 100.0, ("batched", 0): 150.0, ("batched", 512): 170.0, ("plain", 512): 90.0}

    def fake_time(idx, q, k_, gamma, mode, block, repeats, group=1):
        # query groups of 2 help the batched 512-thread scan by 10%
        g = 1.1 if (mode, block, group) == ("batched", 512, 2) else (0.9 if group == 2 else 1.0)
        return speed[(mode, block)] * g * (2.0 if idx.window == 8192 else 1.0) / (gamma / 100.0), None

    monkeypatch.setattr(autotune.sindi, "Index", FakeIndex)
    monkeypatch.setattr(autotune, "_time_search", fake_time)
    monkeypatch.setattr(torch.cuda, "get_device_properties",
                        lambda dev: types.SimpleNamespace(name="fake GPU", multi_processor_count=152))
    q = (_FakeTensor(np.zeros(n_q + 1)), _FakeTensor(np.zeros(1)), _FakeTensor(np.zeros(1)))
    docs = (_FakeTensor(np.zeros(1001)), _FakeTensor(np.zeros(5)), _FakeTensor(np.zeros(5)))
    cache = str(tmp_path / "tune.json")
    res = autotune.autotune(*docs, 64, *q, k=k, alpha=0.5, windows=[4096, 8192], gammas=(100, 200, 300, 500),
                            blocks=(0, 512), modes=("plain", "batched"), cache=cache, groups=(1, 2))
    ch = res["choice"]
    # window 8192 reaches the target at gamma 200: 170 * 1.1 * 2 / 2 = 187 QPS (batched, 512 threads, groups of
    # 2) beats window 4096 at gamma 300 (62.3); the plain schedule is timed without groups
    assert (ch["window"], ch["gamma"], ch["mode"], ch["block"], ch["group"]) == (8192, 200, "batched", 512, 2)
    assert {r["group"] for r in res["table"] if r.get("mode") == "plain"} == {1}
    assert ch["recall"] == 1.0 and res["gpu"] == "fake GPU"
    tried = {(r["window"], r["gamma"]) for r in res["table"] if "qps" not in r}
    assert tried == {(4096, 100), (4096, 200), (4096, 300), (8192, 100), (8192, 200)}
    monkeypatch.setattr(autotune, "_time_search", lambda *a, **kw: (_ for _ in ()).throw(AssertionError("timed")))
    again = autotune.autotune(*docs, 64, *q, k=k, alpha=0.5, windows=[4096, 8192], gammas=(100, 200, 300, 500),
                              blocks=(0, 512), modes=("plain", "batched"), cache=cache, groups=(1, 2))
    assert again["choice"] == ch                          # served from the cache, nothing timed
    none = autotune.autotune(*docs, 64, *q, k=k, alpha=0.5, windows=[4096], gammas=(100, 200), blocks=(0,),
                             modes=("plain",))
    assert none["choice"] is None and len(none["table"]) == 2


def test_bench_clock_summary(tmp_path):
    """The clock record of the timed region: median SM clock, the maximum, and the throttle reasons that
    were active in any sample (nvidia-smi's csv,noheader,nounits rows; unreadable rows are skipped)."""
    import bench

    path = tmp_path / "clocks.csv"
    path.write_text(
        "0, 2070, 2070, 910.1, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active\n"
        "0, 1980, 2070, 1390.0, 0x0000000000000004, Not Active, Not Active, Not Active, Active\n"
        "0, [N/A], 2070, [N/A], [N/A], [N/A], [N/A], [N/A], [N/A]\n"
        "0, 2040, 2070, 1200.0, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active\n")
    c = bench.Clocks.__new__(bench.Clocks)
    c.proc, c.path = object(), str(path)
    s = c.summary()
    assert s == {"sm_mhz": 2040.0, "sm_max_mhz": 2070.0, "samples": 3, "reasons": ["sw_power_cap"]}
    c2 = bench.Clocks.__new__(bench.Clocks)
    c2.proc, c2.path = None, str(tmp_path / "none.csv")
    assert c2.summary()["reasons"] == ["nvidia-smi unavailable"]


def test_bench_hbm_peak_source(tmp_path, monkeypatch):
    """The roofline's HBM denominator: the measured copy rate when the peaks file has it, else the stated
    fallback, and the line says which."""
    import json

    import bench

    good = tmp_path / "peaks.json"
    good.write_text(json.dumps({"hbm_gbs": 6780.7, "bf16_tflops": 1890.1}))
    monkeypatch.setattr(bench, "PEAKS_FILE", str(good))
    assert bench.measured_hbm_peak() == (6780.7, "measured")
    monkeypatch.setattr(bench, "PEAKS_FILE", str(tmp_path / "missing.json"))
    assert bench.measured_hbm_peak() == (bench.FALLBACK_HBM_GBS, "fallback")
    bad = tmp_path / "bad.json"
    bad.write_text("{}")
    monkeypatch.setattr(bench, "PEAKS_FILE", str(bad))
    assert bench.measured_hbm_peak()[1] == "fallback"
    assert bench.FALLBACK_HBM_GBS == 6800.0


def test_generator_rows_do_not_depend_on_thread_count():
    """Rows come from a counter-based generator keyed by (seed, row): one thread or many draw the same
    matrix."""
    import subprocess
    import sys

    code = ("import sys, hashlib; sys.path.insert(0, %r); import datagen; "
            "w = datagen.WORKLOADS['pruned-1m'].scaled(n_docs=30000); ip, ix, v = datagen.docs(w); "
            "print(hashlib.sha256(ip.tobytes() + ix.tobytes() + v.tobytes()).hexdigest())" % ROOT)
    out = []
    for threads in ("1", "8"):
        env = dict(os.environ, OMP_NUM_THREADS=threads)
        r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env, timeout=120)
        assert r.returncode == 0, r.stderr
        out.append(r.stdout.strip())
    assert out[0] == out[1] and len(out[0]) == 64


def test_serving_load_generator_is_open_loop():
    """bench_native/serve_load.c against a fake server: one request per scheduled Poisson arrival (rows taken in
    turn), a failed request counted, and latency measured from the scheduled arrival (it includes the server's
    own submit-to-results time)."""
    import ctypes
    import importlib.util
    import threading
    import time

    spec = importlib.util.spec_from_file_location("bench_native_build_t", os.path.join(ROOT, "bench_native", "build.py"))
    bn = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(bn)
    bn.build()
    gen = ctypes.CDLL(bn.LOAD_LIB)
    sys_path = sys.path[:]
    sys.path.insert(0, ROOT)
    try:
        import bench
    finally:
        sys.path[:] = sys_path
    SUBMIT = ctypes.CFUNCTYPE(ctypes.c_int, ctypes.c_void_p, ctypes.POINTER(ctypes.c_int32),
                              ctypes.POINTER(ctypes.c_float), ctypes.c_int32, ctypes.POINTER(ctypes.c_uint64))
    POLL = ctypes.CFUNCTYPE(ctypes.c_int, ctypes.c_void_p, ctypes.c_uint64, ctypes.c_int32,
                            ctypes.POINTER(ctypes.c_uint32), ctypes.POINTER(ctypes.c_float),
                            ctypes.POINTER(ctypes.c_double))
    lock = threading.Lock()
    seen, times = [], []

    def submit(_srv, idx, val, nnz, ticket):
        with lock:
            ticket[0] = len(seen)
            seen.append((nnz, idx[0] if nnz else -1))
            times.append(time.perf_counter())
        return 0

    def poll(_srv, ticket, _wait, _ids, _sc, lat):
        lat[0] = 0.5
        return 6 if ticket == 5 else 0

    fs, fp = SUBMIT(submit), POLL(poll)
    qp = np.array([0, 2, 5, 6], np.int64)
    qx = np.array([10, 11, 20, 21, 22, 30], np.int32)
    qv = np.ones(6, np.float32)
    gen.sindi_load_open_loop.restype = ctypes.c_int
    gen.sindi_load_open_loop.argtypes = [ctypes.c_void_p] * 6 + [ctypes.c_int64, ctypes.c_uint32, ctypes.c_double,
                                                                 ctypes.c_double, ctypes.c_uint64,
                                                                 ctypes.POINTER(bench._LoadResult)]
    res = bench._LoadResult()
    rc = gen.sindi_load_open_loop(ctypes.c_void_p(1), ctypes.cast(fs, ctypes.c_void_p),
                                  ctypes.cast(fp, ctypes.c_void_p), qp.ctypes.data, qx.ctypes.data, qv.ctypes.data,
                                  3, 10, 2000.0, 0.5, 11, ctypes.byref(res))
    assert rc == 0
    assert res.requests == 1000 == len(seen)
    assert res.failed == 1
    assert seen[:6] == [(2, 10), (3, 20), (1, 30), (2, 10), (3, 20), (1, 30)]
    assert res.p50_ms >= 0.5 and res.server_p50_ms == 0.5 and res.p99_ms >= res.p50_ms
    # the arrivals follow the schedule: mean gap 1 / 2000 s (Poisson), not the speed of the submitter
    gaps = np.diff(times)
    assert 0.35e-3 < gaps.mean() < 0.7e-3, gaps.mean()
    assert 1200 < res.achieved_qps < 2600, res.achieved_qps
    # bad arguments are refused before anything is submitted
    assert gen.sindi_load_open_loop(None, None, None, None, None, None, 0, 10, 1.0, 1.0, 1,
                                    ctypes.byref(res)) == -1


def test_window_cost_model_fit():
    """The autotuner's window prior (Sec. 3.4's double power law T = c_rand l^a + c_evict l^-b + c0): exact
    data from known parameters gives back the closed-form optimum l* = (c_evict b / (c_rand a))^(1/(a+b)); noisy
    data stays near it; a curve with no rising term has no optimum and keeps every candidate."""
    from paper_2509_08395_gb300 import autotune as at

    lam = np.array([2048, 4096, 8192, 16384, 32768], np.float64)
    t = 3e-9 * lam ** 0.7 + 2e-3 * lam ** -0.9 + 1e-6
    f = at.fit_window_model(lam, t)
    want = (2e-3 * 0.9 / (3e-9 * 0.7)) ** (1 / 1.6)
    assert abs(f["lambda_star"] / want - 1) < 1e-6, (f, want)
    assert at.windows_near(f["lambda_star"], [2048, 4096, 8192, 16384, 32768]) == [2048, 4096, 8192]
    rng = np.random.default_rng(3)
    fn = at.fit_window_model(lam, t * (1 + 0.01 * rng.standard_normal(len(t))))
    assert 0.5 < fn["lambda_star"] / want < 2.0, fn
    falling = 2e-3 * lam ** -0.9 + 1e-6
    fd = at.fit_window_model(lam, falling)
    assert fd["lambda_star"] is None or fd["lambda_star"] > 1e6, fd
    if fd["lambda_star"] is None:
        assert at.windows_near(None, [4096, 2048]) == [2048, 4096]


def test_checked_build_predicates(tmp_path):
    """The bounds tests of the checked build (csrc/checks.cuh), compiled for the host: each accepts the last
    valid offset or id and refuses the first invalid one."""
    import subprocess

    src = tmp_path / "checks_host.cpp"
    src.write_text(r"""
#include <cstdio>
#include "checks.cuh"
using namespace sindi;
#define T(c) do { if (!(c)) { std::printf("failed: %s\n", #c); return 1; } } while (0)
int main() {
    static_assert(!kChecks, "host build: checks off unless asked for");
    T(segment_in_bounds(0, 0, 0)); T(segment_in_bounds(5, 16, 16)); T(!segment_in_bounds(5, 17, 16));
    T(!segment_in_bounds(9, 8, 16));
    T(group_in_bounds(8, 16)); T(!group_in_bounds(16, 16)); T(!group_in_bounds(4, 16));
    T(slot_in_bounds(4095, 4096)); T(!slot_in_bounds(4096, 4096));
    T(list_in_bounds(0, 0, 1, 1)); T(list_in_bounds(29, 61, 30, 62)); T(!list_in_bounds(30, 0, 30, 62));
    T(!list_in_bounds(-1, 0, 30, 62)); T(!list_in_bounds(0, 62, 30, 62));
    T(doc_in_bounds(999, 1000)); T(!doc_in_bounds(1000, 1000)); T(!doc_in_bounds(0xFFFFFFFFu, 1000));
    T(row_in_bounds(0, 0, 0)); T(row_in_bounds(3, 10, 10)); T(!row_in_bounds(3, 11, 10)); T(!row_in_bounds(5, 4, 10));
    T(!row_in_bounds(-1, 4, 10));
    std::printf("ok\n");
    return 0;
}
""")
    exe = tmp_path / "checks_host"
    inc = os.path.join(ROOT, "paper_2509_08395_gb300", "csrc")
    subprocess.run(["g++", "-std=c++17", "-Wall", "-Werror", "-I", inc, str(src), "-o", str(exe)], check=True)
    r = subprocess.run([str(exe)], capture_output=True, text=True)
    assert r.returncode == 0 and r.stdout.strip() == "ok", r.stdout + r.stderr


def test_fixed_point_rule_compiled_for_the_host(tmp_path):
    """The fixed-point window's arithmetic (csrc/fixed_point.cuh), compiled for the host:
    - exponent_bound brackets every positive float (2^(x-1) <= f < 2^x; subnormal, inf);
    - pow2f is 2^e;
    - fx_exponent_from keeps B * 2^e below 2^30 and every |w| * 2^e below 2^127, within [-126, 126];
    - fx_threshold, brute-forced around every threshold it returns: no sum whose FP32 score reaches the
      bound is below it, it is exact while the bound is within 2^24 units, and at most 129 units low above
      that (also next to -2^31, where a 32-bit margin would wrap)."""
    import subprocess

    src = tmp_path / "fixed_host.cpp"
    src.write_text(r"""
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <random>
#include "fixed_point.cuh"
using namespace sindi;
#define T(c) do { if (!(c)) { std::printf("failed line %d: %s\n", __LINE__, #c); return 1; } } while (0)
static bool qualifies(int64_t n, float thr, int e) { return (float)n * pow2f(-e) >= thr; }
int main() {
    std::mt19937 rng(7);
    // exponent_bound and pow2f
    for (int e = -126; e <= 126; e++) T(pow2f(e) == std::ldexp(1.0f, e));
    std::uniform_real_distribution<double> ex(-125.0, 127.0), fr(1.0, 2.0);
    for (int i = 0; i < 20000; i++) {
        const float f = (float)std::ldexp(fr(rng), (int)std::floor(ex(rng)));
        if (!(f > 0.0f) || std::isinf(f)) continue;
        const int x = exponent_bound(f);
        T(std::ldexp(1.0, x - 1) <= (double)f && (double)f < std::ldexp(1.0, x));
    }
    T(exponent_bound(1.0f) == 1 && exponent_bound(0.75f) == 0 && exponent_bound(2.0f) == 2);
    T(exponent_bound(1e-40f) == -126 && exponent_bound(INFINITY) == 140);
    // fx_exponent_from
    T(fx_exponent_from(0.0f, 1.0f) == 0 && fx_exponent_from(-1.0f, 1.0f) == 0);
    T(fx_exponent_from(1e-38f, 1e-38f) == 126 && fx_exponent_from(1e38f, 1.0f) == -97);  // 1e38 < 2^127
    T(fx_exponent_from(1.0f, 1e30f) == 127 - exponent_bound(1e30f));
    for (int i = 0; i < 20000; i++) {
        const float B = (float)std::ldexp(fr(rng), (int)std::floor(ex(rng)) - 1);
        const float M = (float)std::ldexp(fr(rng), (int)std::floor(ex(rng)) - 1);
        if (!(B > 0.0f) || std::isinf(B) || !(M > 0.0f) || std::isinf(M)) continue;
        const int e = fx_exponent_from(B, M);
        T(e >= -126 && e <= 126);
        if (e > -126) T((double)B * std::ldexp(1.0, e) < std::ldexp(1.0, 30));
        T((double)M * std::ldexp(1.0, e) < std::ldexp(1.0, 127));
    }
    // fx_threshold: specials
    T(fx_threshold(NAN, 0) == INT32_MAX && fx_threshold(-INFINITY, 5) == INT32_MIN);
    T(fx_threshold(INFINITY, 0) == INT32_MAX);
    T(fx_threshold(1.0e-45f, -126) == 1);  // the least positive float: only positive sums
    T(fx_threshold(0.0f, 7) == 0 && fx_threshold(-0.0f, 7) == 0);
    // fx_threshold: brute force around the threshold
    const int es[] = {-126, -60, -3, 0, 5, 30, 90, 126};
    std::uniform_real_distribution<double> lg(-31.5, 31.5), sg(0.0, 1.0);
    int checked = 0;
    for (int e : es) {
        for (int i = 0; i < 400; i++) {
            // bounds at every scale of units, both signs, and at the 2^24 and 2^31 edges
            double units = std::pow(2.0, lg(rng));
            if (i % 10 == 0) units = 16777216.0 + (double)(i % 7) - 3.0;
            if (i % 10 == 1) units = 2147483648.0 - (double)(i % 200);
            const double sign = sg(rng) < 0.5 ? -1.0 : 1.0;
            const float thr = (float)(sign * units * std::ldexp(1.0, -e));
            if (thr == 0.0f || std::isinf(thr)) continue;
            const int32_t t = fx_threshold(thr, e);
            const double X = (double)thr * std::ldexp(1.0, e);
            int64_t lo = (int64_t)t - 400, hi = (int64_t)t + 400;
            if (lo < INT32_MIN) lo = INT32_MIN;
            if (hi > INT32_MAX) hi = INT32_MAX;
            for (int64_t n = lo; n <= hi; n++) {
                if (qualifies(n, thr, e)) T(n >= t);                            // never above the least qualifying sum
                if (std::fabs(X) < 16777216.0 && n >= t) T(qualifies(n, thr, e));   // exact below 2^24 units
                checked++;
            }
            if (X > 16777216.0 && X < 2147483648.0) T((double)t >= std::floor(X) - 129.0);
            if (X < -16777216.0 && X >= -2147483648.0) T((double)t >= std::floor(X) - 129.0 || t == INT32_MIN);
        }
    }
    T(fx_threshold(-2147483648.0f, 0) == INT32_MIN);                  // -2^31 units: no 32-bit wrap
    T(fx_threshold(-2147483520.0f, 0) == INT32_MIN);                  // within 128 of -2^31
    std::printf("ok %d\n", checked);
    return 0;
}
""")
    exe = tmp_path / "fixed_host"
    inc = os.path.join(ROOT, "paper_2509_08395_gb300", "csrc")
    subprocess.run(["g++", "-std=c++17", "-O2", "-Wall", "-Werror", "-I", inc, str(src), "-o", str(exe)], check=True)
    r = subprocess.run([str(exe)], capture_output=True, text=True)
    assert r.returncode == 0 and r.stdout.startswith("ok"), r.stdout + r.stderr
