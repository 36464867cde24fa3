"""Parity at full scale: the 8.8M-document index of the batched and reduced-precision configs (1,075 windows
of 8,192 documents per query, 230M postings, merges far above 16,384 candidates), on sampled queries against
the FP64 oracle (needs a GB300; minutes of host time for the oracle's index)."""
import concurrent.futures

import numpy as np
import pytest

import datagen
import oracle
from parity import check_reranked

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu, pytest.mark.slow]

if not torch.cuda.is_available():  # collected on CPU machines, never run there
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_2509_08395_gb300 as sindi  # noqa: E402

DEV = torch.device("cuda:0")
N_SAMPLE = 10


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


@pytest.fixture(scope="module")
def scale():
    w3, w4 = datagen.WORKLOADS["batched-8.8m"], datagen.WORKLOADS["lowprec-8.8m"]
    ip, ix, v = datagen.docs(w3)
    D = oracle.Dataset(ip, ix, v, w3.dim)
    # one oracle index per posting dtype, built at the same time (the oracle's C calls release the GIL)
    with concurrent.futures.ThreadPoolExecutor(max_workers=2) as ex:
        f32 = ex.submit(oracle.Index, D, window=w3.window, alpha=w3.alpha)
        f16 = ex.submit(oracle.Index, D, window=w4.window, alpha=w4.alpha, dtype="f16")
        I32, I16 = f32.result(), f16.result()
    qs = {}
    for w in (w3, w4):
        qp, qx, qv = datagen.queries(w)
        rows = list(range(0, len(qp) - 1, (len(qp) - 1) // N_SAMPLE))[:N_SAMPLE]
        sqp = np.concatenate([[0], np.cumsum([qp[r + 1] - qp[r] for r in rows])]).astype(np.int64)
        sqx = np.concatenate([qx[qp[r]:qp[r + 1]] for r in rows]).astype(np.int32)
        sqv = np.concatenate([qv[qp[r]:qp[r + 1]] for r in rows]).astype(np.float32)
        qs[w.name] = (sqp, sqx, sqv, oracle.Dataset(sqp, sqx, sqv, w.dim))
    return w3, w4, (ip, ix, v), D, I32, I16, qs


@pytest.mark.parametrize("mode,group", [("plain", 0), ("batched", 0), ("batched", 4)])
def test_batched_8_8m_sampled_queries(scale, mode, group):
    """8.8M docs, alpha 0.5, gamma 500, k 50, window 8,192, queries of 5 to 200 terms: each sampled query's
    reordered top-50 is the exact top-50 of an admissible candidate set of the oracle's Algorithm 4."""
    w3, _, (ip, ix, v), D, I32, _, qs = scale
    qp, qx, qv, Q = qs[w3.name]
    with sindi.Index(dev(ip), dev(ix), dev(v), w3.dim, window=w3.window, alpha=w3.alpha) as idx:
        assert idx.info["n_windows"] == 1075 and idx.info["postings"] == I32.postings
        ids, sc = idx.search(dev(qp), dev(qx), dev(qv), k=w3.k, gamma=w3.gamma, mode=mode, group=group)
        idx.check()
    ids, sc = ids.cpu().numpy().view(np.uint32).astype(np.int64), sc.cpu().numpy()
    touched = sum(check_reranked(ids[r], sc[r], D, Q, r, I32, w3.k, w3.gamma, what=f"{mode} query {r}")
                  for r in range(Q.n))
    assert touched <= 2


def test_lowprec_8_8m_fp16_gamma_1000(scale):
    """The same index with FP16 postings and a reorder pool of 1,000 (batched): the coarse stage against the
    oracle's Algorithm 2 on the same FP16 values, the answer exact FP32 scores of the full vectors."""
    _, w4, (ip, ix, v), D, _, I16, qs = scale
    qp, qx, qv, Q = qs[w4.name]
    with sindi.Index(dev(ip), dev(ix), dev(v), w4.dim, window=w4.window, alpha=w4.alpha, value_dtype="f16") as idx:
        ids, sc = idx.search(dev(qp), dev(qx), dev(qv), k=w4.k, gamma=w4.gamma, mode="batched")
        idx.check()
    ids, sc = ids.cpu().numpy().view(np.uint32).astype(np.int64), sc.cpu().numpy()
    touched = sum(check_reranked(ids[r], sc[r], D, Q, r, I16, w4.k, w4.gamma, what=f"f16 query {r}")
                  for r in range(Q.n))
    assert touched <= 2
