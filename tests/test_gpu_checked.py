"""The checked build (lib/libsindi_checked.so: every offset and id a search kernel follows is tested first and a
failure recorded in the error word, never a trap) on small parity cases: results equal the oracle's and the
error word stays zero (needs a GB300). Each case runs in a child process that loads the checked library."""
import os
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # collected on CPU machines, never run there
    pytest.skip("needs a CUDA device", allow_module_level=True)

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CHECKED = os.path.join(ROOT, "paper_2509_08395_gb300", "lib", "libsindi_checked.so")

CHILD = r"""
import sys
import numpy as np
import torch
sys.path.insert(0, {root!r})
sys.path.insert(0, {tests!r})
import datagen, oracle
from parity import check_ranked, check_reranked
import paper_2509_08395_gb300 as sindi
assert sindi.load()._name.endswith("libsindi_checked.so"), sindi.load()._name
dev = torch.device("cuda:0")
t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
w = datagen.WORKLOADS["pruned-1m"].scaled(n_docs=20_001, n_queries=16)
ip, ix, v = datagen.docs(w)
qp, qx, qv = datagen.queries(w)
D, Q = oracle.Dataset(ip, ix, v, w.dim), oracle.Dataset(qp, qx, qv, w.dim)
cases = {cases}
for window, alpha, dtype, mode, k, gamma, group, block in cases:
    I = oracle.Index(D, window=window, alpha=alpha, dtype=dtype)
    with sindi.Index(t(ip), t(ix), t(v), w.dim, window=window, alpha=alpha, value_dtype=dtype) as idx:
        ids, sc = idx.search(t(qp), t(qx), t(qv), k=k, gamma=gamma, mode=mode, group=group, block=block)
        idx.check()  # raises on any recorded bounds failure
        ids = ids.cpu().numpy().view(np.uint32).astype(np.int64)
        sc = sc.cpu().numpy()
    for r in range(Q.n):
        if gamma == 0:
            oi, os_ = I.search(Q, r, k=k + 64, gamma=0)
            check_ranked(ids[r], sc[r], oi, os_, k, D.n, what=f"{{window}} {{mode}} query {{r}}")
        else:
            check_reranked(ids[r], sc[r], D, Q, r, I, k, gamma, what=f"{{window}} {{mode}} query {{r}}")
print("checked ok", len(cases))
"""


@pytest.mark.parametrize("cases", [
    [(4096, 1.0, "f32", "plain", 20, 0, 0, 0), (2048, 0.5, "f32", "batched", 20, 300, 0, 0)],
    [(1024, 0.5, "f16", "batched", 20, 300, 4, 1024), (300, 0.5, "f8", "plain", 10, 200, 0, 0)],
    [(8192, 0.5, "f32", "plain", 50, 500, 0, 1), (4096, 0.5, "f32", "batched", 50, 0, 0, 256)],
])
def test_checked_build_parity_and_clean_error_word(cases):
    assert os.path.exists(CHECKED), "build lib/libsindi_checked.so first (__graft_entry__.build())"
    code = CHILD.format(root=ROOT, tests=os.path.join(ROOT, "tests"), cases=repr(cases))
    env = dict(os.environ, SINDI_LIBRARY=CHECKED)
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env, timeout=600)
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-3000:]
    assert "checked ok" in r.stdout
