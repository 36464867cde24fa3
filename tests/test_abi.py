"""The C ABI library: it loads without a GPU and exports every function include/*.h declares."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"\b(sindi_\w+)\s*\(", text):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def lib():
    from paper_2509_08395_gb300 import build_native

    path = build_native.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = _declared()
    for n in ("sindi_build", "sindi_search", "sindi_check", "sindi_index_info", "sindi_index_free",
              "sindi_last_error", "sindi_index_export"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in sorted(_declared()) if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_the_header():
    from paper_2509_08395_gb300 import sindi

    assert _declared() <= set(sindi._SIGS)


def test_calls_without_device_fail_cleanly(lib):
    """No compute: argument checks return INVALID_ARG before touching a device."""
    from paper_2509_08395_gb300 import sindi

    L = sindi.load()
    out = ctypes.c_void_p()
    assert L.sindi_build(None, None, None, 10, 4, None, None, ctypes.byref(out)) == sindi.SINDI_ERR_INVALID_ARG
    prm = sindi.sindi_search_params(k=0, gamma=0, beta=1.0, mode=0, block_threads=0)
    assert L.sindi_search(None, None, None, None, 1, ctypes.byref(prm), None, None, None) == \
        sindi.SINDI_ERR_INVALID_ARG
    assert b"NULL" in L.sindi_last_error()
    assert L.sindi_version().startswith(b"sindi-gb300")


def test_index_load_rejects_files_that_are_not_index_files(lib, tmp_path):
    """The header is checked before any device work: foreign, truncated or inconsistent files are
    SINDI_ERR_INVALID_DATA, a missing file INVALID_ARG."""
    from paper_2509_08395_gb300 import sindi

    L = sindi.load()
    out = ctypes.c_void_p()
    junk = tmp_path / "junk.bin"
    junk.write_bytes(b"not an index" * 10)
    assert L.sindi_index_load(str(junk).encode(), None, ctypes.byref(out)) == sindi.SINDI_ERR_INVALID_DATA
    assert out.value is None
    # the right magic and version, a header whose sizes disagree (sigma != ceil(n_docs / lambda))
    import struct
    hdr = struct.pack("<8sIIqiIIidiIqq", b"SINDIGB3", 1, 72, 100, 8, 64, 7, 0, 1.0, 0, 0, 10, 10)
    assert len(hdr) == 72
    bad = tmp_path / "bad.bin"
    bad.write_bytes(hdr)
    assert L.sindi_index_load(str(bad).encode(), None, ctypes.byref(out)) == sindi.SINDI_ERR_INVALID_DATA
    assert b"header" in L.sindi_last_error()
    # a consistent header that claims more postings than uint32 scan positions can address
    big = struct.pack("<8sIIqiIIidiIqq", b"SINDIGB3", 1, 72, 100, 8, 64, 2, 0, 1.0, 0, 0, 1 << 33, 1 << 32)
    bad.write_bytes(big)
    assert L.sindi_index_load(str(bad).encode(), None, ctypes.byref(out)) == sindi.SINDI_ERR_INVALID_DATA
    assert b"inconsistent header" in L.sindi_last_error()
    # a consistent header over a truncated body
    hdr = struct.pack("<8sIIqiIIidiIqq", b"SINDIGB3", 1, 72, 100, 8, 64, 2, 0, 1.0, 0, 0, 10, 10)
    short = tmp_path / "short.bin"
    short.write_bytes(hdr + b"\0" * 16)
    assert L.sindi_index_load(str(short).encode(), None, ctypes.byref(out)) == sindi.SINDI_ERR_INVALID_DATA
    assert b"size" in L.sindi_last_error()
    assert L.sindi_index_load(str(tmp_path / "missing.bin").encode(), None, ctypes.byref(out)) == \
        sindi.SINDI_ERR_INVALID_ARG


def test_binding_checks_buffer_sizes_before_the_call(lib):
    """The C calls get bare pointers; the binding refuses undersized buffers before calling them, and takes
    a stream as a raw handle or as an object with a cuda_stream attribute."""
    import numpy as np
    import pytest
    from paper_2509_08395_gb300 import sindi

    qp, qx, qv = np.array([0, 1, 2], np.int64), np.array([1, 2], np.int32), np.ones(2, np.float32)
    ids, sc = np.empty((2, 10), np.uint32), np.empty((2, 10), np.float32)
    with pytest.raises(ValueError, match="out_ids"):
        sindi.sindi_search(1, qp, qx, qv, 2, ids[:1], sc, k=10)
    with pytest.raises(ValueError, match="out_scores"):
        sindi.sindi_search_noalloc(1, qp, qx, qv, 2, ids, sc[:, :5].copy(), k=10)
    with pytest.raises(ValueError, match="q_indptr"):
        sindi.sindi_search(1, qp, qx, qv, 3, np.empty((3, 10), np.uint32), np.empty((3, 10), np.float32), k=10)
    with pytest.raises(ValueError, match="indptr"):
        sindi.sindi_build(np.zeros(3, np.int64), qx, qv, 5, 4)
    with pytest.raises(ValueError, match="accum"):
        sindi.sindi_search(1, qp, qx, qv, 2, ids, sc, k=10, accum="fp16")
    assert sindi._accum("auto") == 0 and sindi._accum("f32") == 1 and sindi._accum("fixed32") == 2

    class FakeStream:
        cuda_stream = 1234

    assert sindi._stream(FakeStream()) == 1234 and sindi._stream(77) == 77 and sindi._stream(None, qp) is None


def test_entry_points_push_nvtx_ranges(lib, tmp_path):
    """Every entry point opens an NVTX range named for the call (a timeline tool shows which call a kernel
    belongs to). A recording NVTX injection library (tests/nvtx_recorder.c) captures them in a child
    process; the calls fail their argument checks, so nothing touches a device."""
    import shutil
    import subprocess
    import sys

    import pytest

    cuda_inc = "/usr/local/cuda/include"
    if not os.path.exists(os.path.join(cuda_inc, "nvtx3", "nvToolsExt.h")) or not shutil.which("gcc"):
        pytest.skip("needs gcc and the CUDA NVTX headers")
    rec = str(tmp_path / "librecorder.so")
    subprocess.check_call(["gcc", "-O1", "-fPIC", "-shared", f"-I{cuda_inc}",
                           os.path.join(ROOT, "tests", "nvtx_recorder.c"), "-o", rec])
    log = tmp_path / "ranges.txt"
    child = (
        "import ctypes, sys\n"
        f"sys.path.insert(0, {ROOT!r})\n"
        "from paper_2509_08395_gb300 import sindi\n"
        "L = sindi.load()\n"
        "out = ctypes.c_void_p()\n"
        "assert L.sindi_build(None, None, None, 10, 4, None, None, ctypes.byref(out)) != 0\n"
        "prm = sindi.sindi_search_params(k=5, gamma=0, beta=1.0, mode=1, block_threads=0)\n"
        "assert L.sindi_search(None, None, None, None, 3, ctypes.byref(prm), None, None, None) != 0\n"
        "assert L.sindi_index_load(b'/nonexistent/index.bin', None, ctypes.byref(out)) != 0\n"
    )
    env = dict(os.environ, NVTX_INJECTION64_PATH=rec, NVTX_RECORD_PATH=str(log))
    subprocess.run([sys.executable, "-c", child], check=True, env=env, timeout=120)
    lines = log.read_text().splitlines()
    assert lines == ["push sindi_build n_docs=10 dim=4", "pop", "push sindi_search n_queries=3 mode=1", "pop",
                     "push sindi_index_load", "pop"], lines


def test_closing_an_index_closes_its_plans_and_servers_first(lib):
    """A plan or server must not outlive its index: Index.close() closes those still open, then frees."""
    import weakref

    from paper_2509_08395_gb300 import sindi

    order = []

    class Dependent:
        def __init__(self, name):
            self.name = name

        def close(self):
            order.append(self.name)

    idx = sindi.Index.__new__(sindi.Index)
    idx.handle = None                       # nothing to free on the device
    idx._dependents = weakref.WeakSet()
    plan, server = Dependent("plan"), Dependent("server")
    idx._dependents.add(plan)
    idx._dependents.add(server)
    idx.close()
    assert sorted(order) == ["plan", "server"]


def test_build_parameter_checks_come_before_any_device_work(lib):
    """Each invalid build parameter is refused with its status and a message, before the device is touched
    (this machine may have none); valid arguments reach the device check and fail cleanly without one."""
    import numpy as np

    from paper_2509_08395_gb300 import sindi

    L = sindi.load()
    ip = np.array([0, 2, 3], np.int64)
    ix = np.array([0, 1, 2], np.int32)
    v = np.ones(3, np.float32)
    out = ctypes.c_void_p()

    def build(n_docs=2, dim=4, **kw):
        prm = sindi.sindi_build_params(**dict(dict(window=0, value_dtype=0, alpha=1.0, prune=0, prune_n=0), **kw))
        return L.sindi_build(ip.ctypes.data, ix.ctypes.data, v.ctypes.data, n_docs, dim, ctypes.byref(prm), None,
                             ctypes.byref(out))

    invalid = [dict(alpha=0.0), dict(alpha=1.5), dict(alpha=float("nan")), dict(window=32769), dict(value_dtype=3),
               dict(value_dtype=-1), dict(prune=4), dict(prune=-1), dict(prune=1, prune_n=0),
               dict(prune=2, prune_n=0), dict(prune=3, prune_n=0), dict(n_docs=-1), dict(dim=0)]
    for kw in invalid:
        assert build(**kw) == sindi.SINDI_ERR_INVALID_ARG, kw
        assert L.sindi_last_error(), kw
        assert out.value is None
    # an offset table of 2^34 entries or more is refused as unsupported
    assert build(n_docs=(1 << 32) - 2, dim=1 << 20, window=1) == sindi.SINDI_ERR_UNSUPPORTED
    assert b"offset table" in L.sindi_last_error()
    import torch

    if not torch.cuda.is_available():
        assert build() == sindi.SINDI_ERR_CUDA and out.value is None


C_CALLER = r"""
#include <stdio.h>
#include <string.h>
#include "sindi.h"

int main(void) {
    sindi_index* idx = NULL;
    int64_t indptr[3] = {0, 1, 2};
    int32_t indices[2] = {0, 1};
    float values[2] = {1.0f, 2.0f};
    sindi_build_params bad = {0, SINDI_F32, 2.0, SINDI_PRUNE_MASS, 0};   /* alpha out of range */
    sindi_status s = sindi_build(indptr, indices, values, 2, 4, &bad, NULL, &idx);
    if (s != SINDI_ERR_INVALID_ARG || idx != NULL || strlen(sindi_last_error()) == 0) return 1;
    sindi_search_params sp = {10, 0, 1.0, SINDI_MODE_PLAIN, 0};
    if (sindi_search(NULL, NULL, NULL, NULL, 1, &sp, NULL, NULL, NULL) != SINDI_ERR_INVALID_ARG) return 2;
    sindi_index_free(NULL);
    printf("%s\n", sindi_version());
    return 0;
}
"""


def test_plain_c_caller(lib, tmp_path):
    """The header is C (not only C++) and the library links and answers from a C program: argument errors
    come back as status codes with a message, before any device work."""
    import shutil
    import subprocess

    import pytest

    if not shutil.which("gcc"):
        pytest.skip("needs gcc")
    src = tmp_path / "caller.c"
    src.write_text(C_CALLER)
    exe = tmp_path / "caller"
    libdir = os.path.dirname(lib._name)
    subprocess.check_call(["gcc", "-std=c11", "-Wall", "-Werror", f"-I{os.path.join(ROOT, 'include')}", str(src),
                           "-o", str(exe), f"-L{libdir}", "-lsindi", f"-Wl,-rpath,{libdir}"])
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=60)
    assert r.returncode == 0, (r.returncode, r.stderr)
    assert r.stdout.startswith("sindi-gb300")
