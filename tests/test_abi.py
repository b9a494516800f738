"""The C ABI without a GPU: libgr.so loads, exports every entry point that
include/gr.h declares, and rejects invalid arguments with GR_EINVAL before
touching the device."""
import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def gr():
    from paper_1501_05387_gb300 import build
    build.build()
    from paper_1501_05387_gb300 import gr as grmod
    return grmod


def declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if not fn.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", fn)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names |= set(re.findall(r"\b(gr_\w+)\s*\(", text))
    return sorted(names)


def test_header_declares_the_primitives():
    names = declared_functions()
    for required in ["gr_graph_create", "gr_graph_destroy", "gr_bfs", "gr_last_error"]:
        assert required in names


def test_library_exports_every_declared_symbol(gr):
    lib = ctypes.CDLL(gr.LIB_PATH)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, f"declared but not exported: {missing}"
    out = subprocess.check_output(["nm", "-D", "--defined-only", gr.LIB_PATH], text=True)
    exported = {l.split()[-1] for l in out.splitlines() if l.strip()}
    assert set(declared_functions()) <= exported


def _create(gr, row_off, col, w=None):
    out = ctypes.c_void_p()
    n = row_off.size - 1
    st = gr._lib.gr_graph_create(n, col.size, row_off.ctypes.data,
                                 col.ctypes.data if col.size else None,
                                 None if w is None else w.ctypes.data, 0, None,
                                 ctypes.byref(out))
    return st, out


@pytest.mark.parametrize("row_off,col,what", [
    (np.array([1, 2], np.int32), np.array([0, 0], np.int32), "row_off[0]"),
    (np.array([0, 2, 1, 2], np.int32), np.array([0, 1], np.int32), "non-decreasing"),
    (np.array([0, 1, 1], np.int32), np.array([0, 1], np.int32), "row_off[n]"),
    (np.array([0, 1, 2], np.int32), np.array([0, 2], np.int32), "out of range"),
    (np.array([0, 1, 2], np.int32), np.array([0, -1], np.int32), "out of range"),
])
def test_invalid_csr_rejected_on_host(gr, row_off, col, what):
    st, out = _create(gr, row_off, col)
    assert st == gr.GR_EINVAL
    assert what in gr.gr_last_error()
    assert not out.value


def test_invalid_sizes_rejected(gr):
    out = ctypes.c_void_p()
    r = np.zeros(1, np.int32)
    assert gr._lib.gr_graph_create(0, 0, r.ctypes.data, None, None, 0, None,
                                   ctypes.byref(out)) == gr.GR_EINVAL
    assert gr._lib.gr_graph_create(1, 2**31, r.ctypes.data, None, None, 0, None,
                                   ctypes.byref(out)) == gr.GR_EINVAL
    assert gr._lib.gr_graph_create(1, -1, r.ctypes.data, None, None, 0, None,
                                   ctypes.byref(out)) == gr.GR_EINVAL
    assert gr._lib.gr_graph_create(1, 0, None, None, None, 0, None,
                                   ctypes.byref(out)) == gr.GR_EINVAL


def test_null_graph_rejected(gr):
    d = np.zeros(4, np.int32)
    assert gr._lib.gr_bfs(None, 0, d.ctypes.data, None, None, None) == gr.GR_EINVAL
    assert "NULL" in gr.gr_last_error()
    assert gr._lib.gr_graph_destroy(None) == gr.GR_OK


def test_server_rejects_bad_arguments(gr):
    out = ctypes.c_void_p()
    for budget, slots, batch in [(0, 1, 1), (1 << 20, 0, 1), (1 << 20, 65, 1),
                                 (1 << 20, 2, 1), (1 << 20, 4, 64),
                                 (1 << 20, 1, 0), (1 << 20, 1, 65)]:
        assert gr._lib.gr_server_create(budget, slots, batch, ctypes.byref(out)) == gr.GR_EINVAL
        if slots in (2, 4):
            assert "num_slots must be 1" in gr.gr_last_error()
    assert gr._lib.gr_server_destroy(None) == gr.GR_OK


def test_batch_and_bc_reject_bad_arguments(gr):
    srcs = np.zeros(65, np.int32)
    d = np.zeros(4, np.int32)
    assert gr._lib.gr_bfs_batch(None, srcs.ctypes.data, 1, d.ctypes.data, None, None) == gr.GR_EINVAL
    assert gr._lib.gr_bc(None, srcs.ctypes.data, 1, d.ctypes.data, None, None) == gr.GR_EINVAL
    assert gr._lib.gr_sssp_batch(None, srcs.ctypes.data, 1, d.ctypes.data, None, None) == gr.GR_EINVAL
    assert gr._lib.gr_bfs_noalloc(0, 0, None, None, 0, None, None, None) == gr.GR_EINVAL
