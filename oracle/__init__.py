"""CPU oracle (test infrastructure only).

Plain single-threaded C implementations of the definitions the paper's
primitives compute (Sec. 5): queue BFS, Dijkstra SSSP, Brandes BC, union-find
CC and FP64 power-iteration PageRank; and of the operations the paper points
to beyond them: the neighbourhood reduction (Sec. 7) and the bipartite
node rankings HITS, SALSA and personalized PageRank (Sec. 5.5). Only ``tests/``, the smoke check in
``__graft_entry__`` and the CPU-baseline leg of ``bench.py`` may import this
package. It shares no code with the CUDA library and never imports it.

The C source is ``oracle.c``; ``build()`` compiles it with gcc.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

INF_DIST = 0xFFFFFFFF


def build(force: bool = False) -> str:
    """Compile liboracle.so with gcc (no-op when up to date)."""
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", _SRC,
                           "-o", tmp])
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB)
            i32, dbl, vp = ctypes.c_int32, ctypes.c_double, ctypes.c_void_p
            lib.or_bfs.restype = ctypes.c_int
            lib.or_bfs.argtypes = [i32, vp, vp, i32, vp, vp]
            lib.or_sssp.restype = ctypes.c_int
            lib.or_sssp.argtypes = [i32, vp, vp, vp, i32, vp, vp]
            lib.or_bc.restype = ctypes.c_int
            lib.or_bc.argtypes = [i32, vp, vp, vp, i32, vp]
            lib.or_cc.restype = ctypes.c_int
            lib.or_cc.argtypes = [i32, vp, vp, vp, vp]
            lib.or_pagerank.restype = ctypes.c_int
            lib.or_pagerank.argtypes = [i32, vp, vp, dbl, i32, dbl, vp, vp]
            lib.or_neighbor_reduce.restype = ctypes.c_int
            lib.or_neighbor_reduce.argtypes = [i32, vp, vp, vp, i32, vp, i32, vp, vp]
            for name in ("or_hits", "or_salsa"):
                f = getattr(lib, name)
                f.restype = ctypes.c_int
                f.argtypes = [i32, i32, vp, vp, i32, dbl, vp, vp]
            lib.or_ppr.restype = ctypes.c_int
            lib.or_ppr.argtypes = [i32, vp, vp, vp, i32, dbl, i32, dbl, vp, vp]
            _lib = lib
    return _lib


def _csr(row_off, col):
    row_off = np.ascontiguousarray(row_off, dtype=np.int32)
    col = np.ascontiguousarray(col, dtype=np.int32)
    return row_off, col, row_off.shape[0] - 1


def _check(rc, what):
    if rc != 0:
        raise RuntimeError(f"oracle {what} failed with code {rc}")


def bfs(row_off, col, src: int):
    """Queue BFS -> (depth int32[n], parent int32[n])."""
    row_off, col, n = _csr(row_off, col)
    depth = np.empty(n, dtype=np.int32)
    parent = np.empty(n, dtype=np.int32)
    _check(_load().or_bfs(n, row_off.ctypes.data, col.ctypes.data, src,
                          depth.ctypes.data, parent.ctypes.data), "bfs")
    return depth, parent


def sssp(row_off, col, w, src: int):
    """Dijkstra -> (dist uint32[n], pred int32[n])."""
    row_off, col, n = _csr(row_off, col)
    w = np.ascontiguousarray(w, dtype=np.uint32)
    dist = np.empty(n, dtype=np.uint32)
    pred = np.empty(n, dtype=np.int32)
    _check(_load().or_sssp(n, row_off.ctypes.data, col.ctypes.data, w.ctypes.data,
                           src, dist.ctypes.data, pred.ctypes.data), "sssp")
    return dist, pred


def bc(row_off, col, srcs):
    """Brandes BC summed over srcs (no halving, no normalisation) -> f64[n]."""
    row_off, col, n = _csr(row_off, col)
    srcs = np.ascontiguousarray(srcs, dtype=np.int32)
    out = np.empty(n, dtype=np.float64)
    _check(_load().or_bc(n, row_off.ctypes.data, col.ctypes.data, srcs.ctypes.data,
                         srcs.shape[0], out.ctypes.data), "bc")
    return out


def cc(row_off, col):
    """Union-find CC -> (label int32[n] = min vertex id, num_components)."""
    row_off, col, n = _csr(row_off, col)
    label = np.empty(n, dtype=np.int32)
    k = ctypes.c_int32()
    _check(_load().or_cc(n, row_off.ctypes.data, col.ctypes.data, label.ctypes.data,
                         ctypes.byref(k)), "cc")
    return label, k.value


def pagerank(row_off, col, damping: float = 0.85, max_iter: int = 50,
             tol: float = 1e-7):
    """FP64 power iteration -> (rank f64[n], iterations run)."""
    row_off, col, n = _csr(row_off, col)
    rank = np.empty(n, dtype=np.float64)
    it = ctypes.c_int32()
    _check(_load().or_pagerank(n, row_off.ctypes.data, col.ctypes.data, damping,
                               max_iter, tol, rank.ctypes.data, ctypes.byref(it)),
           "pagerank")
    return rank, it.value


REDUCE_SUM, REDUCE_WSUM, REDUCE_MIN, REDUCE_MAX = 0, 1, 2, 3


def neighbor_reduce(row_off, col, op: int, x, w=None, frontier=None):
    """out[v] = sum / weighted sum / min / max of x[u] over the entries
    (v, u) of v's row, for v in frontier (default: every vertex); other
    entries of out are left at 0 (sums) or the identity (min/max)."""
    row_off, col, n = _csr(row_off, col)
    is_sum = op in (REDUCE_SUM, REDUCE_WSUM)
    x = np.ascontiguousarray(x, dtype=np.float64 if is_sum else np.int32)
    if is_sum:
        out = np.zeros(n, dtype=np.float64)
    else:
        out = np.full(n, np.iinfo(np.int32).max if op == REDUCE_MIN else np.iinfo(np.int32).min,
                      dtype=np.int32)
    wp = None
    if w is not None:
        w = np.ascontiguousarray(w, dtype=np.uint32)
        wp = w.ctypes.data
    fp, q = None, 0
    if frontier is not None:
        frontier = np.ascontiguousarray(frontier, dtype=np.int32)
        fp, q = frontier.ctypes.data, frontier.shape[0]
    _check(_load().or_neighbor_reduce(n, row_off.ctypes.data, col.ctypes.data, wp, op, fp, q,
                                      x.ctypes.data, out.ctypes.data), "neighbor_reduce")
    return out


def hits(row_off, col, n_left: int, max_iter: int = 100, tol: float = 1e-10):
    """HITS on a bipartite graph -> (score f64[n]: hub scores on [0, n_left),
    authority scores on [n_left, n), iterations run)."""
    row_off, col, n = _csr(row_off, col)
    out = np.empty(n, dtype=np.float64)
    it = ctypes.c_int32()
    _check(_load().or_hits(n, n_left, row_off.ctypes.data, col.ctypes.data, max_iter, tol,
                           out.ctypes.data, ctypes.byref(it)), "hits")
    return out, it.value


def salsa(row_off, col, n_left: int, max_iter: int = 100, tol: float = 1e-10):
    """SALSA on a bipartite graph -> (score f64[n], iterations run)."""
    row_off, col, n = _csr(row_off, col)
    out = np.empty(n, dtype=np.float64)
    it = ctypes.c_int32()
    _check(_load().or_salsa(n, n_left, row_off.ctypes.data, col.ctypes.data, max_iter, tol,
                            out.ctypes.data, ctypes.byref(it)), "salsa")
    return out, it.value


def ppr(row_off, col, seeds, damping: float = 0.85, max_iter: int = 50, tol: float = 1e-7):
    """Personalized PageRank from distinct seed vertices -> (rank f64[n],
    iterations run)."""
    row_off, col, n = _csr(row_off, col)
    seeds = np.ascontiguousarray(seeds, dtype=np.int32)
    out = np.empty(n, dtype=np.float64)
    it = ctypes.c_int32()
    _check(_load().or_ppr(n, row_off.ctypes.data, col.ctypes.data, seeds.ctypes.data,
                          seeds.shape[0], damping, max_iter, tol, out.ctypes.data,
                          ctypes.byref(it)), "ppr")
    return out, it.value
