"""Seeded synthetic graph inputs (R-MAT, 2D grid, weights, sources).

This module generates inputs only: it contains none of the traversal
arithmetic. Both the CPU oracle (``oracle/``) and the CUDA library read the
CSR arrays it returns. The native code is ``graphgen.cpp``; this file builds
it on first use (g++) and wraps it with ctypes.

Workload shapes follow the paper's evaluation (Sec. 6, Table 1): R-MAT
stands in for the generated scale-free kron_g500-logn21 graph and the 2D grid
with random deletions for the large-diameter mesh graphs (rgg_n_24,
roadnet_CA). Graphs are symmetrised as the paper does for all its datasets;
edge weights are uniform integers, the paper using [1, 64] (Sec. 6).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "graphgen.cpp")
_LIB = os.path.join(_HERE, "libgraphgen.so")
_lock = threading.Lock()
_lib = None

RMAT_ABC = (0.57, 0.19, 0.19)


def build(force: bool = False) -> str:
    """Compile libgraphgen.so next to its source (no-op when up to date)."""
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    subprocess.check_call(["g++", "-O3", "-std=c++17", "-shared", "-fPIC",
                           "-pthread", _SRC, "-o", tmp])
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB)
            P = ctypes.POINTER
            i32, i64, u64, dbl = ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64, ctypes.c_double
            lib.gg_hash3.restype = u64
            lib.gg_hash3.argtypes = [u64, u64, u64]
            lib.gg_rmat_build.restype = ctypes.c_void_p
            lib.gg_rmat_build.argtypes = [i32, i32, dbl, dbl, dbl, u64, i32,
                                          P(i32), P(i64), P(i64)]
            lib.gg_rmat_bipartite_build.restype = ctypes.c_void_p
            lib.gg_rmat_bipartite_build.argtypes = [i32, i32, i32, dbl, dbl, dbl, u64,
                                                    P(i32), P(i32), P(i64)]
            lib.gg_grid_build.restype = ctypes.c_void_p
            lib.gg_grid_build.argtypes = [i32, dbl, u64, P(i32), P(i64), P(i64)]
            lib.gg_csr_copy.restype = None
            lib.gg_csr_copy.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
            lib.gg_csr_free.restype = None
            lib.gg_csr_free.argtypes = [ctypes.c_void_p]
            lib.gg_weights.restype = None
            lib.gg_weights.argtypes = [ctypes.c_void_p, ctypes.c_void_p, i32, u64,
                                       ctypes.c_uint32, ctypes.c_uint32, ctypes.c_void_p]
            lib.gg_sources.restype = i32
            lib.gg_sources.argtypes = [ctypes.c_void_p, i32, i32, u64, ctypes.c_void_p]
            lib.gg_max_degree_vertex.restype = i32
            lib.gg_max_degree_vertex.argtypes = [ctypes.c_void_p, i32]
            _lib = lib
    return _lib


def _ptr(a: np.ndarray) -> int:
    return a.ctypes.data


def hash3(seed: int, stream: int, idx: int) -> int:
    """The counter-based generator every draw of this module uses."""
    return int(_load().gg_hash3(seed, stream, idx))


def _take(h, n: int, m: int):
    lib = _load()
    row_off = np.empty(n + 1, dtype=np.int32)
    col = np.empty(m, dtype=np.int32)
    lib.gg_csr_copy(h, _ptr(row_off), _ptr(col))
    lib.gg_csr_free(h)
    return row_off, col


def rmat(scale: int, edge_factor: int = 16, seed: int = 1, abc=RMAT_ABC,
         permute: bool = False):
    """R-MAT graph with 2**scale vertices and edge_factor * 2**scale raw
    edges, symmetrised, self-loops dropped, per-row sorted and deduplicated.

    Returns (row_off int32[n+1], col int32[m]).
    """
    lib = _load()
    n = ctypes.c_int32()
    m = ctypes.c_int64()
    raw = ctypes.c_int64()
    a, b, c = abc
    h = lib.gg_rmat_build(scale, edge_factor, a, b, c, seed, int(permute),
                          ctypes.byref(n), ctypes.byref(m), ctypes.byref(raw))
    if not h:
        raise ValueError("R-MAT build failed (bad scale or m > INT32_MAX)")
    return _take(h, n.value, m.value)


def rmat_bipartite(scale_left: int, scale_right: int, edge_factor: int = 16, seed: int = 1,
                   abc=RMAT_ABC):
    """Bipartite R-MAT: 2**scale_left hubs (ids [0, n_left)) and
    2**scale_right authorities (ids [n_left, n)), edge_factor * max(sides)
    raw edges, each joining a hub and an authority, stored in both
    directions (sorted, deduplicated). Returns (row_off, col, n_left)."""
    lib = _load()
    n = ctypes.c_int32()
    nl = ctypes.c_int32()
    m = ctypes.c_int64()
    a, b, c = abc
    h = lib.gg_rmat_bipartite_build(scale_left, scale_right, edge_factor, a, b, c, seed,
                                    ctypes.byref(n), ctypes.byref(nl), ctypes.byref(m))
    if not h:
        raise ValueError("bipartite R-MAT build failed (bad scales or m > INT32_MAX)")
    r, col = _take(h, n.value, m.value)
    return r, col, nl.value


def grid(side: int, p_del: float = 0.05, seed: int = 4):
    """side x side 4-neighbour grid, each undirected edge deleted with
    probability p_del. Returns (row_off, col)."""
    lib = _load()
    n = ctypes.c_int32()
    m = ctypes.c_int64()
    kept = ctypes.c_int64()
    h = lib.gg_grid_build(side, p_del, seed, ctypes.byref(n), ctypes.byref(m),
                          ctypes.byref(kept))
    if not h:
        raise ValueError("grid build failed")
    return _take(h, n.value, m.value)


def weights(row_off: np.ndarray, col: np.ndarray, seed: int, wmin: int = 1,
            wmax: int = 64) -> np.ndarray:
    """uint32 weight per CSR entry, uniform in [wmin, wmax], equal for both
    directions of an undirected edge."""
    row_off = np.ascontiguousarray(row_off, dtype=np.int32)
    col = np.ascontiguousarray(col, dtype=np.int32)
    w = np.empty(col.shape[0], dtype=np.uint32)
    _load().gg_weights(_ptr(row_off), _ptr(col), row_off.shape[0] - 1, seed,
                       wmin, wmax, _ptr(w))
    return w


def sources(row_off: np.ndarray, count: int, seed: int) -> np.ndarray:
    """`count` distinct random vertices of non-zero degree."""
    row_off = np.ascontiguousarray(row_off, dtype=np.int32)
    out = np.empty(count, dtype=np.int32)
    got = _load().gg_sources(_ptr(row_off), row_off.shape[0] - 1, count, seed, _ptr(out))
    return out[:got]


def max_degree_vertex(row_off: np.ndarray) -> int:
    """Highest-degree vertex, ties broken toward the smallest id."""
    row_off = np.ascontiguousarray(row_off, dtype=np.int32)
    return int(_load().gg_max_degree_vertex(_ptr(row_off), row_off.shape[0] - 1))


def from_edges(n: int, edges, symmetric: bool = True):
    """Small helper for tests: CSR (sorted, deduplicated, no self-loops) from
    an explicit edge list."""
    rows = [set() for _ in range(n)]
    for u, v in edges:
        if u == v:
            continue
        rows[u].add(v)
        if symmetric:
            rows[v].add(u)
    row_off = np.zeros(n + 1, dtype=np.int32)
    for i in range(n):
        row_off[i + 1] = row_off[i] + len(rows[i])
    col = np.array([v for i in range(n) for v in sorted(rows[i])], dtype=np.int32)
    return row_off, col
