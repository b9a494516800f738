"""Result validators shared by the oracle pins and the GPU parity tests.

A BFS parent array is not unique (any discoverer one level up is valid), so
parents are validated rather than compared, with the checks of the Graph500
BFS validation rules restated here; depth is unique and is compared exactly.
"""
from __future__ import annotations

import numpy as np


def edge_keys(row_off: np.ndarray, col: np.ndarray) -> np.ndarray:
    """Sorted int64 keys u*n+v of every CSR entry (rows sorted ascending)."""
    n = row_off.shape[0] - 1
    src = np.repeat(np.arange(n, dtype=np.int64), np.diff(row_off).astype(np.int64))
    keys = src * n + col.astype(np.int64)
    if keys.size > 1 and not np.all(keys[1:] >= keys[:-1]):
        keys = np.sort(keys)
    return keys


def has_edges(keys: np.ndarray, n: int, u: np.ndarray, v: np.ndarray) -> np.ndarray:
    q = u.astype(np.int64) * n + v.astype(np.int64)
    if keys.size == 0:
        return np.zeros(q.shape, dtype=bool)
    pos = np.minimum(np.searchsorted(keys, q), keys.size - 1)
    return keys[pos] == q


def edge_sources(row_off: np.ndarray) -> np.ndarray:
    n = row_off.shape[0] - 1
    return np.repeat(np.arange(n, dtype=np.int32), np.diff(row_off))


def validate_bfs(row_off, col, src, depth, parent, symmetric=True, keys=None, su=None):
    """Raise AssertionError unless (depth, parent) is a valid BFS tree.
    keys / su: precomputed edge_keys / edge_sources for large graphs."""
    n = row_off.shape[0] - 1
    depth = np.asarray(depth)
    parent = np.asarray(parent)
    assert depth[src] == 0, "depth[src] != 0"
    assert parent[src] == src, "parent[src] != src"
    reached = depth >= 0
    assert np.all(depth >= -1)
    assert np.all(parent[~reached] == -1), "unreached vertex with a parent"
    vs = np.nonzero(reached)[0]
    vs = vs[vs != src]
    p = parent[vs]
    assert np.all((p >= 0) & (p < n)), "parent out of range"
    assert np.all(depth[p] == depth[vs] - 1), "depth[parent] != depth - 1"
    if keys is None:
        keys = edge_keys(row_off, col)
    if vs.size:
        assert np.all(has_edges(keys, n, p, vs)), "(parent, v) is not an edge"
    # every edge spans at most one level and never leaves the reached set
    if su is None:
        su = edge_sources(row_off)
    du = depth[su]
    dv = depth[col]
    both = (du >= 0) & (dv >= 0)
    # an arc (u, v) from a reached u reaches v at most one level later
    assert np.all(dv[both] <= du[both] + 1), "arc spans > 1 level forward"
    assert np.all(~(du >= 0) | (dv >= 0)), "arc from reached to unreached"
    if symmetric:
        assert np.all(np.abs(du[both] - dv[both]) <= 1), "edge spans > 1 level"
        assert np.all((du >= 0) == (dv >= 0)), "reachability differs across an edge"


def validate_sssp_pred(row_off, col, w, src, dist, pred, keys=None):
    """pred[v] must sit on a shortest-path edge into v (dist[u]+w == dist[v])."""
    n = row_off.shape[0] - 1
    INF = np.uint32(0xFFFFFFFF)
    assert dist[src] == 0 and pred[src] == src
    reached = dist != INF
    assert np.all(pred[~reached] == -1)
    vs = np.nonzero(reached)[0]
    vs = vs[vs != src]
    p = pred[vs]
    assert np.all((p >= 0) & (p < n))
    if keys is None:
        keys = edge_keys(row_off, col)
    q = p.astype(np.int64) * n + vs.astype(np.int64)
    pos = np.searchsorted(keys, q)
    assert np.all(keys[np.minimum(pos, keys.size - 1)] == q), "(pred, v) is not an edge"
    # the weight of that edge: keys are in CSR order when rows are sorted
    we = w[pos].astype(np.int64)
    assert np.all(dist[p].astype(np.int64) + we == dist[vs].astype(np.int64))


def manhattan(side: int, src: int) -> np.ndarray:
    r0, c0 = divmod(src, side)
    r, c = np.divmod(np.arange(side * side), side)
    return (np.abs(r - r0) + np.abs(c - c0)).astype(np.int32)


def floyd_warshall(n: int, row_off, col, w=None) -> np.ndarray:
    """All-pairs shortest distances by brute force (np.inf if unreachable)."""
    d = np.full((n, n), np.inf)
    np.fill_diagonal(d, 0.0)
    for u in range(n):
        for e in range(row_off[u], row_off[u + 1]):
            v = col[e]
            wt = 1.0 if w is None else float(w[e])
            if u != v:
                d[u, v] = min(d[u, v], wt)
    for k in range(n):
        d = np.minimum(d, d[:, k:k + 1] + d[k:k + 1, :])
    return d


def brute_force_bc(n: int, row_off, col, srcs) -> np.ndarray:
    """BC by enumerating every shortest path explicitly (small graphs only):
    sum over s in srcs and t != s of (#shortest s-t paths through v) /
    (#shortest s-t paths), for v not in {s, t}."""
    d = floyd_warshall(n, row_off, col)
    adj = [list(col[row_off[u]:row_off[u + 1]]) for u in range(n)]
    bc = np.zeros(n)
    for s in srcs:
        for t in range(n):
            if t == s or not np.isfinite(d[s, t]):
                continue
            paths = []

            def walk(path):
                u = path[-1]
                if u == t:
                    paths.append(list(path))
                    return
                for v in adj[u]:
                    if d[s, v] == d[s, u] + 1 and d[v, t] == d[u, t] - 1:
                        path.append(v)
                        walk(path)
                        path.pop()
            walk([s])
            cnt = np.zeros(n)
            for p in paths:
                for v in p[1:-1]:
                    cnt[v] += 1
            bc += cnt / len(paths)
    return bc


def relative_l1(a, b) -> float:
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.abs(a - b).sum() / np.abs(b).sum())
