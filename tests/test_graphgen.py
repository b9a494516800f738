"""The seeded input generator: determinism, CSR well-formedness, R-MAT shape,
grid structure, weights and source selection."""
import hashlib
import os

import numpy as np
import pytest

import graphgen as gg

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _csr_ok(row_off, col, n):
    assert row_off.shape == (n + 1,) and row_off[0] == 0 and row_off[-1] == col.size
    assert np.all(np.diff(row_off) >= 0)
    assert np.all((col >= 0) & (col < n))
    src = np.repeat(np.arange(n), np.diff(row_off))
    assert not np.any(src == col), "self-loop"
    # rows strictly ascending (sorted + deduplicated)
    same_row = src[1:] == src[:-1]
    assert np.all(col[1:][same_row] > col[:-1][same_row])
    # symmetric: the set of (u,v) keys equals the set of (v,u) keys
    k1 = np.sort(src.astype(np.int64) * n + col)
    k2 = np.sort(col.astype(np.int64) * n + src)
    assert np.array_equal(k1, k2)


def test_rmat_s10_wellformed_and_deterministic():
    r1, c1 = gg.rmat(10, 16, seed=7)
    r2, c2 = gg.rmat(10, 16, seed=7)
    assert np.array_equal(r1, r2) and np.array_equal(c1, c2)
    _csr_ok(r1, c1, 1024)
    r3, _ = gg.rmat(10, 16, seed=8)
    assert not np.array_equal(r1, r3)


def test_rmat_thread_count_independent(monkeypatch):
    # output depends only on (seed, stream, index), not on the schedule
    r1, c1 = gg.rmat(16, 8, seed=3)
    import subprocess, sys, json
    code = ("import graphgen as gg, hashlib;r,c=gg.rmat(16,8,seed=3);"
            "print(hashlib.sha256(r.tobytes()+c.tobytes()).hexdigest())")
    env = dict(os.environ, GG_THREADS="1",
               PYTHONPATH=os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    out = subprocess.check_output([sys.executable, "-c", code], env=env, text=True).strip()
    assert out == hashlib.sha256(r1.tobytes() + c1.tobytes()).hexdigest()


def test_rmat_skew_hubs_at_low_ids():
    # with a > b = c > d and no permutation, vertex 0 is the quadrant-(0,0)
    # attractor: it gets the largest expected degree
    r, c = gg.rmat(14, 16, seed=1)
    deg = np.diff(r)
    assert gg.max_degree_vertex(r) == int(np.argmax(deg))
    assert int(np.argmax(deg)) < 16
    assert deg.max() > 50 * deg[deg > 0].mean()
    # edge count before dedupe is n * edge_factor; after symmetrising at most 2x
    assert c.size <= 2 * 16 * (1 << 14)


def test_rmat_permutation_is_a_relabeling():
    r0, c0 = gg.rmat(12, 8, seed=5)
    r1, c1 = gg.rmat(12, 8, seed=5, permute=True)
    assert c0.size == c1.size
    assert np.array_equal(np.sort(np.diff(r0)), np.sort(np.diff(r1)))
    _csr_ok(r1, c1, 1 << 12)


def test_rmat_s14_golden_hash():
    r, c = gg.rmat(14, 16, seed=1)
    h = hashlib.sha256(r.tobytes() + c.tobytes()).hexdigest()
    with open(os.path.join(GOLDEN, "rmat_s14_seed1.txt")) as f:
        rec = dict(line.split("=", 1) for line in f.read().split() if "=" in line)
    assert int(rec["m"]) == c.size
    assert rec["sha256"] == h


def test_grid_full_and_deleted():
    side = 37
    r, c = gg.grid(side, p_del=0.0, seed=4)
    n = side * side
    _csr_ok(r, c, n)
    assert c.size == 2 * 2 * side * (side - 1)
    rr, cc = np.divmod(np.arange(n), side)
    src = np.repeat(np.arange(n), np.diff(r))
    # neighbours are exactly the 4-neighbourhood
    assert np.all(np.abs(rr[src] - rr[c]) + np.abs(cc[src] - cc[c]) == 1)
    r2, c2 = gg.grid(side, p_del=0.05, seed=4)
    _csr_ok(r2, c2, n)
    kept = c2.size // 2
    total = 2 * side * (side - 1)
    # Bernoulli(0.05) deletions: within 6 sigma of the mean
    sd = np.sqrt(total * 0.05 * 0.95)
    assert abs((total - kept) - 0.05 * total) < 6 * sd


def test_weights_symmetric_and_in_range():
    r, c = gg.rmat(12, 16, seed=2)
    w = gg.weights(r, c, seed=3, wmin=1, wmax=64)
    assert w.min() >= 1 and w.max() <= 64
    assert np.unique(w).size == 64
    n = r.size - 1
    src = np.repeat(np.arange(n), np.diff(r))
    k = src.astype(np.int64) * n + c
    kt = c.astype(np.int64) * n + src
    order = np.argsort(kt)
    # weight of (u,v) equals weight of (v,u)
    assert np.array_equal(w[np.argsort(k)], w[order])


def test_sources_distinct_nonisolated():
    r, c = gg.rmat(14, 16, seed=2)
    s = gg.sources(r, 16, seed=2)
    assert s.size == 16 and np.unique(s).size == 16
    assert np.all(np.diff(r)[s] > 0)
    assert np.array_equal(s, gg.sources(r, 16, seed=2))


@pytest.mark.parametrize("sl,sr,ef", [(8, 8, 8), (10, 6, 4), (5, 9, 16)])
def test_rmat_bipartite_shape(sl, sr, ef):
    r, c, nl = gg.rmat_bipartite(sl, sr, ef, seed=7)
    n = r.size - 1
    assert nl == 1 << sl and n == (1 << sl) + (1 << sr)
    rows = np.repeat(np.arange(n), np.diff(r))
    assert np.all((rows < nl) != (c < nl))  # every entry joins a hub and an authority
    keys = set(zip(rows.tolist(), c.tolist()))
    assert all((v, u) in keys for u, v in keys)  # both directions stored
    for v in range(0, n, max(1, n // 50)):
        row = c[r[v]:r[v + 1]]
        assert np.all(np.diff(row) > 0)  # sorted, no duplicates
    assert c.size // 2 <= ef * max(1 << sl, 1 << sr)
    r2, c2, _ = gg.rmat_bipartite(sl, sr, ef, seed=7)
    assert np.array_equal(r, r2) and np.array_equal(c, c2)
    r3, c3, _ = gg.rmat_bipartite(sl, sr, ef, seed=8)
    assert not np.array_equal(c, c3)
    # R-MAT skew: the lowest ids carry the most links on each side
    deg = np.diff(r)
    assert deg[:nl][: nl // 8].mean() > deg[:nl].mean()
