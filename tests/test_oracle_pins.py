"""Pins for the CPU oracle against facts fixed outside it: closed forms,
brute force on tiny graphs, invariants, exact fixed points and independent
library routines (networkx, scipy). Each primitive is pinned so that a
dropped term, a wrong sign or index, or a transposed operand fails a test.
"""
import itertools

import numpy as np
import pytest

import graphgen as gg
import oracle
from checks import (brute_force_bc, floyd_warshall, manhattan, relative_l1,
                    validate_bfs, validate_sssp_pred)


def path_graph(n):
    return gg.from_edges(n, [(i, i + 1) for i in range(n - 1)])


def cycle_graph(n):
    return gg.from_edges(n, [(i, (i + 1) % n) for i in range(n)])


def star_graph(n):
    return gg.from_edges(n, [(0, i) for i in range(1, n)])


def complete_graph(n):
    return gg.from_edges(n, [(i, j) for i in range(n) for j in range(i + 1, n)])


def hypercube(d):
    n = 1 << d
    return gg.from_edges(n, [(v, v ^ (1 << b)) for v in range(n) for b in range(d)])


def torus(side):
    e = []
    for r in range(side):
        for c in range(side):
            v = r * side + c
            e.append((v, r * side + (c + 1) % side))
            e.append((v, ((r + 1) % side) * side + c))
    return gg.from_edges(side * side, e)


def random_graph(n, p, seed):
    rng = np.random.default_rng(seed)
    e = [(i, j) for i in range(n) for j in range(i + 1, n) if rng.random() < p]
    return gg.from_edges(n, e)


# ------------------------------------------------------------------ BFS
@pytest.mark.parametrize("src", [0, 5, 40 * 40 - 1, 20 * 40 + 17])
def test_bfs_full_grid_is_manhattan(src):
    side = 40
    r, c = gg.grid(side, p_del=0.0)
    depth, parent = oracle.bfs(r, c, src)
    assert np.array_equal(depth, manhattan(side, src))
    validate_bfs(r, c, src, depth, parent)


def test_bfs_deleted_grid_bounds():
    side = 64
    r, c = gg.grid(side, p_del=0.05, seed=4)
    src = 0
    depth, parent = oracle.bfs(r, c, src)
    md = manhattan(side, src)
    reached = depth >= 0
    assert np.all(depth[reached] >= md[reached])
    # the grid is bipartite: every path length has the parity of Manhattan
    assert np.all((depth[reached] - md[reached]) % 2 == 0)
    validate_bfs(r, c, src, depth, parent)


def test_bfs_closed_forms():
    n = 9
    r, c = path_graph(n)
    d, _ = oracle.bfs(r, c, 3)
    assert list(d) == [abs(i - 3) for i in range(n)]
    r, c = cycle_graph(n)
    d, _ = oracle.bfs(r, c, 0)
    assert list(d) == [min(i, n - i) for i in range(n)]
    r, c = star_graph(n)
    d, p = oracle.bfs(r, c, 4)
    assert list(d) == [1] + [0 if i == 4 else 2 for i in range(1, n)]
    assert p[0] == 4 and all(p[i] == 0 for i in range(1, n) if i != 4)
    r, c = complete_graph(6)
    d, p = oracle.bfs(r, c, 2)
    assert list(d) == [1, 1, 0, 1, 1, 1] and all(p[i] == 2 for i in range(6))


def test_bfs_isolated_and_disconnected():
    r, c = gg.from_edges(6, [(0, 1), (1, 2), (4, 5)])
    d, p = oracle.bfs(r, c, 3)
    assert list(d) == [-1, -1, -1, 0, -1, -1] and list(p) == [-1, -1, -1, 3, -1, -1]
    d, p = oracle.bfs(r, c, 5)
    assert list(d) == [-1, -1, -1, -1, 1, 0]


def test_bfs_directed_input():
    # directed 0->1->2, 2->0 absent in reverse: depth follows arc direction
    r = np.array([0, 1, 2, 2], np.int32)
    c = np.array([1, 2], np.int32)
    d, p = oracle.bfs(r, c, 1)
    assert list(d) == [-1, 0, 1] and list(p) == [-1, 1, 1]


def all_graphs(n):
    pairs = list(itertools.combinations(range(n), 2))
    for mask in range(1 << len(pairs)):
        yield gg.from_edges(n, [pairs[i] for i in range(len(pairs)) if mask >> i & 1])


def test_bfs_exhaustive_small_graphs():
    for n in range(1, 6):
        for r, c in all_graphs(n):
            fw = floyd_warshall(n, r, c)
            for s in range(n):
                d, p = oracle.bfs(r, c, s)
                exp = np.where(np.isfinite(fw[s]), fw[s], -1).astype(np.int32)
                assert np.array_equal(d, exp)
                validate_bfs(r, c, s, d, p)


@pytest.mark.parametrize("seed", range(20))
def test_bfs_random_vs_floyd_warshall(seed):
    n = 12
    r, c = random_graph(n, 0.25, seed)
    fw = floyd_warshall(n, r, c)
    for s in range(n):
        d, p = oracle.bfs(r, c, s)
        assert np.array_equal(d, np.where(np.isfinite(fw[s]), fw[s], -1))
        validate_bfs(r, c, s, d, p)


def test_bfs_rmat_vs_networkx():
    nx = pytest.importorskip("networkx")
    r, c = gg.rmat(12, 16, seed=11)
    n = r.size - 1
    G = nx.Graph()
    G.add_nodes_from(range(n))
    src = np.repeat(np.arange(n), np.diff(r))
    G.add_edges_from(zip(src.tolist(), c.tolist()))
    s = gg.max_degree_vertex(r)
    d, p = oracle.bfs(r, c, s)
    ref = nx.single_source_shortest_path_length(G, s)
    exp = np.full(n, -1)
    for v, dv in ref.items():
        exp[v] = dv
    assert np.array_equal(d, exp)
    validate_bfs(r, c, s, d, p)


def test_bfs_s14_golden_levels():
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "rmat_s14_seed1.txt")
    rec = dict(l.split("=", 1) for l in open(path).read().split() if "=" in l)
    r, c = gg.rmat(14, 16, seed=1)
    d, _ = oracle.bfs(r, c, int(rec["src"]))
    levels = [int(x) for x in rec["bfs_levels"].split(",")]
    assert list(np.bincount(d[d >= 0])) == levels


# ----------------------------------------------------------------- SSSP
def test_sssp_unit_weights_on_grid_is_manhattan():
    side = 30
    r, c = gg.grid(side, p_del=0.0)
    w = np.ones(c.size, np.uint32)
    dist, pred = oracle.sssp(r, c, w, 7)
    assert np.array_equal(dist.astype(np.int64), manhattan(side, 7))
    validate_sssp_pred(r, c, w, 7, dist, pred)


def test_sssp_path_prefix_sums():
    n = 10
    r, c = path_graph(n)
    # weight of edge {i, i+1} = i + 1, both directions
    src = np.repeat(np.arange(n), np.diff(r))
    w = (np.minimum(src, c) + 1).astype(np.uint32)
    dist, pred = oracle.sssp(r, c, w, 0)
    assert list(dist) == [i * (i + 1) // 2 for i in range(n)]
    assert list(pred) == [0] + list(range(n - 1))


def test_sssp_prefers_lighter_longer_path():
    # 0-1 weight 10; 0-2-1 weights 3+4: dist(1) = 7 via 2
    r, c = gg.from_edges(3, [(0, 1), (0, 2), (1, 2)])
    src = np.repeat(np.arange(3), np.diff(r))
    wt = {frozenset((0, 1)): 10, frozenset((0, 2)): 3, frozenset((1, 2)): 4}
    w = np.array([wt[frozenset((int(a), int(b)))] for a, b in zip(src, c)], np.uint32)
    dist, pred = oracle.sssp(r, c, w, 0)
    assert list(dist) == [0, 7, 3] and list(pred) == [0, 2, 0]


@pytest.mark.parametrize("seed", range(15))
def test_sssp_random_vs_floyd_warshall(seed):
    n = 12
    r, c = random_graph(n, 0.3, seed)
    w = gg.weights(r, c, seed=seed, wmin=1, wmax=9)
    fw = floyd_warshall(n, r, c, w)
    for s in range(n):
        dist, pred = oracle.sssp(r, c, w, s)
        exp = np.where(np.isfinite(fw[s]), fw[s], 0xFFFFFFFF).astype(np.uint32)
        assert np.array_equal(dist, exp)
        validate_sssp_pred(r, c, w, s, dist, pred)
        # pred is the smallest shortest-path in-neighbour
        for v in range(n):
            if v == s or dist[v] == 0xFFFFFFFF:
                continue
            cands = [u for u in range(n) for e in range(r[u], r[u + 1])
                     if c[e] == v and fw[s, u] + w[e] == fw[s, v]]
            assert pred[v] == min(cands)


def test_sssp_rmat_vs_scipy_dijkstra():
    sp = pytest.importorskip("scipy.sparse")
    csgraph = pytest.importorskip("scipy.sparse.csgraph")
    r, c = gg.rmat(13, 16, seed=9)
    w = gg.weights(r, c, seed=3)
    n = r.size - 1
    A = sp.csr_matrix((w.astype(np.float64), c, r), shape=(n, n))
    s = int(gg.sources(r, 1, seed=9)[0])
    ref = csgraph.dijkstra(A, directed=True, indices=s)
    dist, pred = oracle.sssp(r, c, w, s)
    exp = np.where(np.isfinite(ref), ref, 0xFFFFFFFF).astype(np.uint32)
    assert np.array_equal(dist, exp)
    validate_sssp_pred(r, c, w, s, dist, pred)


# ------------------------------------------------------------------- BC
def test_bc_closed_forms():
    n = 9
    r, c = path_graph(n)
    bc = oracle.bc(r, c, np.arange(n))
    assert np.allclose(bc, [2 * i * (n - 1 - i) for i in range(n)], rtol=0, atol=1e-12)
    r, c = star_graph(n)
    bc = oracle.bc(r, c, np.arange(n))
    assert np.allclose(bc, [(n - 1) * (n - 2)] + [0] * (n - 1))
    r, c = complete_graph(7)
    assert np.all(oracle.bc(r, c, np.arange(7)) == 0)
    # odd cycle C_{2k+1}: every vertex is interior to 2*(d-1) ordered
    # shortest paths of each length d = 2..k, i.e. k*(k-1) in total
    k = 4
    r, c = cycle_graph(2 * k + 1)
    assert np.allclose(oracle.bc(r, c, np.arange(2 * k + 1)), k * (k - 1))
    # even cycle C_6: antipodal pairs have two shortest paths
    r, c = cycle_graph(6)
    # pairs at distance 2: 12 ordered, 1 interior vertex each -> 12/6 = 2 per
    # vertex; distance 3: 6 ordered pairs, 2 paths with 2 interior vertices
    # each, weight 1/2 -> 6*2/6 = 2 per vertex
    assert np.allclose(oracle.bc(r, c, np.arange(6)), 4.0)


def test_bc_single_source_path():
    # from source 0 on a path, vertex i is interior to the paths to i+1..n-1
    n = 7
    r, c = path_graph(n)
    bc = oracle.bc(r, c, [0])
    assert np.allclose(bc, [0] + [n - 1 - i for i in range(1, n)])


@pytest.mark.parametrize("seed", range(12))
def test_bc_random_vs_path_enumeration(seed):
    n = 9
    r, c = random_graph(n, 0.35, seed)
    srcs = [0, 3, 5] if seed % 2 else list(range(n))
    assert np.allclose(oracle.bc(r, c, srcs), brute_force_bc(n, r, c, srcs),
                       rtol=1e-12, atol=1e-12)


def test_bc_rmat_vs_networkx_subset():
    nx = pytest.importorskip("networkx")
    r, c = gg.rmat(10, 8, seed=13)
    n = r.size - 1
    G = nx.DiGraph()  # both directions stored: directed counting, no halving
    G.add_nodes_from(range(n))
    src = np.repeat(np.arange(n), np.diff(r))
    G.add_edges_from(zip(src.tolist(), c.tolist()))
    srcs = gg.sources(r, 8, seed=13)
    ref = nx.betweenness_centrality_subset(G, sources=srcs.tolist(),
                                           targets=list(range(n)), normalized=False)
    exp = np.array([ref[v] for v in range(n)])
    got = oracle.bc(r, c, srcs)
    assert np.allclose(got, exp, rtol=1e-10, atol=1e-9)


# ------------------------------------------------------------------- CC
def test_cc_closed_form_union_of_pieces():
    # path 0..3, triangle 4..6, isolated 7, edge 8-9 (given as 9->8 first)
    r, c = gg.from_edges(10, [(0, 1), (1, 2), (2, 3), (4, 5), (5, 6), (6, 4), (9, 8)])
    label, k = oracle.cc(r, c)
    assert list(label) == [0, 0, 0, 0, 4, 4, 4, 7, 8, 8] and k == 4


def test_cc_exhaustive_small_graphs():
    for n in range(1, 6):
        for r, c in all_graphs(n):
            fw = floyd_warshall(n, r, c)
            label, k = oracle.cc(r, c)
            exp = [int(np.nonzero(np.isfinite(fw[v]))[0].min()) for v in range(n)]
            assert list(label) == exp
            assert k == len(set(exp))


def test_cc_rmat_vs_scipy_and_invariants():
    sp = pytest.importorskip("scipy.sparse")
    csgraph = pytest.importorskip("scipy.sparse.csgraph")
    r, c = gg.rmat(14, 4, seed=21)
    n = r.size - 1
    A = sp.csr_matrix((np.ones(c.size), c, r), shape=(n, n))
    k_ref, comp = csgraph.connected_components(A, directed=False)
    label, k = oracle.cc(r, c)
    assert k == k_ref
    # min vertex id per scipy component
    mins = np.full(k_ref, n)
    np.minimum.at(mins, comp, np.arange(n))
    assert np.array_equal(label, mins[comp])
    assert np.all(label <= np.arange(n))
    assert np.array_equal(label[label], label)
    src = np.repeat(np.arange(n), np.diff(r))
    assert np.all(label[src] == label[c])


def test_cc_grid_with_deletions_vs_scipy():
    sp = pytest.importorskip("scipy.sparse")
    csgraph = pytest.importorskip("scipy.sparse.csgraph")
    side = 80
    r, c = gg.grid(side, p_del=0.3, seed=4)
    n = side * side
    A = sp.csr_matrix((np.ones(c.size), c, r), shape=(n, n))
    k_ref, comp = csgraph.connected_components(A, directed=False)
    label, k = oracle.cc(r, c)
    mins = np.full(k_ref, n)
    np.minimum.at(mins, comp, np.arange(n))
    assert k == k_ref and np.array_equal(label, mins[comp])


# ------------------------------------------------------------- PageRank
@pytest.mark.parametrize("make", [lambda: cycle_graph(11), lambda: complete_graph(9),
                                  lambda: hypercube(5), lambda: torus(6)])
def test_pagerank_regular_graphs_uniform(make):
    r, c = make()
    n = r.size - 1
    rank, it = oracle.pagerank(r, c, 0.85, 50, 0.0)
    assert it == 50
    assert np.allclose(rank, 1.0 / n, rtol=0, atol=1e-15)


def test_pagerank_one_iteration_by_hand():
    # star with centre 0 and three leaves, one iteration from r = 1/4:
    # centre: 0.15/4 + 0.85 * 3 * (1/4) / 1 = 0.675
    # leaf:   0.15/4 + 0.85 * (1/4) / 3 = 0.1083333...
    r, c = star_graph(4)
    rank, it = oracle.pagerank(r, c, 0.85, 1, 0.0)
    assert it == 1
    assert np.allclose(rank, [0.675] + [0.0375 + 0.85 / 12] * 3, rtol=0, atol=1e-15)


def test_pagerank_dangling_by_hand():
    # vertices 0-1 joined, 2 isolated (dangling): one iteration from 1/3
    # D = 1/3; r0 = r1 = 0.05 + 0.85 * (1/3 + 1/9), r2 = 0.05 + 0.85/9
    r, c = gg.from_edges(3, [(0, 1)])
    rank, _ = oracle.pagerank(r, c, 0.85, 1, 0.0)
    a = 0.05 + 0.85 * (1 / 3 + 1 / 9)
    assert np.allclose(rank, [a, a, 0.05 + 0.85 / 9], rtol=0, atol=1e-15)
    assert abs(rank.sum() - 1) < 1e-15


def exact_pagerank(r, c, d):
    """Fixed point of the iteration, solved directly:
    (I - d*(P + u*dang^T)) x = (1-d)/n * 1, P[v,u] = 1/deg(u) per edge u->v."""
    n = r.size - 1
    deg = np.diff(r)
    P = np.zeros((n, n))
    for u in range(n):
        for e in range(r[u], r[u + 1]):
            P[c[e], u] += 1.0 / deg[u]
    dang = (deg == 0).astype(np.float64)
    M = P + np.outer(np.full(n, 1.0 / n), dang)
    return np.linalg.solve(np.eye(n) - d * M, np.full(n, (1 - d) / n))


@pytest.mark.parametrize("seed", range(8))
def test_pagerank_converges_to_exact_fixed_point(seed):
    n = 40
    r, c = random_graph(n, 0.08, seed)  # sparse: some isolated (dangling) vertices
    rank, it = oracle.pagerank(r, c, 0.85, 1000, 1e-15)
    exact = exact_pagerank(r, c, 0.85)
    assert np.allclose(rank, exact, rtol=1e-12, atol=1e-14)
    assert abs(rank.sum() - 1.0) < 1e-12


def test_pagerank_directed_fixed_point():
    # directed arcs exercise the in-edge sum and out-degree normalisation
    r = np.array([0, 2, 3, 3, 4], np.int32)
    c = np.array([1, 2, 2, 0], np.int32)  # 0->1, 0->2, 1->2, 3->0; 2 dangling
    rank, _ = oracle.pagerank(r, c, 0.85, 2000, 1e-16)
    assert np.allclose(rank, exact_pagerank(r, c, 0.85), rtol=1e-12)


def test_pagerank_rmat_vs_networkx():
    nx = pytest.importorskip("networkx")
    r, c = gg.rmat(11, 8, seed=17)
    n = r.size - 1
    G = nx.DiGraph()
    G.add_nodes_from(range(n))
    src = np.repeat(np.arange(n), np.diff(r))
    G.add_edges_from(zip(src.tolist(), c.tolist()))
    ref = nx.pagerank(G, alpha=0.85, tol=1e-14, max_iter=1000)
    rank, _ = oracle.pagerank(r, c, 0.85, 1000, 1e-15)
    assert relative_l1(rank, [ref[v] for v in range(n)]) < 1e-9


def test_pagerank_stop_rule():
    r, c = gg.rmat(10, 8, seed=3)
    rank50, it50 = oracle.pagerank(r, c, 0.85, 50, 0.0)
    assert it50 == 50
    rank_tol, it_tol = oracle.pagerank(r, c, 0.85, 500, 1e-7)
    assert it_tol < 500
    # the run stopped at the first iteration whose L1 change fell below tol
    prev, _ = oracle.pagerank(r, c, 0.85, it_tol - 1, 0.0)
    assert np.abs(rank_tol - prev).sum() < 1e-7
    prev2, _ = oracle.pagerank(r, c, 0.85, it_tol - 2, 0.0)
    assert np.abs(prev - prev2).sum() >= 1e-7


def test_oracle_rejects_bad_arguments():
    r, c = path_graph(4)
    with pytest.raises(RuntimeError):
        oracle.bfs(r, c, 4)
    with pytest.raises(RuntimeError):
        oracle.sssp(r, c, np.ones(c.size, np.uint32), -1)
    with pytest.raises(RuntimeError):
        oracle.pagerank(r, c, 1.5, 10, 0.0)
