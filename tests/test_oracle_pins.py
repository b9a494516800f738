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


# ------------------------------------------------- neighbourhood reduce
def csr_matrix(r, c, data=None):
    sp = pytest.importorskip("scipy.sparse")
    n = r.size - 1
    return sp.csr_matrix((np.ones(c.size) if data is None else data, c, r), shape=(n, n))


def test_neighbor_reduce_sum_of_ones_is_degree():
    r, c = gg.rmat(9, 8, seed=2)
    out = oracle.neighbor_reduce(r, c, oracle.REDUCE_SUM, np.ones(r.size - 1))
    assert np.array_equal(out, np.diff(r).astype(np.float64))


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_neighbor_reduce_sums_vs_scipy(seed):
    r, c = gg.rmat(10, 8, seed=seed)
    n = r.size - 1
    rng = np.random.default_rng(seed)
    x = rng.standard_normal(n)
    w = gg.weights(r, c, seed=seed, wmin=1, wmax=64)
    assert np.allclose(oracle.neighbor_reduce(r, c, oracle.REDUCE_SUM, x),
                       csr_matrix(r, c) @ x, rtol=1e-12, atol=1e-12)
    assert np.allclose(oracle.neighbor_reduce(r, c, oracle.REDUCE_WSUM, x, w=w),
                       csr_matrix(r, c, w.astype(np.float64)) @ x, rtol=1e-12, atol=1e-12)
    # unit weights: the weighted sum is the sum
    assert np.array_equal(
        oracle.neighbor_reduce(r, c, oracle.REDUCE_WSUM, x, w=np.ones(c.size, np.uint32)),
        oracle.neighbor_reduce(r, c, oracle.REDUCE_SUM, x))


def test_neighbor_reduce_min_label_propagation_gives_components():
    """Repeated min over the closed neighbourhood reaches, at its fixed
    point, the smallest vertex id of each component (scipy's components)."""
    csg = pytest.importorskip("scipy.sparse.csgraph")
    r, c = gg.grid(30, p_del=0.35, seed=5)
    n = r.size - 1
    label = np.arange(n, dtype=np.int32)
    for _ in range(4 * n):
        nb = oracle.neighbor_reduce(r, c, oracle.REDUCE_MIN, label)
        new = np.minimum(label, nb)
        if np.array_equal(new, label):
            break
        label = new
    _, comp = csg.connected_components(csr_matrix(r, c), directed=False)
    first = {}
    for v in range(n):
        first.setdefault(comp[v], v)
    assert np.array_equal(label, np.array([first[comp[v]] for v in range(n)], np.int32))


def test_neighbor_reduce_min_max_closed_forms_and_identity():
    n = 9
    r, c = gg.from_edges(n, [(i, i + 1) for i in range(n - 2)])  # path 0..7, 8 isolated
    ids = np.arange(n, dtype=np.int32)
    mx = oracle.neighbor_reduce(r, c, oracle.REDUCE_MAX, ids)
    mn = oracle.neighbor_reduce(r, c, oracle.REDUCE_MIN, ids)
    assert list(mx[:7]) == [v + 1 for v in range(7)] and mx[7] == 6
    assert list(mn[1:8]) == [v - 1 for v in range(1, 8)] and mn[0] == 1
    assert mx[8] == np.iinfo(np.int32).min and mn[8] == np.iinfo(np.int32).max
    s = oracle.neighbor_reduce(r, c, oracle.REDUCE_SUM, ids.astype(np.float64))
    assert s[8] == 0.0 and s[0] == 1.0 and s[3] == 6.0


def test_neighbor_reduce_frontier_and_brute_force():
    rng = np.random.default_rng(11)
    r, c = gg.rmat(7, 6, seed=4)
    n = r.size - 1
    xi = rng.integers(-1000, 1000, n).astype(np.int32)
    frontier = np.array([5, 0, 77, 5, n - 1], np.int32)
    for op in (oracle.REDUCE_MIN, oracle.REDUCE_MAX):
        full = oracle.neighbor_reduce(r, c, op, xi)
        part = oracle.neighbor_reduce(r, c, op, xi, frontier=frontier)
        ident = np.iinfo(np.int32).max if op == oracle.REDUCE_MIN else np.iinfo(np.int32).min
        for v in range(n):
            nb = [int(xi[u]) for u in c[r[v]:r[v + 1]]]
            want = (min(nb) if op == oracle.REDUCE_MIN else max(nb)) if nb else ident
            assert full[v] == want
            assert part[v] == (want if v in set(frontier.tolist()) else ident)


# ---------------------------------------------- bipartite node ranking
def complete_bipartite(a, b):
    return gg.from_edges(a + b, [(l, a + j) for l in range(a) for j in range(b)])


def bipartite_matrix(r, c, n_left):
    n = r.size - 1
    A = np.zeros((n_left, n - n_left))
    for l in range(n_left):
        for u in c[r[l]:r[l + 1]]:
            A[l, u - n_left] = 1.0
    return A


@pytest.mark.parametrize("a,b", [(1, 1), (3, 5), (6, 2)])
def test_hits_complete_bipartite_uniform(a, b):
    r, c = complete_bipartite(a, b)
    s, it = oracle.hits(r, c, a, 50, 1e-14)
    assert np.allclose(s[:a], 1.0 / np.sqrt(a), rtol=1e-14)
    assert np.allclose(s[a:], 1.0 / np.sqrt(b), rtol=1e-14)
    assert it <= 2


@pytest.mark.parametrize("seed", range(5))
def test_hits_is_the_dominant_singular_pair(seed):
    """Authorities: the dominant eigenvector of A^T A; hubs: that of A A^T
    (numpy eigh), on connected random bipartite graphs."""
    rng = np.random.default_rng(seed)
    nl, nr = 7, 9
    edges = [(l, nl + j) for l in range(nl) for j in range(nr) if rng.random() < 0.45]
    edges += [(l, nl + (l % nr)) for l in range(nl)] + [(j % nl, nl + j) for j in range(nr)]
    r, c = gg.from_edges(nl + nr, edges)
    s, _ = oracle.hits(r, c, nl, 5000, 1e-15)
    A = bipartite_matrix(r, c, nl)
    for M, part in ((A.T @ A, s[nl:]), (A @ A.T, s[:nl])):
        vals, vecs = np.linalg.eigh(M)
        v = np.abs(vecs[:, -1])
        assert vals[-1] - vals[-2] > 1e-3  # a unique dominant direction
        assert np.allclose(part, v / np.linalg.norm(v), atol=1e-9)


def test_hits_first_iteration_by_hand():
    # hubs 0, 1; authorities 2, 3, 4; links 0-2, 0-3, 1-3, 1-4
    r, c = gg.from_edges(5, [(0, 2), (0, 3), (1, 3), (1, 4)])
    s, it = oracle.hits(r, c, 2, 1, 0.0)
    h0 = 1 / np.sqrt(2)
    a = np.array([h0, 2 * h0, h0])
    a /= np.linalg.norm(a)
    h = np.array([a[0] + a[1], a[1] + a[2]])
    h /= np.linalg.norm(h)
    assert it == 1 and np.allclose(s, np.concatenate([h, a]), rtol=1e-15)


def test_salsa_degree_closed_form_connected():
    r, c, nl = gg.rmat_bipartite(7, 6, 8, seed=5)
    csg = pytest.importorskip("scipy.sparse.csgraph")
    ncomp, comp = csg.connected_components(csr_matrix(r, c), directed=False)
    deg = np.diff(r).astype(np.float64)
    s, it = oracle.salsa(r, c, nl, 20000, 1e-15)
    # per component C (with links): hubs get (linked hubs of C / linked hubs)
    # * deg / |E_C|, authorities (the same share) * deg / |E_C|
    linked = (deg[:nl] > 0).sum()
    want = np.zeros_like(s)
    for k in range(ncomp):
        vs = np.nonzero(comp == k)[0]
        e_c = deg[vs].sum() / 2
        if e_c == 0:
            continue
        share = (deg[vs[vs < nl]] > 0).sum() / linked
        want[vs] = share * deg[vs] / e_c
    assert np.allclose(s, want, atol=1e-12)
    assert abs(s[:nl].sum() - 1) < 1e-12 and abs(s[nl:].sum() - 1) < 1e-12


def test_salsa_first_iteration_by_hand():
    r, c = gg.from_edges(5, [(0, 2), (0, 3), (1, 3), (1, 4)])
    s, _ = oracle.salsa(r, c, 2, 1, 0.0)
    h0 = np.array([0.5, 0.5])
    a = np.array([h0[0] / 2, h0[0] / 2 + h0[1] / 2, h0[1] / 2])
    h = np.array([a[0] / 1 + a[1] / 2, a[1] / 2 + a[2] / 1])
    assert np.allclose(s, np.concatenate([h, a]), rtol=1e-15)


def test_ppr_all_seeds_is_pagerank():
    r, c = gg.rmat(10, 8, seed=7)
    n = r.size - 1
    a, ia = oracle.ppr(r, c, np.arange(n), 0.85, 60, 0.0)
    b, ib = oracle.pagerank(r, c, 0.85, 60, 0.0)
    assert ia == ib == 60 and np.allclose(a, b, rtol=1e-13, atol=1e-16)


@pytest.mark.parametrize("seed", range(6))
def test_ppr_exact_fixed_point(seed):
    n = 30
    r, c = random_graph(n, 0.1, seed)
    deg = np.diff(r)
    seeds = np.array(sorted({int(x) for x in np.random.default_rng(seed).integers(0, n, 3)}))
    t = np.zeros(n)
    t[seeds] = 1.0 / seeds.size
    P = np.zeros((n, n))
    for u in range(n):
        for v in c[r[u]:r[u + 1]]:
            P[v, u] += 1.0 / deg[u]
    M = P + np.outer(t, (deg == 0).astype(np.float64))
    exact = np.linalg.solve(np.eye(n) - 0.85 * M, (1 - 0.85) * t)
    got, _ = oracle.ppr(r, c, seeds, 0.85, 3000, 1e-16)
    assert np.allclose(got, exact, rtol=1e-11, atol=1e-15)
    assert abs(got.sum() - 1.0) < 1e-12


def test_ppr_vs_networkx_personalization():
    nx = pytest.importorskip("networkx")
    r, c, nl = gg.rmat_bipartite(8, 7, 8, seed=9)
    n = r.size - 1
    G = nx.DiGraph()
    G.add_nodes_from(range(n))
    G.add_edges_from(zip(np.repeat(np.arange(n), np.diff(r)).tolist(), c.tolist()))
    seeds = [int(v) for v in np.nonzero(np.diff(r)[:nl] > 0)[0][:4]]
    ref = nx.pagerank(G, alpha=0.85, personalization={s: 1.0 for s in seeds},
                      tol=1e-14, max_iter=2000)
    got, _ = oracle.ppr(r, c, seeds, 0.85, 2000, 1e-15)
    assert relative_l1(got, [ref[v] for v in range(n)]) < 1e-9


def test_bipartite_oracles_reject_bad_input():
    r, c = gg.from_edges(4, [(0, 1), (0, 2), (2, 3)])  # 0-2 joins two hubs when n_left = 3
    with pytest.raises(RuntimeError):
        oracle.hits(r, c, 3)
    with pytest.raises(RuntimeError):
        oracle.salsa(r, c, 3)
    with pytest.raises(RuntimeError):
        oracle.ppr(r, c, [1, 1])  # repeated seed
