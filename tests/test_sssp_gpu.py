"""SSSP parity: distances bit-exact against Dijkstra, predecessors equal to
the oracle's canonical choice (smallest shortest-path in-neighbour), for any
near/far bucket width."""
import numpy as np
import pytest

import graphgen as gg
import oracle
from checks import manhattan, validate_sssp_pred

pytestmark = pytest.mark.gpu

INF = 0xFFFFFFFF


def run_sssp(gr, g, src, o=None, with_pred=True):
    import torch
    dist = torch.empty(g.n, dtype=torch.int32, device="cuda")
    pred = torch.empty(g.n, dtype=torch.int32, device="cuda") if with_pred else None
    gr.gr_sssp(g, src, dist, pred, o)
    torch.cuda.synchronize()
    gr.gr_sssp_stats(g)  # raises on a device-side cap or timeout
    d = dist.cpu().numpy().view(np.uint32)
    return d, (pred.cpu().numpy() if with_pred else None)


def check(gr, r, c, w, g, src, o=None):
    ref_d, ref_p = oracle.sssp(r, c, w, src)
    d, p = run_sssp(gr, g, src, o)
    bad = np.nonzero(d != ref_d)[0]
    assert bad.size == 0, f"dist mismatch at {bad[:10]}: {d[bad[:10]]} vs {ref_d[bad[:10]]}"
    assert np.array_equal(p, ref_p)


def opts(gr, delta=0, mode="auto", direction="auto", alpha=0.0):
    m = {"auto": gr.GR_MODE_AUTO, "launch": gr.GR_MODE_LAUNCH, "graph": gr.GR_MODE_GRAPH,
         "persistent": gr.GR_MODE_PERSISTENT}[mode]
    d = {"auto": gr.GR_DIR_AUTO, "push": gr.GR_DIR_PUSH, "pull": gr.GR_DIR_PULL}[direction]
    return gr.gr_opts(delta=delta, mode=m, direction=d, alpha=alpha)


@pytest.fixture(scope="module")
def s14w(cuda_lib):
    r, c = gg.rmat(14, 16, seed=1)
    w = gg.weights(r, c, seed=3)
    g = cuda_lib.gr_graph_create(r, c, w)
    yield r, c, w, g
    g.close()


@pytest.mark.parametrize("delta", [0, 1, 8, 64, 0xFFFFFFFF])
@pytest.mark.parametrize("mode", ["graph", "launch", "persistent"])
def test_rmat_s14_delta_invariance(cuda_lib, s14w, delta, mode):
    r, c, w, g = s14w
    for src in [gg.max_degree_vertex(r)] + list(gg.sources(r, 3, seed=7)):
        check(cuda_lib, r, c, w, g, int(src), opts(cuda_lib, delta, mode))


@pytest.mark.parametrize("delta", [0, 8, 0xFFFFFFFF])
@pytest.mark.parametrize("mode", ["graph", "launch", "persistent"])
@pytest.mark.parametrize("direction,alpha", [("pull", 0.0), ("auto", 2.0), ("auto", 1.25),
                                             ("push", 0.0)])
def test_rmat_s14_pull_relaxation(cuda_lib, s14w, delta, mode, direction, alpha):
    """Direction-optimising SSSP: relaxations in pull form (every one, or
    those whose near frontier holds m / alpha edges) give Dijkstra's
    distances and the canonical predecessors, like push."""
    r, c, w, g = s14w
    o = opts(cuda_lib, delta, mode, direction, alpha)
    pulls = []
    for src in [gg.max_degree_vertex(r)] + list(gg.sources(r, 2, seed=9)):
        check(cuda_lib, r, c, w, g, int(src), o)
        pulls.append(cuda_lib.gr_sssp_pull_stats(g))
    if direction == "pull":
        assert min(pulls) > 0
    if direction == "push":
        assert max(pulls) == 0


def test_pull_relaxation_edge_cases(cuda_lib):
    """Forced pull on graphs with isolated vertices, zero weights, a
    disconnected part and a hub whose row spans several chunks; a directed
    CSR rejects forced pull."""
    gr = cuda_lib
    rng = np.random.default_rng(3)
    hub = [(0, v) for v in range(1, 3000)]
    extra = [(int(a), int(b)) for a, b in rng.integers(1, 3000, size=(4000, 2)) if a != b]
    far = [(3100 + i, 3101 + i) for i in range(50)]  # a separate path
    r, c = gg.from_edges(3200, hub + extra + far)
    for wmin, wmax in [(0, 3), (1, 64)]:
        w = gg.weights(r, c, seed=5, wmin=wmin, wmax=wmax)
        with gr.gr_graph_create(r, c, w) as g:
            for src in [0, 17, 3100, 3150, 3199]:
                check(gr, r, c, w, g, src, opts(gr, 0, "persistent", "pull"))
                check(gr, r, c, w, g, src, opts(gr, 0xFFFFFFFF, "graph", "pull"))
    rd = np.array([0, 1, 2, 2], np.int32)
    cd = np.array([1, 2], np.int32)
    with gr.gr_graph_create(rd, cd, np.ones(2, np.uint32)) as g:
        import torch
        d = torch.empty(3, dtype=torch.int32, device="cuda")
        with pytest.raises(gr.GrError) as ei:
            gr.gr_sssp(g, 0, d, None, opts(gr, 0, "auto", "pull"))
        assert ei.value.status == gr.GR_EINVAL


def test_unit_weights_equal_bfs_depth_on_grid(cuda_lib):
    side = 50
    r, c = gg.grid(side, p_del=0.0)
    w = np.ones(c.size, np.uint32)
    with cuda_lib.gr_graph_create(r, c, w) as g:
        d, p = run_sssp(cuda_lib, g, 77)
        assert np.array_equal(d.astype(np.int64), manhattan(side, 77))
        validate_sssp_pred(r, c, w, 77, d, p)


@pytest.mark.parametrize("side,p_del", [(40, 0.05), (23, 0.3)])
def test_grid_weighted(cuda_lib, side, p_del):
    r, c = gg.grid(side, p_del=p_del, seed=4)
    w = gg.weights(r, c, seed=5, wmin=1, wmax=16)
    with cuda_lib.gr_graph_create(r, c, w) as g:
        for src in [0, side * side // 2]:
            for delta in [0, 1, 16, 0xFFFFFFFF]:
                for mode in ["graph", "persistent"]:
                    check(cuda_lib, r, c, w, g, src, opts(cuda_lib, delta, mode))


@pytest.mark.parametrize("n", [1, 2, 33, 257])
def test_ragged_paths(cuda_lib, n):
    r, c = gg.from_edges(n, [(i, i + 1) for i in range(n - 1)])
    w = gg.weights(r, c, seed=n, wmin=1, wmax=64)
    with cuda_lib.gr_graph_create(r, c, w) as g:
        for src in sorted({0, n // 2, n - 1}):
            check(cuda_lib, r, c, w, g, src, opts(cuda_lib, 4))
            check(cuda_lib, r, c, w, g, src, opts(cuda_lib, 4, "persistent"))


def test_zero_and_large_weights(cuda_lib):
    # zero weights are allowed (non-negative); a huge weight makes a target
    # unreachable when the sum does not fit below 0xFFFFFFFF
    r, c = gg.from_edges(5, [(0, 1), (1, 2), (2, 3), (3, 4)])
    src = np.repeat(np.arange(5), np.diff(r))
    for big, d4 in [(0xFFFFFFF0, 0xFFFFFFF5), (0xFFFFFFF9, 0xFFFFFFFE), (0xFFFFFFFA, INF)]:
        # 5 + big: the largest representable distance is 0xFFFFFFFE
        key = {(0, 1): 0, (1, 2): 5, (2, 3): 0, (3, 4): big}
        w = np.array([key[(min(a, b), max(a, b))] for a, b in zip(src, c)], np.uint32)
        with cuda_lib.gr_graph_create(r, c, w) as g:
            d, p = run_sssp(cuda_lib, g, 0)
            assert list(d) == [0, 0, 5, 5, d4]
            assert list(p) == [0, 0, 1, 2, 3 if d4 != INF else -1]


def test_disconnected_and_isolated(cuda_lib):
    r, c = gg.from_edges(8, [(0, 1), (1, 2), (4, 5)])
    w = gg.weights(r, c, seed=1)
    with cuda_lib.gr_graph_create(r, c, w) as g:
        for s in range(8):
            check(cuda_lib, r, c, w, g, s)


def test_directed_weighted(cuda_lib):
    # 0->1 (9), 0->2 (2), 2->1 (3), 1->3 (1), 3->0 (1)
    r = np.array([0, 2, 3, 4, 5], np.int32)
    c = np.array([1, 2, 3, 1, 0], np.int32)
    w = np.array([9, 2, 1, 3, 1], np.uint32)
    with cuda_lib.gr_graph_create(r, c, w) as g:
        for s in range(4):
            check(cuda_lib, r, c, w, g, s)


def test_requires_weights(cuda_lib):
    import torch
    r, c = gg.from_edges(3, [(0, 1)])
    with cuda_lib.gr_graph_create(r, c) as g:
        d = torch.empty(3, dtype=torch.int32, device="cuda")
        with pytest.raises(cuda_lib.GrError) as ei:
            cuda_lib.gr_sssp(g, 0, d)
        assert ei.value.status == cuda_lib.GR_EINVAL


def test_host_outputs(cuda_lib, s14w):
    r, c, w, g = s14w
    s = int(gg.sources(r, 1, seed=3)[0])
    d = np.empty(g.n, np.uint32)
    p = np.empty(g.n, np.int32)
    cuda_lib.gr_sssp(g, s, d, p)
    import torch
    torch.cuda.synchronize()
    ref_d, ref_p = oracle.sssp(r, c, w, s)
    assert np.array_equal(d, ref_d) and np.array_equal(p, ref_p)


@pytest.mark.slow
def test_rmat_s22_sampled_sources(cuda_lib):
    """R-MAT scale 22, seed 2, weights U[1,64] from seed 3: distances of 3 of
    the 16 benchmark sources bit-exact against Dijkstra."""
    r, c = gg.rmat(22, 16, seed=2)
    w = gg.weights(r, c, seed=3)
    with cuda_lib.gr_graph_create(r, c, w) as g:
        for s in gg.sources(r, 16, seed=2)[:3]:
            ref_d, ref_p = oracle.sssp(r, c, w, int(s))
            d, p = run_sssp(cuda_lib, g, int(s))
            assert np.array_equal(d, ref_d)
            assert np.array_equal(p, ref_p)


# ------------------------------------------------------- batched searches
# gr_sssp_batch runs k searches as one near/far search over k disjoint copies
# of the graph; every lane must equal Dijkstra from its own source.

def run_batch(gr, g, srcs, o=None):
    import torch
    k = len(srcs)
    dist = torch.empty(k * g.n, dtype=torch.int32, device="cuda")
    gr.gr_sssp_batch(g, srcs, dist, o)
    torch.cuda.synchronize()
    gr.gr_sssp_batch_stats(g)  # raises on a device-side cap or timeout
    return dist.cpu().numpy().view(np.uint32).reshape(k, g.n)


def check_batch(gr, r, c, w, g, srcs, o=None, cache=None, d=None):
    if d is None:
        d = run_batch(gr, g, srcs, o)
    cache = {} if cache is None else cache
    for lane, s in enumerate(srcs):
        s = int(s)
        if s not in cache:
            cache[s] = oracle.sssp(r, c, w, s)[0]
        bad = np.nonzero(d[lane] != cache[s])[0]
        assert bad.size == 0, (f"lane {lane} (source {s}): dist mismatch at {bad[:10]}: "
                               f"{d[lane][bad[:10]]} vs {cache[s][bad[:10]]}")


@pytest.fixture(scope="module")
def s14_sources(s14w):
    r = s14w[0]
    isolated = int(np.nonzero(np.diff(r) == 0)[0][0])
    top = int(gg.max_degree_vertex(r))
    # 64 lanes: a repeated source and an isolated one among them
    return [top, isolated] + [int(x) for x in gg.sources(r, 61, seed=11)] + [top]


@pytest.mark.parametrize("delta", [0, 1, 0xFFFFFFFF])
@pytest.mark.parametrize("mode", ["launch", "graph", "persistent"])
def test_batch_rmat_s14(cuda_lib, s14w, s14_sources, delta, mode):
    r, c, w, g = s14w
    cache = {}
    for k in (1, 5, 64):
        check_batch(cuda_lib, r, c, w, g, s14_sources[:k], opts(cuda_lib, delta, mode), cache)


@pytest.mark.parametrize("mode", ["launch", "persistent"])
def test_batch_grid_low_degree(cuda_lib, mode):
    """A mesh (maximum degree 4: one thread per frontier vertex) with 5 %
    of its edges deleted; corners, centre and random sources."""
    side = 64
    r, c = gg.grid(side, p_del=0.05, seed=4)
    w = gg.weights(r, c, seed=5, wmin=1, wmax=16)
    srcs = [0, side - 1, side * side - 1, side * side // 2 + side // 2]
    srcs += [int(x) for x in gg.sources(r, 12, seed=8)]
    with cuda_lib.gr_graph_create(r, c, w) as g:
        cache = {}
        for delta in (0, 1, 16):
            check_batch(cuda_lib, r, c, w, g, srcs, opts(cuda_lib, delta, mode), cache)


@pytest.mark.parametrize("n", [1, 2, 33, 257])
def test_batch_ragged_paths(cuda_lib, n):
    r, c = gg.from_edges(n, [(i, i + 1) for i in range(n - 1)])
    w = gg.weights(r, c, seed=n, wmin=1, wmax=64)
    srcs = sorted({0, n // 2, n - 1}) + [0]
    with cuda_lib.gr_graph_create(r, c, w) as g:
        for mode in ("launch", "persistent"):
            check_batch(cuda_lib, r, c, w, g, srcs, opts(cuda_lib, 4, mode))


def test_batch_directed_zero_weights_and_disconnected(cuda_lib):
    # directed, with a zero-weight edge and an unreachable part (5, 6)
    r = np.array([0, 2, 3, 4, 5, 5, 6, 6], np.int32)
    c = np.array([1, 2, 3, 1, 0, 6], np.int32)
    w = np.array([9, 0, 1, 3, 1, 7], np.uint32)
    with cuda_lib.gr_graph_create(r, c, w) as g:
        check_batch(cuda_lib, r, c, w, g, list(range(7)))


def test_batch_equals_single_rmat_s16(cuda_lib):
    """24 lanes on a larger graph (merge-path relaxation over several chunks
    per iteration) against gr_sssp one source at a time and Dijkstra."""
    import torch
    r, c = gg.rmat(16, 16, seed=9)
    w = gg.weights(r, c, seed=10)
    srcs = [int(x) for x in gg.sources(r, 24, seed=12)]
    with cuda_lib.gr_graph_create(r, c, w) as g:
        d = run_batch(cuda_lib, g, srcs)
        for lane, s in enumerate(srcs[:6]):
            one, _ = run_sssp(cuda_lib, g, s, with_pred=False)
            assert np.array_equal(d[lane], one)
        check_batch(cuda_lib, r, c, w, g, srcs, d=d)
        torch.cuda.synchronize()


def test_batch_host_output_and_regrow(cuda_lib, s14w, s14_sources):
    """Host (pageable) output; the workspace grows from 4 to 16 lanes and is
    reused for 2."""
    import torch
    r, c, w, g = s14w
    cache = {}
    h = np.full(4 * g.n, 7, np.uint32)
    cuda_lib.gr_sssp_batch(g, s14_sources[:4], h)
    torch.cuda.synchronize()
    check_batch(cuda_lib, r, c, w, g, s14_sources[:4], cache=cache, d=h.reshape(4, g.n))
    check_batch(cuda_lib, r, c, w, g, s14_sources[10:26], cache=cache)
    check_batch(cuda_lib, r, c, w, g, s14_sources[30:32], cache=cache)


def test_batch_bad_arguments(cuda_lib, s14w):
    import torch
    r, c, w, g = s14w
    d = torch.empty(65 * g.n, dtype=torch.int32, device="cuda")
    for srcs in ([], list(range(65)), [0, g.n], [-1]):
        with pytest.raises(cuda_lib.GrError) as ei:
            cuda_lib.gr_sssp_batch(g, srcs, d)
        assert ei.value.status == cuda_lib.GR_EINVAL
    r2, c2 = gg.from_edges(3, [(0, 1)])
    with cuda_lib.gr_graph_create(r2, c2) as g2:
        with pytest.raises(cuda_lib.GrError) as ei:
            cuda_lib.gr_sssp_batch(g2, [0], d)
        assert ei.value.status == cuda_lib.GR_EINVAL


def _kary_tree(k, depth):
    n = sum(k ** i for i in range(depth + 1))
    edges = [(v, k * v + j) for v in range(n) for j in range(1, k + 1) if k * v + j < n]
    return gg.from_edges(n, edges)


@pytest.mark.parametrize("delta", [0xFFFFFFFF, 16, 1])
def test_low_degree_tree(cuda_lib, delta):
    # a 15-ary tree of depth 4 (max degree 16, the per-thread relaxation):
    # near frontiers of 1, 15, 225, 3375 and 50625 vertices with one bucket
    r, c = _kary_tree(15, 4)
    w = gg.weights(r, c, seed=21, wmin=1, wmax=64)
    n = r.size - 1
    with cuda_lib.gr_graph_create(r, c, w) as g:
        for src in [0, n - 1]:
            check(cuda_lib, r, c, w, g, src, opts(cuda_lib, delta, "persistent"))


def test_low_degree_random_graph_large_far_pile(cuda_lib):
    # a random graph of degree <= 4 with bucket width 1: a far pile of
    # hundreds of thousands of vertices, split over and over
    n = 400_000
    rng = np.random.default_rng(12)
    e = np.concatenate([np.stack([np.arange(n), rng.permutation(n)], 1) for _ in range(2)])
    r, c = gg.from_edges(n, [tuple(x) for x in e.tolist()])
    w = gg.weights(r, c, seed=22, wmin=1, wmax=64)
    with cuda_lib.gr_graph_create(r, c, w) as g:
        for delta in [1, 0xFFFFFFFF]:
            check(cuda_lib, r, c, w, g, 5, opts(cuda_lib, delta, "persistent"))


@pytest.mark.parametrize("delta", [0, 16, 300])
def test_mesh_persistent_equals_graph_driver(cuda_lib, delta):
    side = 300
    r, c = gg.grid(side, p_del=0.05, seed=4)
    w = gg.weights(r, c, seed=23, wmin=1, wmax=16)
    with cuda_lib.gr_graph_create(r, c, w) as g:
        src = side * side // 2 + side // 3
        check(cuda_lib, r, c, w, g, src, opts(cuda_lib, delta, "persistent"))
        # the same search through the CUDA-graph driver gives the same answer
        d_graph, _ = run_sssp(cuda_lib, g, src, opts(cuda_lib, delta, "graph"))
        d_pers, _ = run_sssp(cuda_lib, g, src, opts(cuda_lib, delta, "persistent"))
        assert np.array_equal(d_graph, d_pers)
