"""BFS parity: the CUDA path against the CPU oracle on seeded inputs.
Depth is compared bit-exactly; parents are validated (any vertex one level
up with an edge to the child is a correct parent)."""
import numpy as np
import pytest

import graphgen as gg
import oracle
from checks import manhattan, validate_bfs

pytestmark = pytest.mark.gpu

DIRS = ["auto", "push", "pull"]
MODES = ["graph", "launch", "persistent"]


def opts(gr, direction="auto", mode="auto", **kw):
    d = {"auto": gr.GR_DIR_AUTO, "push": gr.GR_DIR_PUSH, "pull": gr.GR_DIR_PULL}[direction]
    m = {"auto": gr.GR_MODE_AUTO, "launch": gr.GR_MODE_LAUNCH, "graph": gr.GR_MODE_GRAPH,
         "persistent": gr.GR_MODE_PERSISTENT}[mode]
    o = gr.gr_opts(direction=d, mode=m)
    for k, v in kw.items():
        setattr(o, k, v)
    return o


def run_bfs(gr, g, src, o=None, with_parent=True):
    import torch
    depth = torch.empty(g.n, dtype=torch.int32, device="cuda")
    parent = torch.empty(g.n, dtype=torch.int32, device="cuda") if with_parent else None
    gr.gr_bfs(g, src, depth, parent, o)
    torch.cuda.synchronize()
    return depth.cpu().numpy(), (parent.cpu().numpy() if with_parent else None)


def check(gr, r, c, g, src, o=None, symmetric=True):
    ref, _ = oracle.bfs(r, c, src)
    d, p = run_bfs(gr, g, src, o)
    assert np.array_equal(d, ref), f"depth mismatch at {np.nonzero(d != ref)[0][:10]}"
    validate_bfs(r, c, src, d, p, symmetric=symmetric)


@pytest.fixture(scope="module")
def s14(cuda_lib):
    r, c = gg.rmat(14, 16, seed=1)
    g = cuda_lib.gr_graph_create(r, c)
    yield r, c, g
    g.close()


@pytest.mark.parametrize("direction", DIRS)
@pytest.mark.parametrize("mode", MODES)
def test_rmat_s14_max_degree_source(cuda_lib, s14, direction, mode):
    r, c, g = s14
    src = gg.max_degree_vertex(r)
    check(cuda_lib, r, c, g, src, opts(cuda_lib, direction, mode))


def test_rmat_s14_many_sources_and_isolated(cuda_lib, s14):
    r, c, g = s14
    info = cuda_lib.gr_graph_info(g)
    assert info["symmetric"] and info["num_isolated"] == int((np.diff(r) == 0).sum())
    srcs = list(gg.sources(r, 12, seed=5))
    srcs.append(int(np.nonzero(np.diff(r) == 0)[0][0]))  # an isolated source
    srcs.append(r.size - 2)                               # last vertex
    for s in srcs:
        check(cuda_lib, r, c, g, int(s))


def test_depth_only_and_stats(cuda_lib, s14):
    r, c, g = s14
    src = gg.max_degree_vertex(r)
    d, _ = run_bfs(cuda_lib, g, src, None, with_parent=False)
    ref, _ = oracle.bfs(r, c, src)
    assert np.array_equal(d, ref)
    levels, pulls = cuda_lib.gr_bfs_stats(g)
    assert levels == ref.max() + 1
    assert 0 <= pulls < levels


@pytest.mark.parametrize("side,p_del", [(64, 0.0), (61, 0.05), (33, 0.3)])
@pytest.mark.parametrize("mode", ["graph", "launch", "persistent"])
def test_grid(cuda_lib, side, p_del, mode):
    r, c = gg.grid(side, p_del=p_del, seed=4)
    with cuda_lib.gr_graph_create(r, c) as g:
        for src in [0, side * side // 2 + side // 3]:
            o = opts(cuda_lib, "auto", mode)
            check(cuda_lib, r, c, g, src, o)
            if p_del == 0.0:
                d, _ = run_bfs(cuda_lib, g, src, o)
                assert np.array_equal(d, manhattan(side, src))


@pytest.mark.parametrize("n", [1, 2, 31, 32, 33, 100, 1000])
def test_ragged_paths_and_stars(cuda_lib, n):
    for edges in ([(i, i + 1) for i in range(n - 1)], [(0, i) for i in range(1, n)]):
        r, c = gg.from_edges(n, edges)
        with cuda_lib.gr_graph_create(r, c) as g:
            for src in sorted({0, n // 2, n - 1}):
                for d in DIRS:
                    check(cuda_lib, r, c, g, src, opts(cuda_lib, d))


def test_no_edges(cuda_lib):
    r = np.zeros(70, np.int32)
    c = np.zeros(0, np.int32)
    with cuda_lib.gr_graph_create(r, c) as g:
        d, p = run_bfs(cuda_lib, g, 42)
        assert d[42] == 0 and p[42] == 42 and (d >= 0).sum() == 1 and (p >= 0).sum() == 1


def test_self_loops_and_duplicates_in_user_csr(cuda_lib):
    # rows: 0 -> {0, 1, 1, 2}, 1 -> {0, 0, 2}, 2 -> {0, 1, 2, 3}, 3 -> {2}
    r = np.array([0, 4, 7, 11, 12], np.int32)
    c = np.array([0, 1, 1, 2, 0, 0, 2, 0, 1, 2, 3, 2], np.int32)
    with cuda_lib.gr_graph_create(r, c) as g:
        assert cuda_lib.gr_graph_info(g)["symmetric"]
        for src in range(4):
            for d in DIRS:
                ref, _ = oracle.bfs(r, c, src)
                dd, pp = run_bfs(cuda_lib, g, src, opts(cuda_lib, d))
                assert np.array_equal(dd, ref)


def test_directed_graph_push_only(cuda_lib):
    # directed chain with a back arc: 0->1->2->3, 3->1; 4->0
    r = np.array([0, 1, 2, 3, 4, 5], np.int32)
    c = np.array([1, 2, 3, 1, 0], np.int32)
    with cuda_lib.gr_graph_create(r, c) as g:
        assert not cuda_lib.gr_graph_info(g)["symmetric"]
        for src in range(5):
            check(cuda_lib, r, c, g, src, None, symmetric=False)
        with pytest.raises(cuda_lib.GrError) as ei:
            run_bfs(cuda_lib, g, 0, opts(cuda_lib, "pull"))
        assert ei.value.status == cuda_lib.GR_EINVAL


def test_invalid_source(cuda_lib, s14):
    import torch
    r, c, g = s14
    d = torch.empty(g.n, dtype=torch.int32, device="cuda")
    for bad in [-1, g.n]:
        with pytest.raises(cuda_lib.GrError) as ei:
            cuda_lib.gr_bfs(g, bad, d)
        assert ei.value.status == cuda_lib.GR_EINVAL


def test_host_output_buffers(cuda_lib, s14):
    import torch
    r, c, g = s14
    src = gg.max_degree_vertex(r)
    ref, _ = oracle.bfs(r, c, src)
    # pinned host tensors
    d = torch.empty(g.n, dtype=torch.int32).pin_memory()
    p = torch.empty(g.n, dtype=torch.int32).pin_memory()
    cuda_lib.gr_bfs(g, src, d, p)
    torch.cuda.synchronize()
    assert np.array_equal(d.numpy(), ref)
    validate_bfs(r, c, src, d.numpy(), p.numpy())
    # pageable numpy arrays
    d2 = np.empty(g.n, np.int32)
    cuda_lib.gr_bfs(g, src, d2, None)
    torch.cuda.synchronize()
    assert np.array_equal(d2, ref)


@pytest.mark.parametrize("mode", ["auto", "graph", "persistent"])
def test_multi_pinned_outputs_on_a_side_stream(cuda_lib, s14, mode):
    """k searches with page-locked host outputs: more searches than staging
    sets, so a set is reused only after its copies finished; synchronising
    the call's own stream (not the device) must be enough to read them."""
    import torch
    r, c, g = s14
    srcs = [int(s) for s in gg.sources(r, 7, seed=11)] + [gg.max_degree_vertex(r)]
    d = [torch.full((g.n,), -7, dtype=torch.int32).pin_memory() for _ in srcs]
    p = [torch.full((g.n,), -7, dtype=torch.int32).pin_memory() for _ in srcs]
    st = torch.cuda.Stream()
    cuda_lib.gr_bfs_multi(g, srcs, d, p, opts(cuda_lib, "auto", mode), st)
    st.synchronize()
    for s, di, pi in zip(srcs, d, p):
        ref, _ = oracle.bfs(r, c, s)
        assert np.array_equal(di.numpy(), ref)
        validate_bfs(r, c, s, di.numpy(), pi.numpy())


def test_multi_mixed_outputs(cuda_lib, s14):
    """Host (pinned and pageable) and device outputs in one call, parents
    missing for some sources, the same source twice."""
    import torch
    r, c, g = s14
    srcs = [int(s) for s in gg.sources(r, 4, seed=12)]
    srcs = srcs + [srcs[0]]
    d = [np.empty(g.n, np.int32), torch.empty(g.n, dtype=torch.int32, device="cuda"),
         torch.empty(g.n, dtype=torch.int32).pin_memory(), np.empty(g.n, np.int32),
         torch.empty(g.n, dtype=torch.int32, device="cuda")]
    p = [None, torch.empty(g.n, dtype=torch.int32).pin_memory(),
         torch.empty(g.n, dtype=torch.int32, device="cuda"), np.empty(g.n, np.int32), None]
    cuda_lib.gr_bfs_multi(g, srcs, d, p)
    torch.cuda.synchronize()

    def host(x):
        return x.cpu().numpy() if hasattr(x, "cpu") else x

    for s, di, pi in zip(srcs, d, p):
        ref, _ = oracle.bfs(r, c, s)
        assert np.array_equal(host(di), ref)
        if pi is not None:
            validate_bfs(r, c, s, host(di), host(pi))
    # without any parent outputs; then k = 0 does nothing
    d1 = [torch.empty(g.n, dtype=torch.int32).pin_memory() for _ in srcs[:3]]
    cuda_lib.gr_bfs_multi(g, srcs[:3], d1)
    torch.cuda.synchronize()
    for s, di in zip(srcs[:3], d1):
        assert np.array_equal(di.numpy(), oracle.bfs(r, c, s)[0])
    cuda_lib.gr_bfs_multi(g, [], [])


def test_multi_checks_everything_before_enqueueing(cuda_lib, s14):
    import torch
    r, c, g = s14
    good = int(gg.sources(r, 1, seed=13)[0])
    d = [torch.full((g.n,), -7, dtype=torch.int32).pin_memory() for _ in range(3)]
    for bad in [-1, g.n]:
        with pytest.raises(cuda_lib.GrError) as ei:
            cuda_lib.gr_bfs_multi(g, [good, good, bad], d)
        assert ei.value.status == cuda_lib.GR_EINVAL
    torch.cuda.synchronize()
    assert all(int(x[0]) == -7 for x in d)  # nothing ran, not even the good sources
    with pytest.raises(cuda_lib.GrError) as ei:
        cuda_lib.gr_bfs_multi(g, [good, good], [d[0], None])
    assert ei.value.status == cuda_lib.GR_EINVAL


def test_device_resident_inputs_and_streams(cuda_lib):
    import torch
    r, c = gg.rmat(12, 8, seed=3)
    rt = torch.from_numpy(r).cuda()
    ct = torch.from_numpy(c).cuda()
    with cuda_lib.gr_graph_create(rt, ct) as g:
        s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
        srcs = gg.sources(r, 6, seed=1)
        outs = []
        for i, s in enumerate(srcs):
            st = s1 if i % 2 else s2
            d = torch.empty(g.n, dtype=torch.int32, device="cuda")
            with torch.cuda.stream(st):
                cuda_lib.gr_bfs(g, int(s), d, None, None, st)
            outs.append(d)
        torch.cuda.synchronize()
        for s, d in zip(srcs, outs):
            assert np.array_equal(d.cpu().numpy(), oracle.bfs(r, c, int(s))[0])


def test_tuning_knobs_do_not_change_depth(cuda_lib, s14):
    r, c, g = s14
    src = int(gg.sources(r, 1, seed=9)[0])
    ref, _ = oracle.bfs(r, c, src)
    for mode in ["graph", "persistent"]:
        for alpha, beta in [(1.0, 1.0), (1000.0, 2.0), (2.0, 1000.0), (0.01, 0.01)]:
            d, p = run_bfs(cuda_lib, g, src, opts(cuda_lib, "auto", mode, alpha=alpha, beta=beta))
            assert np.array_equal(d, ref)
            validate_bfs(r, c, src, d, p)


@pytest.mark.slow
def test_rmat_s22_sixteen_sources(cuda_lib):
    """The benchmark's configuration: R-MAT scale 22, edge factor 16, seed 2,
    16 random non-isolated sources, default (tuned) options."""
    r, c = gg.rmat(22, 16, seed=2)
    from checks import edge_keys, edge_sources
    keys = edge_keys(r, c)
    su = edge_sources(r)
    with cuda_lib.gr_graph_create(r, c) as g:
        for s in gg.sources(r, 16, seed=2):
            ref, _ = oracle.bfs(r, c, int(s))
            d, p = run_bfs(cuda_lib, g, int(s))
            assert np.array_equal(d, ref)
            validate_bfs(r, c, int(s), d, p, keys=keys, su=su)


@pytest.mark.parametrize("mode", ["graph", "persistent"])
@pytest.mark.parametrize("direction", DIRS)
def test_trace_frontier_sizes_match_oracle_levels(cuda_lib, s14, direction, mode):
    # every frontier is exact (each vertex enters once), so the traced
    # frontier sizes equal the oracle's vertex count per depth
    r, c, g = s14
    src = gg.max_degree_vertex(r)
    run_bfs(cuda_lib, g, src, opts(cuda_lib, direction, mode))
    tr = cuda_lib.gr_bfs_trace(g)
    ref, _ = oracle.bfs(r, c, src)
    hist = np.bincount(ref[ref >= 0])
    assert [f for _, f, _, _ in tr] == list(hist)
    deg = np.diff(r)
    for lvl, (d, f, e, t) in enumerate(tr):
        assert e == int(deg[ref == lvl].sum())
        assert d == (0 if direction == "push" or lvl == 0 else d)
    if direction == "pull":
        assert all(d == 1 for d, _, _, _ in tr[1:])
    times = [t for _, _, _, t in tr]
    assert all(b >= a for a, b in zip(times, times[1:]))


def _kary_tree(k, depth):
    # complete k-ary tree, vertices in level order: children of v are
    # k*v + 1 .. k*v + k
    n = sum(k ** i for i in range(depth + 1))
    edges = [(v, k * v + j) for v in range(n) for j in range(1, k + 1) if k * v + j < n]
    return gg.from_edges(n, edges)


@pytest.mark.parametrize("src_kind", ["root", "leaf", "middle"])
def test_low_degree_cluster_overflow_and_handoff(cuda_lib, src_kind):
    # a 15-ary tree of depth 4 (max degree 16: the low-degree path): from the
    # root the frontiers are 1, 15, 225, 3375, 50625, so a level's claims
    # overflow the per-CTA buffers of the one-cluster driver into the global
    # queue, and the last frontier is handed to the grid kernel
    r, c = _kary_tree(15, 4)
    n = r.size - 1
    src = {"root": 0, "leaf": n - 1, "middle": 1 + 15 + 7}[src_kind]
    with cuda_lib.gr_graph_create(r, c) as g:
        for mode in ["persistent", "auto", "graph"]:
            check(cuda_lib, r, c, g, src, opts(cuda_lib, "auto", mode))
        ref, _ = oracle.bfs(r, c, src)
        run_bfs(cuda_lib, g, src, opts(cuda_lib, "auto", "persistent"))
        assert cuda_lib.gr_bfs_stats(g)[0] == int(ref.max()) + 1
        tr = cuda_lib.gr_bfs_trace(g)
        assert [f for _, f, _, _ in tr] == list(np.bincount(ref[ref >= 0]))
        deg = np.diff(r)
        assert [e for _, _, e, _ in tr] == [int(deg[ref == l].sum()) for l in range(len(tr))]


def test_low_degree_random_graph_grows_past_the_cluster(cuda_lib):
    # two random permutations as edges: degree <= 4, frontiers grow ~3x per
    # level until they leave the cluster driver
    n = 300_000
    rng = np.random.default_rng(11)
    e = np.concatenate([np.stack([np.arange(n), rng.permutation(n)], 1) for _ in range(2)])
    r, c = gg.from_edges(n, [tuple(x) for x in e.tolist()])
    with cuda_lib.gr_graph_create(r, c) as g:
        for src in [0, 123_457]:
            check(cuda_lib, r, c, g, src, opts(cuda_lib, "auto", "persistent"))
            ref, _ = oracle.bfs(r, c, src)
            run_bfs(cuda_lib, g, src, opts(cuda_lib, "auto", "persistent"), with_parent=False)
            tr = cuda_lib.gr_bfs_trace(g)
            assert [f for _, f, _, _ in tr] == list(np.bincount(ref[ref >= 0]))[:len(tr)]


@pytest.mark.parametrize("side", [64, 300])
def test_mesh_trace_matches_oracle_levels(cuda_lib, side):
    r, c = gg.grid(side, p_del=0.05, seed=4)
    with cuda_lib.gr_graph_create(r, c) as g:
        src = side * side // 2 + side // 3
        ref, _ = oracle.bfs(r, c, src)
        check(cuda_lib, r, c, g, src, opts(cuda_lib, "auto", "persistent"))
        tr = cuda_lib.gr_bfs_trace(g)
        hist = list(np.bincount(ref[ref >= 0]))
        assert [f for _, f, _, _ in tr] == hist[:len(tr)]
        assert cuda_lib.gr_bfs_stats(g)[0] == len(hist)
