"""Batched (64-lane) BFS and Brandes BC parity. Batched depths equal the
oracle's queue BFS per source bit-exactly; BC (FP64) is within 1e-9
relative error of the oracle per vertex and exactly 0 where the oracle's is."""
import numpy as np
import pytest

import graphgen as gg
import oracle

pytestmark = pytest.mark.gpu

BC_RTOL = 1e-9


def run_batch(gr, g, srcs):
    import torch
    d = torch.empty(len(srcs) * g.n, dtype=torch.int32, device="cuda")
    gr.gr_bfs_batch(g, srcs, d)
    torch.cuda.synchronize()
    return d.cpu().numpy().reshape(len(srcs), g.n)


def run_bc(gr, g, srcs, host=False):
    import torch
    if host:
        out = np.empty(g.n, np.float64)
        gr.gr_bc(g, srcs, out)
        return out
    out = torch.empty(g.n, dtype=torch.float64, device="cuda")
    gr.gr_bc(g, srcs, out)
    torch.cuda.synchronize()
    return out.cpu().numpy()


def check_bc(got, ref):
    zero = ref == 0
    assert np.all(got[zero] == 0), "nonzero BC where the oracle has 0"
    rel = np.abs(got[~zero] - ref[~zero]) / np.abs(ref[~zero])
    assert rel.size == 0 or rel.max() <= BC_RTOL, f"max rel err {rel.max()}"


@pytest.mark.parametrize("k", [1, 7, 32, 63, 64])
def test_batch_bfs_rmat(cuda_lib, k):
    r, c = gg.rmat(13, 16, seed=4)
    srcs = gg.sources(r, k, seed=k)
    with cuda_lib.gr_graph_create(r, c) as g:
        d = run_batch(cuda_lib, g, srcs)
        for i, s in enumerate(srcs):
            assert np.array_equal(d[i], oracle.bfs(r, c, int(s))[0])


def test_batch_bfs_repeats_isolated_and_grid(cuda_lib):
    r, c = gg.grid(45, p_del=0.1, seed=4)
    srcs = [0, 0, 7, 2024, 45 * 45 - 1]
    with cuda_lib.gr_graph_create(r, c) as g:
        d = run_batch(cuda_lib, g, srcs)
        for i, s in enumerate(srcs):
            assert np.array_equal(d[i], oracle.bfs(r, c, s)[0])
    r, c = gg.from_edges(40, [(1, 2), (2, 3)])
    with cuda_lib.gr_graph_create(r, c) as g:
        d = run_batch(cuda_lib, g, [0, 2, 39])
        for i, s in enumerate([0, 2, 39]):
            assert np.array_equal(d[i], oracle.bfs(r, c, s)[0])


@pytest.mark.parametrize("n", [63, 64, 65, 66, 130, 300])
def test_batch_bfs_long_paths(cuda_lib, n):
    # the depths of the first 64 levels come from the kept level masks, those
    # of deeper levels are written as they are reached: cover both and the
    # boundary between them
    r, c = gg.from_edges(n, [(i, i + 1) for i in range(n - 1)])
    srcs = [0, n // 2, n - 1, 0]
    with cuda_lib.gr_graph_create(r, c) as g:
        d = run_batch(cuda_lib, g, srcs)
        for i, s in enumerate(srcs):
            assert np.array_equal(d[i], np.abs(np.arange(n) - s).astype(np.int32))


@pytest.mark.parametrize("tail", [10, 15, 16, 17, 40])
def test_batch_bfs_kept_level_boundary(cuda_lib, tail):
    """A hub with 20 leaves (so the graph is not mesh-like and a batch keeps
    the lane masks of its first levels) and a path hanging off it: depths of
    the kept levels come from the end-of-run pass, deeper ones are written as
    they are reached; sources on the path, the hub and a leaf."""
    edges = [(0, i) for i in range(1, 21)]
    prev = 0
    for i in range(tail):
        edges.append((prev, 21 + i))
        prev = 21 + i
    n = 21 + tail
    r, c = gg.from_edges(n, edges)
    srcs = [0, 5, n - 1, 21 + tail // 2, n - 1]
    with cuda_lib.gr_graph_create(r, c) as g:
        d = run_batch(cuda_lib, g, srcs)
        levels = cuda_lib.gr_bfs_batch_stats(g)
        for i, s in enumerate(srcs):
            assert np.array_equal(d[i], oracle.bfs(r, c, s)[0])
    assert levels == max(int(oracle.bfs(r, c, s)[0].max()) for s in srcs) + 1


def test_batch_bfs_bad_args(cuda_lib):
    import torch
    r, c = gg.from_edges(5, [(0, 1)])
    with cuda_lib.gr_graph_create(r, c) as g:
        d = torch.empty(65 * 5, dtype=torch.int32, device="cuda")
        for srcs in [[], list(range(5)) * 13, [5], [-1]]:
            with pytest.raises(cuda_lib.GrError) as ei:
                cuda_lib.gr_bfs_batch(g, srcs, d)
            assert ei.value.status == cuda_lib.GR_EINVAL


def test_bc_closed_forms(cuda_lib):
    n = 9
    for edges, expect in [
        ([(i, i + 1) for i in range(n - 1)], [2 * i * (n - 1 - i) for i in range(n)]),
        ([(0, i) for i in range(1, n)], [(n - 1) * (n - 2)] + [0] * (n - 1)),
    ]:
        r, c = gg.from_edges(n, edges)
        with cuda_lib.gr_graph_create(r, c) as g:
            got = run_bc(cuda_lib, g, list(range(n)))
            assert np.allclose(got, expect, rtol=1e-12, atol=0)
    r, c = gg.from_edges(6, [(i, (i + 1) % 6) for i in range(6)])
    with cuda_lib.gr_graph_create(r, c) as g:
        assert np.allclose(run_bc(cuda_lib, g, list(range(6))), 4.0, rtol=1e-12)


@pytest.mark.parametrize("scale,ef,k", [(10, 8, 5), (12, 16, 64), (13, 16, 100)])
def test_bc_rmat(cuda_lib, scale, ef, k):
    r, c = gg.rmat(scale, ef, seed=scale)
    srcs = gg.sources(r, k, seed=3)
    with cuda_lib.gr_graph_create(r, c) as g:
        check_bc(run_bc(cuda_lib, g, srcs), oracle.bc(r, c, srcs))
        check_bc(run_bc(cuda_lib, g, srcs, host=True), oracle.bc(r, c, srcs))


def test_bc_small_random_and_repeated_sources(cuda_lib):
    rng = np.random.default_rng(5)
    for t in range(6):
        n = 30
        e = [(i, j) for i in range(n) for j in range(i + 1, n) if rng.random() < 0.12]
        r, c = gg.from_edges(n, e)
        srcs = list(rng.integers(0, n, 10)) + [3, 3]
        with cuda_lib.gr_graph_create(r, c) as g:
            check_bc(run_bc(cuda_lib, g, srcs), oracle.bc(r, c, srcs))


def test_bc_no_sources_and_overflow(cuda_lib):
    r, c = gg.from_edges(4, [(0, 1), (1, 2)])
    with cuda_lib.gr_graph_create(r, c) as g:
        assert np.all(run_bc(cuda_lib, g, []) == 0)
    # opposite corners of a full 1100 x 1100 grid: C(2198, 1099) shortest
    # paths overflow FP64
    side = 1100
    r, c = gg.grid(side, p_del=0.0)
    import torch
    with cuda_lib.gr_graph_create(r, c) as g:
        out = torch.empty(g.n, dtype=torch.float64, device="cuda")
        with pytest.raises(cuda_lib.GrError) as ei:
            cuda_lib.gr_bc(g, [0], out)
        assert ei.value.status == cuda_lib.GR_EINVAL


def directed_rmat(scale, seed, keep=0.6):
    """R-MAT with each directed entry kept with probability `keep`: a
    non-symmetric CSR with dense levels and vertices without out-edges."""
    r, c = gg.rmat(scale, 16, seed=seed)
    rng = np.random.default_rng(seed)
    keep_e = rng.random(c.size) < keep
    rows = np.repeat(np.arange(r.size - 1), np.diff(r))
    deg = np.bincount(rows[keep_e], minlength=r.size - 1)
    r2 = np.zeros_like(r)
    r2[1:] = np.cumsum(deg)
    return r2.astype(np.int32), c[keep_e].astype(np.int32)


def test_batch_bfs_and_bc_directed(cuda_lib):
    """On a directed CSR every batched level pushes along out-edges; depths
    equal the oracle's per source, BC equals directed Brandes."""
    r, c = directed_rmat(12, 7)
    srcs = gg.sources(r, 64, seed=7)
    with cuda_lib.gr_graph_create(r, c) as g:
        assert not cuda_lib.gr_graph_info(g)["symmetric"]
        d = run_batch(cuda_lib, g, srcs)
        for i in (0, 17, 40, 63):
            assert np.array_equal(d[i], oracle.bfs(r, c, int(srcs[i]))[0]), f"lane {i}"
        check_bc(run_bc(cuda_lib, g, srcs), oracle.bc(r, c, srcs))


@pytest.mark.parametrize("diamonds", [60, 70])
def test_bc_path_counts_past_2_to_the_64(cuda_lib, diamonds):
    """A chain of diamonds doubles the number of shortest paths at each
    diamond: 2^60 paths fit the exact uint64 counts, 2^70 do not and the
    batch is counted again in FP64 (where powers of two are exact)."""
    edges, c0 = [], 0
    for i in range(diamonds):
        a, b, c1 = 3 * i + 1, 3 * i + 2, 3 * i + 3
        edges += [(c0, a), (c0, b), (a, c1), (b, c1)]
        c0 = c1
    n = c0 + 1
    r, c = gg.from_edges(n, edges)
    srcs = [0, n - 1, 1, 3 * (diamonds // 2)]
    with cuda_lib.gr_graph_create(r, c) as g:
        check_bc(run_bc(cuda_lib, g, srcs), oracle.bc(r, c, srcs))


def _oracle_bc_part(args):
    scale, seed, srcs = args
    import graphgen
    import oracle as orc
    r, c = graphgen.rmat(scale, 16, seed=seed)
    return orc.bc(r, c, srcs)


def oracle_bc_parallel(scale, seed, srcs, procs=16):
    """The oracle's BC summed over sources, the sources split over a pool of
    spawned processes (each regenerates the seeded graph)."""
    import multiprocessing as mp
    parts = [list(map(int, srcs[i::procs])) for i in range(procs)]
    parts = [p for p in parts if p]
    with mp.get_context("spawn").Pool(len(parts)) as pool:
        res = pool.map(_oracle_bc_part, [(scale, seed, p) for p in parts])
    return np.sum(res, axis=0)


@pytest.mark.slow
def test_bc_rmat_s23_64_sources(cuda_lib):
    """R-MAT scale 23, seed 5, 64 random sources in one lane batch, FP64,
    relative error <= 1e-9 per vertex against Brandes on the CPU."""
    r, c = gg.rmat(23, 16, seed=5)
    srcs = gg.sources(r, 64, seed=5)
    with cuda_lib.gr_graph_create(r, c) as g:
        got = run_bc(cuda_lib, g, srcs)
    check_bc(got, oracle_bc_parallel(23, 5, srcs))
