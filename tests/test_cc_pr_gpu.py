"""CC and PageRank parity. CC labels are bit-exact (smallest vertex id per
component); PageRank (FP32 on the device) is within relative L1 1e-5 of the
FP64 oracle run for the same number of iterations."""
import numpy as np
import pytest

import graphgen as gg
import oracle
from checks import relative_l1

pytestmark = pytest.mark.gpu

PR_TOL = 1e-5


def run_cc(gr, g, host=False):
    import torch
    if host:
        lab = np.empty(g.n, np.int32)
        k = gr.gr_cc(g, lab)
        return lab, k
    lab = torch.empty(g.n, dtype=torch.int32, device="cuda")
    k = gr.gr_cc(g, lab)
    return lab.cpu().numpy(), k


def run_pr(gr, g, damping=0.85, max_iter=50, tol=1e-7, mode=None):
    import torch
    rank = torch.empty(g.n, dtype=torch.float32, device="cuda")
    o = None if mode is None else gr.gr_opts(mode=mode)
    it = gr.gr_pagerank(g, rank, damping, max_iter, tol, o)
    return rank.cpu().numpy(), it


# ------------------------------------------------------------------- CC
@pytest.mark.parametrize("scale,ef,seed", [(10, 2, 1), (14, 16, 1), (16, 4, 21)])
def test_cc_rmat(cuda_lib, scale, ef, seed):
    r, c = gg.rmat(scale, ef, seed=seed)
    ref, k_ref = oracle.cc(r, c)
    with cuda_lib.gr_graph_create(r, c) as g:
        lab, k = run_cc(cuda_lib, g)
        assert np.array_equal(lab, ref) and k == k_ref
        lab2, k2 = run_cc(cuda_lib, g, host=True)
        assert np.array_equal(lab2, ref) and k2 == k_ref


@pytest.mark.parametrize("side,p_del", [(64, 0.05), (100, 0.45), (37, 0.7)])
def test_cc_grid(cuda_lib, side, p_del):
    r, c = gg.grid(side, p_del=p_del, seed=4)
    ref, k_ref = oracle.cc(r, c)
    with cuda_lib.gr_graph_create(r, c) as g:
        lab, k = run_cc(cuda_lib, g)
        assert np.array_equal(lab, ref) and k == k_ref


@pytest.mark.parametrize("n", [1, 2, 31, 33, 1000])
def test_cc_paths_reversed_ids(cuda_lib, n):
    # a path whose ids decrease along it, plus isolated tail vertices
    edges = [(n - 1 - i, n - 2 - i) for i in range(max(0, n - 1) // 2)]
    r, c = gg.from_edges(n, edges)
    ref, k_ref = oracle.cc(r, c)
    with cuda_lib.gr_graph_create(r, c) as g:
        lab, k = run_cc(cuda_lib, g)
        assert np.array_equal(lab, ref) and k == k_ref


def test_cc_directed_is_weak(cuda_lib):
    # arcs 3->1, 1->0, 5->4 ; 2 isolated: weak components {0,1,3}, {2}, {4,5}
    r = np.array([0, 0, 1, 1, 2, 2, 3], np.int32)
    c = np.array([0, 1, 4], np.int32)
    ref, k_ref = oracle.cc(r, c)
    with cuda_lib.gr_graph_create(r, c) as g:
        lab, k = run_cc(cuda_lib, g)
        assert list(lab) == [0, 0, 2, 0, 4, 4] and k == 3
        assert np.array_equal(lab, ref) and k == k_ref


# ------------------------------------------------------------- PageRank
@pytest.mark.parametrize("scale,ef,seed", [(10, 8, 3), (14, 16, 1), (16, 16, 5)])
def test_pagerank_rmat(cuda_lib, scale, ef, seed):
    r, c = gg.rmat(scale, ef, seed=seed)
    with cuda_lib.gr_graph_create(r, c) as g:
        rank, it = run_pr(cuda_lib, g)
        ref, _ = oracle.pagerank(r, c, 0.85, it, 0.0)
        assert relative_l1(rank, ref) <= PR_TOL
        assert abs(rank.astype(np.float64).sum() - 1.0) < 1e-4


def test_pagerank_stop_rule_and_modes(cuda_lib):
    r, c = gg.rmat(12, 8, seed=3)
    with cuda_lib.gr_graph_create(r, c) as g:
        rank_g, it_g = run_pr(cuda_lib, g, max_iter=500, tol=1e-6)
        rank_l, it_l = run_pr(cuda_lib, g, max_iter=500, tol=1e-6, mode=cuda_lib.GR_MODE_LAUNCH)
        assert 1 < it_g < 500 and abs(it_g - it_l) <= 1
        ref, _ = oracle.pagerank(r, c, 0.85, it_g, 0.0)
        assert relative_l1(rank_g, ref) <= PR_TOL
        rank0, it0 = run_pr(cuda_lib, g, max_iter=0)
        assert it0 == 0 and np.allclose(rank0, 1.0 / g.n)
        rank3, it3 = run_pr(cuda_lib, g, max_iter=3, tol=0.0)
        ref3, _ = oracle.pagerank(r, c, 0.85, 3, 0.0)
        assert it3 == 3 and relative_l1(rank3, ref3) <= 1e-6


@pytest.mark.parametrize("side", [16, 33])
def test_pagerank_regular_torus_uniform(cuda_lib, side):
    e = []
    for rr in range(side):
        for cc in range(side):
            v = rr * side + cc
            e += [(v, rr * side + (cc + 1) % side), (v, ((rr + 1) % side) * side + cc)]
    r, c = gg.from_edges(side * side, e)
    with cuda_lib.gr_graph_create(r, c) as g:
        rank, it = run_pr(cuda_lib, g, max_iter=50, tol=0.0)
        assert it == 50
        assert np.allclose(rank, 1.0 / (side * side), rtol=1e-5)


def test_pagerank_directed_and_dangling(cuda_lib):
    rng = np.random.default_rng(0)
    n = 3000
    src = rng.integers(0, n, 20000)
    dst = rng.integers(0, n, 20000)
    keep = src % 7 != 0            # vertices = 0 mod 7 have no out-arcs (dangling)
    src, dst = src[keep], dst[keep]
    order = np.lexsort((dst, src))
    src, dst = src[order], dst[order]
    r = np.zeros(n + 1, np.int32)
    np.add.at(r, src + 1, 1)
    r = np.cumsum(r).astype(np.int32)
    c = dst.astype(np.int32)
    with cuda_lib.gr_graph_create(r, c) as g:
        assert not cuda_lib.gr_graph_info(g)["symmetric"]
        rank, it = run_pr(cuda_lib, g, max_iter=40, tol=0.0)
        ref, _ = oracle.pagerank(r, c, 0.85, 40, 0.0)
        assert relative_l1(rank, ref) <= PR_TOL


def test_pagerank_bad_args(cuda_lib):
    import torch
    r, c = gg.from_edges(4, [(0, 1)])
    with cuda_lib.gr_graph_create(r, c) as g:
        rank = torch.empty(4, dtype=torch.float32, device="cuda")
        for kw in [dict(damping=0.0), dict(damping=1.0), dict(max_iter=-1), dict(tol=-1.0)]:
            args = dict(damping=0.85, max_iter=10, tol=0.0)
            args.update(kw)
            with pytest.raises(cuda_lib.GrError) as ei:
                cuda_lib.gr_pagerank(g, rank, **args)
            assert ei.value.status == cuda_lib.GR_EINVAL


@pytest.mark.slow
def test_pagerank_cc_rmat_s23(cuda_lib):
    """R-MAT scale 23, seed 5: PageRank (d = 0.85, 50 iterations or L1 change
    < 1e-7) within 1e-5 relative L1 of the FP64 oracle; CC labels exact."""
    r, c = gg.rmat(23, 16, seed=5)
    with cuda_lib.gr_graph_create(r, c) as g:
        rank, it = run_pr(cuda_lib, g)
        ref, _ = oracle.pagerank(r, c, 0.85, it, 0.0)
        assert relative_l1(rank, ref) <= PR_TOL
        lab, k = run_cc(cuda_lib, g)
        ref_l, k_ref = oracle.cc(r, c)
        assert np.array_equal(lab, ref_l) and k == k_ref
