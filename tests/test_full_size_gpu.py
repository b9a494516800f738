"""Parity at the full sizes of the specified workloads, with the tuned default
options the benchmark suite uses: the 4096 x 4096 mesh with 5 % of its edges
deleted (BFS, SSSP, CC) and R-MAT scale 23 (CC, PageRank, the 64-lane batched
BFS). Depths, distances and labels are compared with the oracle element by
element; BFS parents are validated; PageRank is within relative L1 1e-5 of
the FP64 oracle run for the same number of iterations."""
import numpy as np
import pytest

import graphgen as gg
import oracle
from checks import edge_keys, edge_sources, relative_l1, validate_bfs, validate_sssp_pred

pytestmark = pytest.mark.gpu

PR_TOL = 1e-5


def dev_empty(n, dtype):
    import torch
    return torch.empty(n, dtype=dtype, device="cuda")


def host(t):
    import torch
    torch.cuda.synchronize()
    return t.cpu().numpy()


@pytest.fixture(scope="module")
def mesh(cuda_lib):
    r, c = gg.grid(4096, p_del=0.05, seed=4)
    w = gg.weights(r, c, seed=4, wmin=1, wmax=16)
    g = cuda_lib.gr_graph_create(r, c, w)
    yield r, c, w, g
    g.close()


@pytest.fixture(scope="module")
def rmat23(cuda_lib):
    r, c = gg.rmat(23, 16, seed=5)
    g = cuda_lib.gr_graph_create(r, c)
    yield r, c, g
    g.close()


def test_mesh_bfs(cuda_lib, mesh):
    import torch
    r, c, _, g = mesh
    keys, su = edge_keys(r, c), edge_sources(r)
    d = dev_empty(g.n, torch.int32)
    p = dev_empty(g.n, torch.int32)
    for s in gg.sources(r, 2, seed=4):
        cuda_lib.gr_bfs(g, int(s), d, p)
        dh, ph = host(d), host(p)
        ref, _ = oracle.bfs(r, c, int(s))
        assert np.array_equal(dh, ref)
        validate_bfs(r, c, int(s), dh, ph, keys=keys, su=su)


def test_mesh_sssp(cuda_lib, mesh):
    import torch
    r, c, w, g = mesh
    s = int(gg.sources(r, 1, seed=4)[0])
    d = dev_empty(g.n, torch.int32)
    p = dev_empty(g.n, torch.int32)
    cuda_lib.gr_sssp(g, s, d, p)
    dh = host(d).view(np.uint32)
    ph = host(p)
    ref, ref_pred = oracle.sssp(r, c, w, s)
    assert np.array_equal(dh, ref)
    assert np.array_equal(ph, ref_pred)
    validate_sssp_pred(r, c, w, s, dh, ph)


def test_mesh_cc(cuda_lib, mesh):
    import torch
    r, c, _, g = mesh
    lab = dev_empty(g.n, torch.int32)
    k = cuda_lib.gr_cc(g, lab)
    ref, ref_k = oracle.cc(r, c)
    assert np.array_equal(host(lab), ref)
    assert k == ref_k


def test_rmat23_cc(cuda_lib, rmat23):
    import torch
    r, c, g = rmat23
    lab = dev_empty(g.n, torch.int32)
    k = cuda_lib.gr_cc(g, lab)
    ref, ref_k = oracle.cc(r, c)
    assert np.array_equal(host(lab), ref)
    assert k == ref_k


def test_rmat23_pagerank_ten_iterations(cuda_lib, rmat23):
    import torch
    r, c, g = rmat23
    rank = dev_empty(g.n, torch.float32)
    it = cuda_lib.gr_pagerank(g, rank, damping=0.85, max_iter=10, tol=0.0)
    assert it == 10
    ref, ref_it = oracle.pagerank(r, c, 0.85, 10, 0.0)
    assert ref_it == 10
    assert relative_l1(host(rank), ref) <= PR_TOL


def test_rmat23_batched_bfs_64_lanes(cuda_lib, rmat23):
    import torch
    r, c, g = rmat23
    srcs = gg.sources(r, 64, seed=5)
    d = dev_empty(64 * g.n, torch.int32)
    cuda_lib.gr_bfs_batch(g, srcs, d)
    dh = host(d).reshape(64, g.n)
    for i in (0, 21, 42, 63):
        ref, _ = oracle.bfs(r, c, int(srcs[i]))
        assert np.array_equal(dh[i], ref), f"lane {i}"
