"""Neighbourhood gather-reduce operator and the bipartite rankings (HITS,
SALSA, personalized PageRank) against the CPU oracle: min and max exact,
FP64 sums within a bound derived from the summation, rankings within a
relative L1 of 1e-10 of the oracle run for the GPU's iteration count."""
import numpy as np
import pytest

import graphgen as gg
import oracle
from checks import relative_l1

pytestmark = pytest.mark.gpu

EPS = np.finfo(np.float64).eps


def sum_bound(r, c, x, w=None):
    """Per-vertex bound on |GPU sum - oracle sum|: both are sums of the same
    deg(v) terms in different orders, each within deg * eps of the exact
    sum (times the sum of absolute terms)."""
    n = r.size - 1
    deg = np.diff(r)
    terms = np.abs(x[c]) * (1.0 if w is None else w.astype(np.float64))
    abs_sum = np.zeros(n)
    np.add.at(abs_sum, np.repeat(np.arange(n), deg), terms)
    return 2.0 * (deg + 1) * EPS * abs_sum + 1e-300


def directed_subset(scale, seed, keep=0.6):
    r, c = gg.rmat(scale, 8, seed=seed)
    rng = np.random.default_rng(seed)
    rows = np.repeat(np.arange(r.size - 1), np.diff(r))
    k = rng.random(c.size) < keep
    r2 = np.zeros_like(r)
    np.cumsum(np.bincount(rows[k], minlength=r.size - 1), out=r2[1:])
    return r2.astype(np.int32), c[k].astype(np.int32)


GRAPHS = {
    "rmat14": lambda: gg.rmat(14, 16, seed=1),
    "grid61": lambda: gg.grid(61, p_del=0.05, seed=4),
    "directed12": lambda: directed_subset(12, 5),
    "hub": lambda: gg.from_edges(5000, [(0, v) for v in range(1, 5000)] +
                                 [(v, v + 1) for v in range(1, 4999, 3)]),
}


@pytest.mark.parametrize("name", list(GRAPHS))
@pytest.mark.parametrize("use_frontier", [False, True])
def test_neighbor_reduce_matches_oracle(cuda_lib, name, use_frontier):
    import torch
    gr = cuda_lib
    r, c = GRAPHS[name]()
    n = r.size - 1
    rng = np.random.default_rng(n)
    w = gg.weights(r, c, seed=3, wmin=1, wmax=64)
    xf = rng.standard_normal(n)
    xi = rng.integers(-10**6, 10**6, n).astype(np.int32)
    frontier = None
    if use_frontier:
        frontier = rng.permutation(n)[: max(1, n // 3)].astype(np.int32)
        frontier = np.concatenate([[0], frontier[frontier != 0]]).astype(np.int32)  # the hub
    fdev = None if frontier is None else torch.from_numpy(frontier).cuda()
    with gr.gr_graph_create(r, c, w) as g:
        for op in (gr.GR_REDUCE_SUM, gr.GR_REDUCE_WSUM, gr.GR_REDUCE_MIN, gr.GR_REDUCE_MAX):
            is_sum = op in (gr.GR_REDUCE_SUM, gr.GR_REDUCE_WSUM)
            x = xf if is_sum else xi
            want = oracle.neighbor_reduce(r, c, op, x, w=w if op == gr.GR_REDUCE_WSUM else None,
                                          frontier=frontier)
            # entries outside the frontier keep their value: start from a
            # sentinel and expect it there
            sentinel = 12345.0 if is_sum else 7
            expected = want.copy()
            if frontier is not None:
                outside = np.ones(n, bool)
                outside[frontier] = False
                expected[outside] = sentinel
            for host_out in (False, True):
                init = np.full(n, sentinel, dtype=np.float64 if is_sum else np.int32)
                out = init if host_out else torch.from_numpy(init).cuda()
                gr.gr_neighbor_reduce(g, op, torch.from_numpy(x).cuda(), out, fdev)
                torch.cuda.synchronize()
                got = out if host_out else out.cpu().numpy()
                if is_sum:
                    bound = sum_bound(r, c, x, w if op == gr.GR_REDUCE_WSUM else None)
                    assert np.all(np.abs(got - expected) <= bound), (op, host_out)
                else:
                    assert np.array_equal(got, expected), (op, host_out)


def test_neighbor_reduce_edge_cases(cuda_lib):
    import torch
    gr = cuda_lib
    r, c = gg.from_edges(1, [])  # one vertex, no entries
    with gr.gr_graph_create(r, c) as g:
        out = torch.full((1,), 5, dtype=torch.int32, device="cuda")
        gr.gr_neighbor_reduce(g, gr.GR_REDUCE_MIN, torch.zeros(1, dtype=torch.int32, device="cuda"), out)
        assert int(out.item()) == np.iinfo(np.int32).max
        outf = torch.full((1,), 5.0, dtype=torch.float64, device="cuda")
        gr.gr_neighbor_reduce(g, gr.GR_REDUCE_SUM, torch.ones(1, dtype=torch.float64, device="cuda"), outf)
        assert float(outf.item()) == 0.0
        with pytest.raises(gr.GrError) as ei:  # no weights
            gr.gr_neighbor_reduce(g, gr.GR_REDUCE_WSUM, torch.ones(1, dtype=torch.float64, device="cuda"), outf)
        assert ei.value.status == gr.GR_EINVAL
    r, c = gg.rmat(10, 8, seed=2)
    with gr.gr_graph_create(r, c) as g:
        x = torch.ones(g.n, dtype=torch.float64, device="cuda")
        out = torch.full((g.n,), 3.0, dtype=torch.float64, device="cuda")
        empty = torch.empty(0, dtype=torch.int32, device="cuda")
        gr.gr_neighbor_reduce(g, gr.GR_REDUCE_SUM, x, out, empty)
        assert torch.all(out == 3.0)  # an empty frontier changes nothing
        with pytest.raises(gr.GrError) as ei:  # x in host memory
            gr.gr_neighbor_reduce(g, gr.GR_REDUCE_SUM, np.ones(g.n), out)
        assert ei.value.status == gr.GR_EINVAL
        with pytest.raises(gr.GrError):
            gr.gr_neighbor_reduce(g, 9, x, out)


def bipartite_graphs():
    yield "rmat_bip_12_10", gg.rmat_bipartite(12, 10, 8, seed=3)
    yield "rmat_bip_9_13", gg.rmat_bipartite(9, 13, 4, seed=4)
    r, c = gg.from_edges(9, [(0, 5), (1, 5), (1, 6), (2, 7), (3, 7), (3, 8)])  # 4 isolated hub
    yield "small_components", (r, c, 5)


@pytest.mark.parametrize("kind", ["hits", "salsa"])
def test_bipartite_rankings_match_oracle(cuda_lib, kind):
    import torch
    gr = cuda_lib
    run = gr.gr_hits if kind == "hits" else gr.gr_salsa
    ref_fn = oracle.hits if kind == "hits" else oracle.salsa
    for name, (r, c, nl) in bipartite_graphs():
        with gr.gr_graph_create(r, c) as g:
            for max_iter, tol in ((1, 0.0), (7, 0.0), (200, 1e-9)):
                for host_out in (False, True):
                    out = (np.empty(g.n) if host_out
                           else torch.empty(g.n, dtype=torch.float64, device="cuda"))
                    it = run(g, nl, out, max_iter=max_iter, tol=tol)
                    got = out if host_out else out.cpu().numpy()
                    want, it_ref = ref_fn(r, c, nl, it, 0.0)  # the GPU's iteration count
                    assert it_ref == it
                    assert relative_l1(got, want) < 1e-10, (name, max_iter, tol)
                    if tol == 0.0:
                        assert it == max_iter
                    else:
                        # the stop rule: the oracle stops within one iteration
                        _, it_own = ref_fn(r, c, nl, max_iter, tol)
                        assert abs(it_own - it) <= 1, (name, it_own, it)


def test_hits_complete_bipartite_closed_form(cuda_lib):
    import torch
    gr = cuda_lib
    a, b = 6, 11
    r, c = gg.from_edges(a + b, [(l, a + j) for l in range(a) for j in range(b)])
    with gr.gr_graph_create(r, c) as g:
        out = torch.empty(g.n, dtype=torch.float64, device="cuda")
        gr.gr_hits(g, a, out, max_iter=10, tol=1e-14)
        s = out.cpu().numpy()
        assert np.allclose(s[:a], 1 / np.sqrt(a), rtol=1e-14)
        assert np.allclose(s[a:], 1 / np.sqrt(b), rtol=1e-14)
        gr.gr_salsa(g, a, out, max_iter=10, tol=1e-14)
        s = out.cpu().numpy()
        assert np.allclose(s[:a], 1 / a, rtol=1e-14) and np.allclose(s[a:], 1 / b, rtol=1e-14)


def test_bipartite_rejects_bad_input(cuda_lib):
    import torch
    gr = cuda_lib
    r, c = gg.from_edges(4, [(0, 1), (0, 2), (2, 3)])
    with gr.gr_graph_create(r, c) as g:
        out = torch.empty(4, dtype=torch.float64, device="cuda")
        for fn in (gr.gr_hits, gr.gr_salsa):
            with pytest.raises(gr.GrError) as ei:
                fn(g, 3, out)  # 0-2 joins two hubs
            assert ei.value.status == gr.GR_EINVAL
            with pytest.raises(gr.GrError):
                fn(g, 5, out)  # n_left > n


@pytest.mark.parametrize("which", ["rmat14", "bipartite", "grid61"])
def test_ppr_matches_oracle(cuda_lib, which):
    import torch
    gr = cuda_lib
    if which == "rmat14":
        r, c = gg.rmat(14, 16, seed=1)
    elif which == "bipartite":
        r, c, _ = gg.rmat_bipartite(12, 10, 8, seed=3)
    else:
        r, c = gg.grid(61, p_del=0.05, seed=4)
    n = r.size - 1
    with gr.gr_graph_create(r, c) as g:
        for seeds in ([int(gg.max_degree_vertex(r))], list(gg.sources(r, 5, seed=2)),
                      [0, n - 1]):  # a possibly isolated seed (dangling mass)
            out = torch.empty(n, dtype=torch.float64, device="cuda")
            it = gr.gr_ppr(g, seeds, out, 0.85, 50, 1e-9)
            want, it_ref = oracle.ppr(r, c, seeds, 0.85, it, 0.0)
            assert it_ref == it
            got = out.cpu().numpy()
            assert relative_l1(got, want) < 1e-10
            assert abs(got.sum() - 1.0) < 1e-9


def test_ppr_rejects_bad_input(cuda_lib):
    import torch
    gr = cuda_lib
    r, c = gg.rmat(8, 8, seed=1)
    with gr.gr_graph_create(r, c) as g:
        out = torch.empty(g.n, dtype=torch.float64, device="cuda")
        for seeds in ([1, 1], [-1], [g.n], []):
            with pytest.raises(gr.GrError) as ei:
                gr.gr_ppr(g, seeds, out)
            assert ei.value.status == gr.GR_EINVAL
    rd = np.array([0, 1, 2, 2], np.int32)
    cd = np.array([1, 2], np.int32)
    with gr.gr_graph_create(rd, cd) as g:
        out = torch.empty(3, dtype=torch.float64, device="cuda")
        with pytest.raises(gr.GrError) as ei:
            gr.gr_ppr(g, [0], out)  # directed CSR
        assert ei.value.status == gr.GR_EINVAL


@pytest.mark.slow
def test_bipartite_rmat_20_18_full_size(cuda_lib):
    """A bipartite R-MAT of 2^20 hubs and 2^18 authorities (edge factor 16):
    HITS, SALSA and PPR against the oracle, 20 iterations."""
    import torch
    gr = cuda_lib
    r, c, nl = gg.rmat_bipartite(20, 18, 16, seed=6)
    with gr.gr_graph_create(r, c) as g:
        out = torch.empty(g.n, dtype=torch.float64, device="cuda")
        for fn, ref in ((gr.gr_hits, oracle.hits), (gr.gr_salsa, oracle.salsa)):
            it = fn(g, nl, out, max_iter=20, tol=0.0)
            want, _ = ref(r, c, nl, it, 0.0)
            assert relative_l1(out.cpu().numpy(), want) < 1e-10
        seeds = list(gg.sources(r, 8, seed=6))
        it = gr.gr_ppr(g, seeds, out, 0.85, 20, 0.0)
        want, _ = oracle.ppr(r, c, seeds, 0.85, it, 0.0)
        assert relative_l1(out.cpu().numpy(), want) < 1e-10
