"""Query server: every result served in the mix (BFS and SSSP batched,
admitted under a memory budget) equals the same query run alone, bit for
bit. The server runs one worker slot (gr_server_create refuses more)."""
import numpy as np
import pytest

import graphgen as gg

pytestmark = pytest.mark.gpu


def alone(gr, g, kind, src):
    import torch
    out = torch.empty(g.n, dtype=torch.int32, device="cuda")
    if kind == gr.GR_QUERY_BFS:
        gr.gr_bfs(g, src, out, None)
    elif kind == gr.GR_QUERY_SSSP:
        gr.gr_sssp(g, src, out, None)
    else:
        gr.gr_cc(g, out, count=False)
    torch.cuda.synchronize()
    return out.cpu().numpy()


@pytest.fixture(scope="module")
def pool(cuda_lib):
    gr = cuda_lib
    graphs = []
    for scale, ef, seed in [(12, 8, 101), (14, 16, 102), (13, 32, 103)]:
        r, c = gg.rmat(scale, ef, seed=seed)
        w = gg.weights(r, c, seed=seed, wmin=1, wmax=64)
        graphs.append((gr.gr_graph_create(r, c, w), True))
    r, c = gg.grid(96, p_del=0.05, seed=104)
    w = gg.weights(r, c, seed=104, wmin=1, wmax=64)
    graphs.append((gr.gr_graph_create(r, c, w), False))
    yield graphs
    for g, _ in graphs:
        g.close()


def make_requests(gr, graphs, count, seed):
    rng = np.random.default_rng(seed)
    reqs = []
    for _ in range(count):
        gi = int(rng.integers(0, len(graphs)))
        u = rng.random()
        kind = gr.GR_QUERY_BFS if u < 0.6 else (gr.GR_QUERY_SSSP if u < 0.9 else gr.GR_QUERY_CC)
        src = int(rng.integers(0, graphs[gi][0].n))
        reqs.append((gi, kind, src))
    return reqs


@pytest.mark.parametrize("slots,batch,budget", [
    (1, 1, 1 << 30), (1, 64, 1 << 30), (1, 16, 200_000)])
def test_mix_equals_alone(cuda_lib, pool, slots, batch, budget):
    gr = cuda_lib
    reqs = make_requests(gr, pool, 240, seed=slots * 7 + batch)
    outs = [np.full(pool[gi][0].n, -7, np.int32) for gi, _, _ in reqs]
    with gr.gr_server_create(budget, slots, batch) as srv:
        ids = [gr.gr_server_add_graph(srv, g, b) for g, b in pool]
        tickets = [gr.gr_server_submit(srv, ids[gi], kind, src, out)
                   for (gi, kind, src), out in zip(reqs, outs)]
        lat = [gr.gr_server_wait(srv, t, 120000) for t in tickets]
        st = gr.gr_server_stats(srv)
    assert st["completed"] == len(reqs) and st["failed"] == 0
    assert all(x >= 0 for x in lat)
    if batch == 1:
        assert st["mean_batch"] == 1.0
    cache = {}
    for (gi, kind, src), out in zip(reqs, outs):
        key = (gi, kind, src if kind != gr.GR_QUERY_CC else 0)
        if key not in cache:
            cache[key] = alone(gr, pool[gi][0], kind, src)
        assert np.array_equal(out, cache[key]), f"request {key} differs in the mix"


def test_batching_happens_and_device_outputs(cuda_lib, pool):
    import torch
    gr = cuda_lib
    g = pool[1][0]
    with gr.gr_server_create(1 << 30, 1, 64) as srv:
        gid = gr.gr_server_add_graph(srv, g, True)
        outs = [torch.empty(g.n, dtype=torch.int32, device="cuda") for _ in range(100)]
        # the first submit starts the worker; the rest queue behind it
        tickets = [gr.gr_server_submit(srv, gid, gr.GR_QUERY_BFS, s, o)
                   for s, o in zip(range(0, 100 * 37, 37), outs)]
        gr.gr_server_drain(srv, 120000)
        st = gr.gr_server_stats(srv)
    assert st["completed"] == 100
    assert st["launches"] < 100 and st["mean_batch"] > 1.0
    for s, o in zip(range(0, 100 * 37, 37), outs[:10]):
        assert np.array_equal(o.cpu().numpy(), alone(gr, g, gr.GR_QUERY_BFS, s))


@pytest.mark.parametrize("depth,batched", [(8, True), (0, False)])
def test_batching_depth(cuda_lib, pool, depth, batched):
    """A graph registered with batchable = 8 batches its BFS requests once 8
    are queued; with 0 it never batches. Results equal the queries alone."""
    import torch
    gr = cuda_lib
    g = pool[3][0]  # the grid
    srcs = list(range(0, 20 * 97, 97))
    with gr.gr_server_create(1 << 30, 1, 64) as srv:
        gid = gr.gr_server_add_graph(srv, g, depth)
        outs = [torch.empty(g.n, dtype=torch.int32, device="cuda") for _ in srcs]
        for s, o in zip(srcs, outs):
            gr.gr_server_submit(srv, gid, gr.GR_QUERY_BFS, s, o)
        gr.gr_server_drain(srv, 120000)
        st = gr.gr_server_stats(srv)
    assert st["completed"] == len(srcs) and st["failed"] == 0
    assert (st["launches"] < len(srcs)) == batched
    for s, o in zip(srcs, outs):
        assert np.array_equal(o.cpu().numpy(), alone(gr, g, gr.GR_QUERY_BFS, s))


@pytest.mark.parametrize("gi", [1, 3])
def test_sssp_batching(cuda_lib, pool, gi):
    """Queued same-graph SSSP requests run as lanes of one batched search
    (an R-MAT graph and the grid); results equal the queries alone."""
    gr = cuda_lib
    g = pool[gi][0]
    srcs = [(i * 53) % g.n for i in range(30)]
    outs = [np.full(g.n, -7, np.int32) for _ in srcs]
    with gr.gr_server_create(1 << 30, 1, 64) as srv:
        gid = gr.gr_server_add_graph(srv, g, 8)
        for s, o in zip(srcs, outs):
            gr.gr_server_submit(srv, gid, gr.GR_QUERY_SSSP, s, o)
        gr.gr_server_drain(srv, 120000)
        st = gr.gr_server_stats(srv)
    assert st["completed"] == len(srcs) and st["failed"] == 0
    assert st["launches"] < len(srcs) and st["mean_batch"] > 1.0
    for s, o in zip(srcs, outs):
        assert np.array_equal(o, alone(gr, g, gr.GR_QUERY_SSSP, s))


@pytest.mark.parametrize("gi", [0, 3])
def test_cc_requests_share_one_run(cuda_lib, pool, gi):
    """Queued CC requests of a graph share one run and its one result
    buffer; every request gets the labels of CC run alone, on the host and
    on the device."""
    import torch
    gr = cuda_lib
    g = pool[gi][0]
    outs = [np.full(g.n, -7, np.int32) for _ in range(12)]
    outs += [torch.full((g.n,), -7, dtype=torch.int32, device="cuda") for _ in range(4)]
    with gr.gr_server_create(1 << 30, 1, 64) as srv:
        gid = gr.gr_server_add_graph(srv, g, 1)
        for o in outs:
            gr.gr_server_submit(srv, gid, gr.GR_QUERY_CC, 0, o)
        gr.gr_server_drain(srv, 120000)
        st = gr.gr_server_stats(srv)
    assert st["completed"] == len(outs) and st["failed"] == 0
    assert st["launches"] < len(outs) and st["mean_batch"] > 1.0
    ref = alone(gr, g, gr.GR_QUERY_CC, 0)
    for o in outs:
        got = o.cpu().numpy() if isinstance(o, torch.Tensor) else o
        assert np.array_equal(got, ref)


def test_bad_requests(cuda_lib, pool):
    gr = cuda_lib
    g = pool[0][0]
    with gr.gr_server_create(1 << 20, 1, 8) as srv:
        gid = gr.gr_server_add_graph(srv, g, True)
        for args in [(gid + 5, gr.GR_QUERY_BFS, 0), (gid, 9, 0), (gid, gr.GR_QUERY_BFS, g.n)]:
            with pytest.raises(gr.GrError) as ei:
                gr.gr_server_submit(srv, *args)
            assert ei.value.status == gr.GR_EINVAL
        with pytest.raises(gr.GrError) as ei:
            gr.gr_server_wait(srv, 12345, 0)
        assert ei.value.status == gr.GR_EINVAL
        with pytest.raises(gr.GrError) as ei:
            gr.gr_server_add_graph(srv, g, 65)
        assert ei.value.status == gr.GR_EINVAL
    with pytest.raises(gr.GrError):
        gr.gr_server_create(0, 1, 1)
