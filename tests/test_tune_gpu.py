"""Autotuner: tuned settings come from the candidate sets, are used by
default afterwards, and never change results."""
import numpy as np
import pytest

import graphgen as gg
import oracle

pytestmark = pytest.mark.gpu


def test_prior_from_degree_statistics(cuda_lib):
    gr = cuda_lib
    r, c = gg.grid(40, p_del=0.05, seed=4)
    with gr.gr_graph_create(r, c) as g:
        t = gr.gr_tuned_opts(g)
        assert t["direction"] == gr.GR_DIR_PUSH and t["blocks_per_sm"] == 1
    r, c = gg.rmat(12, 16, seed=2)
    with gr.gr_graph_create(r, c) as g:
        t = gr.gr_tuned_opts(g)
        assert t["direction"] == gr.GR_DIR_AUTO


@pytest.mark.parametrize("kind", ["rmat", "grid"])
def test_autotune_keeps_results(cuda_lib, kind):
    import torch
    gr = cuda_lib
    if kind == "rmat":
        r, c = gg.rmat(15, 16, seed=3)
    else:
        r, c = gg.grid(120, p_del=0.05, seed=4)
    w = gg.weights(r, c, seed=9)
    srcs = gg.sources(r, 4, seed=1)
    with gr.gr_graph_create(r, c, w) as g:
        gr.gr_autotune(g, srcs, gr.GR_TUNE_BFS | gr.GR_TUNE_SSSP)
        t = gr.gr_tuned_opts(g)
        assert t["mode"] in (gr.GR_MODE_PERSISTENT, gr.GR_MODE_GRAPH)
        assert t["blocks_per_sm"] in (0, 1, 2)
        assert t["bfs_ms"] > 0 and t["sssp_ms"] > 0
        # the bucket width is one of the tuner's candidates: multiples of
        # the mean weight, or a single bucket
        mw = max(1.0, int(w.sum(dtype=np.uint64)) / w.size)
        cands = {int(max(1.0, min(4.0e9, f * mw))) for f in (0.5, 1, 2, 4, 8, 32, 64)}
        assert t["delta"] in cands | {0xFFFFFFFF}
        for s in list(srcs) + [int(gg.sources(r, 8, seed=5)[-1])]:
            d = torch.empty(g.n, dtype=torch.int32, device="cuda")
            gr.gr_bfs(g, int(s), d, None)
            dist = torch.empty(g.n, dtype=torch.int32, device="cuda")
            gr.gr_sssp(g, int(s), dist, None)
            torch.cuda.synchronize()
            assert np.array_equal(d.cpu().numpy(), oracle.bfs(r, c, int(s))[0])
            assert np.array_equal(dist.cpu().numpy().view(np.uint32),
                                  oracle.sssp(r, c, w, int(s))[0])


def test_autotune_bad_args(cuda_lib):
    gr = cuda_lib
    r, c = gg.rmat(8, 4, seed=1)
    with gr.gr_graph_create(r, c) as g:
        for srcs, what in [([], 1), ([g.n], 1), ([0], 8), ([0], gr.GR_TUNE_SSSP)]:
            with pytest.raises(gr.GrError) as ei:
                gr.gr_autotune(g, srcs, what)
            assert ei.value.status == gr.GR_EINVAL
