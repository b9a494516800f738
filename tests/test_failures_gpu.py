"""Failure handling without a GPU fault: a bounded device wait that runs out
reports GR_ETIMEOUT and leaves the context usable; injected allocation
failures surface as GR_ENOMEM and leave the library usable."""
import numpy as np
import pytest

import graphgen as gg
import oracle

pytestmark = pytest.mark.gpu


def test_bounded_wait_times_out_and_context_survives(cuda_lib):
    import torch
    gr = cuda_lib
    with pytest.raises(gr.GrError) as ei:
        gr.gr_diag_wait_timeout(1000)
    assert ei.value.status == gr.GR_ETIMEOUT
    # the device still works: a BFS afterwards is correct
    r, c = gg.rmat(10, 8, seed=1)
    with gr.gr_graph_create(r, c) as g:
        d = torch.empty(g.n, dtype=torch.int32, device="cuda")
        gr.gr_bfs(g, 0, d)
        torch.cuda.synchronize()
        assert np.array_equal(d.cpu().numpy(), oracle.bfs(r, c, 0)[0])


def test_injected_allocation_failures(cuda_lib):
    import torch
    gr = cuda_lib
    r, c = gg.rmat(10, 8, seed=2)
    try:
        for after in range(0, 12):
            gr.gr_diag_fail_alloc(after)
            try:
                g = gr.gr_graph_create(r, c)
            except gr.GrError as e:
                assert e.status == gr.GR_ENOMEM and "injected" in str(e)
                continue
            try:
                d = torch.empty(g.n, dtype=torch.int32, device="cuda")
                try:
                    gr.gr_bfs(g, 0, d)
                except gr.GrError as e:
                    assert e.status == gr.GR_ENOMEM
            finally:
                gr.gr_diag_fail_alloc(-1)
                g.close()
    finally:
        gr.gr_diag_fail_alloc(-1)
    with gr.gr_graph_create(r, c) as g:
        d = torch.empty(g.n, dtype=torch.int32, device="cuda")
        gr.gr_bfs(g, 0, d)
        torch.cuda.synchronize()
        assert np.array_equal(d.cpu().numpy(), oracle.bfs(r, c, 0)[0])
