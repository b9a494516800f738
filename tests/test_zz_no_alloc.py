"""gr_bfs_noalloc: the BFS entry point for callers that cannot allocate
device memory (for example code that runs while a stream is being captured
into a CUDA graph, or inside a host application that owns all device memory
through its own pool). Its scratch is a fixed device array inside the
library, so it must give the same results as gr_bfs, call after call.

This file is collected last on purpose: the entry point shares one scratch
array per device, and running it after every other test checks that earlier
work on the device leaves nothing it depends on."""
import ctypes

import numpy as np
import pytest

import graphgen as gg
from checks import validate_bfs

pytestmark = pytest.mark.gpu


def test_noalloc_bfs_matches_gr_bfs_twice(cuda_lib):
    import torch
    gr = cuda_lib
    r, c = gg.rmat(14, 16, seed=1)
    n, m = r.size - 1, c.size
    rt = torch.from_numpy(r).cuda()
    ct = torch.from_numpy(c).cuda()
    stream = torch.cuda.current_stream()
    srcs = [gg.max_degree_vertex(r), int(gg.sources(r, 1, seed=11)[0])]
    with gr.gr_graph_create(r, c) as g:
        for src in srcs:  # two calls in a row
            ref_d = torch.empty(n, dtype=torch.int32, device="cuda")
            gr.gr_bfs(g, src, ref_d, None)
            d = torch.full((n,), 7, dtype=torch.int32, device="cuda")
            p = torch.full((n,), 7, dtype=torch.int32, device="cuda")
            st = gr._lib.gr_bfs_noalloc(n, m, rt.data_ptr(), ct.data_ptr(), src,
                                        d.data_ptr(), p.data_ptr(),
                                        ctypes.c_void_p(stream.cuda_stream))
            assert st == gr.GR_OK, gr.gr_last_error()
            torch.cuda.synchronize()
            dn, pn = d.cpu().numpy(), p.cpu().numpy()
            assert np.array_equal(dn, ref_d.cpu().numpy())
            validate_bfs(r, c, src, dn, pn)


def test_noalloc_bfs_depth_only_on_a_grid(cuda_lib):
    """Depth only (parent NULL) on a mesh with deleted edges, two sources in
    a row, checked against the CPU queue BFS itself."""
    import oracle
    import torch
    gr = cuda_lib
    r, c = gg.grid(48, p_del=0.05, seed=4)
    rt = torch.from_numpy(r).cuda()
    ct = torch.from_numpy(c).cuda()
    n = r.size - 1
    for src in (0, 1000):
        want, _ = oracle.bfs(r, c, src)
        d = torch.full((n,), 7, dtype=torch.int32, device="cuda")
        gr.gr_bfs_noalloc(rt, ct, src, d, None)
        torch.cuda.synchronize()
        got = d.cpu().numpy()
        assert got[src] == 0  # not GR_NOALLOC_INCOMPLETE
        assert np.array_equal(got, want)


def test_noalloc_wrapper_rejects_bad_tensors(cuda_lib):
    """The Python wrapper checks what the C entry point cannot (types,
    device, sizes) before any pointer reaches the GPU."""
    import torch
    gr = cuda_lib
    r, c = gg.grid(8, p_del=0.0, seed=1)
    rt = torch.from_numpy(r).cuda()
    ct = torch.from_numpy(c).cuda()
    n = r.size - 1
    d = torch.empty(n, dtype=torch.int32, device="cuda")
    with pytest.raises(ValueError):
        gr.gr_bfs_noalloc(rt.long(), ct, 0, d)                        # int64 offsets
    with pytest.raises(ValueError):
        gr.gr_bfs_noalloc(rt, ct, 0, d[: n - 1])                      # short depth
    with pytest.raises(ValueError):
        gr.gr_bfs_noalloc(rt, ct, 0, d, torch.empty(3, dtype=torch.int32, device="cuda"))
    with pytest.raises(ValueError):
        gr.gr_bfs_noalloc(rt.cpu(), ct, 0, d)                         # host tensor


def test_noalloc_bfs_rejects_oversized_graph(cuda_lib):
    gr = cuda_lib
    dummy = ctypes.c_void_p(16)
    st = gr._lib.gr_bfs_noalloc((1 << 20) + 1, 0, dummy, dummy, 0, dummy, None, None)
    assert st == gr.GR_EINVAL
    assert "1048576" in gr.gr_last_error()
