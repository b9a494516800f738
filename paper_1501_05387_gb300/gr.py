"""Python binding of libgr.so, the C ABI declared in include/gr.h.

Argument marshalling only: every step of every primitive runs in the CUDA
library. Functions keep the C names; tensors (torch, CUDA or pinned host) or
numpy arrays are passed as raw pointers together with the current torch
stream. A missing libgr.so raises ImportError: there is no fallback.
"""
from __future__ import annotations

import atexit
import ctypes
import os
import weakref

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# GR_LIBRARY selects another build of the same ABI (the GR_CHECKED
# diagnostic build, libgr_checked.so); default: libgr.so next to this file
LIB_PATH = os.environ.get("GR_LIBRARY") or os.path.join(_HERE, "libgr.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(
        f"{LIB_PATH} is not built; run paper_1501_05387_gb300.build.build() "
        "(or __graft_entry__.build()) first")

_lib = ctypes.CDLL(LIB_PATH)

GR_OK, GR_EINVAL, GR_ENOMEM, GR_ECUDA, GR_ETIMEOUT, GR_EBUSY = range(6)
STATUS_NAMES = {0: "GR_OK", 1: "GR_EINVAL", 2: "GR_ENOMEM", 3: "GR_ECUDA",
                4: "GR_ETIMEOUT", 5: "GR_EBUSY"}
GR_DIR_AUTO, GR_DIR_PUSH, GR_DIR_PULL = 0, 1, 2
GR_MODE_AUTO, GR_MODE_LAUNCH, GR_MODE_GRAPH, GR_MODE_PERSISTENT = 0, 1, 2, 3
GR_QUERY_BFS, GR_QUERY_SSSP, GR_QUERY_CC = 0, 1, 2
GR_NOALLOC_INCOMPLETE = -2
GR_REDUCE_SUM, GR_REDUCE_WSUM, GR_REDUCE_MIN, GR_REDUCE_MAX = 0, 1, 2, 3
GR_TUNE_BFS, GR_TUNE_SSSP = 1, 2


class gr_opts(ctypes.Structure):
    _fields_ = [("direction", ctypes.c_int32), ("mode", ctypes.c_int32),
                ("block", ctypes.c_int32), ("chunk", ctypes.c_int32),
                ("alpha", ctypes.c_float), ("beta", ctypes.c_float),
                ("delta", ctypes.c_uint32), ("max_iters", ctypes.c_int32)]


class GrError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        msg = _lib.gr_last_error().decode(errors="replace")
        super().__init__(f"{where}: {STATUS_NAMES.get(status, status)}: {msg}")


_vp, _i32, _i64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
_P = ctypes.POINTER


def _sig(name, args, res=ctypes.c_int):
    f = getattr(_lib, name)
    f.argtypes = args
    f.restype = res
    return f


_sig("gr_last_error", [], ctypes.c_char_p)
_sig("gr_graph_create", [_i32, _i64, _vp, _vp, _vp, ctypes.c_int, _vp, _P(_vp)])
_sig("gr_graph_destroy", [_vp])
_sig("gr_graph_info", [_vp, _P(_i32), _P(_i64), _P(_i32), _P(_i32), _P(_i32), _P(_i32)])
_sig("gr_bfs", [_vp, _i32, _vp, _vp, _P(gr_opts), _vp])
_sig("gr_bfs_multi", [_vp, _i32, _vp, _vp, _vp, _P(gr_opts), _vp])
_sig("gr_bfs_stats", [_vp, _P(_i32), _P(_i32)])
_sig("gr_bfs_trace", [_vp, _i32, _vp, _vp, _vp, _vp, _P(_i32)])
_sig("gr_sssp", [_vp, _i32, _vp, _vp, _P(gr_opts), _vp])
_sig("gr_sssp_pull_stats", [_vp, _P(_i32)])
_sig("gr_sssp_stats", [_vp, _P(_i32), _P(_i32), _P(_i64)])
_sig("gr_bfs_batch", [_vp, _vp, _i32, _vp, _P(gr_opts), _vp])
_sig("gr_bfs_batch_stats", [_vp, _P(_i32)])
_sig("gr_sssp_batch", [_vp, _vp, _i32, _vp, _P(gr_opts), _vp])
_sig("gr_sssp_batch_stats", [_vp, _P(_i32), _P(_i32), _P(_i64)])
_sig("gr_bc", [_vp, _vp, _i32, _vp, _P(gr_opts), _vp])
_sig("gr_autotune", [_vp, _vp, _i32, _i32, _vp])
_sig("gr_tuned_opts", [_vp, _P(gr_opts), _P(ctypes.c_double), _P(ctypes.c_double)])
_sig("gr_tuned_sssp", [_vp, _P(_i32), _P(_i32), _P(ctypes.c_uint32)])
_sig("gr_diag_wait_timeout", [_i64, _vp])
_sig("gr_diag_fail_alloc", [_i64])
_sig("gr_diag_guard", [_P(_i32), _P(_i64), _P(_i64)])
_sig("gr_server_create", [ctypes.c_size_t, _i32, _i32, _P(_vp)])
_sig("gr_server_add_graph", [_vp, _vp, _i32, _P(_i32)])
_sig("gr_server_submit", [_vp, _i32, _i32, _i32, _vp, _P(ctypes.c_uint64)])
_sig("gr_server_wait", [_vp, ctypes.c_uint64, _i32, _P(ctypes.c_double)])
_sig("gr_server_drain", [_vp, _i32])
_sig("gr_server_stats", [_vp, _P(_i64), _P(_i64), _P(_i64), _P(ctypes.c_double),
                         _P(ctypes.c_double), _P(ctypes.c_double), _P(ctypes.c_double)])
_sig("gr_server_destroy", [_vp])
_sig("gr_bfs_noalloc", [_i32, _i64, _vp, _vp, _i32, _vp, _vp, _vp])
_sig("gr_neighbor_reduce", [_vp, _i32, _vp, _i32, _vp, _vp, _vp])
_sig("gr_hits", [_vp, _i32, _i32, ctypes.c_double, _vp, _P(_i32), _vp])
_sig("gr_salsa", [_vp, _i32, _i32, ctypes.c_double, _vp, _P(_i32), _vp])
_sig("gr_ppr", [_vp, _vp, _i32, ctypes.c_double, _i32, ctypes.c_double, _vp, _P(_i32), _vp])
_sig("gr_cc", [_vp, _vp, _P(_i32), _P(gr_opts), _vp])
_sig("gr_pagerank", [_vp, ctypes.c_float, _i32, ctypes.c_double, _vp, _P(_i32),
                     _P(gr_opts), _vp])


def _check(status: int, where: str):
    if status != GR_OK:
        raise GrError(status, where)


def _is_torch(x) -> bool:
    return type(x).__module__.startswith("torch")


def _ptr(x, dtype=None):
    """Raw pointer of a contiguous torch tensor or numpy array (or None)."""
    if x is None:
        return None
    if _is_torch(x):
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return x.data_ptr()
    if isinstance(x, np.ndarray):
        if not x.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        if dtype is not None and x.dtype != dtype:
            raise TypeError(f"expected {dtype}, got {x.dtype}")
        return x.ctypes.data
    if isinstance(x, int):
        return x
    raise TypeError(f"unsupported buffer type {type(x)}")


def _on_device(x) -> bool:
    return _is_torch(x) and x.is_cuda


def _stream(stream):
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available():
                return torch.cuda.current_stream().cuda_stream
        except Exception:
            pass
        return None
    if hasattr(stream, "cuda_stream"):
        return stream.cuda_stream
    return int(stream)


def _opts(opts):
    if opts is None:
        return None
    if isinstance(opts, gr_opts):
        return ctypes.byref(opts)
    o = gr_opts()
    for k, v in dict(opts).items():
        setattr(o, k, v)
    return ctypes.byref(o)


class Graph:
    """Owning wrapper of a gr_graph handle."""

    def __init__(self, handle: int, n: int, m: int):
        self.handle = handle
        self.n = n
        self.m = m

    def close(self):
        if self.handle:
            _lib.gr_graph_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def gr_graph_create(row_off, col, w=None, stream=None) -> Graph:
    """Create a graph from a CSR held in numpy arrays (host) or torch tensors
    (all on the device or all on the host)."""
    n = int(row_off.shape[0]) - 1
    m = int(col.shape[0])
    dev = _on_device(row_off)
    if dev != _on_device(col) or (w is not None and dev != _on_device(w)):
        raise ValueError("row_off, col and w must all be on the host or all on the device")
    out = _vp()
    st = _lib.gr_graph_create(n, m, _ptr(row_off, np.int32), _ptr(col, np.int32),
                              _ptr(w, np.uint32), int(dev), _stream(stream),
                              ctypes.byref(out))
    _check(st, "gr_graph_create")
    return Graph(out.value, n, m)


def gr_graph_destroy(g: Graph):
    g.close()


def gr_graph_info(g: Graph) -> dict:
    n, mx, iso, sym, hw = _i32(), _i32(), _i32(), _i32(), _i32()
    m = _i64()
    _check(_lib.gr_graph_info(g.handle, ctypes.byref(n), ctypes.byref(m), ctypes.byref(mx),
                              ctypes.byref(iso), ctypes.byref(sym), ctypes.byref(hw)),
           "gr_graph_info")
    return {"n": n.value, "m": m.value, "max_degree": mx.value,
            "num_isolated": iso.value, "symmetric": bool(sym.value),
            "has_weights": bool(hw.value)}


def gr_bfs(g: Graph, src: int, depth, parent=None, opts=None, stream=None):
    """BFS from src into depth[n] (and parent[n] if given), int32."""
    _check(_lib.gr_bfs(g.handle, int(src), _ptr(depth, np.int32), _ptr(parent, np.int32),
                       _opts(opts), _stream(stream)), "gr_bfs")


def gr_bfs_multi(g: Graph, srcs, depths, parents=None, opts=None, stream=None):
    """len(srcs) searches, each as gr_bfs, into depths[i] (and parents[i]
    when parents is given; an entry may be None). Host outputs are copied
    out while the next search runs."""
    srcs = np.ascontiguousarray(np.asarray(srcs, dtype=np.int32))
    k = int(srcs.size)
    if len(depths) != k or (parents is not None and len(parents) != k):
        raise ValueError("one depth (and parent) output per source")
    dp = (ctypes.c_void_p * max(k, 1))(*[_ptr(d, np.int32) for d in depths])
    pp = None
    if parents is not None:
        pp = (ctypes.c_void_p * max(k, 1))(*[_ptr(p, np.int32) for p in parents])
    _check(_lib.gr_bfs_multi(g.handle, k, srcs.ctypes.data if k else None, dp, pp,
                             _opts(opts), _stream(stream)), "gr_bfs_multi")


def gr_bfs_stats(g: Graph):
    lv, pl = _i32(), _i32()
    _check(_lib.gr_bfs_stats(g.handle, ctypes.byref(lv), ctypes.byref(pl)), "gr_bfs_stats")
    return lv.value, pl.value


def gr_bfs_trace(g: Graph, cap: int = 64):
    """Per-level trace of the last BFS: list of (dir, frontier, edges, end_us)."""
    d = np.zeros(cap, np.int32)
    f = np.zeros(cap, np.int32)
    e = np.zeros(cap, np.int64)
    t = np.zeros(cap, np.float64)
    nl = _i32()
    _check(_lib.gr_bfs_trace(g.handle, cap, d.ctypes.data, f.ctypes.data, e.ctypes.data,
                             t.ctypes.data, ctypes.byref(nl)), "gr_bfs_trace")
    k = min(cap, nl.value)
    return [(int(d[i]), int(f[i]), int(e[i]), float(t[i])) for i in range(k)]


def gr_sssp(g: Graph, src: int, dist, pred=None, opts=None, stream=None):
    """SSSP from src into dist[n] (uint32; torch.int32 tensors are accepted
    and hold the same bits) and pred[n] (int32) if given."""
    _check(_lib.gr_sssp(g.handle, int(src), _ptr(dist, np.uint32), _ptr(pred, np.int32),
                        _opts(opts), _stream(stream)), "gr_sssp")


def gr_sssp_stats(g: Graph):
    it, ph = _i32(), _i32()
    rl = _i64()
    _check(_lib.gr_sssp_stats(g.handle, ctypes.byref(it), ctypes.byref(ph), ctypes.byref(rl)),
           "gr_sssp_stats")
    return it.value, ph.value, rl.value


def gr_sssp_pull_stats(g: Graph) -> int:
    """Relaxations of the last gr_sssp on g that ran in pull form."""
    p = _i32()
    _check(_lib.gr_sssp_pull_stats(g.handle, ctypes.byref(p)), "gr_sssp_pull_stats")
    return p.value


def gr_sssp_batch(g: Graph, srcs, dist, opts=None, stream=None):
    """k SSSP searches (k = len(srcs), up to 64) in one run into dist[k*n]
    (uint32, source-major; torch.int32 tensors hold the same bits)."""
    srcs = np.ascontiguousarray(np.asarray(srcs, dtype=np.int32))
    _check(_lib.gr_sssp_batch(g.handle, srcs.ctypes.data if srcs.size else None,
                              int(srcs.size), _ptr(dist, np.uint32), _opts(opts),
                              _stream(stream)), "gr_sssp_batch")


def gr_sssp_batch_stats(g: Graph):
    it, ph = _i32(), _i32()
    rl = _i64()
    _check(_lib.gr_sssp_batch_stats(g.handle, ctypes.byref(it), ctypes.byref(ph),
                                    ctypes.byref(rl)), "gr_sssp_batch_stats")
    return it.value, ph.value, rl.value


def gr_bfs_batch(g: Graph, srcs, depth, opts=None, stream=None):
    """Batched BFS from up to 64 sources into depth[k*n] (int32,
    source-major)."""
    srcs = np.ascontiguousarray(np.asarray(srcs, dtype=np.int32))
    _check(_lib.gr_bfs_batch(g.handle, srcs.ctypes.data, int(srcs.size), _ptr(depth, np.int32),
                             _opts(opts), _stream(stream)), "gr_bfs_batch")


def gr_bfs_batch_stats(g: Graph) -> int:
    """Levels of the last batched BFS on g (synchronises; GrError with
    GR_ETIMEOUT if it stopped at a device-side limit)."""
    lv = _i32()
    _check(_lib.gr_bfs_batch_stats(g.handle, ctypes.byref(lv)), "gr_bfs_batch_stats")
    return lv.value


def gr_bc(g: Graph, srcs, bc, opts=None, stream=None):
    """Brandes BC summed over srcs (no halving, no normalisation) into
    bc[n] (float64)."""
    srcs = np.ascontiguousarray(np.asarray(srcs, dtype=np.int32))
    _check(_lib.gr_bc(g.handle, srcs.ctypes.data if srcs.size else None, int(srcs.size),
                      _ptr(bc, np.float64), _opts(opts), _stream(stream)), "gr_bc")


def gr_bfs_noalloc(row_off, col, src: int, depth, parent=None, stream=None):
    """BFS without any device allocation (see include/gr.h): row_off, col,
    depth and parent are contiguous int32 CUDA tensors on the current device,
    owned by the caller; depth and parent hold at least n entries. The C
    entry point does not validate the CSR and reads these pointers on the
    device, so their types, device and sizes are checked here."""
    import torch
    dev = torch.cuda.current_device()
    for name, t in (("row_off", row_off), ("col", col), ("depth", depth), ("parent", parent)):
        if t is None and name == "parent":
            continue
        if not _is_torch(t) or not t.is_cuda or t.device.index != dev:
            raise ValueError(f"{name} must be a CUDA tensor on the current device (cuda:{dev})")
        if t.dtype != torch.int32 or not t.is_contiguous() or t.dim() != 1:
            raise ValueError(f"{name} must be a contiguous 1-D int32 tensor")
    n = int(row_off.shape[0]) - 1
    if n < 1:
        raise ValueError("row_off must hold n + 1 >= 2 entries")
    if depth.numel() < n or (parent is not None and parent.numel() < n):
        raise ValueError(f"depth and parent must hold at least n = {n} entries")
    _check(_lib.gr_bfs_noalloc(n, int(col.shape[0]), _ptr(row_off), _ptr(col), int(src),
                               _ptr(depth), _ptr(parent), _stream(stream)), "gr_bfs_noalloc")


def gr_neighbor_reduce(g: Graph, op: int, x, out, frontier=None, stream=None):
    """out[v] = sum / weighted sum (float64) or min / max (int32) of x[u]
    over the entries (v, u) of v's row, for every vertex or the distinct
    vertices of a device int32 frontier tensor."""
    q = 0 if frontier is None else int(frontier.numel())
    if frontier is not None and q == 0:
        return  # an empty frontier reduces nothing (its data pointer may be NULL)
    _check(_lib.gr_neighbor_reduce(g.handle, int(op), _ptr(frontier), q, _ptr(x), _ptr(out),
                                   _stream(stream)), "gr_neighbor_reduce")


def gr_hits(g: Graph, n_left: int, score, max_iter=100, tol=1e-10, stream=None, count=True):
    """HITS hub (on [0, n_left)) and authority scores into score[n]
    (float64); returns the iterations run (synchronises) when count."""
    it = _i32()
    _check(_lib.gr_hits(g.handle, int(n_left), int(max_iter), float(tol), _ptr(score),
                        ctypes.byref(it) if count else None, _stream(stream)), "gr_hits")
    return it.value if count else None


def gr_salsa(g: Graph, n_left: int, score, max_iter=100, tol=1e-10, stream=None, count=True):
    """SALSA hub and authority scores into score[n] (float64)."""
    it = _i32()
    _check(_lib.gr_salsa(g.handle, int(n_left), int(max_iter), float(tol), _ptr(score),
                         ctypes.byref(it) if count else None, _stream(stream)), "gr_salsa")
    return it.value if count else None


def gr_ppr(g: Graph, seeds, rank, damping=0.85, max_iter=50, tol=1e-7, stream=None,
           count=True):
    """Personalized PageRank from distinct seeds into rank[n] (float64)."""
    seeds = np.ascontiguousarray(np.asarray(seeds, dtype=np.int32))
    it = _i32()
    _check(_lib.gr_ppr(g.handle, seeds.ctypes.data, int(seeds.size), float(damping),
                       int(max_iter), float(tol), _ptr(rank),
                       ctypes.byref(it) if count else None, _stream(stream)), "gr_ppr")
    return it.value if count else None


def gr_cc(g: Graph, label, opts=None, stream=None, count=True):
    """CC labels (int32, smallest vertex id per component) into label[n];
    returns the number of components (synchronises) when count is true."""
    k = _i32()
    _check(_lib.gr_cc(g.handle, _ptr(label, np.int32), ctypes.byref(k) if count else None,
                      _opts(opts), _stream(stream)), "gr_cc")
    return k.value if count else None


def gr_pagerank(g: Graph, rank, damping=0.85, max_iter=50, tol=1e-7, opts=None,
                stream=None, count=True):
    """PageRank (float32) into rank[n]; returns the iterations run
    (synchronises) when count is true."""
    it = _i32()
    _check(_lib.gr_pagerank(g.handle, float(damping), int(max_iter), float(tol),
                            _ptr(rank, np.float32), ctypes.byref(it) if count else None,
                            _opts(opts), _stream(stream)), "gr_pagerank")
    return it.value if count else None


def gr_autotune(g: Graph, srcs, what: int = 1, stream=None):
    """Measure candidate settings on sample sources; keep the fastest."""
    srcs = np.ascontiguousarray(np.asarray(srcs, dtype=np.int32))
    _check(_lib.gr_autotune(g.handle, srcs.ctypes.data, int(srcs.size), int(what),
                            _stream(stream)), "gr_autotune")


def gr_tuned_opts(g: Graph):
    o = gr_opts()
    b, s = ctypes.c_double(), ctypes.c_double()
    _check(_lib.gr_tuned_opts(g.handle, ctypes.byref(o), ctypes.byref(b), ctypes.byref(s)),
           "gr_tuned_opts")
    return {"mode": o.mode, "direction": o.direction, "alpha": o.alpha, "beta": o.beta, "blocks_per_sm": o.block,
            "delta": o.delta, "bfs_ms": b.value, "sssp_ms": s.value}


def gr_tuned_sssp(g: Graph):
    m, b = _i32(), _i32()
    d = ctypes.c_uint32()
    _check(_lib.gr_tuned_sssp(g.handle, ctypes.byref(m), ctypes.byref(b), ctypes.byref(d)),
           "gr_tuned_sssp")
    return {"mode": m.value, "blocks_per_sm": b.value, "delta": d.value}


_live_servers = weakref.WeakSet()


@atexit.register
def _close_servers():
    # join every server's workers before the interpreter exits, so that no
    # device work is in flight when the process ends
    for srv in list(_live_servers):
        try:
            srv.close()
        except Exception:
            pass


class Server:
    """Owning wrapper of a gr_server handle."""

    def __init__(self, handle: int):
        self.handle = handle
        self.graphs = []  # keep the graphs alive as long as the server
        _live_servers.add(self)

    def close(self):
        if self.handle:
            _lib.gr_server_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def gr_server_create(budget_bytes: int, num_slots: int = 1, max_batch: int = 64) -> Server:
    out = _vp()
    _check(_lib.gr_server_create(int(budget_bytes), int(num_slots), int(max_batch),
                                 ctypes.byref(out)), "gr_server_create")
    return Server(out.value)


def gr_server_add_graph(s: Server, g: Graph, batchable: int = 1) -> int:
    """Register g; batchable = the number of queued same-graph BFS requests
    from which they run as lanes of one batch (0: never; True counts as 1)."""
    gid = _i32()
    _check(_lib.gr_server_add_graph(s.handle, g.handle, int(batchable), ctypes.byref(gid)),
           "gr_server_add_graph")
    s.graphs.append(g)
    return gid.value


def gr_server_submit(s: Server, graph_id: int, kind: int, src: int = 0, out=None) -> int:
    t = ctypes.c_uint64()
    _check(_lib.gr_server_submit(s.handle, int(graph_id), int(kind), int(src), _ptr(out),
                                 ctypes.byref(t)), "gr_server_submit")
    return t.value


def gr_server_wait(s: Server, ticket: int, timeout_ms: int = -1) -> float:
    lat = ctypes.c_double()
    _check(_lib.gr_server_wait(s.handle, ctypes.c_uint64(ticket), int(timeout_ms),
                               ctypes.byref(lat)), "gr_server_wait")
    return lat.value


def gr_server_drain(s: Server, timeout_ms: int = -1):
    _check(_lib.gr_server_drain(s.handle, int(timeout_ms)), "gr_server_drain")


def gr_server_stats(s: Server) -> dict:
    c, f, l = _i64(), _i64(), _i64()
    q, p50, p99, mb = (ctypes.c_double() for _ in range(4))
    _check(_lib.gr_server_stats(s.handle, ctypes.byref(c), ctypes.byref(f), ctypes.byref(l),
                                ctypes.byref(q), ctypes.byref(p50), ctypes.byref(p99),
                                ctypes.byref(mb)), "gr_server_stats")
    return {"completed": c.value, "failed": f.value, "launches": l.value, "qps": q.value,
            "p50_ms": p50.value, "p99_ms": p99.value, "mean_batch": mb.value}


def gr_server_destroy(s: Server):
    s.close()


def gr_diag_wait_timeout(spin_limit: int, stream=None):
    _check(_lib.gr_diag_wait_timeout(int(spin_limit), _stream(stream)), "gr_diag_wait_timeout")


def gr_diag_guard():
    site, idx, bound = _i32(), _i64(), _i64()
    _check(_lib.gr_diag_guard(ctypes.byref(site), ctypes.byref(idx), ctypes.byref(bound)),
           "gr_diag_guard")
    return site.value, idx.value, bound.value


def gr_diag_fail_alloc(after: int):
    _check(_lib.gr_diag_fail_alloc(int(after)), "gr_diag_fail_alloc")


def gr_last_error() -> str:
    return _lib.gr_last_error().decode(errors="replace")
