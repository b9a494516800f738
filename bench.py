"""Benchmark: BFS GTEPS on R-MAT scale 22 (edge factor 16, seed 2, 16 random
non-isolated sources), with the HBM roofline fraction of the BFS level loop,
an end-to-end number through the C ABI with host buffers, and the CPU oracle
as a reported baseline.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gr|reference]

A step is 16 BFS traversals (one per source) with depth and parent outputs.
TEPS follow the paper's convention (Sec. 6, Table 3): edges of the whole
graph (directed CSR entries) per traversal time. The L2 cache is flushed by
writing a 256 MB buffer before every step, outside the timed events.
Under torchrun (N > 1) every rank runs the same 16 traversals on its own GPU
(replicas, weak scaling) and the slowest rank's time is reported.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

SCALE, EDGE_FACTOR, GRAPH_SEED, SOURCE_SEED, NUM_SOURCES = 22, 16, 2, 2, 16
WORKLOAD = "rmat22_bfs"
METRIC = "BFS GTEPS (R-MAT s22, 16 sources)"
L2_FLUSH_BYTES = 256 << 20

# DRAM traffic of one traversal (k_bfs_init + k_bfs_do), from one ncu capture
# (dram__bytes_read.sum + dram__bytes_write.sum) of the 16 timed traversals
# of this benchmark at R-MAT s21 with cold caches, scaled to other scales by
# the edge count. It is reported only while the traversal's sources hash to
# the value they had when it was measured (null after any change).
TRAFFIC_S21 = {"bytes_per_traversal": 42946576, "m": 63540402,
               "sources_sha256": "8bc6ed50d34737c70fca1725f04d33978108aaa840032d1a7ffaeac6703dc284"}
TRAFFIC_SOURCES = ("paper_1501_05387_gb300/csrc/bfs.cu", "paper_1501_05387_gb300/csrc/advance.cuh",
                   "paper_1501_05387_gb300/csrc/gr_internal.cuh")


def traversal_sources_sha256():
    import hashlib
    h = hashlib.sha256()
    for f in TRAFFIC_SOURCES:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def measured_traffic(m):
    t = TRAFFIC_S21
    if t["bytes_per_traversal"] is None or t["sources_sha256"] != traversal_sources_sha256():
        return None
    return t["bytes_per_traversal"] * m / t["m"]


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gr", choices=["gr", "reference"])
    ap.add_argument("--cpu-sample-sources", type=int, default=8)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--serving", action="store_true",
                    help="run the query-server benchmark (plain vs continuous batching) also "
                         "with more than one rank (at N=1 it runs unless --no-serving)")
    ap.add_argument("--no-serving", action="store_true",
                    help="skip the query-server benchmark")
    ap.add_argument("--serving-requests", type=int, default=1000)
    ap.add_argument("--serving-full", action="store_true",
                    help="serve 20000 requests over the 24-graph pool (slow)")
    ap.add_argument("--suite", action="store_true",
                    help="instead of the BFS line, measure every primitive on its workload "
                         "(SSSP s22, grid 4096^2 BFS/SSSP/CC, s23 PageRank/CC/BC/batched BFS)")
    ap.add_argument("--suite-part", default="all",
                    choices=["all", "sssp", "grid", "rmat", "pagerank", "cc", "bfs64", "bc64",
                             "reduce", "bipartite"],
                    help="run one part of the suite (profiling runs)")
    ap.add_argument("--suite-scale", type=int, default=0,
                    help="R-MAT scale of the suite part (profiling runs; 0: the specified one)")
    ap.add_argument("--scale", type=int, default=SCALE,
                    help="R-MAT scale (profiling runs only; the metric is quoted at 22)")
    ap.add_argument("--mode", default="auto", choices=["auto", "graph", "launch", "persistent"],
                    help="BFS level-loop driver (profiling runs: 'launch' exposes "
                         "every kernel to ncu)")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def max_over_ranks(x: float, world: int, device=None) -> float:
    """The slowest rank's value (a max all-reduce); x itself at N = 1."""
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(units_per_rank: float, world: int, seconds: float) -> float:
    """Whole-job rate under weak scaling: every rank processes the same
    number of units; the job takes as long as the slowest rank."""
    return world * units_per_rank / seconds


def make_inputs(scale=SCALE):
    import graphgen as gg
    r, c = gg.rmat(scale, EDGE_FACTOR, seed=GRAPH_SEED)
    srcs = gg.sources(r, NUM_SOURCES, seed=SOURCE_SEED)
    return r, c, srcs


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during a region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.dev), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.thread.join(timeout=2)
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in self.lines:
            parts = [p.strip() for p in l.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                mx = float(parts[1])
            except ValueError:
                continue
            for nm, val in zip(names, parts[3:7]):
                if val.lower() in ("active", "1", "yes"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


def bfs_bytes(r, depth_list, m):
    """Algorithmic bytes of one BFS: each column index of the reached
    vertices read once (4 B), the row offsets once (4 B each), and a depth
    and a parent write per reached vertex (8 B)."""
    out = []
    deg = np.diff(r).astype(np.int64)
    n = r.size - 1
    for d in depth_list:
        reached = d >= 0
        m_reached = int(deg[reached].sum())
        out.append(4 * m_reached + 4 * (n + 1) + 8 * int(reached.sum()))
    return out


# ----------------------------------------------------------------- serving
def serving_pool(full: bool):
    """The resident graph pool: R-MAT graphs (a,b,c) = (0.57,0.19,0.19) and
    grids with 5 % deletions, uint32 weights in [1, 64]. full=True is the
    24-graph pool (12 R-MAT scale 16 + i mod 7, edge factor 8/16/32 by i mod
    3, seed 100 + i; 12 grids of side 512/1024/2048/4096 x 3 deletion seeds);
    otherwise a 6-graph subset that builds in seconds."""
    import graphgen as gg
    specs = []
    if full:
        for i in range(12):
            specs.append(("rmat", 16 + i % 7, (8, 16, 32)[i % 3], 100 + i))
        for j, side in enumerate([512, 1024, 2048, 4096]):
            for k in range(3):
                specs.append(("grid", side, 0, 200 + 3 * j + k))
    else:
        specs = [("rmat", 16, 8, 100), ("rmat", 18, 16, 101), ("rmat", 20, 16, 102),
                 ("rmat", 17, 32, 103), ("grid", 512, 0, 200), ("grid", 1024, 0, 201)]
    out = []
    for kind, a, b, seed in specs:
        if kind == "rmat":
            r, c = gg.rmat(a, b, seed=seed)
        else:
            r, c = gg.grid(a, p_del=0.05, seed=seed)
        w = gg.weights(r, c, seed=seed + 1000, wmin=1, wmax=64)
        out.append((kind, a, b, seed, r, c, w))
    return out


def serving_requests(pool, count, seed=6):
    """Seeded request mix: 60 % BFS, 30 % SSSP, 10 % CC, uniform graph, random
    non-isolated source; Poisson arrivals are drawn per run (unit rate here,
    scaled by the run's rate)."""
    rng = np.random.default_rng(seed)
    reqs = []
    for _ in range(count):
        gi = int(rng.integers(0, len(pool)))
        u = rng.random()
        kind = 0 if u < 0.6 else (1 if u < 0.9 else 2)
        r = pool[gi][4]
        deg = np.diff(r)
        while True:
            s = int(rng.integers(0, r.size - 1))
            if deg[s] > 0:
                break
        reqs.append((gi, kind, s))
    gaps = rng.exponential(1.0, size=count)
    return reqs, np.cumsum(gaps)


def run_serving(gr, graphs, batchable, reqs, unit_arrivals, rate, slots, batch, budget,
                drain_s=300.0):
    """Submit reqs at Poisson times (rate per second) to a fresh server and
    wait for all; returns the server's stats. The server is always
    destroyed (its workers joined) before returning, also on errors, so no
    device work outlives the call."""
    srv = gr.gr_server_create(budget, slots, batch)
    try:
        ids = [gr.gr_server_add_graph(srv, g, b) for g, b in zip(graphs, batchable)]
        arrivals = unit_arrivals / rate
        t0 = time.perf_counter()
        for (gi, kind, src), at in zip(reqs, arrivals):
            now = time.perf_counter() - t0
            if at > now:
                time.sleep(at - now)
            gr.gr_server_submit(srv, ids[gi], kind, src, None)
        gr.gr_server_drain(srv, int(drain_s * 1000))
        st = gr.gr_server_stats(srv)
        if st["failed"]:
            raise RuntimeError(f"{st['failed']} of {len(reqs)} requests failed: "
                               f"{gr.gr_last_error()}")
        return st
    finally:
        srv.close()


def serving_bench(gr, full=False, count=2000):
    """Plain path (no batching) vs served path (continuous batching of up to
    64 BFS or SSSP lanes per launch) on the same seeded request stream, both
    on the server's one worker slot. Every phase must complete all its
    requests."""
    slots = 1
    pool = serving_pool(full)
    graphs = [gr.gr_graph_create(r, c, w) for (_, _, _, _, r, c, w) in pool]
    try:
        # every graph batches whatever is queued (a batched traversal is one
        # persistent kernel, on grids as on R-MAT graphs)
        batchable = [1 for _ in pool]
        # per-graph tuning (BFS driver / thresholds, SSSP bucket width) on
        # one sample source each, as a deployment would do once per graph
        for (_, _, _, _, r, _, _), g in zip(pool, graphs):
            src = [int(np.argmax(np.diff(r)))]
            gr.gr_autotune(g, src, gr.GR_TUNE_BFS | gr.GR_TUNE_SSSP)
        reqs, unit = serving_requests(pool, count)
        # the budget covers result buffers and the slots' kept workspaces;
        # with batching those reach about 6 GB on the 6-graph subset and
        # about 40 GB on the 24-graph pool (batched SSSP scratch on the
        # 2048^2 and 4096^2 grids), past which admission could no longer
        # batch
        budget = (64 << 30) if full else (16 << 30)
        warm = [(gi, k, int(np.argmax(np.diff(pool[gi][4]))))
                for gi in range(len(pool)) for k in range(3)]
        for sl, batch in [(1, 1), (slots, 64)]:
            run_serving(gr, graphs, batchable, warm, np.arange(len(warm), dtype=float), 1e9,
                        sl, batch, budget)
        # throughput: both paths see the whole stream at once (saturated);
        # latency: both at 0.7x their own saturated throughput
        # a phase may take as long as its requests run one at a time on the
        # largest graphs (the 4096^2 grids' SSSP: about 70 ms each)
        drain = max(300.0, 0.1 * len(reqs))
        plain = run_serving(gr, graphs, batchable, reqs, unit, 1e9, 1, 1, budget, drain)
        served = run_serving(gr, graphs, batchable, reqs, unit, 1e9, slots, 64, budget, drain)
        plain_lat = run_serving(gr, graphs, batchable, reqs, unit, 0.7 * plain["qps"], 1, 1,
                                budget, drain)
        served_lat = run_serving(gr, graphs, batchable, reqs, unit, 0.7 * served["qps"], slots,
                                 64, budget, drain)
        # and at the plain path's latency-run load (the same arrival times;
        # the full pool skips it: its arrivals alone take as long as the
        # plain latency run)
        served_eq = None if full else run_serving(gr, graphs, batchable, reqs, unit,
                                                  0.7 * plain["qps"], slots, 64, budget, drain)
    finally:
        for g in graphs:
            g.close()
    pick = lambda st: None if st is None else {k: st[k] for k in ("qps", "p50_ms", "p99_ms",
                                                                 "mean_batch", "launches")}
    return {"requests": count, "graphs": len(pool),
            "pool": "24-graph pool" if full else "6-graph subset (R-MAT s16-s20, grids 512/1024)",
            "mix": "60/30/10 BFS/SSSP/CC, Poisson arrivals seed 6",
            "plain": {"saturated": pick(plain), "at_0.7x_capacity": pick(plain_lat)},
            "served": {"saturated": pick(served), "at_0.7x_capacity": pick(served_lat),
                       "at_plain_0.7x_load": pick(served_eq),
                       "slots": slots, "max_batch": 64,
                       "batching_depth": "BFS: whatever same-graph requests are queued, up to "
                                         "64 lanes; SSSP: whatever is queued, up to the "
                                         "graph's lane limit"},
            "speedup_qps": served["qps"] / max(plain["qps"], 1e-9)}


# ------------------------------------------------------------------- suite
def _timed_calls(fn, calls, flush, warm=1):
    """Mean CUDA-event milliseconds of fn() over `calls` calls on the current
    stream, the L2 flushed (outside the events) before each call."""
    import torch
    stream = torch.cuda.current_stream()
    for _ in range(warm):
        fn()
    torch.cuda.synchronize()
    ms = []
    for _ in range(calls):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        fn()
        b.record(stream)
        b.synchronize()
        ms.append(a.elapsed_time(b))
    return float(np.mean(ms)), ms


def _roof(bytes_per_call, ms, peak, model):
    gbs = bytes_per_call / (ms * 1e-3) / 1e9
    return {"bound": "hbm", "achieved": gbs, "peak": peak, "unit": "GB/s", "frac": gbs / peak,
            "bytes_per_call": float(bytes_per_call), "bytes_model": model}


def run_suite(args):
    """Every primitive on the workload it is specified on, timed with CUDA
    events (L2 flushed before each call), with its edge-byte roofline."""
    import torch
    import graphgen as gg
    from paper_1501_05387_gb300 import build
    build.build()
    from paper_1501_05387_gb300 import gr
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.int32, device=dev)
    try:
        peak = float(json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["hbm_gbs"])
    except Exception:
        peak = 6800.0
    out = []

    def reach_bytes(r, reached, per_edge, per_vertex):
        deg = np.diff(r).astype(np.int64)
        n = r.size - 1
        return per_edge * int(deg[reached].sum()) + 4 * (n + 1) + per_vertex * int(reached.sum())

    part = args.suite_part
    want = lambda *names: part == "all" or part in names

    # --- SSSP on R-MAT s22 (weights [1,64], seed 3), the BFS sources
    if want("sssp"):
        suite_sssp(args, gr, gg, torch, dev, flush, peak, out, reach_bytes)
    if want("grid"):
        suite_grid(args, gr, gg, torch, dev, flush, peak, out, reach_bytes)
    if want("rmat", "pagerank", "cc", "bfs64", "bc64", "reduce"):
        suite_rmat(args, gr, gg, torch, dev, flush, peak, out, want)
    if want("bipartite"):
        suite_bipartite(args, gr, gg, torch, dev, flush, peak, out)
    print(json.dumps({"suite": out, "peak_hbm_gbs": peak}), flush=True)


INF32 = 0xFFFFFFFF


def suite_sssp(args, gr, gg, torch, dev, flush, peak, out, reach_bytes):
    INF = INF32
    scale = args.suite_scale or 22
    r, c = gg.rmat(scale, 16, seed=2)
    w = gg.weights(r, c, seed=3, wmin=1, wmax=64)
    srcs = gg.sources(r, 16, seed=2)
    n, m = r.size - 1, c.size
    g = gr.gr_graph_create(r, c, w)
    # launch mode (host-enqueued iterations, one bucket as the tuner picks on
    # R-MAT s22) only for profiling runs, where the kernels must be separate
    # launches
    o = gr.gr_opts(mode=gr.GR_MODE_LAUNCH, delta=0xFFFFFFFF) if args.mode == "launch" else None
    if o is None:
        gr.gr_autotune(g, [int(np.argmax(np.diff(r)))], gr.GR_TUNE_SSSP)
    dist = torch.empty(n, dtype=torch.int32, device=dev)
    per, byts = [], []
    for s in srcs:
        ms, _ = _timed_calls(lambda: gr.gr_sssp(g, int(s), dist, opts=o), 2, flush)
        d = dist.cpu().numpy().view(np.uint32)
        per.append(ms)
        byts.append(reach_bytes(r, d != INF, 8, 4))
    mean = float(np.mean(per))
    it, ph, rl = gr.gr_sssp_stats(g)
    out.append({"workload": f"rmat{scale}_sssp", "primitive": "sssp", "calls": 2 * len(srcs),
                "last_call": {"iterations": it, "phases": ph, "edges_relaxed_per_m": rl / m},
                "ms_per_call": mean, "throughput": m / (mean * 1e-3) / 1e9, "unit": "GTEPS",
                "tuned": gr.gr_tuned_opts(g), "tuned_sssp": gr.gr_tuned_sssp(g),
                "roofline": _roof(float(np.mean(byts)), mean, peak,
                                  "8 B per column+weight entry of the reached vertices, "
                                  "4 B per row offset, 4 B per reached distance")})
    g.close()


def suite_grid(args, gr, gg, torch, dev, flush, peak, out, reach_bytes):
    INF = INF32
    # --- 4096^2 grid, 5 % deletions (seed 4), weights [1,16]: BFS, SSSP, CC
    r, c = gg.grid(4096, p_del=0.05, seed=4)
    w = gg.weights(r, c, seed=4, wmin=1, wmax=16)
    n, m = r.size - 1, c.size
    g = gr.gr_graph_create(r, c, w)
    srcs = gg.sources(r, 4, seed=4)
    depth = torch.empty(n, dtype=torch.int32, device=dev)
    parent = torch.empty(n, dtype=torch.int32, device=dev)
    per, byts, levels, single_depth = [], [], [], []
    for s in srcs:
        ms, _ = _timed_calls(lambda: gr.gr_bfs(g, int(s), depth, parent), 1, flush)
        levels.append(gr.gr_bfs_stats(g)[0])
        per.append(ms)
        d = depth.cpu().numpy()
        single_depth.append(d.copy())
        byts.append(reach_bytes(r, d >= 0, 4, 8))
    mean = float(np.mean(per))
    out.append({"workload": "grid4096_bfs", "primitive": "bfs", "calls": len(srcs),
                "ms_per_call": mean, "throughput": m / (mean * 1e-3) / 1e9, "unit": "GTEPS",
                "levels": levels, "us_per_level": 1e3 * mean / float(np.mean(levels)),
                "tuned": gr.gr_tuned_opts(g),
                "roofline": _roof(float(np.mean(byts)), mean, peak,
                                  "4 B per column entry of the reached vertices, 4 B per "
                                  "row offset, 8 B depth+parent per reached vertex")})
    # the same traversals batched: 64 sources (the four above first) as bit
    # lanes of one persistent traversal, against one at a time
    del parent
    kb = 64
    srcs_b = [int(x) for x in srcs] + [int(x) for x in gg.sources(r, kb + 8, seed=24)
                                        if int(x) not in set(int(y) for y in srcs)][:kb - len(srcs)]
    depth_b = torch.empty(kb * n, dtype=torch.int32, device=dev)
    ms_b, _ = _timed_calls(lambda: gr.gr_bfs_batch(g, srcs_b, depth_b), 1, flush)
    lv_b = gr.gr_bfs_batch_stats(g)
    db = depth_b.view(kb, n)
    equal = [bool(np.array_equal(db[i].cpu().numpy(), single_depth[i])) for i in range(len(srcs))]
    out.append({"workload": f"grid4096_bfs_batch{kb}", "primitive": "batched bfs", "calls": 1,
                "sources": kb, "ms_per_call": ms_b, "ms_per_source": ms_b / kb,
                "queries_per_s": kb / (ms_b * 1e-3),
                "speedup_vs_single": (kb / ms_b) / (1.0 / mean), "levels": lv_b,
                "us_per_level": 1e3 * ms_b / lv_b,
                "lanes_equal_single": equal,
                "throughput": kb * m / (ms_b * 1e-3) / 1e9, "unit": "GTEPS (k*m per call)"})
    del depth_b, db
    # SSSP bucket width and driver tuned once on two sample sources
    gr.gr_autotune(g, [int(srcs[0]), int(srcs[1])], gr.GR_TUNE_SSSP)
    per, byts, iters, single = [], [], [], []
    dist_g = torch.empty(n, dtype=torch.int32, device=dev)
    for s in srcs[:2]:
        ms, _ = _timed_calls(lambda: gr.gr_sssp(g, int(s), dist_g), 1, flush)
        iters.append(gr.gr_sssp_stats(g)[0])
        per.append(ms)
        single.append(dist_g.cpu().numpy().view(np.uint32).copy())
        byts.append(reach_bytes(r, single[-1] != INF, 8, 4))
    mean = float(np.mean(per))
    out.append({"workload": "grid4096_sssp", "primitive": "sssp", "calls": 2,
                "tuned_delta": gr.gr_tuned_opts(g)["delta"],
                "tuned_sssp": gr.gr_tuned_sssp(g),
                "ms_per_call": mean, "throughput": m / (mean * 1e-3) / 1e9, "unit": "GTEPS",
                "iterations": iters,
                "roofline": _roof(float(np.mean(byts)), mean, peak,
                                  "8 B per column+weight entry of the reached vertices, "
                                  "4 B per row offset, 4 B per reached distance")})
    # the same searches batched: 16 sources (the two above first) as one
    # search over 16 copies of the graph
    k = 16
    srcs_k = [int(x) for x in srcs[:2]] + [int(x) for x in gg.sources(r, k + 2, seed=14)
                                           if int(x) not in (int(srcs[0]), int(srcs[1]))][:k - 2]
    dist_k = torch.empty(k * n, dtype=torch.int32, device=dev)
    ms_k, _ = _timed_calls(lambda: gr.gr_sssp_batch(g, srcs_k, dist_k), 1, flush)
    it_k = gr.gr_sssp_batch_stats(g)[0]
    dk = dist_k.cpu().numpy().view(np.uint32).reshape(k, n)
    out.append({"workload": f"grid4096_sssp_batch{k}", "primitive": "sssp (batched)",
                "calls": 1, "sources": k, "ms_per_call": ms_k, "ms_per_source": ms_k / k,
                "queries_per_s": k / (ms_k * 1e-3),
                "speedup_vs_single": (k / ms_k) / (1.0 / mean), "iterations": it_k,
                "lanes_equal_single": [bool(np.array_equal(dk[i], single[i])) for i in range(2)],
                "throughput": k * m / (ms_k * 1e-3) / 1e9, "unit": "GTEPS (k*m per call)"})
    del dist_k
    label = torch.empty(n, dtype=torch.int32, device=dev)
    ms, _ = _timed_calls(lambda: gr.gr_cc(g, label, count=False), 3, flush)
    out.append({"workload": "grid4096_cc", "primitive": "cc", "calls": 3, "ms_per_call": ms,
                "throughput": m / (ms * 1e-3) / 1e9, "unit": "G edges/s",
                "components": gr.gr_cc(g, label),
                "roofline": _roof(4 * m + 4 * (n + 1) + 8 * n, ms, peak,
                                  "4 B per column entry, 4 B per row offset, label write "
                                  "at init and after pointer jumping")})
    g.close()


def suite_bipartite(args, gr, gg, torch, dev, flush, peak, out):
    # --- bipartite R-MAT: 2^22 hubs, 2^20 authorities, edge factor 16 (seed
    # 7): HITS, SALSA and personalized PageRank, 20 iterations each
    sl = args.suite_scale or 22
    sr = sl - 2
    r, c, nl = gg.rmat_bipartite(sl, sr, 16, seed=7)
    n, m = r.size - 1, c.size
    g = gr.gr_graph_create(r, c)
    score = torch.empty(n, dtype=torch.float64, device=dev)
    iters = 20
    per_iter = 2 * (4 * m + 4 * (n + 1)) + 3 * 8 * n

    def row(name, fn, bytes_model):
        ms, _ = _timed_calls(fn, 2, flush)
        out.append({"workload": f"bipartite{sl}x{sr}_{name}", "primitive": name, "calls": 2,
                    "iterations": iters, "ms_per_call": ms, "ms_per_iteration": ms / iters,
                    "throughput": iters * m / (ms * 1e-3) / 1e9,
                    "unit": "G entries/s (entries x iterations)", "n": n, "n_left": nl, "m": m,
                    "roofline": _roof(iters * per_iter, ms, peak, bytes_model)})

    model = ("per iteration the two gather passes read every column entry and row offset "
             "once; scores, sums and score/degree written and read once per vertex (8 B)")
    row("hits", lambda: gr.gr_hits(g, nl, score, max_iter=iters, tol=0.0, count=False), model)
    row("salsa", lambda: gr.gr_salsa(g, nl, score, max_iter=iters, tol=0.0, count=False), model)
    seeds = [int(v) for v in gg.sources(r, 8, seed=7)]
    per_iter = 4 * m + 4 * (n + 1) + 4 * 8 * n
    row("ppr", lambda: gr.gr_ppr(g, seeds, score, 0.85, iters, 0.0, count=False),
        "per iteration one gather pass over every column entry and row offset; rank, "
        "rank/degree, sums and teleport once per vertex (8 B)")
    g.close()


def suite_rmat(args, gr, gg, torch, dev, flush, peak, out, want):
    # --- R-MAT s23 (seed 5): PageRank, CC, batched BFS and BC over 64 sources
    scale = args.suite_scale or 23
    tag = f"rmat{scale}"
    r, c = gg.rmat(scale, 16, seed=5)
    n, m = r.size - 1, c.size
    g = gr.gr_graph_create(r, c)
    srcs64 = gg.sources(r, 64, seed=5)
    lv = 0
    if want("rmat", "pagerank"):
        suite_pagerank(gr, torch, dev, flush, peak, out, g, n, m, tag, args.mode)
    if want("rmat", "cc"):
        label = torch.empty(n, dtype=torch.int32, device=dev)
        ms, _ = _timed_calls(lambda: gr.gr_cc(g, label, count=False), 3, flush)
        out.append({"workload": f"{tag}_cc", "primitive": "cc", "calls": 3, "ms_per_call": ms,
                    "throughput": m / (ms * 1e-3) / 1e9, "unit": "G edges/s",
                    "roofline": _roof(4 * m + 4 * (n + 1) + 8 * n, ms, peak,
                                      "4 B per column entry, 4 B per row offset, label write "
                                      "at init and after pointer jumping")})
    if want("rmat", "reduce"):
        # the gather-reduce operator over every vertex: FP64 sum and int32 min
        x = torch.rand(n, dtype=torch.float64, device=dev)
        outr = torch.empty(n, dtype=torch.float64, device=dev)
        ms, _ = _timed_calls(lambda: gr.gr_neighbor_reduce(g, gr.GR_REDUCE_SUM, x, outr), 3,
                             flush)
        out.append({"workload": f"{tag}_reduce_sum", "primitive": "gather-reduce (sum, f64)",
                    "calls": 3, "ms_per_call": ms, "throughput": m / (ms * 1e-3) / 1e9,
                    "unit": "G entries/s",
                    "roofline": _roof(4 * m + 4 * (n + 1) + 16 * n, ms, peak,
                                      "4 B per column entry, 4 B per row offset, x read and "
                                      "out written once (8 B each per vertex)")})
        xi = torch.randint(0, 1 << 30, (n,), dtype=torch.int32, device=dev)
        outi = torch.empty(n, dtype=torch.int32, device=dev)
        ms, _ = _timed_calls(lambda: gr.gr_neighbor_reduce(g, gr.GR_REDUCE_MIN, xi, outi), 3,
                             flush)
        out.append({"workload": f"{tag}_reduce_min", "primitive": "gather-reduce (min, i32)",
                    "calls": 3, "ms_per_call": ms, "throughput": m / (ms * 1e-3) / 1e9,
                    "unit": "G entries/s",
                    "roofline": _roof(4 * m + 4 * (n + 1) + 8 * n, ms, peak,
                                      "4 B per column entry, 4 B per row offset, x read and "
                                      "out written once (4 B each per vertex)")})
        del x, outr, xi, outi
    lv = None
    if want("rmat", "bfs64"):
        depth64 = torch.empty(64 * n, dtype=torch.int32, device=dev)
        ms, _ = _timed_calls(lambda: gr.gr_bfs_batch(g, srcs64, depth64), 2, flush)
        lv = int(depth64.view(64, n).max().item()) + 1
        out.append({"workload": f"{tag}_bfs64", "primitive": "batched bfs (64 lanes)",
                    "calls": 2, "ms_per_call": ms, "levels": lv,
                    "throughput": 64 * m / (ms * 1e-3) / 1e9, "unit": "GTEPS",
                    "roofline": _roof(lv * (4 * m + 4 * (n + 1) + 24 * n) + 4 * 64 * n, ms,
                                      peak,
                                      "per level a sweep of every column entry and row "
                                      "offset with three 8 B lane masks per vertex; 4 B "
                                      "per lane depth written")})
        del depth64
    if want("rmat", "bc64"):
        # with --suite-part bc64 the BC calls are the process's first
        # batched kernels (profiling runs skip a known number of launches)
        bc = torch.empty(n, dtype=torch.float64, device=dev)
        ms, _ = _timed_calls(lambda: gr.gr_bc(g, srcs64, bc), 1, flush)
        if lv is None:  # levels of the 64 traversals, for the bytes model
            depth64 = torch.empty(64 * n, dtype=torch.int32, device=dev)
            gr.gr_bfs_batch(g, srcs64, depth64)
            lv = int(depth64.view(64, n).max().item()) + 1
            del depth64
        out.append({"workload": f"{tag}_bc64", "primitive": "bc (64 sources, FP64)", "calls": 1,
                    "ms_per_call": ms, "levels": lv,
                    "throughput": 64 * 2 * m / (ms * 1e-3) / 1e9,
                    "unit": "GTEPS (2|E| per source)",
                    "roofline": _roof(2 * lv * (4 * m + 4 * (n + 1) + 16 * n) + 4 * 512 * n,
                                      ms, peak,
                                      "forward and backward: per level a sweep of every column "
                                      "entry and row offset with two 8 B lane masks per vertex; "
                                      "sigma and dependency rows (512 B per vertex) written and "
                                      "read once each")})
    g.close()


def suite_pagerank(gr, torch, dev, flush, peak, out, g, n, m, tag, mode="auto"):
    rank = torch.empty(n, dtype=torch.float32, device=dev)
    # launch mode (host-enqueued iterations) only for profiling runs: ncu
    # cannot profile the kernels inside a graph's while loop one by one
    o = gr.gr_opts(mode=gr.GR_MODE_LAUNCH) if mode == "launch" else None
    it = gr.gr_pagerank(g, rank, opts=o)
    ms, _ = _timed_calls(lambda: gr.gr_pagerank(g, rank, opts=o, count=False), 2, flush)
    per_iter = 4 * m + 4 * (n + 1) + 12 * n
    out.append({"workload": f"{tag}_pagerank", "primitive": "pagerank", "calls": 2,
                "ms_per_call": ms, "iterations": it,
                "throughput": it / (ms * 1e-3), "unit": "iterations/s",
                "roofline": _roof(per_iter * it, ms, peak,
                                  "per iteration: 4 B per column entry, 4 B per row offset, "
                                  "contribution write, rank read+write (12 B per vertex)")})


def host_cpu():
    """The host's logical core count (nproc) and CPU model (lscpu)."""
    info = {"host_cores": os.cpu_count()}
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            key, _, val = line.partition(":")
            if key.strip() in ("Model name", "Vendor ID", "Architecture") and val.strip():
                info[key.strip().lower().replace(" ", "_")] = val.strip()
    except (OSError, subprocess.SubprocessError):
        pass
    return info


def cpu_baseline(r, c, srcs, m, k):
    import oracle
    t0 = time.perf_counter()
    for s in srcs[:k]:
        oracle.bfs(r, c, int(s))
    dt = time.perf_counter() - t0
    out = {"value": m * k / dt / 1e9, "unit": "GTEPS", "cores": 1, "kind": "oracle",
           "sample": f"{k} of the {NUM_SOURCES} sources, single-threaded queue BFS, "
                     f"{dt:.2f} s wall"}
    out.update(host_cpu())
    return out


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    r, c, srcs = make_inputs()
    m = int(c.size)
    import oracle
    oracle.bfs(r, c, int(srcs[0]))  # warm the page cache / build
    per_step = max(1, min(len(srcs), 2))  # bounded sample per step
    for k in range(args.warmup):  # untimed
        oracle.bfs(r, c, int(srcs[k % len(srcs)]))
    times = []
    for k in range(args.steps):
        t0 = time.perf_counter()
        for j in range(per_step):
            oracle.bfs(r, c, int(srcs[(k * per_step + j) % len(srcs)]))
        times.append(time.perf_counter() - t0)
    total = sum(times)
    value = m * per_step * args.steps / total / 1e9
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "GTEPS",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * total / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "graph": f"R-MAT s{SCALE} ef{EDGE_FACTOR} seed {GRAPH_SEED}",
                       "n": int(r.size - 1), "m": m,
                       "sources_per_step": per_step},
            "cpu_baseline": dict({"value": value, "unit": "GTEPS", "cores": 1, "kind": "oracle",
                                  "sample": f"{per_step} traversals per step"}, **host_cpu()),
            "e2e": {"value": value, "unit": "GTEPS", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_gr(args):
    import torch
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    from paper_1501_05387_gb300 import build
    if rank == 0:
        build.build()
    if world > 1:
        torch.distributed.barrier()
    from paper_1501_05387_gb300 import gr

    r, c, srcs = make_inputs(args.scale)
    n, m = int(r.size - 1), int(c.size)
    g = gr.gr_graph_create(r, c)
    mode = {"auto": gr.GR_MODE_AUTO, "graph": gr.GR_MODE_GRAPH,
            "launch": gr.GR_MODE_LAUNCH, "persistent": gr.GR_MODE_PERSISTENT}[args.mode]
    bfs_opts = gr.gr_opts(mode=mode)
    dev = torch.device("cuda", local)
    depth = [torch.empty(n, dtype=torch.int32, device=dev) for _ in srcs]
    parent = [torch.empty(n, dtype=torch.int32, device=dev) for _ in srcs]
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream()

    def step(events=None):
        for i, s in enumerate(srcs):
            if events is not None:
                events[i][0].record(stream)
            gr.gr_bfs(g, int(s), depth[i], parent[i], bfs_opts)
            if events is not None:
                events[i][1].record(stream)

    for _ in range(max(3, args.warmup)):
        flush.zero_()
        step()
    torch.cuda.synchronize()
    depth_host = [d.cpu().numpy() for d in depth]
    levels = []
    traces = []
    for s in srcs:  # levels per traversal (for the launch count)
        gr.gr_bfs(g, int(s), depth[0], None, bfs_opts)
        levels.append(gr.gr_bfs_stats(g)[0])
        traces.append(gr.gr_bfs_trace(g))
    # our kernels per traversal: init + one per level (graph / launch mode)
    # or init + one persistent kernel
    launches_per_step = sum(2 if args.mode in ("auto", "persistent") else 1 + lv
                            for lv in levels)

    clocks = ClockSampler(local)
    ev = [[[torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)]
           for _ in srcs] for _ in range(args.steps)]
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks.start()
    time.sleep(0.3)
    wall0 = time.perf_counter()
    for k in range(args.steps):
        flush.zero_()
        step(ev[k])
    torch.cuda.synchronize()
    wall = time.perf_counter() - wall0
    clk = clocks.stop()
    if world > 1:
        torch.distributed.barrier()
    per_bfs = np.array([[a.elapsed_time(b) for a, b in ev[k]] for k in range(args.steps)])  # ms
    step_ms = per_bfs.sum(axis=1)
    total_s = max_over_ranks(float(step_ms.sum()) / 1e3, world, dev)
    value = job_throughput(m * len(srcs) * args.steps, world, total_s) / 1e9

    # roofline of the BFS level loop (one gr_bfs call = one launch of the
    # device-side while-loop graph)
    bytes_per_bfs = bfs_bytes(r, depth_host, m)
    mean_bfs_s = float(per_bfs.mean()) / 1e3
    achieved = float(np.mean(bytes_per_bfs)) / mean_bfs_s / 1e9
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    peak = float(peaks.get("hbm_gbs", 6800.0))
    roofline = {"bound": "hbm", "kernel": "gr_bfs traversal (init + level loop)",
                "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "peak_source": "measured" if "hbm_gbs" in peaks else "fallback",
                "frac_of_nominal_8TBs": achieved / 8000.0,
                "algorithmic_bytes_per_launch": float(np.mean(bytes_per_bfs)),
                "traffic": measured_traffic(m),
                "traffic_source": "ncu dram bytes of k_bfs_init + k_bfs_do at R-MAT s21, "
                                  "16 traversals, scaled by the edge count"}

    # end to end: the same traversals through the C ABI into page-locked
    # host buffers (gr_bfs_multi: each result is copied out while the next
    # traversal runs); the call's stream is synchronised before the clock
    # stops, so every depth and parent is in host memory
    e2e_times = [float("nan")]
    if not args.no_e2e:
        hd = [torch.empty(n, dtype=torch.int32).pin_memory() for _ in srcs]
        hp = [torch.empty(n, dtype=torch.int32).pin_memory() for _ in srcs]
        src_list = [int(s) for s in srcs]
        for _ in range(2):
            gr.gr_bfs_multi(g, src_list, hd, hp, bfs_opts, stream)
        stream.synchronize()
        # context for the end-to-end number: one result's device-to-host
        # copy into page-locked memory, alone (best of 5, CUDA events)
        d2h_ms = []
        for _ in range(5):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            hd[0].copy_(depth[0], non_blocking=True)
            e1.record(stream)
            e1.synchronize()
            d2h_ms.append(e0.elapsed_time(e1))
        d2h_gbs = 4 * n / (min(d2h_ms) * 1e-3) / 1e9
        e2e_times = []
        for k in range(args.steps):
            flush.zero_()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            gr.gr_bfs_multi(g, src_list, hd, hp, bfs_opts, stream)
            stream.synchronize()
            e2e_times.append(time.perf_counter() - t0)
        for i in (0, len(srcs) - 1):  # the host copies hold the results
            if not np.array_equal(hd[i].numpy(), depth_host[i]):
                raise RuntimeError("end-to-end depths differ from the device-timed run")
    e2e_total = max_over_ranks(sum(e2e_times), world, dev)
    e2e = {"value": job_throughput(m * len(srcs) * args.steps, world, e2e_total) / 1e9,
           "unit": "GTEPS",
           "h2d_bytes_per_step": 4 * len(srcs),
           "d2h_bytes_per_step": 2 * 4 * n * len(srcs),
           "call": "gr_bfs_multi into page-locked host depth+parent buffers (copies "
                   "overlap the next traversal)"}
    if not args.no_e2e:
        e2e["ms_per_step"] = [round(1e3 * t, 3) for t in e2e_times]
        e2e["d2h_copy_gbs"] = round(d2h_gbs, 1)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(r, c, srcs, m, args.cpu_sample_sources)
    serving = None
    if rank == 0 and not args.no_serving and (args.serving or world == 1):
        g.close()
        g = None
        try:
            serving = serving_bench(gr, full=args.serving_full,
                                    count=20000 if args.serving_full else args.serving_requests)
        except Exception as e:  # the BFS line is still reported
            serving = {"error": f"{type(e).__name__}: {e}"}

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "GTEPS", "n_gpus": world,
                "steps": args.steps, "warmup": max(3, args.warmup),
                "ms_per_step": 1e3 * total_s / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "int32",
                "data": "synthetic",
                "config": {"workload": WORKLOAD if args.scale == SCALE else f"rmat{args.scale}_bfs",
                           "graph": f"R-MAT s{args.scale} ef{EDGE_FACTOR} (a,b,c)=(0.57,0.19,0.19) seed {GRAPH_SEED}",
                           "mode": args.mode,
                           "n": n, "m": m, "sources": [int(s) for s in srcs],
                           "outputs": "depth+parent int32",
                           "l2": "256 MB flush before each step (outside the events)",
                           "parallelism": f"replicas x{world}"},
                "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e,
                "clocks": clk, "gpu_launches": launches_per_step * args.steps,
                "serving": serving,
                "bfs_ms": {"mean": float(per_bfs.mean()), "p50": float(np.median(per_bfs)),
                           "p99": float(np.percentile(per_bfs, 99)),
                           "min": float(per_bfs.min()), "max": float(per_bfs.max())},
                "levels": levels, "wall_s_timed_loop": wall,
                "trace_first_source": [
                    {"dir": "pull" if d else "push", "frontier": f, "edges": e,
                     "end_us": round(t, 2)} for d, f, e, t in traces[0]]}
        print(json.dumps(line), flush=True)
    if g is not None:
        g.close()
    if world > 1:
        torch.distributed.destroy_process_group()


def main():
    args = parse()
    if args.suite:
        run_suite(args)
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gr(args)


if __name__ == "__main__":
    main()
