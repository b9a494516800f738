// Query server: continuous batching of graph queries on resident graphs.
//
// Not part of the paper (which evaluates one query at a time); it serves
// BFS / SSSP / CC queries on graphs kept resident on the device:
//
//   * requests enter a FIFO queue (gr_server_submit);
//   * a worker thread (the slot) owns a CUDA stream and, per graph, its own
//     scratch workspaces, and runs one batch at a time;
//   * admission and batching (server_core.hpp): a batch is admitted while
//     its result buffers and any workspace it must create fit in the
//     device-memory budget next to the workspaces already kept;
//   * same-graph BFS requests are batched: the slot takes up to max_batch
//     queued BFS requests for the graph (in arrival order) and runs them as
//     bit lanes of one batched traversal; on high-diameter graphs only once
//     enough of them are queued;
//   * same-graph SSSP requests are batched the same way, as lanes of one
//     near/far search over copies of the graph (sssp_batch_run), as many as
//     the graph's lane limit allows;
//   * a result is copied to the caller's buffer (device or host) given at
//     submission, then its server buffer is released.
//
// With max_batch = 1 the same code is the plain path: one query per launch
// sequence, in arrival order, on one stream.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <thread>
#include <unordered_map>
#include <vector>

#include "gr_internal.cuh"
#include "server_core.hpp"

namespace gr {

namespace {

double now_ms() {
  using clk = std::chrono::steady_clock;
  static const clk::time_point t0 = clk::now();
  return std::chrono::duration<double, std::milli>(clk::now() - t0).count();
}

struct Request {
  uint64_t ticket = 0;
  int32_t graph = 0;
  int32_t kind = 0;
  int32_t src = 0;
  void *out = nullptr;
  bool out_on_device = false;
  double t_submit = 0.0;
  double t_start = 0.0;
  double t_done = 0.0;
  gr_status status = GR_OK;
  bool done = false;
  int32_t batch = 1;  // lanes of the launch that served it
};

struct SlotGraphState {
  BfsWorkspace *bfs = nullptr;
  SsspWorkspace *sssp = nullptr;
  CcWorkspace *cc = nullptr;
  BatchWorkspace *batch = nullptr;
  SsspWorkspace *sssp_batch = nullptr;  // for the graph's sssp_lanes lanes
  ~SlotGraphState() {
    free_bfs(bfs);
    free_sssp(sssp);
    free_sssp(sssp_batch);
    free_cc(cc);
    free_batch(batch);
  }
};

// Scratch one slot's batched SSSP workspace may take on a graph; the lane
// limit of the graph follows from it.
constexpr size_t kSsspBatchBytes = size_t(4) << 30;

// Longest a batch's device work may take before its slot gives up on it.
constexpr double kBatchLimitMs = 120000.0;

// Wait for the slot's stream with a time limit (a stream that never drains
// must not stall the slot's thread, and with it server shutdown, forever).
gr_status wait_stream(cudaStream_t s, double limit_ms) {
  const double t0 = now_ms();
  for (int polls = 0;; ++polls) {
    const cudaError_t e = cudaStreamQuery(s);
    if (e == cudaSuccess) return GR_OK;
    if (e != cudaErrorNotReady) return cuda_fail(e, "server stream");
    if (now_ms() - t0 > limit_ms)
      return fail(GR_ETIMEOUT, "device work of the batch did not finish within the slot's limit");
    if (polls < 2000) std::this_thread::yield();
    else std::this_thread::sleep_for(std::chrono::microseconds(100));
  }
}

gr_status copy_out(const Request &r, const void *dev, size_t bytes, cudaStream_t s) {
  if (!r.out) return GR_OK;
  GR_CUDA(cudaMemcpyAsync(r.out, dev, bytes,
                          r.out_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                          s));
  return GR_OK;
}

}  // namespace

struct Server {
  serve::Admission adm;  // under mu
  int device = 0;
  std::vector<gr_graph *> graphs;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::unordered_map<uint64_t, Request> reqs;  // all known requests
  uint64_t next_ticket = 1;
  bool stopping = false;
  std::vector<std::thread> workers;
  std::vector<double> latencies;  // completed requests (ms, submit -> done)
  uint64_t completed = 0, failed = 0, launches = 0, batched_lanes = 0;
  double t_first_submit = -1.0, t_last_done = 0.0;
  std::string last_error;

  void worker();
};

namespace {

// The device side of one batch on the slot (serve::run_batch's Dev).
struct SlotDev {
  gr_graph *g;
  SlotGraphState &st;
  const std::vector<Request> &rs;
  int32_t sssp_lanes;
  cudaStream_t s;
  DevMem &buf;
  std::string &broken;  // set once the slot's stream stopped draining

  bool many() const { return rs.size() > 1; }

  gr_status prepare(size_t need) {
    if (!s) return fail(GR_ECUDA, "server slot has no stream");
    if (!broken.empty()) return fail(GR_ECUDA, broken);
    // every earlier batch of this slot has been waited for (run_batch), so
    // the buffer is free to reallocate
    if (buf.bytes < need) GR_TRY(buf.alloc(need, "server result buffer"));
    return GR_OK;
  }

  gr_status enqueue() {
    const Request &first = rs[0];
    const size_t nbytes = sizeof(int32_t) * (size_t)g->n;
    // the graph's tuned settings are read under its lock, which also orders
    // this batch against public calls on the graph from other threads
    std::lock_guard<std::mutex> lock(g->mu);
    const gr_opts &o = default_opts();
    if (first.kind == GR_QUERY_BFS && many()) {
      if (!st.batch) GR_TRY(batch_ws_create(g, &st.batch));
      std::vector<int32_t> srcs;
      for (auto &r : rs) srcs.push_back(r.src);
      GR_TRY(bfs_batch_run(g, st.batch, srcs.data(), (int32_t)srcs.size(), buf.as<int32_t>(),
                           g->n + 1, s));
    } else if (first.kind == GR_QUERY_BFS) {
      if (!st.bfs) GR_TRY(bfs_ws_create(g, s, &st.bfs));
      GR_TRY(bfs_run(g, st.bfs, first.src, buf.as<int32_t>(), nullptr, o, s));
    } else if (first.kind == GR_QUERY_SSSP && many()) {
      if (!st.sssp_batch) GR_TRY(sssp_ws_create(g, s, &st.sssp_batch, sssp_lanes));
      std::vector<int32_t> srcs;
      for (auto &r : rs) srcs.push_back(r.src);
      GR_TRY(sssp_batch_run(g, st.sssp_batch, srcs.data(), (int32_t)srcs.size(),
                            buf.as<uint32_t>(), o, s));
    } else if (first.kind == GR_QUERY_SSSP) {
      if (!st.sssp) GR_TRY(sssp_ws_create(g, s, &st.sssp));
      GR_TRY(sssp_run(g, st.sssp, first.src, buf.as<uint32_t>(), nullptr, o, s));
    } else {
      // the CC requests of a batch share one run
      if (!st.cc) GR_TRY(cc_ws_create(g, &st.cc));
      GR_TRY(cc_run(g, st.cc, buf.as<int32_t>(), s));
    }
    const bool shared = first.kind == GR_QUERY_CC;
    for (size_t i = 0; i < rs.size(); ++i)
      GR_TRY(copy_out(rs[i], buf.as<char>() + (shared ? 0 : i * nbytes), nbytes, s));
    return GR_OK;
  }

  gr_status wait_idle() {
    const gr_status w = wait_stream(s, kBatchLimitMs);
    if (w == GR_ETIMEOUT) broken = std::string("server slot unusable: ") + gr_last_error();
    return w;
  }

  // a traversal that stopped at a device-side limit (level or iteration
  // cap, a timed-out wait) fails its request
  gr_status check_device_errors() {
    const int32_t kind = rs[0].kind;
    if (kind == GR_QUERY_BFS) return many() ? batch_read_ctl_error(st.batch, s)
                                            : bfs_read_ctl_error(st.bfs, s);
    if (kind == GR_QUERY_SSSP) return sssp_read_ctl_error(many() ? st.sssp_batch : st.sssp, s);
    return GR_OK;
  }
};

}  // namespace

void Server::worker() {
  cudaSetDevice(device);
  cudaStream_t s = nullptr;
  // a slot without a stream still drains its requests, failing them, so
  // that waiters never hang
  if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) {
    s = nullptr;
    cudaGetLastError();
  }
  // per-graph workspaces and the result staging of this slot; held by
  // pointer so that a slot whose stream stopped draining can leave them
  // (freeing memory that queued work may still use would wait on it)
  auto *state = new std::map<int32_t, SlotGraphState>();
  auto *buf = new DevMem();
  std::string broken;
  for (;;) {
    std::vector<Request> rs;
    {
      std::unique_lock<std::mutex> lock(mu);
      std::vector<uint64_t> batch;
      cv_work.wait(lock, [&] {
        if (stopping) return true;
        batch = adm.take_batch();
        return !batch.empty();
      });
      if (batch.empty()) break;  // stopping
      const double t = now_ms();
      for (uint64_t tk : batch) {
        reqs[tk].t_start = t;
        rs.push_back(reqs[tk]);
      }
    }
    // requests of a batch share kind and graph
    const Request &first = rs[0];
    gr_graph *g = graphs[first.graph];
    int32_t sssp_lanes;
    {
      std::lock_guard<std::mutex> lock(mu);
      sssp_lanes = adm.graphs[first.graph].sssp_lanes;
    }
    SlotDev dev{g, (*state)[first.graph], rs, sssp_lanes, s, *buf, broken};
    const gr_status status = serve::run_batch(
        dev, sizeof(int32_t) * (size_t)g->n * serve::Admission::result_units(first.kind, rs.size()));
    std::string err;
    if (status != GR_OK)
      err = std::string(gr_last_error()) + " [batch: kind " + std::to_string(first.kind) +
            ", graph " + std::to_string(first.graph) + ", lanes " + std::to_string(rs.size()) +
            ", first source " + std::to_string(first.src) + "]";
    const double t = now_ms();
    {
      std::lock_guard<std::mutex> lock(mu);
      for (auto &r : rs) {
        Request &q = reqs[r.ticket];
        q.done = true;
        q.status = status;
        q.t_done = t;
        q.batch = (int32_t)rs.size();
        if (status == GR_OK) {
          ++completed;
          latencies.push_back(t - q.t_submit);
        } else {
          ++failed;
          last_error = err;
        }
      }
      adm.release(first.graph, first.kind, rs.size());
      const serve::WsKind w = serve::ws_kind(first.kind, rs.size() > 1);
      const SlotGraphState &st = (*state)[first.graph];
      const void *ws = w == serve::kWsBfs ? (const void *)st.bfs
                       : w == serve::kWsBfsBatch ? (const void *)st.batch
                       : w == serve::kWsSssp ? (const void *)st.sssp
                       : w == serve::kWsSsspBatch ? (const void *)st.sssp_batch
                                                  : (const void *)st.cc;
      if (!ws) adm.ws_not_created(first.graph, w);
      ++launches;
      batched_lanes += rs.size();
      t_last_done = std::max(t_last_done, t);
    }
    cv_done.notify_all();
    cv_work.notify_all();
  }
  if (broken.empty()) {
    delete state;
    delete buf;
    if (s) cudaStreamDestroy(s);
  }
}

}  // namespace gr

struct gr_server {
  gr::Server impl;
};

using namespace gr;

extern "C" {

gr_status gr_server_create(size_t budget_bytes, int32_t num_slots, int32_t max_batch,
                           gr_server **out) {
  clear_error();
  if (!out) return fail(GR_EINVAL, "out must not be NULL");
  *out = nullptr;
  if (num_slots != 1)
    return fail(GR_EINVAL,
                "num_slots must be 1: the server runs one worker slot (several slots running "
                "traversals at once are disabled until a device fault seen with them is "
                "explained)");
  if (max_batch < 1 || max_batch > 64) return fail(GR_EINVAL, "max_batch must be in [1, 64]");
  if (budget_bytes == 0) return fail(GR_EINVAL, "budget_bytes must be > 0");
  std::unique_ptr<gr_server> srv(new gr_server());
  Server &S = srv->impl;
  GR_CUDA(cudaGetDevice(&S.device));
  S.adm.budget = budget_bytes;
  S.adm.max_batch = max_batch;
  *out = srv.release();
  return GR_OK;
}

gr_status gr_server_add_graph(gr_server *srv, gr_graph *g, int32_t batchable,
                              int32_t *graph_id) {
  clear_error();
  if (!srv || !g || !graph_id) return fail(GR_EINVAL, "server, graph and graph_id must not be NULL");
  if (batchable < 0 || batchable > 64) return fail(GR_EINVAL, "batchable must be in [0, 64]");
  Server &S = srv->impl;
  std::lock_guard<std::mutex> lock(S.mu);
  if (!S.workers.empty()) return fail(GR_EBUSY, "add graphs before the first submit");
  serve::GraphInfo e;
  e.n = g->n;
  e.min_batch = batchable;
  if (g->has_weights) {
    const size_t per_lane = sssp_ws_bytes(g, 1) + sizeof(uint32_t) * (size_t)g->n;
    const size_t by_mem = std::max<size_t>(1, kSsspBatchBytes / per_lane);
    e.sssp_lanes = (int32_t)std::min<size_t>(by_mem, (size_t)sssp_batch_max_lanes(g));
  }
  e.ws_bytes[serve::kWsBfs] = bfs_ws_bytes(g);
  e.ws_bytes[serve::kWsBfsBatch] = batch_ws_bytes(g);
  e.ws_bytes[serve::kWsSssp] = g->has_weights ? sssp_ws_bytes(g) : 0;
  e.ws_bytes[serve::kWsSsspBatch] = g->has_weights ? sssp_ws_bytes(g, e.sssp_lanes) : 0;
  e.ws_bytes[serve::kWsCc] = cc_ws_bytes(g);
  S.adm.graphs.push_back(e);
  S.graphs.push_back(g);
  *graph_id = (int32_t)S.graphs.size() - 1;
  return GR_OK;
}

gr_status gr_server_submit(gr_server *srv, int32_t graph_id, int32_t kind, int32_t src,
                           void *out, uint64_t *ticket) {
  clear_error();
  if (!srv || !ticket) return fail(GR_EINVAL, "server and ticket must not be NULL");
  Server &S = srv->impl;
  std::unique_lock<std::mutex> lock(S.mu);
  if (graph_id < 0 || graph_id >= (int32_t)S.graphs.size())
    return fail(GR_EINVAL, "unknown graph id");
  gr_graph *g = S.graphs[graph_id];
  if (kind != GR_QUERY_BFS && kind != GR_QUERY_SSSP && kind != GR_QUERY_CC)
    return fail(GR_EINVAL, "unknown query kind");
  if (kind != GR_QUERY_CC && (src < 0 || src >= g->n)) return fail(GR_EINVAL, "source out of range");
  if (kind == GR_QUERY_SSSP && !g->has_weights) return fail(GR_EINVAL, "SSSP needs weights");
  if (sizeof(int32_t) * (size_t)g->n > S.adm.budget)
    return fail(GR_EINVAL, "a single result does not fit the memory budget");
  if (S.stopping) return fail(GR_EBUSY, "server is shutting down");
  Request r;
  r.ticket = S.next_ticket++;
  r.graph = graph_id;
  r.kind = kind;
  r.src = src;
  r.out = out;
  if (out) {
    cudaPointerAttributes attr;
    if (cudaPointerGetAttributes(&attr, out) == cudaSuccess)
      r.out_on_device = attr.type == cudaMemoryTypeDevice || attr.type == cudaMemoryTypeManaged;
    else
      cudaGetLastError();
  }
  r.t_submit = now_ms();
  if (S.t_first_submit < 0) S.t_first_submit = r.t_submit;
  S.reqs[r.ticket] = r;
  S.adm.pending[r.ticket] = serve::Pending{graph_id, kind};
  S.adm.queue.push_back(r.ticket);
  *ticket = r.ticket;
  if (S.workers.empty()) S.workers.emplace_back([&S] { S.worker(); });
  lock.unlock();
  S.cv_work.notify_one();
  return GR_OK;
}

gr_status gr_server_wait(gr_server *srv, uint64_t ticket, int32_t timeout_ms,
                         double *latency_ms) {
  clear_error();
  if (!srv) return fail(GR_EINVAL, "server must not be NULL");
  Server &S = srv->impl;
  std::unique_lock<std::mutex> lock(S.mu);
  auto it = S.reqs.find(ticket);
  if (it == S.reqs.end()) return fail(GR_EINVAL, "unknown ticket");
  auto pred = [&] { return S.reqs[ticket].done; };
  if (timeout_ms < 0) {
    S.cv_done.wait(lock, pred);
  } else if (!S.cv_done.wait_for(lock, std::chrono::milliseconds(timeout_ms), pred)) {
    return fail(GR_ETIMEOUT, "request not finished within the timeout");
  }
  Request &r = S.reqs[ticket];
  if (latency_ms) *latency_ms = r.t_done - r.t_submit;
  const gr_status st = r.status;
  if (st != GR_OK) set_error(S.last_error);
  S.reqs.erase(ticket);
  return st;
}

gr_status gr_server_drain(gr_server *srv, int32_t timeout_ms) {
  clear_error();
  if (!srv) return fail(GR_EINVAL, "server must not be NULL");
  Server &S = srv->impl;
  std::unique_lock<std::mutex> lock(S.mu);
  auto pred = [&] {
    if (!S.adm.queue.empty()) return false;
    for (auto &kv : S.reqs)
      if (!kv.second.done) return false;
    return true;
  };
  if (timeout_ms < 0) {
    S.cv_done.wait(lock, pred);
  } else if (!S.cv_done.wait_for(lock, std::chrono::milliseconds(timeout_ms), pred)) {
    return fail(GR_ETIMEOUT, "requests still pending after the timeout");
  }
  // forget finished requests nobody waits for
  for (auto it = S.reqs.begin(); it != S.reqs.end();)
    it = it->second.done ? S.reqs.erase(it) : std::next(it);
  return GR_OK;
}

gr_status gr_server_stats(gr_server *srv, int64_t *completed, int64_t *failed,
                          int64_t *launches, double *qps, double *p50_ms, double *p99_ms,
                          double *mean_batch) {
  clear_error();
  if (!srv) return fail(GR_EINVAL, "server must not be NULL");
  Server &S = srv->impl;
  std::lock_guard<std::mutex> lock(S.mu);
  std::vector<double> lat = S.latencies;
  std::sort(lat.begin(), lat.end());
  auto pct = [&](double p) {
    if (lat.empty()) return 0.0;
    size_t i = (size_t)std::min<double>(lat.size() - 1, std::ceil(p * lat.size()) - 1);
    return lat[i];
  };
  if (completed) *completed = (int64_t)S.completed;
  if (failed) *failed = (int64_t)S.failed;
  if (launches) *launches = (int64_t)S.launches;
  const double span = S.t_last_done - S.t_first_submit;
  if (qps) *qps = span > 0 ? S.completed / (span * 1e-3) : 0.0;
  if (p50_ms) *p50_ms = pct(0.50);
  if (p99_ms) *p99_ms = pct(0.99);
  if (mean_batch) *mean_batch = S.launches ? (double)S.batched_lanes / S.launches : 0.0;
  return GR_OK;
}

gr_status gr_server_destroy(gr_server *srv) {
  clear_error();
  if (!srv) return GR_OK;
  Server &S = srv->impl;
  {
    std::lock_guard<std::mutex> lock(S.mu);
    S.stopping = true;
  }
  S.cv_work.notify_all();
  for (auto &t : S.workers) t.join();
  delete srv;
  return GR_OK;
}

}  // extern "C"
