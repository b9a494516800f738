// Query server: continuous batching of graph queries on resident graphs.
//
// Not part of the paper (which evaluates one query at a time); it serves
// BFS / SSSP / CC queries on graphs kept resident on the device:
//
//   * requests enter a FIFO queue (gr_server_submit);
//   * a worker thread per slot owns a CUDA stream and, per graph, its own
//     scratch workspaces, so queries on different slots overlap on the GPU;
//   * admission is by a device-memory budget: a request is started only
//     when its result buffer fits in what the in-flight requests' buffers
//     and the workspaces the slots keep leave free (the oldest request
//     always starts when nothing is in flight); the memory footprint
//     follows the paper's alpha*|E| + beta*|V| model (Sec. 6);
//   * same-graph BFS requests are batched: a worker that takes a BFS request
//     also takes up to max_batch - 1 further queued BFS requests for that
//     graph (in arrival order) and runs them as bit lanes of one batched
//     traversal; on high-diameter graphs (many levels) only once enough of
//     them are queued;
//   * same-graph SSSP requests are batched the same way, as lanes of one
//     near/far search over copies of the graph (sssp_batch_run), as many as
//     the graph's lane limit allows;
//   * a result is copied to the caller's buffer (device or host) given at
//     submission, then its server buffer is released.
//
// With one slot and max_batch = 1 the same code is the plain path: one query
// per launch sequence, in arrival order, on one stream, no overlap.
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
  SsspWorkspace *sssp_batch = nullptr;  // for GraphEntry::sssp_lanes lanes
  ~SlotGraphState() {
    free_bfs(bfs);
    free_sssp(sssp);
    free_sssp(sssp_batch);
    free_cc(cc);
    free_batch(batch);
  }
};

struct GraphEntry {
  gr_graph *g = nullptr;
  // a BFS request is run as lanes of a batch when at least this many BFS
  // requests for the graph are queued (0: never batched)
  int32_t min_batch = 1;
  // most SSSP requests one batched search takes (1: never batched)
  int32_t sssp_lanes = 1;
};

// Scratch one slot's batched SSSP workspace may take on a graph; the lane
// limit of the graph follows from it.
constexpr size_t kSsspBatchBytes = size_t(4) << 30;

}  // namespace

struct Server {
  size_t budget = 0;
  size_t in_use = 0;    // result buffers of admitted, unfinished requests
  size_t resident = 0;  // workspaces created by the slots (kept)
  int32_t nslots = 1;
  int32_t max_batch = 64;
  int device = 0;
  std::vector<GraphEntry> graphs;
  std::mutex mu;
  std::mutex setup_mu;  // one slot at a time builds workspaces and level-loop graphs
  std::condition_variable cv_work, cv_done;
  std::deque<uint64_t> queue;                      // tickets waiting
  std::unordered_map<uint64_t, Request> reqs;      // all known requests
  uint64_t next_ticket = 1;
  bool stopping = false;
  std::vector<std::thread> workers;
  std::vector<double> latencies;  // completed requests (ms, submit -> done)
  uint64_t completed = 0, failed = 0, launches = 0, batched_lanes = 0;
  double t_first_submit = -1.0, t_last_done = 0.0;
  std::string last_error;

  size_t result_bytes(const Request &r) const {
    const gr_graph *g = graphs[r.graph].g;
    return sizeof(int32_t) * (size_t)g->n;
  }
  void worker();
};

namespace {

// Pick the next batch for a slot (caller holds the lock): the oldest
// request whose memory fits, plus same-graph BFS requests behind it when
// enough of them are queued for the graph to batch.
std::vector<uint64_t> take_batch(Server &S) {
  std::vector<uint64_t> out;
  for (auto it = S.queue.begin(); it != S.queue.end(); ++it) {
    Request &r = S.reqs[*it];
    const size_t need = S.result_bytes(r);
    if (S.resident + S.in_use + need > S.budget && S.in_use > 0) break;  // wait for memory
    out.push_back(*it);
    S.in_use += need;
    S.queue.erase(it);
    // lanes the batch of r may have
    int32_t cap = 1;
    const GraphEntry &ge = S.graphs[r.graph];
    if (r.kind == GR_QUERY_BFS && S.max_batch > 1 && ge.min_batch > 0) {
      int32_t queued = 1;  // r and the same-graph BFS requests behind it
      for (auto jt = S.queue.begin(); jt != S.queue.end() && queued < ge.min_batch; ++jt) {
        const Request &q = S.reqs[*jt];
        if (q.kind == GR_QUERY_BFS && q.graph == r.graph) ++queued;
      }
      if (queued >= ge.min_batch) cap = S.max_batch;
    } else if (r.kind == GR_QUERY_SSSP && S.max_batch > 1 && ge.min_batch > 0) {
      cap = std::min(S.max_batch, ge.sssp_lanes);
    }
    if (cap > 1) {
      for (auto jt = S.queue.begin(); jt != S.queue.end() && (int32_t)out.size() < cap;) {
        Request &q = S.reqs[*jt];
        if (q.kind == r.kind && q.graph == r.graph) {
          const size_t nq = S.result_bytes(q);
          if (S.resident + S.in_use + nq > S.budget) break;
          S.in_use += nq;
          out.push_back(*jt);
          jt = S.queue.erase(jt);
        } else {
          ++jt;
        }
      }
    }
    break;
  }
  return out;
}

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

void Server::worker() {
  cudaSetDevice(device);
  cudaStream_t s = nullptr;
  // a slot without a stream still drains its requests, failing them, so
  // that waiters never hang
  const cudaError_t se = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
  const std::string stream_err =
      se == cudaSuccess ? std::string() : std::string("server slot stream: ") + cudaGetErrorString(se);
  // per-graph workspaces and the result staging of this slot; held by
  // pointer so that a slot whose stream stopped draining can leave them
  // (freeing memory that queued work may still use would wait on it)
  auto *state = new std::map<int32_t, SlotGraphState>();
  auto *buf_p = new DevMem();
  DevMem &buf = *buf_p;
  std::string broken;  // set when the slot's stream stopped draining
  for (;;) {
    std::vector<uint64_t> batch;
    {
      std::unique_lock<std::mutex> lock(mu);
      cv_work.wait(lock, [&] {
        if (stopping) return true;
        batch = take_batch(*this);
        return !batch.empty();
      });
      if (batch.empty()) break;  // stopping
      for (uint64_t t : batch) reqs[t].t_start = now_ms();
    }
    // requests of a batch share kind and graph
    Request first;
    std::vector<Request> rs;
    {
      std::lock_guard<std::mutex> lock(mu);
      for (uint64_t t : batch) rs.push_back(reqs[t]);
    }
    first = rs[0];
    GraphEntry &ge = graphs[first.graph];
    gr_graph *g = ge.g;
    SlotGraphState &st = (*state)[first.graph];
    const size_t nbytes = sizeof(int32_t) * (size_t)g->n;
    const size_t need = nbytes * rs.size();
    gr_status status = GR_OK;
    std::string err;
    if (!stream_err.empty()) status = fail(GR_ECUDA, stream_err);
    if (status == GR_OK && !broken.empty()) status = fail(GR_ECUDA, broken);
    if (status == GR_OK && buf.bytes < need) status = buf.alloc(need, "server result buffer");
    // with several slots, graph-mode level loops: slots may run traversals
    // at once, so no launch may need the whole GPU to itself (cooperative
    // launches do); a single slot has the GPU to itself and runs each
    // graph's tuned driver
    gr_opts o = default_opts();
    if (nslots > 1) o.mode = GR_MODE_GRAPH;
    size_t ws_new = 0;
    // the first request of a kind on a graph creates this slot's workspace
    // and captures its level-loop graph; slots do that one at a time
    std::unique_lock<std::mutex> setup(setup_mu, std::defer_lock);
    const bool many = rs.size() > 1;
    const bool fresh = (first.kind == GR_QUERY_BFS && many)    ? !st.batch
                       : first.kind == GR_QUERY_BFS            ? !st.bfs
                       : (first.kind == GR_QUERY_SSSP && many) ? !st.sssp_batch
                       : first.kind == GR_QUERY_SSSP           ? !st.sssp
                                                               : !st.cc;
    if (fresh) setup.lock();
    if (status == GR_OK) {
      if (first.kind == GR_QUERY_BFS && rs.size() > 1) {
        if (!st.batch) {
          status = batch_ws_create(g, &st.batch);
          ws_new += batch_ws_bytes(g);
        }
        if (status == GR_OK) {
          std::vector<int32_t> srcs;
          for (auto &r : rs) srcs.push_back(r.src);
          status = bfs_batch_run(g, st.batch, srcs.data(), (int32_t)srcs.size(),
                                 buf.as<int32_t>(), g->n + 1, s);
        }
      } else if (first.kind == GR_QUERY_BFS) {
        if (!st.bfs) {
          status = bfs_ws_create(g, s, &st.bfs);
          ws_new += bfs_ws_bytes(g);
        }
        if (status == GR_OK) status = bfs_run(g, st.bfs, first.src, buf.as<int32_t>(), nullptr, o, s);
      } else if (first.kind == GR_QUERY_SSSP && many) {
        if (!st.sssp_batch) {
          status = sssp_ws_create(g, s, &st.sssp_batch, ge.sssp_lanes);
          ws_new += sssp_ws_bytes(g, ge.sssp_lanes);
        }
        if (status == GR_OK) {
          std::vector<int32_t> srcs;
          for (auto &r : rs) srcs.push_back(r.src);
          // the CUDA-graph driver holds one-lane arguments: host-driven
          // batches stand in for it (sssp_batch_run)
          status = sssp_batch_run(g, st.sssp_batch, srcs.data(), (int32_t)srcs.size(),
                                  buf.as<uint32_t>(), o, s);
        }
      } else if (first.kind == GR_QUERY_SSSP) {
        if (!st.sssp) {
          status = sssp_ws_create(g, s, &st.sssp);
          ws_new += sssp_ws_bytes(g);
        }
        if (status == GR_OK)
          status = sssp_run(g, st.sssp, first.src, buf.as<uint32_t>(), nullptr, o, s);
      } else {
        if (!st.cc) {
          status = cc_ws_create(g, &st.cc);
          ws_new += cc_ws_bytes(g);
        }
        if (status == GR_OK) status = cc_run(g, st.cc, buf.as<int32_t>(), s);
      }
      for (size_t i = 0; status == GR_OK && i < rs.size(); ++i)
        status = copy_out(rs[i], buf.as<char>() + i * nbytes, nbytes, s);
      if (setup.owns_lock()) setup.unlock();
      if (status == GR_OK) {
        status = wait_stream(s, kBatchLimitMs);
        if (status == GR_ETIMEOUT) broken = std::string("server slot unusable: ") + gr_last_error();
      }
      // a traversal that stopped at a device-side limit (level or iteration
      // cap, a timed-out wait) fails its request
      if (status == GR_OK && first.kind == GR_QUERY_BFS && rs.size() == 1)
        status = bfs_read_ctl_error(st.bfs, s);
      if (status == GR_OK && first.kind == GR_QUERY_SSSP)
        status = sssp_read_ctl_error(many ? st.sssp_batch : st.sssp, s);
    }
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
        in_use -= result_bytes(q);
        if (status == GR_OK) {
          ++completed;
          latencies.push_back(t - q.t_submit);
        } else {
          ++failed;
          last_error = err;
        }
      }
      ++launches;
      batched_lanes += rs.size();
      resident += ws_new;  // workspaces stay with the slot
      t_last_done = std::max(t_last_done, t);
    }
    cv_done.notify_all();
    cv_work.notify_all();
  }
  if (broken.empty()) {
    delete state;
    delete buf_p;
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
  if (num_slots < 1 || num_slots > 64) return fail(GR_EINVAL, "num_slots must be in [1, 64]");
  if (max_batch < 1 || max_batch > 64) return fail(GR_EINVAL, "max_batch must be in [1, 64]");
  if (budget_bytes == 0) return fail(GR_EINVAL, "budget_bytes must be > 0");
  std::unique_ptr<gr_server> srv(new gr_server());
  Server &S = srv->impl;
  GR_CUDA(cudaGetDevice(&S.device));
  S.budget = budget_bytes;
  S.nslots = num_slots;
  S.max_batch = max_batch;
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
  GraphEntry e;
  e.g = g;
  e.min_batch = batchable;
  if (g->has_weights) {
    const size_t per_lane = sssp_ws_bytes(g, 1) + sizeof(uint32_t) * (size_t)g->n;
    const size_t by_mem = std::max<size_t>(1, kSsspBatchBytes / per_lane);
    e.sssp_lanes = (int32_t)std::min<size_t>(by_mem, (size_t)sssp_batch_max_lanes(g));
  }
  S.graphs.push_back(e);
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
  gr_graph *g = S.graphs[graph_id].g;
  if (kind != GR_QUERY_BFS && kind != GR_QUERY_SSSP && kind != GR_QUERY_CC)
    return fail(GR_EINVAL, "unknown query kind");
  if (kind != GR_QUERY_CC && (src < 0 || src >= g->n)) return fail(GR_EINVAL, "source out of range");
  if (kind == GR_QUERY_SSSP && !g->has_weights) return fail(GR_EINVAL, "SSSP needs weights");
  if (sizeof(int32_t) * (size_t)g->n > S.budget)
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
  S.queue.push_back(r.ticket);
  *ticket = r.ticket;
  if (S.workers.empty())
    for (int i = 0; i < S.nslots; ++i) S.workers.emplace_back([&S] { S.worker(); });
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
    if (!S.queue.empty()) return false;
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
