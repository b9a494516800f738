// Single-source shortest paths with a near/far frontier split (Alg. 1,
// Sec. 4.5 "Priority queue", Sec. 5.2).
//
// Alg. 1 initialises labels to infinity and label[root] = 0, then loops
// advance (UpdateLabel = atomicMin relaxation), filter (RemoveRedundant, an
// output-queue stamp per vertex) and the priority-queue split until the
// frontier is empty. Here one iteration of the device-side loop is:
//
//   k_sssp_scan   degree scan of the near frontier (skipped when empty)
//   k_sssp_relax  load-balanced advance; per edge new = dist[u] + w(e),
//                 atomicMin on dist[v]; an improved v goes to the next near
//                 frontier if new < T (deduplicated by a per-iteration stamp,
//                 the RemoveRedundant filter) and to the far pile otherwise
//                 (deduplicated by a per-phase stamp)
//   k_sssp_split  only when the near frontier is empty: the far pile is
//                 split by the raised threshold into near and far; entries
//                 whose distance fell below the old threshold were already
//                 expanded and are dropped
//   k_sssp_end    one thread: swaps buffers, raises T (jumping to the
//                 bucket of the smallest far distance when the next bucket
//                 would be empty), ends the loop when both piles are empty
//
// T starts at delta and grows by delta per phase (delta = UINT32_MAX: one
// bucket, i.e. plain frontier relaxation). Distances do not depend on delta.
// An optional last pass fills pred[v] with the smallest u that has an edge
// (u, v) with dist[u] + w = dist[v].
#include <algorithm>
#include <cstring>

#include "advance.cuh"

namespace gr {

enum : int32_t { kSsspRelax = 0, kSsspSplit = 1 };

struct SsspCtl {
  uint32_t *dist;
  int32_t *pred;
  int32_t src;
  int32_t mode;          // kSsspRelax / kSsspSplit for the current iteration
  int32_t near_parity;   // which near buffer holds the current frontier
  int32_t far_parity;    // which far buffer holds the current pile
  int32_t near_len;
  int32_t near_next_len;  // atomic
  int32_t far_len;        // atomic (relax appends to the current pile)
  int32_t far_next_len;   // atomic (split output)
  int32_t tile_ctr;
  int32_t done;
  int32_t error;
  int32_t iter;           // iteration id, also the near-frontier stamp
  int32_t far_epoch;      // far-pile stamp
  int32_t max_iters;
  int32_t phases;         // number of splits
  uint32_t epoch;         // scan epoch (never reset)
  uint32_t far_min;       // lower bound of far-pile distances (atomicMin)
  uint32_t far_min_next;  // min distance of entries kept by a split
  unsigned long long T;   // near criterion: dist < T
  unsigned long long T_old;
  unsigned long long delta;
  long long relaxations;  // edges expanded (statistics)
};

struct SsspArgs {
  const int32_t *R;
  const int32_t *C;
  const uint32_t *W;
  int32_t n;
  int32_t *nearq[2];
  int32_t *farq[2];
  int32_t *scan;
  int32_t *stamp;
  int32_t *far_stamp;
  unsigned long long *status;
  SsspCtl *ctl;
};

constexpr int kSsspScanThreads = 512, kSsspScanItems = 4;
constexpr int kSsspThreads = 256, kSsspItems = 8;

struct SsspWorkspace {
  DevMem nearq[2], farq[2], scan, stamp, far_stamp, status, ctl;
  cudaGraphExec_t exec = nullptr;
  cudaGraph_t graph = nullptr;
  ~SsspWorkspace() {
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
  }
};

void free_sssp(SsspWorkspace *ws) { delete ws; }

namespace {

__device__ __forceinline__ int32_t *pick(int32_t *const *a, int p) { return p ? a[1] : a[0]; }

__global__ void k_sssp_init(SsspArgs a, int32_t src, uint32_t *dist, int32_t *pred,
                            unsigned long long delta, int32_t max_iters) {
  const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t v = tid; v < a.n; v += stride) {
    dist[v] = v == src ? 0u : 0xFFFFFFFFu;
    a.stamp[v] = -1;
    a.far_stamp[v] = -1;
  }
  if (tid == 0) {
    SsspCtl *c = a.ctl;
    a.nearq[0][0] = src;
    c->dist = dist;
    c->pred = pred;
    c->src = src;
    c->mode = kSsspRelax;
    c->near_parity = 0;
    c->far_parity = 0;
    c->near_len = 1;
    c->near_next_len = 0;
    c->far_len = 0;
    c->far_next_len = 0;
    c->tile_ctr = 0;
    c->done = 0;
    c->error = kDevOk;
    c->iter = 0;
    c->far_epoch = 0;
    c->max_iters = max_iters;
    c->phases = 0;
    c->far_min = 0xFFFFFFFFu;
    c->far_min_next = 0xFFFFFFFFu;
    c->delta = delta;
    c->T = delta;
    c->T_old = 0;
    c->relaxations = 0;
  }
}

__global__ void __launch_bounds__(kSsspScanThreads) k_sssp_scan(SsspArgs a) {
  SsspCtl *c = a.ctl;
  if (c->done || c->error || c->mode != kSsspRelax) return;
  ScanState st{a.status, &c->tile_ctr, &c->error, c->epoch};
  long long total;
  if (frontier_degree_scan<kSsspScanThreads, kSsspScanItems>(
          a.R, pick(a.nearq, c->near_parity), c->near_len, a.scan, st, &total))
    c->relaxations += total;
}

struct RelaxF {
  const uint32_t *W;
  uint32_t *dist;
  int32_t *stamp;
  int32_t *far_stamp;
  uint32_t *far_min;
  unsigned long long T;
  int32_t iter;
  int32_t far_epoch;
  __device__ __forceinline__ int operator()(int32_t u, int32_t v, int32_t e) const {
    const unsigned long long nd = (unsigned long long)dist[u] + W[e];
    if (nd >= 0xFFFFFFFFull) return 0;  // not representable: no path improvement
    const uint32_t nd32 = (uint32_t)nd;
    if (nd32 >= dist[v]) return 0;  // plain-load cull
    const uint32_t old = atomicMin(dist + v, nd32);
    if (nd32 >= old) return 0;
    if (nd < T) return atomicExch(stamp + v, iter) != iter ? 1 : 0;
    atomicMin(far_min, nd32);
    return atomicExch(far_stamp + v, far_epoch) != far_epoch ? 2 : 0;
  }
};

__global__ void __launch_bounds__(kSsspThreads) k_sssp_relax(SsspArgs a) {
  SsspCtl *c = a.ctl;
  if (c->done || c->error || c->mode != kSsspRelax) return;
  const int32_t np = c->near_parity;
  RelaxF f{a.W, c->dist, a.stamp, a.far_stamp, &c->far_min, c->T, c->iter, c->far_epoch};
  lb_advance<kSsspThreads, kSsspItems, 2>(a.R, a.C, pick(a.nearq, np), c->near_len, a.scan, f,
                                          pick(a.nearq, np ^ 1), &c->near_next_len,
                                          pick(a.farq, c->far_parity), &c->far_len);
}

__global__ void __launch_bounds__(kSsspThreads) k_sssp_split(SsspArgs a) {
  SsspCtl *c = a.ctl;
  if (c->done || c->error || c->mode != kSsspSplit) return;
  const int32_t *F = pick(a.farq, c->far_parity);
  int32_t *Fn = pick(a.farq, c->far_parity ^ 1);
  int32_t *Nn = pick(a.nearq, c->near_parity ^ 1);
  const int32_t len = c->far_len;
  const unsigned long long T = c->T, T_old = c->T_old;
  const int32_t iter = c->iter, epoch = c->far_epoch + 1;
  const uint32_t *dist = c->dist;
  __shared__ int32_t s_out0[kSsspThreads], s_out1[kSsspThreads];
  __shared__ int32_t s_cnt[2], s_base[2];
  uint32_t local_min = 0xFFFFFFFFu;
  const int64_t rounds = (len + (int64_t)gridDim.x * kSsspThreads - 1) /
                         ((int64_t)gridDim.x * kSsspThreads);
  for (int64_t r = 0; r < rounds; ++r) {
    const int64_t i = (r * gridDim.x + blockIdx.x) * kSsspThreads + threadIdx.x;
    if (threadIdx.x < 2) s_cnt[threadIdx.x] = 0;
    __syncthreads();
    int code = 0;
    int32_t v = 0;
    if (i < len) {
      v = F[i];
      const uint32_t d = dist[v];
      if ((unsigned long long)d < T_old) {
        code = 0;  // stale: improved below the old threshold and expanded
      } else if ((unsigned long long)d < T) {
        code = atomicExch(a.stamp + v, iter) != iter ? 1 : 0;
      } else {
        local_min = min(local_min, d);
        code = atomicExch(a.far_stamp + v, epoch) != epoch ? 2 : 0;
      }
    }
    warp_append(code, v, s_out0, &s_cnt[0], s_out1, &s_cnt[1]);
    __syncthreads();
    if (threadIdx.x < 2) {
      const int32_t cnt = s_cnt[threadIdx.x];
      s_base[threadIdx.x] =
          cnt ? atomicAdd(threadIdx.x ? &c->far_next_len : &c->near_next_len, cnt) : 0;
    }
    __syncthreads();
    for (int32_t k = threadIdx.x; k < s_cnt[0]; k += kSsspThreads) Nn[s_base[0] + k] = s_out0[k];
    for (int32_t k = threadIdx.x; k < s_cnt[1]; k += kSsspThreads) Fn[s_base[1] + k] = s_out1[k];
    __syncthreads();
  }
  for (int o = 16; o > 0; o >>= 1) local_min = min(local_min, __shfl_xor_sync(0xffffffffu, local_min, o));
  if ((threadIdx.x & 31) == 0 && local_min != 0xFFFFFFFFu) atomicMin(&c->far_min_next, local_min);
}

__device__ __forceinline__ unsigned long long bucket_end(uint32_t d, unsigned long long delta) {
  return ((unsigned long long)d / delta + 1ull) * delta;
}

__device__ __forceinline__ void sssp_end_body(SsspCtl *c) {
  if (c->done) return;
  if (c->error) {
    c->done = 1;
    return;
  }
  if (c->mode == kSsspRelax) {
    c->near_len = c->near_next_len;
    c->near_parity ^= 1;
  } else {
    c->near_len = c->near_next_len;
    c->near_parity ^= 1;
    c->far_len = c->far_next_len;
    c->far_parity ^= 1;
    c->far_epoch += 1;
    c->far_min = c->far_min_next;
    c->phases += 1;
  }
  c->near_next_len = 0;
  c->far_next_len = 0;
  c->far_min_next = 0xFFFFFFFFu;
  c->tile_ctr = 0;
  c->epoch += 1;
  c->iter += 1;
  if (c->near_len > 0) {
    c->mode = kSsspRelax;
  } else if (c->far_len > 0) {
    c->mode = kSsspSplit;
    c->T_old = c->T;
    unsigned long long t = c->T + c->delta;
    const unsigned long long j = bucket_end(c->far_min, c->delta);
    c->T = t > j ? t : j;
  } else {
    c->done = 1;
    return;
  }
  if (c->iter >= c->max_iters) {
    c->error = kDevOverflow;
    c->done = 1;
  }
}

__global__ void k_sssp_end(SsspArgs a, cudaGraphConditionalHandle h, int32_t use_cond) {
  if (threadIdx.x != 0) return;
  sssp_end_body(a.ctl);
  if (use_cond) cudaGraphSetConditional(h, a.ctl->done ? 0u : 1u);
}

// pred[v] = smallest u with an edge (u, v) and dist[u] + w = dist[v]
__global__ void k_sssp_pred_init(int32_t *pred, int32_t n) {
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n;
       v += (int64_t)gridDim.x * blockDim.x)
    pred[v] = INT32_MAX;
}

__global__ void k_sssp_pred(const int32_t *R, const int32_t *C, const uint32_t *W,
                            const uint32_t *dist, int32_t *pred, int32_t n, int32_t src) {
  const int64_t gw = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int lane = threadIdx.x & 31;
  for (int64_t uu = gw; uu < n; uu += nw) {
    const int32_t u = (int32_t)uu;
    const uint32_t du = dist[u];
    if (du == 0xFFFFFFFFu) continue;
    for (int32_t e = R[u] + lane; e < R[u + 1]; e += 32) {
      const int32_t v = C[e];
      const uint32_t dv = dist[v];
      if (v != src && dv != 0xFFFFFFFFu && (unsigned long long)du + W[e] == dv)
        atomicMin(pred + v, u);
    }
  }
}

__global__ void k_sssp_pred_fin(int32_t *pred, int32_t n, int32_t src) {
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n;
       v += (int64_t)gridDim.x * blockDim.x)
    pred[v] = v == src ? src : (pred[v] == INT32_MAX ? -1 : pred[v]);
}

}  // namespace

static gr_status ensure_sssp_ws(gr_graph *g, cudaStream_t s) {
  if (g->sssp) return GR_OK;
  std::unique_ptr<SsspWorkspace> ws(new SsspWorkspace());
  const size_t n = (size_t)g->n;
  for (int i = 0; i < 2; ++i) {
    GR_TRY(ws->nearq[i].alloc(sizeof(int32_t) * (n + 1), "SSSP near queue"));
    GR_TRY(ws->farq[i].alloc(sizeof(int32_t) * (n + 1), "SSSP far pile"));
  }
  GR_TRY(ws->scan.alloc(sizeof(int32_t) * (n + 2), "SSSP degree scan"));
  GR_TRY(ws->stamp.alloc(sizeof(int32_t) * n, "SSSP near stamps"));
  GR_TRY(ws->far_stamp.alloc(sizeof(int32_t) * n, "SSSP far stamps"));
  const size_t ntiles = n / (kSsspScanThreads * kSsspScanItems) + 2;
  GR_TRY(ws->status.alloc(sizeof(unsigned long long) * ntiles, "scan status"));
  GR_TRY(ws->ctl.alloc(sizeof(SsspCtl), "SSSP control"));
  GR_CUDA(cudaMemsetAsync(ws->status.p, 0, ws->status.bytes, s));
  SsspCtl init;
  std::memset(&init, 0, sizeof(init));
  init.epoch = 1;
  GR_CUDA(cudaMemcpyAsync(ws->ctl.p, &init, sizeof(init), cudaMemcpyHostToDevice, s));
  GR_CUDA(cudaStreamSynchronize(s));
  g->sssp = ws.release();
  return GR_OK;
}

static SsspArgs sssp_args(gr_graph *g) {
  SsspWorkspace *ws = g->sssp;
  SsspArgs a;
  a.R = g->row_off.as<int32_t>();
  a.C = g->col.as<int32_t>();
  a.W = g->w.as<uint32_t>();
  a.n = g->n;
  for (int i = 0; i < 2; ++i) {
    a.nearq[i] = ws->nearq[i].as<int32_t>();
    a.farq[i] = ws->farq[i].as<int32_t>();
  }
  a.scan = ws->scan.as<int32_t>();
  a.stamp = ws->stamp.as<int32_t>();
  a.far_stamp = ws->far_stamp.as<int32_t>();
  a.status = ws->status.as<unsigned long long>();
  a.ctl = ws->ctl.as<SsspCtl>();
  return a;
}

static gr_status sssp_enqueue_iter(gr_graph *g, const SsspArgs &a, cudaStream_t s,
                                   cudaGraphConditionalHandle h, int use_cond) {
  k_sssp_scan<<<g->num_sms * 2, kSsspScanThreads, 0, s>>>(a);
  k_sssp_relax<<<g->num_sms * 4, kSsspThreads, 0, s>>>(a);
  k_sssp_split<<<g->num_sms * 4, kSsspThreads, 0, s>>>(a);
  k_sssp_end<<<1, 32, 0, s>>>(a, h, use_cond);
  GR_CUDA(cudaGetLastError());
  return GR_OK;
}

static gr_status build_sssp_graph(gr_graph *g) {
  SsspWorkspace *ws = g->sssp;
  if (ws->exec) return GR_OK;
  cudaGraph_t graph;
  GR_CUDA(cudaGraphCreate(&graph, 0));
  cudaGraphConditionalHandle h;
  GR_CUDA(cudaGraphConditionalHandleCreate(&h, graph, 1, cudaGraphCondAssignDefault));
  cudaGraphNodeParams cp = {};
  cp.type = cudaGraphNodeTypeConditional;
  cp.conditional.handle = h;
  cp.conditional.type = cudaGraphCondTypeWhile;
  cp.conditional.size = 1;
  cudaGraphNode_t node;
  GR_CUDA(cudaGraphAddNode(&node, graph, nullptr, nullptr, 0, &cp));
  cudaGraph_t body = cp.conditional.phGraph_out[0];
  cudaStream_t cs;
  GR_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
  GR_CUDA(cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0,
                                        cudaStreamCaptureModeThreadLocal));
  gr_status st = sssp_enqueue_iter(g, sssp_args(g), cs, h, 1);
  cudaGraph_t captured;
  cudaError_t e = cudaStreamEndCapture(cs, &captured);
  cudaStreamDestroy(cs);
  if (st != GR_OK) return st;
  GR_CUDA(e);
  GR_CUDA(cudaGraphInstantiate(&ws->exec, graph, 0));
  ws->graph = graph;
  return GR_OK;
}

// default bucket width: a multiple of the mean weight (computed once)
static uint32_t tuned_delta(gr_graph *g) { return g->sssp_delta; }

}  // namespace gr

using namespace gr;

extern "C" {

gr_status gr_sssp(gr_graph *g, int32_t src, uint32_t *dist, int32_t *pred,
                  const gr_opts *opts, void *stream) {
  clear_error();
  if (!g) return fail(GR_EINVAL, "graph must not be NULL");
  if (!g->has_weights) return fail(GR_EINVAL, "SSSP needs edge weights (w was NULL at creation)");
  if (src < 0 || src >= g->n) return fail(GR_EINVAL, "source out of range");
  if (!dist) return fail(GR_EINVAL, "dist must not be NULL");
  const gr_opts &o = opts ? *opts : default_opts();
  if (o.mode < GR_MODE_AUTO || o.mode > GR_MODE_PERSISTENT)
    return fail(GR_EINVAL, "unknown mode");
  std::lock_guard<std::mutex> lock(g->mu);
  cudaStream_t s = (cudaStream_t)stream;
  GR_TRY(begin_call(g, s));
  GR_TRY(ensure_sssp_ws(g, s));
  const unsigned long long delta =
      o.delta == UINT32_MAX ? (1ull << 40) : (o.delta ? o.delta : tuned_delta(g));
  int32_t max_iters = o.max_iters > 0 ? o.max_iters : (int32_t)std::min<long long>(
                                                          INT32_MAX, 8ll * g->n + 1024);
  void *d_dist, *d_pred;
  bool cp_dist, cp_pred;
  GR_TRY(resolve_output(g, 0, dist, sizeof(uint32_t) * (size_t)g->n, &d_dist, &cp_dist));
  GR_TRY(resolve_output(g, 1, pred, sizeof(int32_t) * (size_t)g->n, &d_pred, &cp_pred));
  SsspArgs a = sssp_args(g);
  k_sssp_init<<<g->num_sms * 8, 256, 0, s>>>(a, src, (uint32_t *)d_dist, (int32_t *)d_pred,
                                             delta, max_iters);
  GR_CUDA(cudaGetLastError());
  if (o.mode == GR_MODE_LAUNCH || o.mode == GR_MODE_PERSISTENT) {
    SsspCtl h;
    int32_t enq = 0, batch = 8;
    for (;;) {
      for (int i = 0; i < batch; ++i) GR_TRY(sssp_enqueue_iter(g, a, s, 0, 0));
      enq += batch;
      GR_CUDA(cudaMemcpyAsync(&h, a.ctl, sizeof(h), cudaMemcpyDeviceToHost, s));
      GR_CUDA(cudaStreamSynchronize(s));
      if (h.done || enq > max_iters + 1) break;
      batch = std::min(batch * 2, 256);
    }
  } else {
    GR_TRY(build_sssp_graph(g));
    GR_CUDA(cudaGraphLaunch(g->sssp->exec, s));
  }
  if (d_pred) {
    const int grid = g->num_sms * 8;
    k_sssp_pred_init<<<grid, 256, 0, s>>>((int32_t *)d_pred, g->n);
    k_sssp_pred<<<grid, 256, 0, s>>>(a.R, a.C, a.W, (uint32_t *)d_dist, (int32_t *)d_pred,
                                     g->n, src);
    k_sssp_pred_fin<<<grid, 256, 0, s>>>((int32_t *)d_pred, g->n, src);
    GR_CUDA(cudaGetLastError());
  }
  if (cp_dist)
    GR_CUDA(cudaMemcpyAsync(dist, d_dist, sizeof(uint32_t) * (size_t)g->n,
                            cudaMemcpyDeviceToHost, s));
  if (cp_pred)
    GR_CUDA(cudaMemcpyAsync(pred, d_pred, sizeof(int32_t) * (size_t)g->n,
                            cudaMemcpyDeviceToHost, s));
  GR_TRY(end_call(g, s));
  return GR_OK;
}

gr_status gr_sssp_stats(gr_graph *g, int32_t *iterations, int32_t *phases,
                        int64_t *relaxations) {
  clear_error();
  if (!g) return fail(GR_EINVAL, "graph must not be NULL");
  if (!g->sssp) return fail(GR_EINVAL, "no SSSP has run on this graph");
  std::lock_guard<std::mutex> lock(g->mu);
  GR_CUDA(cudaSetDevice(g->device));
  if (g->has_last) GR_CUDA(cudaEventSynchronize(g->last_done));
  SsspCtl h;
  GR_CUDA(cudaMemcpy(&h, g->sssp->ctl.p, sizeof(h), cudaMemcpyDeviceToHost));
  if (h.error == kDevTimeout) return fail(GR_ETIMEOUT, "a device-side wait timed out");
  if (h.error == kDevOverflow) return fail(GR_ETIMEOUT, "iteration limit reached");
  if (iterations) *iterations = h.iter;
  if (phases) *phases = h.phases;
  if (relaxations) *relaxations = h.relaxations;
  return GR_OK;
}

}  // extern "C"
