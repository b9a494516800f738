// PageRank (Sec. 5.5) in pull form.
//
// The paper keeps every vertex in the frontier, accumulates with atomicAdd
// in an advance (push) and filters out converged vertices. Here each
// iteration gathers over in-neighbourhoods instead (the neighbourhood
// gather-reduce of Sec. 7), which computes the same sums without a scatter:
//
//   k_pr_gather  sum[v] = sum over edges (v, u) of contrib[u], contrib[u] =
//                rank[u] / deg(u), FP32 (merge-path chunks, segmented warp
//                sums, one atomicAdd per owner run)
//   k_pr_update  rank'[v] = (1 - d)/n + d * (sum[v] + D/n), D = rank mass on
//                degree-0 vertices; writes contrib' and clears sum; the
//                dangling mass of rank' and the L1 change sum |rank' - rank|
//                are reduced in FP64
//   k_pr_end     one thread: stops after max_iter iterations or once the L1
//                change is below tol
//
// In-neighbours equal out-neighbours only for a symmetric CSR; a directed
// CSR is transposed once on the device (counting sort by column) and the
// gather runs over the transpose with out-degrees from the original.
#include <algorithm>
#include <cstring>

#include "advance.cuh"

namespace gr {

// Gather tiles: 20 items for each of 96 threads, 8 blocks per SM with the
// L1 cache given the rest of the SM's shared-memory array. Long per-thread
// runs of independent gathers and a large L1 for the hub values beat more,
// smaller blocks (R-MAT s23, 50 iterations: 256 x 8 at 8 blocks per SM and
// the default carveout 1.92 ms per iteration, this 1.47 ms).
constexpr int kPrThreads = 96, kPrItems = 20, kPrBlocksPerSm = 8;

struct PrCtl {
  float *rank;           // output ranks (set per call, read by every kernel)
  double dangling;       // D of the current ranks
  double dangling_next;  // D of the ranks being produced
  double delta;          // L1 change of the last iteration
  double tol;
  float damping;
  int32_t iter;
  int32_t max_iter;
  int32_t done;
};

struct PrWorkspace {
  DevMem contrib, sum, ctl;
  DevMem cb;  // chunk bounds of the gather's merge path (fixed per graph)
  int gather_blocks = 0;  // resident gather blocks (all SMs)
  DevMem tr_off, tr_col;  // transpose (directed graphs only)
  bool has_transpose = false;
  cudaGraphExec_t exec = nullptr;
  cudaGraph_t graph = nullptr;
  ~PrWorkspace() {
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
  }
};

void free_pr(PrWorkspace *ws) { delete ws; }

GR_GUARD_REPORTER(guard_report_pr)

namespace {

struct PrArgs {
  const int32_t *R;   // gather structure (CSR or its transpose)
  const int32_t *C;
  const int32_t *deg; // out-degrees
  int32_t n;
  float *contrib;
  float *sum;
  PrCtl *ctl;
  const int32_t *cb;  // chunk bounds of the gather
};

__global__ void k_pr_init(PrArgs a, float *rank, float damping, int32_t max_iter, double tol,
                          int32_t num_dangling) {
  const float r0 = 1.0f / (float)a.n;
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < a.n;
       v += (int64_t)gridDim.x * blockDim.x) {
    rank[v] = r0;
    const int32_t d = a.deg[v];
    a.contrib[v] = d ? r0 / (float)d : 0.0f;
    a.sum[v] = 0.0f;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    PrCtl *c = a.ctl;
    c->rank = rank;
    c->dangling = (double)num_dangling / (double)a.n;
    c->dangling_next = 0.0;
    c->delta = 0.0;
    c->tol = tol;
    c->damping = damping;
    c->iter = 0;
    c->max_iter = max_iter;
    c->done = max_iter <= 0;
  }
}

struct ContribG {
  const float *contrib;
  __device__ __forceinline__ float operator()(int32_t u, int32_t) const { return __ldg(contrib + u); }
};

__global__ void __launch_bounds__(kPrThreads, kPrBlocksPerSm) k_pr_gather(PrArgs a) {
  if (a.ctl->done) return;
  ContribG g{a.contrib};
  lb_neighbor_reduce<kPrThreads, kPrItems, float>(a.R, a.C, a.n, g, a.sum, a.cb);
}

__global__ void __launch_bounds__(256) k_pr_update(PrArgs a) {
  PrCtl *c = a.ctl;
  if (c->done) return;
  const double d = c->damping;
  const double base = (1.0 - d) / a.n + d * c->dangling / a.n;
  float *rank = c->rank;
  double dang = 0.0, delta = 0.0;
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < a.n;
       v += (int64_t)gridDim.x * blockDim.x) {
    const float rn = (float)(base + d * (double)a.sum[v]);
    const float ro = rank[v];
    const int32_t dg = a.deg[v];
    rank[v] = rn;
    a.contrib[v] = dg ? rn / (float)dg : 0.0f;
    a.sum[v] = 0.0f;
    if (!dg) dang += rn;
    delta += fabs((double)rn - (double)ro);
  }
  __shared__ double s_red[33];
  dang = block_sum(dang, s_red);
  delta = block_sum(delta, s_red);
  if (threadIdx.x == 0) {
    if (dang != 0.0) atomicAdd(&c->dangling_next, dang);
    atomicAdd(&c->delta, delta);
  }
}

__global__ void k_pr_end(PrArgs a, cudaGraphConditionalHandle h, int32_t use_cond) {
  if (threadIdx.x != 0) return;
  PrCtl *c = a.ctl;
  if (!c->done) {
    c->iter += 1;
    c->dangling = c->dangling_next;
    c->dangling_next = 0.0;
    if (c->iter >= c->max_iter || c->delta < c->tol) c->done = 1;
    else c->delta = 0.0;
  }
  if (use_cond) cudaGraphSetConditional(h, c->done ? 0u : 1u);
}

// ---- transpose for directed graphs: counting sort of (u, v) by v
__global__ void k_tr_count(const int32_t *R, const int32_t *C, int32_t n, int32_t *cnt) {
  const int64_t gw = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t u = gw; u < n; u += nw)
    for (int32_t e = R[u] + (threadIdx.x & 31); e < R[u + 1]; e += 32) atomicAdd(cnt + C[e], 1);
}

__global__ void k_tr_fill(const int32_t *R, const int32_t *C, int32_t n, int32_t *pos,
                          int32_t *tcol) {
  const int64_t gw = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t u = gw; u < n; u += nw)
    for (int32_t e = R[u] + (threadIdx.x & 31); e < R[u + 1]; e += 32)
      tcol[atomicAdd(pos + C[e], 1)] = (int32_t)u;
}

// single-block exclusive scan of counts into offsets (one-time setup)
__global__ void k_tr_scan(const int32_t *cnt, int32_t n, int32_t *off, int32_t *pos) {
  __shared__ int32_t s_red[33];
  __shared__ int32_t s_carry;
  if (threadIdx.x == 0) s_carry = 0;
  __syncthreads();
  for (int64_t base = 0; base < n; base += blockDim.x) {
    const int64_t i = base + threadIdx.x;
    const int32_t x = i < n ? cnt[i] : 0;
    int32_t tot;
    const int32_t ex = block_excl_sum(x, s_red, &tot);
    if (i < n) {
      off[i] = s_carry + ex;
      pos[i] = s_carry + ex;
    }
    __syncthreads();
    if (threadIdx.x == 0) s_carry += tot;
    __syncthreads();
  }
  if (threadIdx.x == 0) off[n] = s_carry;
}

}  // namespace

static gr_status ensure_pr_ws(gr_graph *g, cudaStream_t s) {
  if (!g->pr) {
    std::unique_ptr<PrWorkspace> ws(new PrWorkspace());
    GR_TRY(ws->contrib.alloc(sizeof(float) * (size_t)g->n, "PageRank contributions"));
    GR_TRY(ws->sum.alloc(sizeof(float) * (size_t)g->n, "PageRank sums"));
    GR_TRY(ws->ctl.alloc(sizeof(PrCtl), "PageRank control"));
    int per_sm = 1;
    GR_TRY(fit_carveout(k_pr_gather, kPrThreads, kPrBlocksPerSm, g->device, &per_sm));
    ws->gather_blocks = per_sm * g->num_sms;
    g->pr = ws.release();
  }
  PrWorkspace *ws = g->pr;
  if (!g->symmetric && !ws->has_transpose) {
    GR_TRY(ws->tr_off.alloc(sizeof(int32_t) * ((size_t)g->n + 1), "transpose offsets"));
    GR_TRY(ws->tr_col.alloc(sizeof(int32_t) * (size_t)g->m, "transpose columns"));
    DevMem cnt, pos;
    GR_TRY(cnt.alloc(sizeof(int32_t) * (size_t)g->n, "transpose counts"));
    GR_TRY(pos.alloc(sizeof(int32_t) * (size_t)g->n, "transpose cursor"));
    GR_CUDA(cudaMemsetAsync(cnt.p, 0, cnt.bytes, s));
    const int grid = g->num_sms * 8;
    k_tr_count<<<grid, 256, 0, s>>>(g->row_off.as<int32_t>(), g->col.as<int32_t>(), g->n,
                                    cnt.as<int32_t>());
    k_tr_scan<<<1, 1024, 0, s>>>(cnt.as<int32_t>(), g->n, ws->tr_off.as<int32_t>(),
                                 pos.as<int32_t>());
    k_tr_fill<<<grid, 256, 0, s>>>(g->row_off.as<int32_t>(), g->col.as<int32_t>(), g->n,
                                   pos.as<int32_t>(), ws->tr_col.as<int32_t>());
    GR_CUDA(cudaGetLastError());
    GR_CUDA(cudaStreamSynchronize(s));
    ws->has_transpose = true;
  }
  if (!ws->cb.p) {
    // the gather's merge path over all vertices is the same every
    // iteration: its chunk bounds are found once
    const int32_t *R = g->symmetric ? g->row_off.as<int32_t>() : ws->tr_off.as<int32_t>();
    const int32_t chunks = merge_chunks(g->n, g->m, kPrThreads * kPrItems);
    GR_TRY(ws->cb.alloc(sizeof(int32_t) * ((size_t)chunks + 1), "PageRank chunk bounds"));
    k_chunk_bounds<<<(chunks + 256) / 256, 256, 0, s>>>(R, g->n, kPrThreads * kPrItems, chunks,
                                                         ws->cb.as<int32_t>());
    GR_CUDA(cudaGetLastError());
  }
  return GR_OK;
}

static PrArgs pr_args(gr_graph *g) {
  PrWorkspace *ws = g->pr;
  PrArgs a;
  a.R = g->symmetric ? g->row_off.as<int32_t>() : ws->tr_off.as<int32_t>();
  a.C = g->symmetric ? g->col.as<int32_t>() : ws->tr_col.as<int32_t>();
  a.deg = g->degree.as<int32_t>();
  a.n = g->n;
  a.contrib = ws->contrib.as<float>();
  a.sum = ws->sum.as<float>();
  a.ctl = ws->ctl.as<PrCtl>();
  a.cb = ws->cb.as<int32_t>();
  return a;
}

static gr_status pr_enqueue_iter(gr_graph *g, const PrArgs &a, cudaStream_t s,
                                 cudaGraphConditionalHandle h, int use_cond) {
  k_pr_gather<<<g->pr->gather_blocks, kPrThreads, 0, s>>>(a);
  k_pr_update<<<g->num_sms * 4, 256, 0, s>>>(a);
  k_pr_end<<<1, 32, 0, s>>>(a, h, use_cond);
  GR_CUDA(cudaGetLastError());
  return GR_OK;
}

static gr_status build_pr_graph(gr_graph *g) {
  PrWorkspace *ws = g->pr;
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
  gr_status st = pr_enqueue_iter(g, pr_args(g), cs, h, 1);
  cudaGraph_t captured;
  cudaError_t e = cudaStreamEndCapture(cs, &captured);
  cudaStreamDestroy(cs);
  if (st != GR_OK) return st;
  GR_CUDA(e);
  GR_CUDA(cudaGraphInstantiate(&ws->exec, graph, 0));
  ws->graph = graph;
  return GR_OK;
}

}  // namespace gr

using namespace gr;

extern "C" {

gr_status gr_pagerank(gr_graph *g, float damping, int32_t max_iter, double tol, float *rank,
                      int32_t *iters, const gr_opts *opts, void *stream) {
  clear_error();
  if (!g) return fail(GR_EINVAL, "graph must not be NULL");
  if (!(damping > 0.0f && damping < 1.0f)) return fail(GR_EINVAL, "damping must be in (0, 1)");
  if (max_iter < 0) return fail(GR_EINVAL, "max_iter must be >= 0");
  if (!(tol >= 0.0)) return fail(GR_EINVAL, "tol must be >= 0");
  if (!rank) return fail(GR_EINVAL, "rank must not be NULL");
  const gr_opts &o = opts ? *opts : default_opts();
  std::lock_guard<std::mutex> lock(g->mu);
  cudaStream_t s = (cudaStream_t)stream;
  GR_TRY(begin_call(g, s));
  GR_TRY(ensure_pr_ws(g, s));
  void *d_rank;
  bool cp_rank;
  GR_TRY(resolve_output(g, 0, rank, sizeof(float) * (size_t)g->n, &d_rank, &cp_rank));
  PrArgs a = pr_args(g);
  k_pr_init<<<g->num_sms * 8, 256, 0, s>>>(a, (float *)d_rank, damping, max_iter, tol,
                                           g->num_isolated);
  GR_CUDA(cudaGetLastError());
  if (max_iter > 0) {
    if (o.mode == GR_MODE_LAUNCH) {
      PrCtl h;
      for (int32_t it = 0; it < max_iter;) {
        const int32_t batch = std::min<int32_t>(8, max_iter - it);
        for (int32_t i = 0; i < batch; ++i) GR_TRY(pr_enqueue_iter(g, a, s, 0, 0));
        it += batch;
        GR_CUDA(cudaMemcpyAsync(&h, a.ctl, sizeof(h), cudaMemcpyDeviceToHost, s));
        GR_CUDA(cudaStreamSynchronize(s));
        if (h.done) break;
      }
    } else {
      GR_TRY(build_pr_graph(g));
      GR_CUDA(cudaGraphLaunch(g->pr->exec, s));
    }
  }
  if (cp_rank)
    GR_CUDA(cudaMemcpyAsync(rank, d_rank, sizeof(float) * (size_t)g->n,
                            cudaMemcpyDeviceToHost, s));
  if (iters) {
    PrCtl h;
    GR_CUDA(cudaMemcpyAsync(&h, a.ctl, sizeof(h), cudaMemcpyDeviceToHost, s));
    GR_CUDA(cudaStreamSynchronize(s));
    *iters = h.iter;
  }
  GR_TRY(end_call(g, s));
  return GR_OK;
}

}  // extern "C"
