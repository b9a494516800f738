// Breadth-first search over the frontier operators (Sec. 5.1).
//
// One BFS level is a fixed sequence of kernels that read every decision from
// a device-resident control block, so the level loop needs no host round
// trip:
//
//   k_bfs_scan   exclusive scan of the frontier's degrees (the "scanned edge
//                offset queue" of Sec. 4.4), single pass with decoupled
//                look-back; its last tile applies the push->pull rule
//                (Sec. 4.5) because only then are the frontier's edges known.
//   k_bfs_push   advance + filter fused (Sec. 4.3 kernel fusion): merge-path
//                partitioning of frontier vertices and their edges into
//                equal chunks (Sec. 4.4 load-balanced partitioning, merging
//                vertex ends with edge ranks), coalesced column loads, a
//                plain-load visited-bitmap cull, one atomicOr claim per
//                surviving candidate so that each vertex enters the next
//                frontier once (the non-idempotent advance of Sec. 4.5), and
//                a warp-aggregated compaction into the next queue.
//   k_bfs_pull   bottom-up advance (Sec. 4.5): every unvisited vertex scans
//                its neighbours for one in the frontier bitmap and stops at
//                the first. A warp owns 32 consecutive vertices, i.e. one
//                bitmap word, so the visited and next-frontier bitmaps are
//                written with a ballot and a plain store: no atomics.
//   k_bfs_level_end  one thread: swaps queues, applies the pull->push rule,
//                detects the empty frontier and, inside a CUDA graph, sets
//                the while-loop condition.
//
// The level loop runs either as a CUDA graph with a device-side while node
// (GR_MODE_GRAPH) or as host-enqueued batches of levels whose kernels exit at
// once after the traversal finished (GR_MODE_LAUNCH). A cooperative
// persistent kernel (GR_MODE_PERSISTENT) serves graphs with thousands of
// small levels.
#include <cooperative_groups.h>

#include <algorithm>
#include <cstring>

#include "advance.cuh"

namespace gr {

enum : int32_t { kPush = 0, kPull = 1 };

struct BfsCtl {
  int32_t *depth;
  int32_t *parent;
  int32_t src;
  int32_t level;        // depth of the current frontier
  int32_t parity;       // which queue / bitmap holds the current frontier
  int32_t dir;          // direction of the current level
  int32_t q_len;        // current frontier size
  int32_t q_prev;       // previous frontier size
  int32_t next_len;     // next frontier size (atomic counter)
  int32_t tile_ctr;     // scan tile counter (atomic)
  int32_t done;
  int32_t error;
  int32_t pull_levels;
  int32_t policy;       // GR_DIR_*
  int32_t mf_pending;   // 1: frontier edge count not yet known (push level)
  int32_t max_levels;
  uint32_t epoch;       // tags scan tile status words; never reset
  int32_t barrier_gen;  // persistent-kernel grid barrier generation
  int32_t barrier_cnt;  // persistent-kernel grid barrier arrivals
  int32_t pad;
  long long mf;         // edges leaving the current frontier
  long long next_mf;    // edges leaving the next frontier (pull producer)
  long long mu;         // edges of still-unexplored vertices
  float alpha;
  float beta;
};

struct BfsArgs {
  const int32_t *R;
  const int32_t *C;
  int32_t n;
  int32_t nwords;
  long long m;
  const uint32_t *iso;
  int32_t *q[2];
  int32_t *scan;
  uint32_t *visited;
  uint32_t *fb[2];
  unsigned long long *status;
  BfsCtl *ctl;
  int32_t do_bitmap;
};

// launch shapes
constexpr int kScanThreads = 512;
constexpr int kScanItems = 4;
constexpr int kScanTile = kScanThreads * kScanItems;
constexpr int kPushThreads = 256;
constexpr int kPushItems = 8;
constexpr int kPullThreads = 256;
constexpr int kPullFlushRounds = 8;

struct BfsWorkspace {
  DevMem q[2], scan, visited, fb[2], status, ctl;
  PinnedMem h_ctl;
  int32_t ntiles = 0;
  cudaGraphExec_t exec[2] = {nullptr, nullptr};  // by do_bitmap
  cudaGraph_t graph[2] = {nullptr, nullptr};
  ~BfsWorkspace() {
    for (int i = 0; i < 2; ++i) {
      if (exec[i]) cudaGraphExecDestroy(exec[i]);
      if (graph[i]) cudaGraphDestroy(graph[i]);
    }
  }
};

void free_bfs(BfsWorkspace *ws) { delete ws; }

// ------------------------------------------------------------- kernels
namespace {

// select by parity without indexing the parameter arrays (a dynamic index
// would copy the kernel parameters to local memory)
__device__ __forceinline__ int32_t *queue_of(const BfsArgs &a, int p) { return p ? a.q[1] : a.q[0]; }
__device__ __forceinline__ uint32_t *bits_of(const BfsArgs &a, int p) { return p ? a.fb[1] : a.fb[0]; }

__global__ void k_bfs_init(BfsArgs a, int32_t src, int32_t *depth, int32_t *parent,
                           int32_t policy, float alpha, float beta,
                           int32_t max_levels, int32_t preset_iso) {
  int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t v = tid; v < a.n; v += stride) {
    depth[v] = v == src ? 0 : -1;
    if (parent) parent[v] = v == src ? src : -1;
  }
  const int32_t sw = src >> 5;
  const uint32_t sb = 1u << (src & 31);
  for (int64_t w = tid; w < a.nwords; w += stride) {
    uint32_t vis = preset_iso ? a.iso[w] : 0u;
    if (w == sw) vis |= sb;
    a.visited[w] = vis;
    if (a.do_bitmap) a.fb[0][w] = (w == sw) ? sb : 0u;
  }
  if (tid == 0) {
    BfsCtl *c = a.ctl;
    a.q[0][0] = src;
    c->depth = depth;
    c->parent = parent;
    c->src = src;
    c->level = 0;
    c->parity = 0;
    c->dir = kPush;
    c->q_len = 1;
    c->q_prev = 0;
    c->next_len = 0;
    c->tile_ctr = 0;
    c->done = 0;
    c->error = kDevOk;
    c->pull_levels = 0;
    c->policy = policy;
    c->mf_pending = 1;
    c->max_levels = max_levels;
    c->barrier_gen = 0;
    c->barrier_cnt = 0;
    c->mf = 0;
    c->next_mf = 0;
    c->mu = a.m;
    c->alpha = alpha;
    c->beta = beta;
  }
}

__global__ void __launch_bounds__(kScanThreads) k_bfs_scan(BfsArgs a) {
  BfsCtl *c = a.ctl;
  if (c->done || c->error || c->dir != kPush) return;
  const int32_t p = c->parity;
  if (a.do_bitmap) {
    uint32_t *N = bits_of(a, p ^ 1);
    for (int64_t w = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; w < a.nwords;
         w += (int64_t)gridDim.x * blockDim.x)
      N[w] = 0u;
  }
  ScanState st{a.status, &c->tile_ctr, &c->error, c->epoch};
  long long total;
  if (frontier_degree_scan<kScanThreads, kScanItems>(a.R, queue_of(a, p), c->q_len, a.scan,
                                                     st, &total)) {
    // last tile: the frontier's edge count is known; apply push -> pull
    if (c->mf_pending) c->mu -= total;
    c->mf_pending = 0;
    c->mf = total;
    if (c->policy == GR_DIR_AUTO && (float)total > (float)c->mu / c->alpha) c->dir = kPull;
  }
}

// Push functor: plain-load cull on the visited bitmap, then one atomicOr
// claim; the unique winner writes depth/parent and the next-frontier bit.
struct BfsPushF {
  uint32_t *visited;
  uint32_t *next_bits;
  int32_t *depth;
  int32_t *parent;
  int32_t next_level;
  int32_t do_bitmap;
  __device__ __forceinline__ int operator()(int32_t u, int32_t v, int32_t) const {
    const uint32_t mask = 1u << (v & 31);
    uint32_t *vw = visited + (v >> 5);
    if (*vw & mask) return 0;
    if (atomicOr(vw, mask) & mask) return 0;
    depth[v] = next_level;
    if (parent) parent[v] = u;
    if (do_bitmap) atomicOr(next_bits + (v >> 5), mask);
    return 1;
  }
};

__global__ void __launch_bounds__(kPushThreads) k_bfs_push(BfsArgs a) {
  BfsCtl *c = a.ctl;
  if (c->done || c->error || c->dir != kPush) return;
  const int32_t p = c->parity;
  BfsPushF f{a.visited, bits_of(a, p ^ 1), c->depth, c->parent, c->level + 1, a.do_bitmap};
  int32_t unused = 0;
  lb_advance<kPushThreads, kPushItems, 1>(a.R, a.C, queue_of(a, p), c->q_len, a.scan, f,
                                          queue_of(a, p ^ 1), &c->next_len, nullptr, &unused);
}

__global__ void __launch_bounds__(kPullThreads) k_bfs_pull(BfsArgs a) {
  BfsCtl *c = a.ctl;
  if (c->done || c->error || c->dir != kPull) return;
  const int32_t p = c->parity;
  const int32_t L = c->level;
  const uint32_t *F = bits_of(a, p);
  uint32_t *N = bits_of(a, p ^ 1);
  int32_t *Qn = queue_of(a, p ^ 1);
  int32_t *depth = c->depth;
  int32_t *parent = c->parent;

  constexpr int kWarps = kPullThreads / 32;
  constexpr int kCap = kPullThreads * kPullFlushRounds;
  __shared__ int32_t s_out[kCap];
  __shared__ int32_t s_cnt, s_base;
  __shared__ long long s_red[33];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (threadIdx.x == 0) s_cnt = 0;
  __syncthreads();
  const long long words_per_round = (long long)gridDim.x * kWarps;
  const int32_t rounds = (int32_t)((a.nwords + words_per_round - 1) / words_per_round);
  long long local_mf = 0;
  for (int32_t r = 0; r < rounds; ++r) {
    const long long w = ((long long)r * gridDim.x + blockIdx.x) * kWarps + wid;
    if (w < a.nwords) {
      const uint32_t vis = a.visited[w];
      const int32_t v = (int32_t)(w * 32 + lane);
      bool found = false;
      int32_t uf = -1, deg = 0;
      if (v < a.n && !((vis >> lane) & 1u)) {
        const int32_t r0 = a.R[v], r1 = a.R[v + 1];
        for (int32_t e = r0; e < r1; ++e) {
          const int32_t u = a.C[e];
          if (test_bit(F, u)) {
            found = true;
            uf = u;
            break;
          }
        }
        if (found) deg = r1 - r0;
      }
      const uint32_t fm = __ballot_sync(0xffffffffu, found);
      if (lane == 0) {
        N[w] = fm;
        if (fm) a.visited[w] = vis | fm;
      }
      if (found) {
        depth[v] = L + 1;
        if (parent) parent[v] = uf;
        local_mf += deg;
      }
      if (fm) {
        int32_t pos = 0;
        if (lane == 0) pos = atomicAdd(&s_cnt, __popc(fm));
        pos = __shfl_sync(0xffffffffu, pos, 0);
        if (found) s_out[pos + __popc(fm & ((1u << lane) - 1u))] = v;
      }
    }
    if ((r + 1) % kPullFlushRounds == 0 || r == rounds - 1) {
      __syncthreads();
      if (threadIdx.x == 0) s_base = s_cnt ? atomicAdd(&c->next_len, s_cnt) : 0;
      __syncthreads();
      for (int32_t k = threadIdx.x; k < s_cnt; k += kPullThreads) Qn[s_base + k] = s_out[k];
      __syncthreads();
      if (threadIdx.x == 0) s_cnt = 0;
      __syncthreads();
    }
  }
  const long long mf = block_sum(local_mf, s_red);
  if (threadIdx.x == 0 && mf) atomicAdd((unsigned long long *)&c->next_mf, (unsigned long long)mf);
}

__device__ __forceinline__ void level_end_body(const BfsArgs &a) {
  BfsCtl *c = a.ctl;
  if (c->done) return;
  if (c->error) {
    c->done = 1;
    return;
  }
  const int32_t qn = c->next_len;
  const bool was_pull = c->dir == kPull;
  if (was_pull) {
    c->mf = c->next_mf;
    c->mu -= c->next_mf;
    c->pull_levels += 1;
    c->mf_pending = 0;
  } else {
    c->mf_pending = 1;
  }
  c->level += 1;
  c->parity ^= 1;
  c->q_prev = c->q_len;
  c->q_len = qn;
  c->next_len = 0;
  c->next_mf = 0;
  c->tile_ctr = 0;
  c->epoch += 1;
  if (qn == 0) {
    c->done = 1;
    return;
  }
  if (c->level >= c->max_levels) {
    c->error = kDevOverflow;
    c->done = 1;
    return;
  }
  if (c->policy == GR_DIR_PUSH) {
    c->dir = kPush;
  } else if (c->policy == GR_DIR_PULL) {
    c->dir = kPull;
  } else if (was_pull) {
    c->dir = ((float)qn < (float)a.n / c->beta && qn < c->q_prev) ? kPush : kPull;
  } else {
    c->dir = kPush;  // the next scan may still switch to pull
  }
}

__global__ void k_bfs_level_end(BfsArgs a, cudaGraphConditionalHandle h, int32_t use_cond) {
  if (threadIdx.x != 0) return;
  level_end_body(a);
  if (use_cond) cudaGraphSetConditional(h, a.ctl->done ? 0u : 1u);
}

// ------------------------------------------------- persistent (push only)
// One cooperative grid runs every level. Per level each warp takes frontier
// vertices in turn and expands their neighbour lists lane-parallel; winners
// of the visited-bitmap claim are appended with one atomic per warp. Levels
// are separated by a sense-reversing grid barrier whose spin is bounded.
constexpr int kPersThreads = 256;

__device__ __forceinline__ bool grid_barrier(BfsCtl *c, int32_t nblocks, int32_t &gen) {
  __syncthreads();
  bool ok = true;
  if (threadIdx.x == 0) {
    __threadfence();
    const int32_t my_gen = gen;
    if (atomicAdd(&c->barrier_cnt, 1) == nblocks - 1) {
      c->barrier_cnt = 0;
      __threadfence();
      atomicExch(&c->barrier_gen, my_gen + 1);
    } else {
      int64_t spins = 0;
      while (*(volatile int32_t *)&c->barrier_gen == my_gen) {
        if (++spins > kSpinLimit) {
          atomicExch(&c->error, kDevTimeout);
          ok = false;
          break;
        }
        __nanosleep(32);
      }
    }
    __threadfence();
  }
  gen += 1;
  __syncthreads();
  return ok;
}

__global__ void __launch_bounds__(kPersThreads) k_bfs_persistent(BfsArgs a) {
  BfsCtl *c = a.ctl;
  int32_t *depth = c->depth;
  int32_t *parent = c->parent;
  const int32_t nblocks = gridDim.x;
  const int lane = threadIdx.x & 31;
  const long long gwarp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
  int32_t gen = 0;
  __shared__ int32_t s_done;
  for (;;) {
    if (threadIdx.x == 0) s_done = *(volatile int32_t *)&c->done | *(volatile int32_t *)&c->error;
    __syncthreads();
    if (s_done) break;
    const int32_t p = *(volatile int32_t *)&c->parity;
    const int32_t q = *(volatile int32_t *)&c->q_len;
    const int32_t L = *(volatile int32_t *)&c->level;
    const int32_t *Q = queue_of(a, p);
    int32_t *Qn = queue_of(a, p ^ 1);
    for (long long i = gwarp; i < q; i += nwarps) {
      const int32_t u = Q[i];
      const int32_t r0 = a.R[u], r1 = a.R[u + 1];
      for (int32_t eb = r0; eb < r1; eb += 32) {
        const int32_t e = eb + lane;
        bool won = false;
        int32_t v = 0;
        if (e < r1) {
          v = a.C[e];
          const uint32_t mask = 1u << (v & 31);
          uint32_t *vw = a.visited + (v >> 5);
          if (!(*(volatile uint32_t *)vw & mask)) won = !(atomicOr(vw, mask) & mask);
          if (won) {
            depth[v] = L + 1;
            if (parent) parent[v] = u;
          }
        }
        const uint32_t bal = __ballot_sync(0xffffffffu, won);
        if (bal) {
          int32_t pos = 0;
          if (lane == 0) pos = atomicAdd(&c->next_len, __popc(bal));
          pos = __shfl_sync(0xffffffffu, pos, 0);
          if (won) Qn[pos + __popc(bal & ((1u << lane) - 1u))] = v;
        }
      }
    }
    if (!grid_barrier(c, nblocks, gen)) break;
    if (blockIdx.x == 0 && threadIdx.x == 0) level_end_body(a);
    if (!grid_barrier(c, nblocks, gen)) break;
  }
}

}  // namespace

// ---------------------------------------------------------------- host
static gr_status ensure_bfs_ws(gr_graph *g, cudaStream_t s) {
  if (g->bfs) return GR_OK;
  std::unique_ptr<BfsWorkspace> ws(new BfsWorkspace());
  const size_t n = (size_t)g->n;
  GR_TRY(ws->q[0].alloc(sizeof(int32_t) * (n + 1), "BFS queue"));
  GR_TRY(ws->q[1].alloc(sizeof(int32_t) * (n + 1), "BFS queue"));
  GR_TRY(ws->scan.alloc(sizeof(int32_t) * (n + 2), "BFS degree scan"));
  GR_TRY(ws->visited.alloc(sizeof(uint32_t) * g->nwords, "visited bitmap"));
  GR_TRY(ws->fb[0].alloc(sizeof(uint32_t) * g->nwords, "frontier bitmap"));
  GR_TRY(ws->fb[1].alloc(sizeof(uint32_t) * g->nwords, "frontier bitmap"));
  ws->ntiles = (int32_t)((n + kScanTile) / kScanTile) + 1;
  GR_TRY(ws->status.alloc(sizeof(unsigned long long) * ws->ntiles, "scan status"));
  GR_TRY(ws->ctl.alloc(sizeof(BfsCtl), "BFS control"));
  GR_TRY(ws->h_ctl.alloc(sizeof(BfsCtl), "BFS control mirror"));
  GR_CUDA(cudaMemsetAsync(ws->status.p, 0, ws->status.bytes, s));
  BfsCtl init;
  std::memset(&init, 0, sizeof(init));
  init.epoch = 1;
  GR_CUDA(cudaMemcpyAsync(ws->ctl.p, &init, sizeof(init), cudaMemcpyHostToDevice, s));
  GR_CUDA(cudaStreamSynchronize(s));
  g->bfs = ws.release();
  return GR_OK;
}

static BfsArgs make_args(gr_graph *g, int32_t do_bitmap) {
  BfsWorkspace *ws = g->bfs;
  BfsArgs a;
  a.R = g->row_off.as<int32_t>();
  a.C = g->col.as<int32_t>();
  a.n = g->n;
  a.nwords = g->nwords;
  a.m = g->m;
  a.iso = g->isolated_bits.as<uint32_t>();
  a.q[0] = ws->q[0].as<int32_t>();
  a.q[1] = ws->q[1].as<int32_t>();
  a.scan = ws->scan.as<int32_t>();
  a.visited = ws->visited.as<uint32_t>();
  a.fb[0] = ws->fb[0].as<uint32_t>();
  a.fb[1] = ws->fb[1].as<uint32_t>();
  a.status = ws->status.as<unsigned long long>();
  a.ctl = ws->ctl.as<BfsCtl>();
  a.do_bitmap = do_bitmap;
  return a;
}

struct Grids {
  int scan, push, pull;
};

static Grids grids_for(const gr_graph *g) {
  Grids gr_;
  gr_.scan = g->num_sms * 2;
  gr_.push = g->num_sms * 4;
  gr_.pull = g->num_sms * 8;
  return gr_;
}

static gr_status enqueue_level(const BfsArgs &a, const Grids &gd, cudaStream_t s,
                               cudaGraphConditionalHandle h, int use_cond) {
  k_bfs_scan<<<gd.scan, kScanThreads, 0, s>>>(a);
  k_bfs_push<<<gd.push, kPushThreads, 0, s>>>(a);
  if (a.do_bitmap) k_bfs_pull<<<gd.pull, kPullThreads, 0, s>>>(a);
  k_bfs_level_end<<<1, 32, 0, s>>>(a, h, use_cond);
  GR_CUDA(cudaGetLastError());
  return GR_OK;
}

static gr_status build_level_graph(gr_graph *g, int32_t do_bitmap) {
  BfsWorkspace *ws = g->bfs;
  if (ws->exec[do_bitmap]) return GR_OK;
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
  BfsArgs a = make_args(g, do_bitmap);
  gr_status st = enqueue_level(a, grids_for(g), cs, h, 1);
  cudaGraph_t captured;
  cudaError_t e = cudaStreamEndCapture(cs, &captured);
  cudaStreamDestroy(cs);
  if (st != GR_OK) return st;
  GR_CUDA(e);
  cudaGraphExec_t exec;
  GR_CUDA(cudaGraphInstantiate(&exec, graph, 0));
  ws->graph[do_bitmap] = graph;
  ws->exec[do_bitmap] = exec;
  return GR_OK;
}

static int32_t resolve_policy(const gr_graph *g, const gr_opts &o) {
  if (o.direction == GR_DIR_PUSH) return GR_DIR_PUSH;
  if (o.direction == GR_DIR_PULL) return GR_DIR_PULL;
  return g->symmetric ? GR_DIR_AUTO : GR_DIR_PUSH;
}

// mode AUTO: graphs whose traversals are long chains of small frontiers
// (low maximum degree, large n) run the persistent kernel; others the
// device-side while loop.
static int32_t resolve_mode(const gr_graph *g, const gr_opts &o, int32_t policy) {
  if (o.mode != GR_MODE_AUTO) return o.mode;
  if (policy == GR_DIR_PUSH && g->max_degree <= 32 && g->n >= (1 << 16))
    return GR_MODE_PERSISTENT;
  return GR_MODE_GRAPH;
}

}  // namespace gr

using namespace gr;

extern "C" {

gr_status gr_bfs(gr_graph *g, int32_t src, int32_t *depth, int32_t *parent,
                 const gr_opts *opts, void *stream) {
  clear_error();
  if (!g) return fail(GR_EINVAL, "graph must not be NULL");
  if (src < 0 || src >= g->n) return fail(GR_EINVAL, "source out of range");
  if (!depth) return fail(GR_EINVAL, "depth must not be NULL");
  const gr_opts &o = opts ? *opts : default_opts();
  if (o.direction < GR_DIR_AUTO || o.direction > GR_DIR_PULL)
    return fail(GR_EINVAL, "unknown direction policy");
  if (o.mode < GR_MODE_AUTO || o.mode > GR_MODE_PERSISTENT)
    return fail(GR_EINVAL, "unknown mode");
  if (o.direction == GR_DIR_PULL && !g->symmetric)
    return fail(GR_EINVAL, "pull traversal needs a symmetric CSR (in-neighbours = out-neighbours)");
  if (o.alpha < 0.f || o.beta < 0.f) return fail(GR_EINVAL, "alpha/beta must be >= 0");
  std::lock_guard<std::mutex> lock(g->mu);
  cudaStream_t s = (cudaStream_t)stream;
  GR_TRY(begin_call(g, s));
  GR_TRY(ensure_bfs_ws(g, s));
  const int32_t policy = resolve_policy(g, o);
  const int32_t mode = resolve_mode(g, o, policy);
  if (mode == GR_MODE_PERSISTENT && policy != GR_DIR_PUSH)
    return fail(GR_EINVAL, "the persistent BFS kernel runs push levels only");
  const int32_t do_bitmap = policy != GR_DIR_PUSH;
  const float alpha = o.alpha > 0.f ? o.alpha : 14.f;
  const float beta = o.beta > 0.f ? o.beta : 24.f;
  int32_t max_levels = g->n + 1;
  if (o.max_iters > 0) max_levels = std::min(max_levels, o.max_iters);

  void *d_depth, *d_parent;
  bool cp_depth, cp_parent;
  GR_TRY(resolve_output(g, 0, depth, sizeof(int32_t) * (size_t)g->n, &d_depth, &cp_depth));
  GR_TRY(resolve_output(g, 1, parent, sizeof(int32_t) * (size_t)g->n, &d_parent, &cp_parent));

  BfsArgs a = make_args(g, do_bitmap);
  const int init_grid = g->num_sms * 8;
  k_bfs_init<<<init_grid, 256, 0, s>>>(a, src, (int32_t *)d_depth, (int32_t *)d_parent,
                                       policy, alpha, beta, max_levels,
                                       (g->symmetric && do_bitmap) ? 1 : 0);
  GR_CUDA(cudaGetLastError());

  if (mode == GR_MODE_GRAPH) {
    GR_TRY(build_level_graph(g, do_bitmap));
    GR_CUDA(cudaGraphLaunch(g->bfs->exec[do_bitmap], s));
  } else if (mode == GR_MODE_PERSISTENT) {
    int per_sm = 0;
    GR_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_bfs_persistent,
                                                          kPersThreads, 0));
    int blocks = std::max(1, std::min(per_sm, 4)) * g->num_sms;
    void *args[] = {&a};
    GR_CUDA(cudaLaunchCooperativeKernel((void *)k_bfs_persistent, blocks, kPersThreads,
                                        args, 0, s));
  } else {
    // host-driven: enqueue batches of levels, then check the done flag
    const Grids gd = grids_for(g);
    BfsCtl *h = g->bfs->h_ctl.as<BfsCtl>();
    int32_t levels_enqueued = 0;
    int32_t batch = 4;
    for (;;) {
      for (int i = 0; i < batch; ++i) GR_TRY(enqueue_level(a, gd, s, 0, 0));
      levels_enqueued += batch;
      GR_CUDA(cudaMemcpyAsync(h, g->bfs->ctl.p, sizeof(BfsCtl), cudaMemcpyDeviceToHost, s));
      GR_CUDA(cudaStreamSynchronize(s));
      if (h->done || levels_enqueued > max_levels) break;
      batch = std::min(batch * 2, 64);
    }
  }
  if (cp_depth)
    GR_CUDA(cudaMemcpyAsync(depth, d_depth, sizeof(int32_t) * (size_t)g->n,
                            cudaMemcpyDeviceToHost, s));
  if (cp_parent)
    GR_CUDA(cudaMemcpyAsync(parent, d_parent, sizeof(int32_t) * (size_t)g->n,
                            cudaMemcpyDeviceToHost, s));
  GR_TRY(end_call(g, s));
  return GR_OK;
}

gr_status gr_bfs_stats(gr_graph *g, int32_t *levels, int32_t *pull_levels) {
  clear_error();
  if (!g) return fail(GR_EINVAL, "graph must not be NULL");
  if (!g->bfs) return fail(GR_EINVAL, "no BFS has run on this graph");
  std::lock_guard<std::mutex> lock(g->mu);
  GR_CUDA(cudaSetDevice(g->device));
  if (g->has_last) GR_CUDA(cudaEventSynchronize(g->last_done));
  BfsCtl h;
  GR_CUDA(cudaMemcpy(&h, g->bfs->ctl.p, sizeof(BfsCtl), cudaMemcpyDeviceToHost));
  if (h.error == kDevTimeout) return fail(GR_ETIMEOUT, "a device-side wait timed out");
  if (h.error == kDevOverflow) return fail(GR_ETIMEOUT, "level limit reached");
  if (levels) *levels = h.level;
  if (pull_levels) *pull_levels = h.pull_levels;
  return GR_OK;
}

}  // extern "C"

// ------------------------------------------------- no-allocation variant
// BFS for callers that must not allocate device memory. Its scratch (the
// control block, two frontier queues and the visited bitmap) lives in one
// file-scope device array sized for kNoAllocMaxVertices vertices; every GPU
// that loads this library holds that array until the process exits.
namespace gr {
namespace {

constexpr int32_t kNoAllocMaxVertices = 1 << 20;
constexpr size_t kNoAllocCtlBytes = 256;  // BfsCtl, padded to 256 bytes
constexpr size_t kNoAllocQueueBytes = sizeof(int32_t) * ((size_t)kNoAllocMaxVertices + 1);
constexpr size_t kNoAllocQueueBytesAligned = (kNoAllocQueueBytes + 255) & ~size_t(255);
constexpr size_t kNoAllocVisitedBytes = sizeof(uint32_t) * (kNoAllocMaxVertices / 32);
constexpr size_t kNoAllocScratchBytes =
    kNoAllocCtlBytes + 2 * kNoAllocQueueBytesAligned + kNoAllocVisitedBytes;
static_assert(sizeof(BfsCtl) <= kNoAllocCtlBytes, "control block does not fit its slot");

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

// device address of g_noalloc_scratch, looked up once per device
constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
void *g_noalloc_addr[kMaxDevices] = {};
int g_noalloc_sms[kMaxDevices] = {};
int g_noalloc_blocks_per_sm[kMaxDevices] = {};

gr_status noalloc_setup(int dev, void **addr, int *sms, int *per_sm) {
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_addr[dev]) {
    void *p = nullptr;
    GR_CUDA(cudaGetSymbolAddress(&p, g_noalloc_scratch));
    int nsm = 0, occ = 0;
    GR_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    GR_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_bfs_persistent,
                                                          kPersThreads, 0));
    g_noalloc_sms[dev] = nsm;
    g_noalloc_blocks_per_sm[dev] = std::max(1, std::min(occ, 4));
    g_noalloc_addr[dev] = p;
  }
  *addr = g_noalloc_addr[dev];
  *sms = g_noalloc_sms[dev];
  *per_sm = g_noalloc_blocks_per_sm[dev];
  return GR_OK;
}

}  // namespace
}  // namespace gr

extern "C" gr_status gr_bfs_noalloc(int32_t n, int64_t m, const int32_t *row_off,
                                    const int32_t *col, int32_t src, int32_t *depth,
                                    int32_t *parent, void *stream) {
  using namespace gr;
  clear_error();
  if (n < 1 || n > kNoAllocMaxVertices)
    return fail(GR_EINVAL, "n must be in [1, " + std::to_string(kNoAllocMaxVertices) +
                               "]: gr_bfs_noalloc has a fixed scratch for at most that "
                               "many vertices (use gr_graph_create + gr_bfs above it)");
  if (m < 0 || m > INT32_MAX) return fail(GR_EINVAL, "m must be in [0, INT32_MAX]");
  if (!row_off || (m > 0 && !col)) return fail(GR_EINVAL, "row_off/col must not be NULL");
  if (!depth) return fail(GR_EINVAL, "depth must not be NULL");
  if (src < 0 || src >= n) return fail(GR_EINVAL, "source out of range");
  int dev = 0;
  GR_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) return fail(GR_EINVAL, "device ordinal too large");
  void *base = nullptr;
  int sms = 0, per_sm = 0;
  GR_TRY(noalloc_setup(dev, &base, &sms, &per_sm));
  unsigned char *p = (unsigned char *)base;
  BfsArgs a;
  std::memset(&a, 0, sizeof(a));
  a.R = row_off;
  a.C = col;
  a.n = n;
  a.nwords = (n + 31) / 32;
  a.m = m;
  a.ctl = (BfsCtl *)p;
  a.q[0] = (int32_t *)(p + kNoAllocCtlBytes);
  a.q[1] = (int32_t *)(p + kNoAllocCtlBytes + kNoAllocQueueBytesAligned);
  a.visited = (uint32_t *)(p + kNoAllocCtlBytes + 2 * kNoAllocQueueBytesAligned);
  a.do_bitmap = 0;
  cudaStream_t s = (cudaStream_t)stream;
  // the init kernel clears the control block and the visited bitmap
  k_bfs_init<<<sms * 4, 256, 0, s>>>(a, src, depth, parent, GR_DIR_PUSH, 14.f, 24.f, n + 1, 0);
  GR_CUDA(cudaGetLastError());
  void *args[] = {&a};
  GR_CUDA(cudaLaunchCooperativeKernel((void *)k_bfs_persistent, per_sm * sms, kPersThreads,
                                      args, 0, s));
  return GR_OK;
}
