// Neighbourhood gather-reduce as an operator of its own (Sec. 7), and the
// bipartite node rankings built on it (Sec. 5.5 "Bipartite graphs": HITS,
// SALSA and personalized PageRank, the three rankings of the who-to-follow
// computation the paper cites).
//
//   gr_neighbor_reduce  out[v] = sum / weighted sum / min / max of x[u] over
//                the entries (v, u) of v's row, for every vertex or for the
//                vertices of a frontier list (lb_gather_reduce; a frontier's
//                degree scan is computed first, three kernels).
//   gr_hits, gr_salsa   on a bipartite graph stored symmetrically (hubs
//                [0, n_left), authorities [n_left, n)): one iteration is the
//                2-hop traversal hub -> authority -> hub, two gather-reduce
//                passes over the two vertex ranges (each authority gathers
//                from its hubs, then each hub from its authorities), with a
//                normalisation sweep after each pass.
//   gr_ppr       personalized PageRank: per iteration one gather-reduce over
//                all vertices and one update sweep (teleport and dangling
//                mass to the seeds).
//
// Each ranking runs as one cooperative persistent kernel: the passes and
// sweeps of an iteration are separated by the bounded grid barrier, global
// sums (squared norms, the L1 change, the dangling mass) are reduced in FP64
// per block and added with one atomic per block into slots that alternate
// between iterations, and every block takes the same stop decision from
// them. Scores are FP64.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "advance.cuh"

namespace gr {

// Gather tiles of 12 items for each of 96 threads, 8 blocks per SM, the
// rest of the SM's shared-memory array left to L1 (R-MAT s23 gather-reduce,
// FP64 sum: 256 x 8 at 4 blocks per SM with the default carveout 3.48 ms,
// with the fitted carveout 1.96 ms, this tile 1.57 ms).
constexpr int kRkThreads = 96, kRkItems = 12;
constexpr int kRkBlocksPerSm = 8;

struct RankCtl {
  GridBarrier bar;
  double red[2][4];  // per iteration parity: squared norms, L1 change, dangling mass
  int32_t iters;
  int32_t error;
  int32_t linked;    // SALSA: hubs with links
};

struct RankWorkspace {
  DevMem cur, tmp, dv, tele, ctl, seeds;
  DevMem fscan, part;   // gr_neighbor_reduce: a frontier's degree scan, block partials
  int32_t bip_left = -1;  // n_left the graph was last checked to be bipartite for
  // chunk bounds of the gather's merge paths: all vertices (fixed per
  // graph), and the hub and authority ranges of the last n_left
  DevMem cb_all, cb_hub, cb_auth;
  int32_t cb_left = -1;
};

void free_rank(RankWorkspace *ws) { delete ws; }

namespace {

// ------------------------------------------------------ gather functors
struct GatherF64 {
  const double *x;
  __device__ __forceinline__ double operator()(int32_t u, int32_t) const { return x[u]; }
};
struct GatherWF64 {
  const double *x;
  const uint32_t *w;
  __device__ __forceinline__ double operator()(int32_t u, int32_t e) const {
    return (double)w[e] * x[u];
  }
};
struct GatherI32 {
  const int32_t *x;
  __device__ __forceinline__ int32_t operator()(int32_t u, int32_t) const { return x[u]; }
};

// ---------------------------------------------- gr_neighbor_reduce kernels
template <class T>
__global__ void k_nr_fill(T *out, const int32_t *Q, int32_t count, T val) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count;
       i += (int64_t)gridDim.x * blockDim.x)
    out[Q ? Q[i] : i] = val;
}

// Exclusive scan of the frontier's degrees in three steps: per-tile sums,
// one block scanning the tile sums, then each tile's scan with its offset.
constexpr int kScanTile = 1024;  // entries per tile (4 per thread)

__global__ void k_scan_tiles(const int32_t *R, const int32_t *Q, int32_t q, int32_t *part) {
  __shared__ int32_t red[33];
  const int64_t base = (int64_t)blockIdx.x * kScanTile;
  int32_t local = 0;
  for (int j = 0; j < kScanTile / 256; ++j) {
    const int64_t i = base + j * 256 + threadIdx.x;
    if (i < q) {
      const int32_t v = Q[i];
      local += R[v + 1] - R[v];
    }
  }
  const int32_t total = block_sum(local, red);
  if (threadIdx.x == 0) part[blockIdx.x] = total;
}

__global__ void k_scan_parts(int32_t *part, int32_t tiles) {
  __shared__ int32_t red[33];
  int32_t carry = 0;
  for (int32_t b = 0; b < tiles; b += 256) {  // block-uniform
    const int32_t i = b + threadIdx.x;
    const int32_t x = i < tiles ? part[i] : 0;
    int32_t total;
    const int32_t ex = block_excl_sum(x, red, &total);
    if (i < tiles) part[i] = carry + ex;
    carry += total;
  }
}

__global__ void k_scan_apply(const int32_t *R, const int32_t *Q, int32_t q, const int32_t *part,
                             int32_t *S) {
  __shared__ int32_t red[33];
  constexpr int PER = kScanTile / 256;
  const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * PER;
  int32_t d[PER];
  int32_t local = 0;
#pragma unroll
  for (int j = 0; j < PER; ++j) {
    const int64_t i = base + j;
    d[j] = 0;
    if (i < q) {
      const int32_t v = Q[i];
      d[j] = R[v + 1] - R[v];
    }
    local += d[j];
  }
  int32_t total;
  int32_t run = part[blockIdx.x] + block_excl_sum(local, red, &total);
#pragma unroll
  for (int j = 0; j < PER; ++j) {
    const int64_t i = base + j;
    if (i < q) S[i] = run;
    run += d[j];
    if (i == q - 1) S[q] = run;
  }
}

template <class T, class OP, bool FRONTIER, class G>
__global__ void __launch_bounds__(kRkThreads, kRkBlocksPerSm) k_nr_gather(const int32_t *R, const int32_t *C,
                                                           const int32_t *Q, const int32_t *S,
                                                           int32_t q, G g, T *out,
                                                           const int32_t *cb) {
  lb_gather_reduce<kRkThreads, kRkItems, T, OP, FRONTIER>(R, C, Q, S, q, 0, g, out, cb);
}

// ------------------------------------------------------ ranking kernels
struct RankArgs {
  const int32_t *R;
  const int32_t *C;
  int32_t n;
  int32_t n_left;
  double *cur;   // scores
  double *tmp;   // gathered sums (zero before each gather)
  double *dv;    // score / degree (SALSA, PPR)
  const double *tele;  // teleport vector (PPR)
  double damping;
  double tol;
  int32_t max_iter;
  RankCtl *ctl;
  const int32_t *cb_all, *cb_hub, *cb_auth;  // chunk bounds of the gathers' ranges
};

// Block-wide FP64 sum, added to *dst by thread 0.
__device__ __forceinline__ void block_add(double v, double *smem, double *dst) {
  const double t = block_sum(v, smem);
  if (threadIdx.x == 0 && t != 0.0) atomicAdd(dst, t);
}

__device__ __forceinline__ double read_slot(const double *p) { return *(const volatile double *)p; }

template <int KIND>  // 0: HITS, 1: SALSA
__global__ void __launch_bounds__(kRkThreads, kRkBlocksPerSm) k_bipartite_do(RankArgs a) {
  __shared__ double red[33];
  RankCtl *c = a.ctl;
  const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int32_t nl = a.n_left, n = a.n;
  int32_t gen = 0;
  int32_t it = 0;
  while (it < a.max_iter) {
    double *slot = c->red[it & 1];
    // authorities gather from their hubs: h[l] (HITS) or h[l] / deg(l) (SALSA)
    {
      GatherF64 gf{KIND == 0 ? a.cur : a.dv};
      lb_gather_reduce<kRkThreads, kRkItems, double, ReduceSum<double>, false>(
          a.R, a.C, nullptr, a.R + nl, n - nl, nl, gf, a.tmp, a.cb_auth);
    }
    if (!grid_sync(&c->bar, &c->error, gen)) return;
    if (blockIdx.x == 0 && threadIdx.x < 4) c->red[(it + 1) & 1][threadIdx.x] = 0.0;
    double inv = 1.0;
    if (KIND == 0) {
      double ss = 0.0;
      for (int64_t r = nl + tid; r < n; r += stride) ss += a.tmp[r] * a.tmp[r];
      block_add(ss, red, &slot[0]);
      if (!grid_sync(&c->bar, &c->error, gen)) return;
      const double t = read_slot(&slot[0]);
      inv = t > 0.0 ? 1.0 / sqrt(t) : 1.0;
    }
    {
      double delta = 0.0;
      for (int64_t r = nl + tid; r < n; r += stride) {
        const double x = a.tmp[r] * inv;
        delta += fabs(x - a.cur[r]);
        a.cur[r] = x;
        if (KIND == 1) {
          const int32_t d = a.R[r + 1] - a.R[r];
          a.dv[r] = d ? x / d : 0.0;
        }
        a.tmp[r] = 0.0;
      }
      block_add(delta, red, &slot[2]);
    }
    if (!grid_sync(&c->bar, &c->error, gen)) return;
    // hubs gather from the new authorities
    {
      GatherF64 gf{KIND == 0 ? a.cur : a.dv};
      lb_gather_reduce<kRkThreads, kRkItems, double, ReduceSum<double>, false>(
          a.R, a.C, nullptr, a.R, nl, 0, gf, a.tmp, a.cb_hub);
    }
    if (!grid_sync(&c->bar, &c->error, gen)) return;
    inv = 1.0;
    if (KIND == 0) {
      double ss = 0.0;
      for (int64_t l = tid; l < nl; l += stride) ss += a.tmp[l] * a.tmp[l];
      block_add(ss, red, &slot[1]);
      if (!grid_sync(&c->bar, &c->error, gen)) return;
      const double t = read_slot(&slot[1]);
      inv = t > 0.0 ? 1.0 / sqrt(t) : 1.0;
    }
    {
      double delta = 0.0;
      for (int64_t l = tid; l < nl; l += stride) {
        const double x = a.tmp[l] * inv;
        delta += fabs(x - a.cur[l]);
        a.cur[l] = x;
        if (KIND == 1) {
          const int32_t d = a.R[l + 1] - a.R[l];
          a.dv[l] = d ? x / d : 0.0;
        }
        a.tmp[l] = 0.0;
      }
      block_add(delta, red, &slot[2]);
    }
    if (!grid_sync(&c->bar, &c->error, gen)) return;
    ++it;
    if (read_slot(&slot[2]) < a.tol) break;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) c->iters = it;
}

__global__ void __launch_bounds__(kRkThreads, kRkBlocksPerSm) k_ppr_do(RankArgs a) {
  __shared__ double red[33];
  RankCtl *c = a.ctl;
  const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const double d = a.damping;
  int32_t gen = 0;
  int32_t it = 0;
  // dangling mass of the starting ranks (the teleport vector)
  double dangling = read_slot(&c->red[1][3]);
  while (it < a.max_iter) {
    double *slot = c->red[it & 1];
    {
      GatherF64 gf{a.dv};
      lb_gather_reduce<kRkThreads, kRkItems, double, ReduceSum<double>, false>(
          a.R, a.C, nullptr, a.R, a.n, 0, gf, a.tmp, a.cb_all);
    }
    if (!grid_sync(&c->bar, &c->error, gen)) return;
    if (blockIdx.x == 0 && threadIdx.x < 4) c->red[(it + 1) & 1][threadIdx.x] = 0.0;
    double delta = 0.0, dang = 0.0;
    for (int64_t v = tid; v < a.n; v += stride) {
      const double t = a.tele[v];
      const double x = (1.0 - d) * t + d * (a.tmp[v] + dangling * t);
      delta += fabs(x - a.cur[v]);
      a.cur[v] = x;
      const int32_t deg = a.R[v + 1] - a.R[v];
      a.dv[v] = deg ? x / deg : 0.0;
      if (!deg) dang += x;
      a.tmp[v] = 0.0;
    }
    block_add(delta, red, &slot[2]);
    block_add(dang, red, &slot[3]);
    if (!grid_sync(&c->bar, &c->error, gen)) return;
    ++it;
    dangling = read_slot(&slot[3]);
    if (read_slot(&slot[2]) < a.tol) break;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) c->iters = it;
}

// Initial scores: HITS h = 1/sqrt(n_left) on the hubs; SALSA h = 1/(hubs
// with links) on those hubs; PPR the teleport vector. tmp = 0; the ranking
// kernel's reduction slots and barrier reset; dv = score / degree.
__global__ void k_rank_init(RankArgs a, int32_t kind) {
  const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  double h0 = 0.0;
  if (kind == 0 && a.n_left > 0) h0 = 1.0 / sqrt((double)a.n_left);
  if (kind == 1) {
    const int32_t linked = *(volatile int32_t *)&a.ctl->linked;
    h0 = linked ? 1.0 / (double)linked : 0.0;
  }
  for (int64_t v = tid; v < a.n; v += stride) {
    const int32_t deg = a.R[v + 1] - a.R[v];
    double x;
    if (kind == 0) x = v < a.n_left ? h0 : 0.0;
    else if (kind == 1) x = (v < a.n_left && deg) ? h0 : 0.0;
    else x = a.tele[v];
    a.cur[v] = x;
    a.tmp[v] = 0.0;
    if (a.dv) a.dv[v] = deg ? x / deg : 0.0;
  }
  if (tid == 0) {
    RankCtl *c = a.ctl;
    grid_barrier_reset(&c->bar);
    for (int i = 0; i < 4; ++i) c->red[0][i] = 0.0;
    c->iters = 0;
    c->error = kDevOk;
  }
}

// PPR: teleport vector (1 / seeds on each seed, zero elsewhere beforehand)
// and its dangling mass. One block.
__global__ void k_ppr_seeds(const int32_t *R, const int32_t *seeds, int32_t ns, double *tele,
                            double *dangling_out) {
  double dang = 0.0;
  for (int32_t i = threadIdx.x; i < ns; i += blockDim.x) {
    const int32_t v = seeds[i];
    tele[v] = 1.0 / ns;
    if (R[v + 1] == R[v]) dang += 1.0 / ns;
  }
  __shared__ double red[33];
  const double t = block_sum(dang, red);
  if (threadIdx.x == 0) *dangling_out = t;
}

// SALSA's starting hubs: those with links (ctl->linked, zero beforehand).
__global__ void k_count_linked(const int32_t *R, int32_t n_left, int32_t *linked) {
  __shared__ int32_t red[33];
  int32_t cnt = 0;
  for (int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; l < n_left;
       l += (int64_t)gridDim.x * blockDim.x)
    cnt += R[l + 1] > R[l];
  const int32_t t = block_sum(cnt, red);
  if (threadIdx.x == 0 && t) atomicAdd(linked, t);
}

// Every entry joins a hub and an authority.
__global__ void k_check_bipartite(const int32_t *R, const int32_t *C, int32_t n, int32_t nl,
                                  int32_t *bad) {
  const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t v = tid; v < n; v += stride)
    for (int32_t e = R[v]; e < R[v + 1]; ++e)
      if ((v < nl) == (C[e] < nl)) {
        atomicOr(bad, 1);
        break;
      }
}

}  // namespace

static gr_status rank_ws(gr_graph *g, RankWorkspace **out) {
  if (!g->rank) g->rank = new RankWorkspace();
  RankWorkspace *ws = g->rank;
  const size_t bytes = sizeof(double) * (size_t)g->n;
  if (!ws->cur.p) {
    GR_TRY(ws->cur.alloc(bytes, "ranking scores"));
    GR_TRY(ws->tmp.alloc(bytes, "ranking sums"));
    GR_TRY(ws->dv.alloc(bytes, "ranking scores per degree"));
    GR_TRY(ws->ctl.alloc(sizeof(RankCtl), "ranking control"));
  }
  *out = ws;
  return GR_OK;
}

// Chunk bounds of the gather's merge path over the vertex range [v0, v1)
// into buf (one search per chunk, on `s`).
static gr_status range_bounds(gr_graph *g, int32_t v0, int32_t v1, DevMem &buf, cudaStream_t s) {
  const int32_t *R = g->row_off.as<int32_t>();
  int32_t r[2] = {0, 0};
  // the range's entry count: two offsets, read once per call
  GR_CUDA(cudaMemcpyAsync(&r[0], R + v0, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  GR_CUDA(cudaMemcpyAsync(&r[1], R + v1, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  GR_CUDA(cudaStreamSynchronize(s));
  const int32_t chunks = merge_chunks(v1 - v0, (long long)r[1] - r[0], kRkThreads * kRkItems);
  if (buf.bytes < sizeof(int32_t) * ((size_t)chunks + 1))
    GR_TRY(buf.alloc(sizeof(int32_t) * ((size_t)chunks + 1), "gather chunk bounds"));
  k_chunk_bounds<<<(chunks + 256) / 256, 256, 0, s>>>(R + v0, v1 - v0, kRkThreads * kRkItems,
                                                       chunks, buf.as<int32_t>());
  GR_CUDA(cudaGetLastError());
  return GR_OK;
}

static gr_status all_bounds(gr_graph *g, RankWorkspace *ws, cudaStream_t s) {
  if (!ws->cb_all.p) GR_TRY(range_bounds(g, 0, g->n, ws->cb_all, s));
  return GR_OK;
}

// One gather-reduce over a range or a frontier, at the tile's resident
// blocks per SM with the rest of the shared-memory array left to L1.
template <class T, class OP, bool FRONTIER, class G>
static gr_status nr_launch(gr_graph *g, cudaStream_t s, const int32_t *R, const int32_t *C,
                           const int32_t *Q, const int32_t *S, int32_t q, G gf, T *out,
                           const int32_t *cb) {
  auto kern = k_nr_gather<T, OP, FRONTIER, G>;
  int per_sm = 1;
  GR_TRY(fit_carveout(kern, kRkThreads, kRkBlocksPerSm, g->device, &per_sm));
  kern<<<per_sm * g->num_sms, kRkThreads, 0, s>>>(R, C, Q, S, q, gf, out, cb);
  GR_CUDA(cudaGetLastError());
  return GR_OK;
}

static gr_status rank_launch(gr_graph *g, void *kern, RankArgs &a, cudaStream_t s) {
  int per_sm = 1;
  GR_TRY(fit_carveout(kern, kRkThreads, kRkBlocksPerSm, g->device, &per_sm));
  const int blocks = per_sm * g->num_sms;
  void *args[] = {&a};
  GR_CUDA(cudaLaunchCooperativeKernel(kern, blocks, kRkThreads, args, 0, s));
  return GR_OK;
}

// Copies the scores to the caller's buffer (device or host) and, with
// iters, synchronises to read the iteration count.
static gr_status rank_finish(gr_graph *g, RankWorkspace *ws, void *user, bool host,
                             int32_t *iters, cudaStream_t s) {
  GR_CUDA(cudaMemcpyAsync(user, ws->cur.p, sizeof(double) * (size_t)g->n,
                          host ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, s));
  if (iters) {
    RankCtl h;
    GR_CUDA(cudaMemcpyAsync(&h, ws->ctl.p, sizeof(RankCtl), cudaMemcpyDeviceToHost, s));
    GR_CUDA(cudaStreamSynchronize(s));
    if (h.error == kDevTimeout) return fail(GR_ETIMEOUT, "a device-side wait timed out");
    *iters = h.iters;
  }
  return GR_OK;
}

static gr_status bipartite_run(gr_graph *g, int kind, int32_t n_left, int32_t max_iter,
                               double tol, double *score, int32_t *iters, void *stream) {
  clear_error();
  if (!g) return fail(GR_EINVAL, "graph must not be NULL");
  if (!score) return fail(GR_EINVAL, "score must not be NULL");
  if (n_left < 0 || n_left > g->n) return fail(GR_EINVAL, "n_left must be in [0, n]");
  if (max_iter < 0 || !(tol >= 0.0)) return fail(GR_EINVAL, "max_iter and tol must be >= 0");
  if (!g->symmetric)
    return fail(GR_EINVAL, "the bipartite graph must be stored in both directions (symmetric CSR)");
  std::lock_guard<std::mutex> lock(g->mu);
  cudaStream_t s = (cudaStream_t)stream;
  GR_TRY(begin_call(g, s));
  RankWorkspace *ws;
  GR_TRY(rank_ws(g, &ws));
  if (ws->bip_left != n_left) {
    DevMem bad;
    GR_TRY(bad.alloc(sizeof(int32_t), "bipartite check"));
    GR_CUDA(cudaMemsetAsync(bad.p, 0, sizeof(int32_t), s));
    k_check_bipartite<<<g->num_sms * 8, 256, 0, s>>>(g->row_off.as<int32_t>(),
                                                     g->col.as<int32_t>(), g->n, n_left,
                                                     bad.as<int32_t>());
    int32_t h = 0;
    GR_CUDA(cudaMemcpyAsync(&h, bad.p, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    GR_CUDA(cudaStreamSynchronize(s));
    if (h) return fail(GR_EINVAL, "an entry joins two vertices on the same side of n_left");
    ws->bip_left = n_left;
  }
  bool host = false;
  GR_TRY(output_on_host(g, score, &host));
  if (ws->cb_left != n_left) {
    GR_TRY(range_bounds(g, 0, n_left, ws->cb_hub, s));
    GR_TRY(range_bounds(g, n_left, g->n, ws->cb_auth, s));
    ws->cb_left = n_left;
  }
  RankArgs a;
  std::memset(&a, 0, sizeof(a));
  a.R = g->row_off.as<int32_t>();
  a.C = g->col.as<int32_t>();
  a.n = g->n;
  a.n_left = n_left;
  a.cb_hub = ws->cb_hub.as<int32_t>();
  a.cb_auth = ws->cb_auth.as<int32_t>();
  a.cur = ws->cur.as<double>();
  a.tmp = ws->tmp.as<double>();
  a.dv = ws->dv.as<double>();
  a.tol = tol;
  a.max_iter = max_iter;
  a.ctl = ws->ctl.as<RankCtl>();
  if (kind == 1) {
    GR_CUDA(cudaMemsetAsync(&a.ctl->linked, 0, sizeof(int32_t), s));
    k_count_linked<<<g->num_sms * 8, 256, 0, s>>>(a.R, n_left, &a.ctl->linked);
  }
  k_rank_init<<<g->num_sms * 8, 256, 0, s>>>(a, kind);
  GR_CUDA(cudaGetLastError());
  if (max_iter > 0)
    GR_TRY(rank_launch(g, kind == 0 ? (void *)k_bipartite_do<0> : (void *)k_bipartite_do<1>, a,
                       s));
  GR_TRY(rank_finish(g, ws, score, host, iters, s));
  GR_TRY(end_call(g, s));
  return GR_OK;
}

}  // namespace gr

using namespace gr;

extern "C" {

gr_status gr_neighbor_reduce(gr_graph *g, int32_t op, const int32_t *frontier, int32_t q,
                             const void *x, void *out, void *stream) {
  clear_error();
  if (!g) return fail(GR_EINVAL, "graph must not be NULL");
  if (op < GR_REDUCE_SUM || op > GR_REDUCE_MAX) return fail(GR_EINVAL, "unknown reduction");
  if (!x || !out) return fail(GR_EINVAL, "x and out must not be NULL");
  if (op == GR_REDUCE_WSUM && !g->has_weights)
    return fail(GR_EINVAL, "the weighted sum needs edge weights");
  if (frontier && (q < 0 || q > g->n)) return fail(GR_EINVAL, "q must be in [0, n]");
  bool x_host = false;
  GR_TRY(output_on_host(g, x, &x_host));
  if (x_host) return fail(GR_EINVAL, "x must be device memory of the graph's device");
  if (frontier) {
    bool f_host = false;
    GR_TRY(output_on_host(g, frontier, &f_host));
    if (f_host) return fail(GR_EINVAL, "frontier must be device memory of the graph's device");
  }
  std::lock_guard<std::mutex> lock(g->mu);
  cudaStream_t s = (cudaStream_t)stream;
  GR_TRY(begin_call(g, s));
  const bool sum = op == GR_REDUCE_SUM || op == GR_REDUCE_WSUM;
  const size_t elem = sum ? sizeof(double) : sizeof(int32_t);
  void *d_out;
  bool cp;
  GR_TRY(resolve_output(g, 0, out, elem * (size_t)g->n, &d_out, &cp));
  // a frontier leaves the other entries as they are: a host output is
  // staged with its current contents
  if (cp && frontier)
    GR_CUDA(cudaMemcpyAsync(d_out, out, elem * (size_t)g->n, cudaMemcpyHostToDevice, s));
  const int32_t count = frontier ? q : g->n;
  const int grid = g->num_sms * 8;
  const int32_t *R = g->row_off.as<int32_t>(), *C = g->col.as<int32_t>();
  // the reduced vertices start at the operation's identity
  if (count > 0) {
    if (sum) k_nr_fill<double><<<grid, 256, 0, s>>>((double *)d_out, frontier, count, 0.0);
    else
      k_nr_fill<int32_t><<<grid, 256, 0, s>>>((int32_t *)d_out, frontier, count,
                                              op == GR_REDUCE_MIN ? INT32_MAX : INT32_MIN);
    GR_CUDA(cudaGetLastError());
  }
  if (count > 0) {
    const int32_t *cb = nullptr;
    if (!frontier) {
      if (!g->rank) g->rank = new RankWorkspace();
      GR_TRY(all_bounds(g, g->rank, s));
      cb = g->rank->cb_all.as<int32_t>();
    }
    if (!frontier) {
      if (op == GR_REDUCE_SUM)
        GR_TRY((nr_launch<double, ReduceSum<double>, false>(
            g, s, R, C, nullptr, R, count, GatherF64{(const double *)x}, (double *)d_out, cb)));
      else if (op == GR_REDUCE_WSUM)
        GR_TRY((nr_launch<double, ReduceSum<double>, false>(
            g, s, R, C, nullptr, R, count, GatherWF64{(const double *)x, g->w.as<uint32_t>()},
            (double *)d_out, cb)));
      else if (op == GR_REDUCE_MIN)
        GR_TRY((nr_launch<int32_t, ReduceMinI32, false>(
            g, s, R, C, nullptr, R, count, GatherI32{(const int32_t *)x}, (int32_t *)d_out, cb)));
      else
        GR_TRY((nr_launch<int32_t, ReduceMaxI32, false>(
            g, s, R, C, nullptr, R, count, GatherI32{(const int32_t *)x}, (int32_t *)d_out, cb)));
    } else {
      RankWorkspace *ws;
      if (!g->rank) g->rank = new RankWorkspace();
      ws = g->rank;
      const int32_t tiles = (count + kScanTile - 1) / kScanTile;
      if (ws->fscan.bytes < sizeof(int32_t) * ((size_t)g->n + 1)) {
        GR_CUDA(cudaStreamSynchronize(s));
        GR_TRY(ws->fscan.alloc(sizeof(int32_t) * ((size_t)g->n + 1), "frontier degree scan"));
      }
      if (ws->part.bytes < sizeof(int32_t) * (size_t)tiles) {
        GR_CUDA(cudaStreamSynchronize(s));
        GR_TRY(ws->part.alloc(sizeof(int32_t) * (size_t)tiles, "frontier scan partials"));
      }
      int32_t *S = ws->fscan.as<int32_t>(), *part = ws->part.as<int32_t>();
      k_scan_tiles<<<tiles, 256, 0, s>>>(R, frontier, count, part);
      k_scan_parts<<<1, 256, 0, s>>>(part, tiles);
      k_scan_apply<<<tiles, 256, 0, s>>>(R, frontier, count, part, S);
      if (op == GR_REDUCE_SUM)
        GR_TRY((nr_launch<double, ReduceSum<double>, true>(
            g, s, R, C, frontier, S, count, GatherF64{(const double *)x}, (double *)d_out,
            nullptr)));
      else if (op == GR_REDUCE_WSUM)
        GR_TRY((nr_launch<double, ReduceSum<double>, true>(
            g, s, R, C, frontier, S, count, GatherWF64{(const double *)x, g->w.as<uint32_t>()},
            (double *)d_out, nullptr)));
      else if (op == GR_REDUCE_MIN)
        GR_TRY((nr_launch<int32_t, ReduceMinI32, true>(
            g, s, R, C, frontier, S, count, GatherI32{(const int32_t *)x}, (int32_t *)d_out,
            nullptr)));
      else
        GR_TRY((nr_launch<int32_t, ReduceMaxI32, true>(
            g, s, R, C, frontier, S, count, GatherI32{(const int32_t *)x}, (int32_t *)d_out,
            nullptr)));
    }
  }
  if (cp) GR_CUDA(cudaMemcpyAsync(out, d_out, elem * (size_t)g->n, cudaMemcpyDeviceToHost, s));
  GR_TRY(end_call(g, s));
  return GR_OK;
}

gr_status gr_hits(gr_graph *g, int32_t n_left, int32_t max_iter, double tol, double *score,
                  int32_t *iters, void *stream) {
  return bipartite_run(g, 0, n_left, max_iter, tol, score, iters, stream);
}

gr_status gr_salsa(gr_graph *g, int32_t n_left, int32_t max_iter, double tol, double *score,
                   int32_t *iters, void *stream) {
  return bipartite_run(g, 1, n_left, max_iter, tol, score, iters, stream);
}

gr_status gr_ppr(gr_graph *g, const int32_t *seeds, int32_t num_seeds, double damping,
                 int32_t max_iter, double tol, double *rank, int32_t *iters, void *stream) {
  clear_error();
  if (!g) return fail(GR_EINVAL, "graph must not be NULL");
  if (!rank || !seeds) return fail(GR_EINVAL, "seeds and rank must not be NULL");
  if (num_seeds < 1 || num_seeds > g->n) return fail(GR_EINVAL, "num_seeds must be in [1, n]");
  if (!(damping > 0.0 && damping < 1.0)) return fail(GR_EINVAL, "damping must lie in (0, 1)");
  if (max_iter < 0 || !(tol >= 0.0)) return fail(GR_EINVAL, "max_iter and tol must be >= 0");
  if (!g->symmetric)
    return fail(GR_EINVAL, "personalized PageRank gathers over rows: the CSR must be symmetric");
  {
    std::vector<int32_t> sorted(seeds, seeds + num_seeds);
    std::sort(sorted.begin(), sorted.end());
    if (sorted.front() < 0 || sorted.back() >= g->n)
      return fail(GR_EINVAL, "seed out of range");
    if (std::adjacent_find(sorted.begin(), sorted.end()) != sorted.end())
      return fail(GR_EINVAL, "seeds must be distinct");
  }
  std::lock_guard<std::mutex> lock(g->mu);
  cudaStream_t s = (cudaStream_t)stream;
  GR_TRY(begin_call(g, s));
  RankWorkspace *ws;
  GR_TRY(rank_ws(g, &ws));
  if (!ws->tele.p) GR_TRY(ws->tele.alloc(sizeof(double) * (size_t)g->n, "PPR teleport"));
  if (ws->seeds.bytes < sizeof(int32_t) * (size_t)num_seeds) {
    GR_CUDA(cudaStreamSynchronize(s));  // the old buffer may still be read
    GR_TRY(ws->seeds.alloc(sizeof(int32_t) * (size_t)num_seeds, "PPR seeds"));
  }
  // pageable source: staged before the call returns, copied in stream order
  GR_CUDA(cudaMemcpyAsync(ws->seeds.p, seeds, sizeof(int32_t) * (size_t)num_seeds,
                          cudaMemcpyHostToDevice, s));
  bool host = false;
  GR_TRY(output_on_host(g, rank, &host));
  GR_TRY(all_bounds(g, ws, s));
  RankArgs a;
  std::memset(&a, 0, sizeof(a));
  a.R = g->row_off.as<int32_t>();
  a.C = g->col.as<int32_t>();
  a.n = g->n;
  a.cur = ws->cur.as<double>();
  a.tmp = ws->tmp.as<double>();
  a.dv = ws->dv.as<double>();
  a.tele = ws->tele.as<double>();
  a.cb_all = ws->cb_all.as<int32_t>();
  a.damping = damping;
  a.tol = tol;
  a.max_iter = max_iter;
  a.ctl = ws->ctl.as<RankCtl>();
  GR_CUDA(cudaMemsetAsync(ws->tele.p, 0, sizeof(double) * (size_t)g->n, s));
  k_ppr_seeds<<<1, 256, 0, s>>>(a.R, ws->seeds.as<int32_t>(), num_seeds, ws->tele.as<double>(),
                                &a.ctl->red[1][3]);
  k_rank_init<<<g->num_sms * 8, 256, 0, s>>>(a, 2);
  GR_CUDA(cudaGetLastError());
  if (max_iter > 0) GR_TRY(rank_launch(g, (void *)k_ppr_do, a, s));
  GR_TRY(rank_finish(g, ws, rank, host, iters, s));
  GR_TRY(end_call(g, s));
  return GR_OK;
}

}  // extern "C"
