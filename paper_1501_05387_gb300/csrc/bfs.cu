// Breadth-first search over the frontier operators (Sec. 5.1).
//
// One BFS level is ONE kernel, k_bfs_level, whose blocks take every decision
// from a device-resident control block, so the level loop needs no host
// round trip:
//
//   push level  advance + filter fused (Sec. 4.3 kernel fusion): merge-path
//               chunks over the frontier's vertex ends and edge ranks (the
//               load-balanced partitioning of Sec. 4.4), coalesced column
//               loads, a plain-load visited-bitmap cull and one atomicOr claim
//               per surviving candidate, so each vertex enters the next
//               frontier once (the non-idempotent advance of Sec. 4.5).
//   pull level  bottom-up advance (Sec. 4.5): every unvisited vertex looks
//               for a neighbour in the frontier bitmap and stops at the first.
//               A warp owns 32 consecutive vertices, one bitmap word, so the
//               visited and next-frontier bitmaps are written with a ballot and
//               a plain store: no atomics. Lanes check their first neighbours
//               with independent loads; vertices left over with longer lists
//               are then scanned by the whole warp, 32 neighbours at a time.
//
// Both emit the next frontier together with its exclusive degree scan (the
// "scanned edge offset queue" of Sec. 4.4): a block compacts its new
// vertices in shared memory, scans their degrees and reserves queue and
// edge ranges with a single 64-bit atomicAdd on a packed (vertices, edges)
// counter, so queue order and scan order agree and no separate scan pass is
// needed. The last block to finish a level applies the push/pull rule
// (Sec. 4.5), swaps the buffers and, inside a CUDA graph, sets the while
// loop's condition.
//
// Drivers: a CUDA graph holding a device-side while loop over k_bfs_level
// (GR_MODE_GRAPH), host-enqueued batches of levels that exit at once after
// the traversal finished (GR_MODE_LAUNCH), and a cooperative persistent
// kernel with a bounded-spin grid barrier for long chains of small push
// frontiers (GR_MODE_PERSISTENT).
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
  int32_t parity;       // which queue / scan array holds the current frontier
  int32_t dir;          // direction of the current level
  int32_t q_len;        // current frontier size
  int32_t q_prev;       // previous frontier size
  int32_t done;
  int32_t error;
  int32_t pull_levels;
  int32_t policy;       // GR_DIR_*
  int32_t max_levels;
  int32_t from_bitmap;  // 1: the current frontier exists only as a bitmap
  int32_t pad_[3];
  // level-kernel blocks finished so far in this traversal; the block whose
  // arrival makes it a multiple of the grid size ends the level
  unsigned long long arrivals;
  // persistent kernel: next-frontier counters, a ring of three so that one
  // can be cleared while the others are in use
  unsigned long long cnt3[3];
  // persistent kernel: largest degree a pull level found, by level (ring)
  int32_t maxdeg3[3];
  int32_t pad3_;
  unsigned long long next_packed;  // [31:0] next frontier size, [63:32] its edges
  long long mf;         // edges leaving the current frontier
  long long mu;         // edges of still-unexplored vertices
  float alpha;
  float beta;
  // per-level trace (first kTraceLevels levels): direction, frontier size
  // and edges of the frontier each level expanded, and globaltimer at the
  // end of the level (the init kernel stamps t_start)
  unsigned long long t_start;
  int32_t tr_dir[64];
  int32_t tr_q[64];
  long long tr_mf[64];
  unsigned long long tr_t[64];
  GridBarrier bar;  // persistent kernels' grid barrier
};
constexpr int kTraceLevels = 64;

__device__ __forceinline__ unsigned long long globaltimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

struct BfsArgs {
  const int32_t *R;
  const int32_t *C;
  int32_t n;
  int32_t nwords;
  long long m;
  const uint32_t *iso;
  const int32_t *first;  // first neighbour per vertex (-1: none); pull levels test it first
  int32_t *q[2];
  int32_t *S[2];        // exclusive degree scan of q[p], S[p][q_len] = edges
  uint32_t *visited;
  uint32_t *fb[3];      // frontier bitmaps, rotating by level (cur, next, spare)
  BfsCtl *ctl;
  int32_t do_bitmap;
  int32_t low_degree;   // push-only on a graph of small maximum degree: per-thread expansion
  // persistent kernel: per-block segments of the vertices a pull level
  // found (and their degrees), compacted into a queue by the next level
  // when it pushes; null in the other drivers
  int32_t *seg_v;
  int32_t *seg_d;
  unsigned long long *seg_cnt;  // per block: [31:0] vertices, [63:32] edges
  int32_t seg_cap;              // entries per block segment
};

// launch shape of the level kernel
constexpr int kLvThreads = 256;
constexpr int kLvItems = 4;                        // merge items per thread (push)
constexpr int kLvChunk = kLvThreads * kLvItems;    // merge items per chunk
constexpr int kLvWarps = kLvThreads / 32;
// neighbours after the first a lane checks alone in a pull level, before the
// warp scans what is left of a long list (R-MAT s22: 0.1827 ms per traversal
// at 3, 0.1815 at 5, 0.1806 at 8, 0.1811 at 12, 0.1809 at 20)
constexpr int kPullLane = 8;
constexpr int kLvBlocksPerSm = 6;
// Largest maximum degree for which push levels expand one frontier vertex per
// thread (mesh-like graphs), and the neighbours a thread loads at once.
constexpr int32_t kLowDegreeMax = 16;
constexpr int kTpvItems = 4;

struct BfsWorkspace {
  DevMem q[2], S[2], visited, fb[3], ctl, seg_v, seg_d, seg_cnt;
  PinnedMem h_ctl;
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

GR_GUARD_REPORTER(guard_report_bfs)

// ------------------------------------------------------------- kernels
namespace {

// select by index without indexing the parameter arrays (a dynamic index
// would copy the kernel parameters to local memory)
__device__ __forceinline__ int32_t *queue_of(const BfsArgs &a, int p) { return p ? a.q[1] : a.q[0]; }
__device__ __forceinline__ int32_t *scan_of(const BfsArgs &a, int p) { return p ? a.S[1] : a.S[0]; }
__device__ __forceinline__ uint32_t *bits_of(const BfsArgs &a, int level) {
  const int k = level % 3;
  return k == 0 ? a.fb[0] : (k == 1 ? a.fb[1] : a.fb[2]);
}

__global__ void k_bfs_init(BfsArgs a, int32_t src, int32_t *depth, int32_t *parent,
                           int32_t policy, float alpha, float beta,
                           int32_t max_levels, int32_t preset_iso) {
  const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
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
    if (a.do_bitmap) {
      a.fb[0][w] = (w == sw) ? sb : 0u;  // frontier of level 0
      a.fb[1][w] = 0u;                   // filled by level 0
    }
  }
  if (tid == 0) {
    BfsCtl *c = a.ctl;
    const int32_t dsrc = a.R[src + 1] - a.R[src];
    a.q[0][0] = src;
    if (a.S[0]) {
      a.S[0][0] = 0;
      a.S[0][1] = dsrc;
    }
    c->depth = depth;
    c->parent = parent;
    c->src = src;
    c->level = 0;
    c->parity = 0;
    c->dir = kPush;
    c->q_len = 1;
    c->q_prev = 0;
    c->done = 0;
    c->error = kDevOk;
    c->pull_levels = 0;
    c->policy = policy;
    c->max_levels = max_levels;
    c->arrivals = 0ull;
    grid_barrier_reset(&c->bar);
    c->next_packed = 0ull;
    c->mf = dsrc;
    c->mu = a.m - dsrc;
    c->alpha = alpha;
    c->beta = beta;
    c->from_bitmap = 0;
    for (int i = 0; i < 3; ++i) {
      c->cnt3[i] = 0ull;
      c->maxdeg3[i] = 0;
    }
    c->t_start = globaltimer();
  }
}

// Shared memory of the level kernel: the push part's merge-path tables and
// the emit buffer (new vertices and their degrees), which the pull part
// reuses.
struct LevelSmem {
  int32_t off[kLvChunk + 1];
  int32_t u[kLvChunk + 1];
  int32_t row[kLvChunk + 1];
  int32_t out[kLvChunk];
  int32_t deg[kLvChunk];
  uint32_t red[33];
  unsigned long long red64[33];
  int32_t sred[kLvWarps];
  int32_t segcnt;
  int32_t i[2];
  int32_t cnt;
  int32_t vbase, ebase;
  int32_t last;
};

// Append (v, deg) to the block's emit buffer, warp-aggregated.
__device__ __forceinline__ void emit(LevelSmem &sm, bool take, int32_t v, int32_t d) {
  const int lane = threadIdx.x & 31;
  const uint32_t b = __ballot_sync(0xffffffffu, take);
  if (!b) return;
  const int leader = __ffs(b) - 1;
  int32_t pos = 0;
  if (lane == leader) pos = atomicAdd(&sm.cnt, __popc(b));
  pos = __shfl_sync(0xffffffffu, pos, leader);
  if (take) {
    const int32_t k = pos + __popc(b & ((1u << lane) - 1u));
    sm.out[k] = v;
    sm.deg[k] = d;
  }
}

// Write the emit buffer to the next queue with its exclusive degree scan,
// reserving both ranges with one packed atomicAdd. Block-uniform call.
__device__ void flush(LevelSmem &sm, unsigned long long *counter, int32_t *Qn, int32_t *Sn,
                      int32_t cap) {
  __syncthreads();
  const int32_t cnt = sm.cnt;
  if (cnt) {  // block-uniform
    constexpr int PER = kLvChunk / kLvThreads;
    const int32_t k0 = threadIdx.x * PER;
    uint32_t local = 0;
#pragma unroll
    for (int j = 0; j < PER; ++j)
      if (k0 + j < cnt) local += (uint32_t)sm.deg[k0 + j];
    uint32_t total;
    uint32_t run = block_excl_sum(local, sm.red, &total);
    if (threadIdx.x == 0) {
      const unsigned long long old = atomicAdd(
          counter, ((unsigned long long)total << 32) | (unsigned long long)cnt);
      sm.vbase = (int32_t)(old & 0xFFFFFFFFull);
      sm.ebase = (int32_t)(old >> 32);
    }
    __syncthreads();
    const int32_t vb = sm.vbase, eb = sm.ebase;
#pragma unroll
    for (int j = 0; j < PER; ++j) {
      const int32_t k = k0 + j;
      if (k < cnt) {
        if (GR_IN(vb + k, cap, 118)) {
          Qn[vb + k] = sm.out[k];
          Sn[vb + k] = eb + (int32_t)run;
        }
        run += (uint32_t)sm.deg[k];
      }
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) sm.cnt = 0;
  __syncthreads();
}

// Push over the frontier Q[0..q) with its exclusive degree scan S (S[q] =
// q_edges); this block takes chunks chunk0, chunk0 + step, ... of the merge
// path. The next frontier goes to the queue of parity p ^ 1.
__device__ void push_range(const BfsArgs &a, BfsCtl *c, LevelSmem &sm, const int32_t *Q,
                           const int32_t *S, int32_t p, int32_t L, int32_t q, int32_t q_edges,
                           unsigned long long *counter, long long chunk0, long long step) {
  int32_t *Qn = queue_of(a, p ^ 1);
  int32_t *Sn = scan_of(a, p ^ 1);
  uint32_t *N = bits_of(a, L + 1);
  int32_t *depth = c->depth;
  int32_t *parent = c->parent;
  const long long total = (long long)q + q_edges;
  const long long nchunks = (total + kLvChunk - 1) / kLvChunk;
  for (long long chunk = chunk0; chunk < nchunks; chunk += step) {
    const long long d0 = chunk * kLvChunk;
    const long long d1 = min(d0 + kLvChunk, total);
    int32_t i0, i1;
    block_chunk_bounds<kLvThreads>(S, q, q_edges, d0, d1, kLvChunk, sm.sred, &i0, &i1);
    const long long j0 = d0 - i0, j1 = d1 - i1;
    const int32_t nv = (i0 <= q - 1) ? (min(i1, q - 1) - i0 + 1) : 0;
    for (int32_t k = threadIdx.x; k < nv; k += kLvThreads) {
      const int32_t i = i0 + k;
      const int32_t u = GR_IN(i, a.n + 1, 110) ? Q[i] : 0;
      sm.off[k] = (i == q) ? q_edges : (GR_IN(i, a.n + 2, 111) ? S[i] : 0);
      sm.u[k] = u;
      sm.row[k] = GR_IN(u, a.n + 1, 112) ? a.R[u] : 0;
    }
    __syncthreads();
    const int32_t ne = (int32_t)(j1 - j0);  // <= kLvChunk: one pass of kLvItems per thread
    // each thread takes kLvItems edges (ranks tid, tid + T, ...) and issues
    // the loads of all of them before using any, so the latency chains of
    // the items overlap
    int32_t v[kLvItems], uo[kLvItems], dv[kLvItems];
    bool won[kLvItems];
#pragma unroll
    for (int j = 0; j < kLvItems; ++j) {
      const int32_t k = j * kLvThreads + threadIdx.x;
      v[j] = -1;
      uo[j] = 0;
      if (k < ne) {
        const int32_t er = (int32_t)(j0 + k);
        int32_t lo = 0, hi = nv - 1;
        while (lo < hi) {
          const int32_t mid = (lo + hi + 1) >> 1;
          if (sm.off[mid] <= er) lo = mid;
          else hi = mid - 1;
        }
        uo[j] = sm.u[lo];
        const long long e = (long long)sm.row[lo] + (er - sm.off[lo]);
        v[j] = GR_IN(e, a.m, 113) ? a.C[e] : -1;
        if (v[j] >= 0 && !GR_IN(v[j], a.n, 114)) v[j] = -1;
      }
    }
    uint32_t vw[kLvItems];
#pragma unroll
    for (int j = 0; j < kLvItems; ++j) vw[j] = v[j] >= 0 ? a.visited[v[j] >> 5] : 0xFFFFFFFFu;
#pragma unroll
    for (int j = 0; j < kLvItems; ++j) {
      won[j] = false;
      if (v[j] >= 0) {
        const uint32_t mask = 1u << (v[j] & 31);
        if (!(vw[j] & mask)) won[j] = !(atomicOr(a.visited + (v[j] >> 5), mask) & mask);
      }
    }
#pragma unroll
    for (int j = 0; j < kLvItems; ++j) {
      dv[j] = 0;
      if (won[j]) {
        depth[v[j]] = L + 1;
        if (parent) parent[v[j]] = uo[j];
        if (a.do_bitmap) atomicOr(N + (v[j] >> 5), 1u << (v[j] & 31));
        dv[j] = a.R[v[j] + 1] - a.R[v[j]];
      }
    }
#pragma unroll
    for (int j = 0; j < kLvItems; ++j) emit(sm, won[j], v[j], dv[j]);
    flush(sm, counter, Qn, Sn, a.n + 1);
  }
}

__device__ __forceinline__ void push_level(const BfsArgs &a, BfsCtl *c, LevelSmem &sm,
                                           int32_t p, int32_t L, int32_t q, int32_t q_edges,
                                           unsigned long long *counter) {
  push_range(a, c, sm, queue_of(a, p), scan_of(a, p), p, L, q, q_edges, counter, blockIdx.x,
             gridDim.x);
}

// Push level for graphs of small maximum degree (meshes): one thread per
// frontier vertex walks its whole neighbour list (the per-thread expansion
// of Sec. 4.4, which is balanced when every degree is small), so the level
// needs neither a merge-path search nor the queue's degree scan. The
// candidates' row offsets are loaded with their visited words, so a
// winner's degree (for the next frontier's edge count) costs no extra round
// trip; winners are appended with one packed atomic per warp.
__device__ void push_level_thread(const BfsArgs &a, BfsCtl *c, int32_t p, int32_t L, int32_t q,
                                  unsigned long long *counter) {
  const int32_t *Q = queue_of(a, p);
  int32_t *Qn = queue_of(a, p ^ 1);
  int32_t *depth = c->depth;
  int32_t *parent = c->parent;
  const int lane = threadIdx.x & 31;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t qr = ((int64_t)q + 31) & ~31ll;  // warp-uniform bound
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < qr; i += stride) {
    int32_t u = 0, r0 = 0, r1 = 0;
    if (i < q) {
      u = Q[i];
      if (GR_IN(u, a.n, 170)) {
        r0 = a.R[u];
        r1 = a.R[u + 1];
      }
    }
    for (int32_t e0 = r0; __any_sync(0xffffffffu, e0 < r1); e0 += kTpvItems) {
      int32_t v[kTpvItems], d0[kTpvItems], d1[kTpvItems];
      uint32_t vw[kTpvItems];
      bool won[kTpvItems];
#pragma unroll
      for (int j = 0; j < kTpvItems; ++j) {
        v[j] = (e0 + j < r1 && GR_IN(e0 + j, a.m, 171)) ? a.C[e0 + j] : -1;
        if (v[j] >= 0 && !GR_IN(v[j], a.n, 172)) v[j] = -1;
      }
#pragma unroll
      for (int j = 0; j < kTpvItems; ++j) {
        vw[j] = 0xFFFFFFFFu;
        d0[j] = d1[j] = 0;
        if (v[j] >= 0) {
          vw[j] = a.visited[v[j] >> 5];
          d0[j] = a.R[v[j]];
          d1[j] = a.R[v[j] + 1];
        }
      }
      uint32_t cnt = 0, deg = 0;
#pragma unroll
      for (int j = 0; j < kTpvItems; ++j) {
        won[j] = false;
        if (v[j] >= 0) {
          const uint32_t mask = 1u << (v[j] & 31);
          if (!(vw[j] & mask)) won[j] = !(atomicOr(a.visited + (v[j] >> 5), mask) & mask);
        }
        if (won[j]) {
          depth[v[j]] = L + 1;
          if (parent) parent[v[j]] = u;
          cnt += 1;
          deg += (uint32_t)(d1[j] - d0[j]);
        }
      }
      // warp-level exclusive scan of (edges, vertices), one packed atomic
      const unsigned long long mine = ((unsigned long long)deg << 32) | cnt;
      unsigned long long incl = mine;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
      }
      const unsigned long long total = __shfl_sync(0xffffffffu, incl, 31);
      if (total) {
        unsigned long long base = 0;
        if (lane == 0) base = atomicAdd(counter, total);
        base = __shfl_sync(0xffffffffu, base, 0);
        int32_t k = (int32_t)((base + (incl - mine)) & 0xFFFFFFFFull);
#pragma unroll
        for (int j = 0; j < kTpvItems; ++j)
          if (won[j]) {
            if (GR_IN(k, a.n + 1, 173)) Qn[k] = v[j];
            ++k;
          }
      }
    }
  }
}

// Pull level: no queue is written; the block counts the vertices it found
// and their edges and adds both to the packed counter once at the end. A
// warp owns kPullWords consecutive bitmap words per step (32 * kPullWords
// vertices, kPullWords per lane) so several load chains are in flight.
constexpr int kPullWords = 2;

__device__ void pull_level(const BfsArgs &a, BfsCtl *c, LevelSmem &sm, int32_t L,
                           unsigned long long *counter, int32_t *maxdeg = nullptr) {
  const uint32_t *F = bits_of(a, L);
  uint32_t *N = bits_of(a, L + 1);
  int32_t *depth = c->depth;
  int32_t *parent = c->parent;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const long long gw = (long long)blockIdx.x * kLvWarps + wid;
  const long long nw = (long long)gridDim.x * kLvWarps;
  const long long groups = (a.nwords + kPullWords - 1) / kPullWords;
  uint32_t found_cnt = 0;
  unsigned long long found_deg = 0;
  uint32_t found_max = 0;
  for (long long gi = gw; gi < groups; gi += nw) {  // warp-uniform loop
    const long long w0 = gi * kPullWords;
    uint32_t vis[kPullWords];
    int32_t v[kPullWords], r0[kPullWords], r1[kPullWords], uf[kPullWords];
    bool act[kPullWords], fnd[kPullWords];
#pragma unroll
    for (int j = 0; j < kPullWords; ++j) {
      const long long w = w0 + j;
      vis[j] = w < a.nwords ? a.visited[w] : 0xFFFFFFFFu;
      v[j] = (int32_t)(w * 32 + lane);
      act[j] = w < a.nwords && v[j] < a.n && !((vis[j] >> lane) & 1u);
      fnd[j] = false;
      uf[j] = -1;
      r0[j] = r1[j] = 0;
    }
    // row bounds and the first neighbour (from the dense first-neighbour
    // array: coalesced, and not waiting for the row offset) of every
    // unvisited vertex, independent loads
    int32_t u1[kPullWords];
#pragma unroll
    for (int j = 0; j < kPullWords; ++j) {
      u1[j] = -1;
      if (act[j]) {
        r0[j] = a.R[v[j]];
        r1[j] = a.R[v[j] + 1];
        u1[j] = a.first[v[j]];
      }
    }
#pragma unroll
    for (int j = 0; j < kPullWords; ++j) {
      if (!GR_IN(r0[j], a.m + 1, 120) || !GR_IN(r1[j], a.m + 1, 121)) {
        r1[j] = r0[j] = 0;
        u1[j] = -1;
      }
      if (u1[j] >= 0 && !GR_IN(u1[j], a.n, 122)) u1[j] = -1;
    }
#pragma unroll
    for (int j = 0; j < kPullWords; ++j)
      if (u1[j] >= 0 && test_bit(F, u1[j])) {
        fnd[j] = true;
        uf[j] = u1[j];
      }
    // the rest of each list: lanes alone up to kPullLane more neighbours,
    // then the whole warp on whatever is left, 32 neighbours at a time
#pragma unroll
    for (int j = 0; j < kPullWords; ++j) {
      if (act[j] && !fnd[j]) {
        const int32_t stop = min(r1[j], r0[j] + 1 + kPullLane);
        for (int32_t e = r0[j] + 1; e < stop; ++e) {
          const int32_t u = a.C[e];
          if (GR_IN(u, a.n, 123) && test_bit(F, u)) {
            fnd[j] = true;
            uf[j] = u;
            break;
          }
        }
      }
      uint32_t longm =
          __ballot_sync(0xffffffffu, act[j] && !fnd[j] && r1[j] - r0[j] > 1 + kPullLane);
      while (longm) {
        const int leader = __ffs(longm) - 1;
        longm &= longm - 1u;
        const int32_t b0 = __shfl_sync(0xffffffffu, r0[j], leader) + 1 + kPullLane;
        const int32_t b1 = __shfl_sync(0xffffffffu, r1[j], leader);
        for (int32_t base = b0; base < b1; base += 32) {
          const int32_t e = base + lane;
          const int32_t u = e < b1 ? a.C[e] : 0;
          const bool hit = e < b1 && GR_IN(u, a.n, 124) && test_bit(F, u);
          const uint32_t hb = __ballot_sync(0xffffffffu, hit);
          if (hb) {
            const int32_t hu = __shfl_sync(0xffffffffu, u, __ffs(hb) - 1);
            if (lane == leader) {
              fnd[j] = true;
              uf[j] = hu;
            }
            break;
          }
        }
      }
      const uint32_t fm = __ballot_sync(0xffffffffu, fnd[j]);
      const long long w = w0 + j;
      if (w < a.nwords && lane == 0) {
        N[w] = fm;
        if (fm) a.visited[w] = vis[j] | fm;
      }
      if (fnd[j]) {
        depth[v[j]] = L + 1;
        if (parent) parent[v[j]] = uf[j];
        ++found_cnt;
        found_deg += (unsigned long long)(r1[j] - r0[j]);
        found_max = max(found_max, (uint32_t)(r1[j] - r0[j]));
      }
      if (a.seg_v && fm) {  // append to this block's segment (shared-memory slot)
        int32_t pos = 0;
        if (lane == 0) pos = atomicAdd(&sm.segcnt, __popc(fm));
        pos = __shfl_sync(0xffffffffu, pos, 0);
        if (fnd[j]) {
          const int64_t kk = pos + __popc(fm & ((1u << lane) - 1u));
          const int64_t k = (int64_t)blockIdx.x * a.seg_cap + kk;
          if (GR_IN(kk, a.seg_cap, 125)) {
            a.seg_v[k] = v[j];
            a.seg_d[k] = r1[j] - r0[j];
          }
        }
      }
    }
  }
  if (maxdeg) {
    const uint32_t wmax = __reduce_max_sync(0xffffffffu, found_max);
    if ((threadIdx.x & 31) == 0 && wmax) atomicMax(maxdeg, (int32_t)wmax);
  }
  // one packed atomicAdd per block: [31:0] vertices, [63:32] their edges
  const unsigned long long packed =
      block_sum((found_deg << 32) | (unsigned long long)found_cnt, (unsigned long long *)sm.red64);
  if (threadIdx.x == 0) {
    if (packed) atomicAdd(counter, packed);
    if (a.seg_v) a.seg_cnt[blockIdx.x] = packed;
  }
}

// Queue + degree scan of the vertices the last pull level found, from the
// per-block segments: every block computes, from the per-block totals, the
// offsets of its segment in the queue and in the edge scan, then compacts
// its own segment. *q_out / *e_out receive the totals.
__device__ void segments_to_queue(const BfsArgs &a, LevelSmem &sm, int32_t *Q, int32_t *S,
                                  int32_t *q_out, int32_t *e_out) {
  const int32_t G = gridDim.x, b = blockIdx.x;
  unsigned long long before = 0, all = 0;
  for (int32_t i = threadIdx.x; i < G; i += kLvThreads) {
    const unsigned long long x = a.seg_cnt[i];
    all += x;
    if (i < b) before += x;
  }
  before = block_sum(before, sm.red64);
  all = block_sum(all, sm.red64);
  *q_out = (int32_t)(all & 0xFFFFFFFFull);
  *e_out = (int32_t)(all >> 32);
  const int32_t vo = (int32_t)(before & 0xFFFFFFFFull);
  uint32_t eo = (uint32_t)(before >> 32);
  const int32_t cb = (int32_t)(a.seg_cnt[b] & 0xFFFFFFFFull);
  const int64_t base = (int64_t)b * a.seg_cap;
  constexpr int PER = kLvChunk / kLvThreads;
  for (int32_t t0 = 0; t0 < cb; t0 += kLvChunk) {  // block-uniform
    const int32_t k0 = t0 + threadIdx.x * PER;
    int32_t dd[PER];
    uint32_t local = 0;
#pragma unroll
    for (int j = 0; j < PER; ++j) {
      dd[j] = (k0 + j < cb && GR_IN(k0 + j, a.seg_cap, 128)) ? a.seg_d[base + k0 + j] : 0;
      local += (uint32_t)dd[j];
    }
    uint32_t tile_total;
    uint32_t run = eo + block_excl_sum(local, sm.red, &tile_total);
#pragma unroll
    for (int j = 0; j < PER; ++j) {
      const int32_t k = k0 + j;
      if (k < cb) {
        if (GR_IN(vo + k, a.n + 1, 126) && GR_IN(k, a.seg_cap, 127)) {
          Q[vo + k] = a.seg_v[base + k];
          S[vo + k] = (int32_t)run;
        }
        run += (uint32_t)dd[j];
      }
    }
    eo += tile_total;
  }
}

// The level after a pull whose vertices all have small degree: every block
// pushes the vertices it found itself (its pull segment), after an in-place
// exclusive scan of their degrees, so the level needs no grid-wide
// compaction and no extra grid barrier. Blocks carry unequal work, bounded by
// the segment sizes and the small degrees.
__device__ void push_own_segment(const BfsArgs &a, BfsCtl *c, LevelSmem &sm, int32_t p,
                                 int32_t L, unsigned long long *counter) {
  const unsigned long long pk = a.seg_cnt[blockIdx.x];
  const int32_t cb = (int32_t)(pk & 0xFFFFFFFFull), eb = (int32_t)(pk >> 32);
  const int64_t base = (int64_t)blockIdx.x * a.seg_cap;
  int32_t *V = a.seg_v + base;
  int32_t *D = a.seg_d + base;
  constexpr int PER = kLvChunk / kLvThreads;
  uint32_t run_base = 0;
  for (int32_t t0 = 0; t0 < cb; t0 += kLvChunk) {  // block-uniform
    const int32_t k0 = t0 + threadIdx.x * PER;
    int32_t dd[PER];
    uint32_t local = 0;
#pragma unroll
    for (int j = 0; j < PER; ++j) {
      dd[j] = (k0 + j < cb && GR_IN(k0 + j, a.seg_cap, 180)) ? D[k0 + j] : 0;
      local += (uint32_t)dd[j];
    }
    uint32_t tile_total;
    uint32_t run = run_base + block_excl_sum(local, sm.red, &tile_total);
#pragma unroll
    for (int j = 0; j < PER; ++j) {
      if (k0 + j < cb && GR_IN(k0 + j, a.seg_cap, 181)) D[k0 + j] = (int32_t)run;
      run += (uint32_t)dd[j];
    }
    run_base += tile_total;
  }
  __syncthreads();
  push_range(a, c, sm, V, D, p, L, cb, eb, counter, 0, 1);
}

// Push level whose frontier exists only as a bitmap (the level after a
// pull): warps walk the frontier bitmap's words, expand each set vertex
// lane-parallel, and append winners with a warp-level degree scan and one
// packed atomicAdd per warp step. Used for the small frontiers after the
// pull phase, where per-warp appends do not contend.
__device__ void push_from_bitmap(const BfsArgs &a, BfsCtl *c, int32_t p, int32_t L,
                                 unsigned long long *counter) {
  const uint32_t *F = bits_of(a, L);
  uint32_t *N = bits_of(a, L + 1);
  int32_t *Qn = queue_of(a, p ^ 1);
  int32_t *Sn = scan_of(a, p ^ 1);
  int32_t *depth = c->depth;
  int32_t *parent = c->parent;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const long long gw = (long long)blockIdx.x * kLvWarps + wid;
  const long long nw = (long long)gridDim.x * kLvWarps;
  for (long long w = gw; w < a.nwords; w += nw) {
    uint32_t fw = F[w];
    while (fw) {
      const int j = __ffs(fw) - 1;
      fw &= fw - 1u;
      const int32_t u = (int32_t)(w * 32 + j);
      const int32_t r0 = a.R[u], r1 = a.R[u + 1];
      for (int32_t base = r0; base < r1; base += 32) {
        const int32_t e = base + lane;
        bool won = false;
        int32_t v = 0, dv = 0;
        if (e < r1 && GR_IN(e, a.m, 130)) {
          v = a.C[e];
          if (GR_IN(v, a.n, 131)) {
            const uint32_t mask = 1u << (v & 31);
            uint32_t *vw = a.visited + (v >> 5);
            if (!(*vw & mask)) won = !(atomicOr(vw, mask) & mask);
            if (won) {
              depth[v] = L + 1;
              if (parent) parent[v] = u;
              if (a.do_bitmap) atomicOr(N + (v >> 5), mask);
              dv = a.R[v + 1] - a.R[v];
            }
          }
        }
        const uint32_t b = __ballot_sync(0xffffffffu, won);
        if (b) {
          const uint32_t incl = warp_incl_sum((uint32_t)dv);
          const uint32_t tot = __shfl_sync(0xffffffffu, incl, 31);
          unsigned long long old = 0;
          if (lane == 0)
            old = atomicAdd(counter,
                            ((unsigned long long)tot << 32) | (unsigned long long)__popc(b));
          old = __shfl_sync(0xffffffffu, old, 0);
          if (won) {
            const int32_t k = (int32_t)(old & 0xFFFFFFFFull) + __popc(b & ((1u << lane) - 1u));
            if (GR_IN(k, a.n + 1, 132)) {
              Qn[k] = v;
              Sn[k] = (int32_t)(old >> 32) + (int32_t)(incl - dv);
            }
          }
        }
      }
    }
  }
}

// Direction of the next level (Sec. 4.5; Beamer et al.'s rule): push ->
// pull when the new frontier's edges exceed the unexplored edges / alpha
// (and are not a negligible share of the graph, so that a tiny frontier
// late in the traversal, when few edges remain unexplored, stays push);
// pull -> push when the frontier has fallen below n / beta vertices and is
// shrinking.
__device__ __forceinline__ int32_t next_direction(int32_t policy, bool was_pull, int32_t qn,
                                                  int32_t q_prev, long long mf, long long mu,
                                                  long long m, int32_t n, float alpha,
                                                  float beta) {
  if (policy == GR_DIR_PUSH) return kPush;
  if (policy == GR_DIR_PULL) return kPull;
  if (was_pull) return ((float)qn < (float)n / beta && qn < q_prev) ? kPush : kPull;
  return ((float)mf > (float)mu / alpha && mf * 1024 > m) ? kPull : kPush;
}

// Run by the last block of a level: install the next frontier and decide
// the next level's direction (Sec. 4.5; Beamer et al.'s rule).
__device__ void level_end(const BfsArgs &a, BfsCtl *c) {
  const unsigned long long packed = *(volatile unsigned long long *)&c->next_packed;
  const int32_t qn = (int32_t)(packed & 0xFFFFFFFFull);
  const long long mf = (long long)(packed >> 32);
  const bool was_pull = c->dir == kPull;
  if (was_pull) c->pull_levels += 1;
  if (c->level < kTraceLevels) {
    c->tr_dir[c->level] = c->dir;
    c->tr_q[c->level] = c->q_len;
    c->tr_mf[c->level] = c->mf;
    c->tr_t[c->level] = globaltimer();
  }
  c->from_bitmap = was_pull;  // a pull leaves only the bitmap of its output
  c->level += 1;
  c->parity ^= 1;
  c->q_prev = c->q_len;
  c->q_len = qn;
  c->next_packed = 0ull;
  c->mf = mf;
  c->mu -= mf;
  if (!was_pull && GR_IN(qn, a.n + 2, 140)) scan_of(a, c->parity)[qn] = (int32_t)mf;
  if (qn == 0) {
    c->done = 1;
    return;
  }
  if (c->level >= c->max_levels) {
    c->error = kDevOverflow;
    c->done = 1;
    return;
  }
  c->dir = next_direction(c->policy, was_pull, qn, c->q_prev, mf, c->mu, a.m, a.n, c->alpha,
                          c->beta);
}

__global__ void __launch_bounds__(kLvThreads, kLvBlocksPerSm)
    k_bfs_level(BfsArgs a, cudaGraphConditionalHandle h, int32_t use_cond) {
  BfsCtl *c = a.ctl;
  if (*(volatile int32_t *)&c->done) {
    // a level kernel after the traversal ended (host-driven batches enqueue
    // a few extra): every block leaves; inside a graph the loop condition is
    // cleared here too, so the while loop cannot outlive the traversal
    if (use_cond && blockIdx.x == 0 && threadIdx.x == 0) cudaGraphSetConditional(h, 0u);
    return;
  }
  __shared__ LevelSmem sm;
  if (threadIdx.x == 0) sm.cnt = 0;
  const int32_t p = c->parity, L = c->level, q = c->q_len, dir = c->dir;
  // clear the bitmap the next level will fill (nobody reads or writes it now)
  if (a.do_bitmap) {
    uint32_t *spare = bits_of(a, L + 2);
    for (int64_t w = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; w < a.nwords;
         w += (int64_t)gridDim.x * blockDim.x)
      spare[w] = 0u;
  }
  __syncthreads();
  if (dir == kPull) pull_level(a, c, sm, L, &c->next_packed);
  else if (c->from_bitmap) push_from_bitmap(a, c, p, L, &c->next_packed);
  else if (a.low_degree) push_level_thread(a, c, p, L, q, &c->next_packed);
  else push_level(a, c, sm, p, L, q, (int32_t)c->mf, &c->next_packed);
  // the last block to finish ends the level
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    const unsigned long long old = atomicAdd(&c->arrivals, 1ull);
    sm.last = (old + 1ull) % gridDim.x == 0ull;
  }
  __syncthreads();
  if (sm.last && threadIdx.x == 0) {
    __threadfence();
    level_end(a, c);
    if (use_cond) cudaGraphSetConditional(h, c->done ? 0u : 1u);
  }
}

// ------------------------------------------- persistent direction-optimising
// The whole traversal in one cooperative kernel: every block runs every
// level and the levels are separated by one bounded-spin grid barrier. After
// the barrier each block reads the level's packed counter and recomputes the
// same next state (direction, sizes, edge counts) in registers, so no second
// barrier is needed to publish it. The counters form a ring of three: the
// one a level fills, the one just read, and the one block 0 clears for the
// next level (its last readers passed the previous barrier).

__device__ __forceinline__ bool grid_barrier(BfsCtl *c, int32_t nblocks, int32_t &gen);

// 6 blocks of 256 threads per SM (40 registers, no spills) took R-MAT s22
// from 0.1976 to 0.1900 ms per traversal against 5 (48 registers); 7 or more
// spill
constexpr int kDoBlocksPerSm = 6;
// After a pull level whose found vertices all have at most this degree, each
// block pushes its own pull segment (no grid-wide compaction).
constexpr int32_t kSegPushMaxDeg = 1024;

__global__ void __launch_bounds__(kLvThreads, kDoBlocksPerSm) k_bfs_do(BfsArgs a) {
  BfsCtl *c = a.ctl;
  __shared__ LevelSmem sm;
  // a traversal the one-cluster driver finished, or one it hands over at
  // level c->level with the frontier in queue c->parity
  if (*(volatile int32_t *)&c->done) return;
  const int32_t policy = c->policy, max_levels = c->max_levels;
  const float alpha = c->alpha, beta = c->beta;
  int32_t level = c->level, parity = c->parity, dir = kPush, q = c->q_len, q_prev = 0,
          from_bitmap = 0;
  long long mf = c->mf, mu = c->mu;
  int32_t gen = 0, pulls = 0;
  int32_t seg_maxdeg = 0;  // largest degree the last pull level found
  if (threadIdx.x == 0) sm.cnt = 0;
  __syncthreads();
  for (;;) {
    const int32_t L = level;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      c->cnt3[(L + 1) % 3] = 0ull;
      c->maxdeg3[(L + 1) % 3] = 0;
    }
    if (a.do_bitmap) {
      uint32_t *spare = bits_of(a, L + 2);
      for (int64_t w = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; w < a.nwords;
           w += (int64_t)gridDim.x * blockDim.x)
        spare[w] = 0u;
    }
    unsigned long long *counter = &c->cnt3[L % 3];
    if (threadIdx.x == 0) sm.segcnt = 0;
    __syncthreads();
    if (dir == kPull) {
      pull_level(a, c, sm, L, counter, &c->maxdeg3[L % 3]);
    } else if (from_bitmap && seg_maxdeg <= kSegPushMaxDeg) {
      push_own_segment(a, c, sm, parity, L, counter);
    } else {
      int32_t qq = q, qe = (int32_t)mf;
      if (from_bitmap) {
        segments_to_queue(a, sm, queue_of(a, parity), scan_of(a, parity), &qq, &qe);
        if (!grid_barrier(c, gridDim.x, gen)) break;
      }
      if (a.low_degree) push_level_thread(a, c, parity, L, qq, counter);
      else push_level(a, c, sm, parity, L, qq, qe, counter);
    }
    // with the two-level barrier of a large grid the level's counter comes
    // with the release; after a one-level barrier every block reads it
    unsigned long long pk = 0ull;
    if (gridDim.x > kFlatBarrierBlocks) {
      if (!grid_sync(&c->bar, &c->error, gen, counter, &pk)) break;
    } else {
      if (!grid_barrier(c, gridDim.x, gen)) break;
      pk = *(volatile unsigned long long *)counter;
    }
    seg_maxdeg = dir == kPull ? *(volatile int32_t *)&c->maxdeg3[L % 3] : 0;
    const int32_t qn = (int32_t)(pk & 0xFFFFFFFFull);
    const long long mfn = (long long)(pk >> 32);
    const bool was_pull = dir == kPull;
    if (blockIdx.x == 0 && threadIdx.x == 0 && L < kTraceLevels) {
      c->tr_dir[L] = dir;
      c->tr_q[L] = q;
      c->tr_mf[L] = mf;
      c->tr_t[L] = globaltimer();
    }
    pulls += was_pull;
    level += 1;
    parity ^= 1;
    q_prev = q;
    q = qn;
    mf = mfn;
    mu -= mfn;
    from_bitmap = was_pull;
    bool done = qn == 0;
    const bool overflow = !done && level >= max_levels;
    if (done || overflow) {
      if (blockIdx.x == 0 && threadIdx.x == 0) {
        c->level = level;
        c->pull_levels = pulls;
        if (overflow) c->error = kDevOverflow;
        c->done = 1;
      }
      break;
    }
    dir = next_direction(policy, was_pull, qn, q_prev, mfn, mu, a.m, a.n, alpha, beta);
  }
}

// ------------------------------------------------------ one-cluster driver
// On graphs of small maximum degree (meshes) a BFS has thousands of levels
// of a few thousand vertices each, and a grid-wide barrier per level costs
// more than the level's work. This driver runs those levels in ONE thread
// block cluster: the CTAs meet at the hardware cluster barrier, and each
// level's new frontier stays in the CTAs' shared memory, where the next level
// reads it through distributed shared memory. Each CTA appends the vertices
// its threads claimed, with their row bounds (so the next level needs no
// row-offset load), to its own buffer (one per level parity); what does not
// fit goes to the global queue of that parity, positioned by the level's
// global counter, so the frontier of a level is the CTAs' buffers followed by
// that queue's first entries. At the end of a level each CTA writes its
// counts into every CTA's shared memory before the barrier, so no level
// starts with a remote load. Once a frontier outgrows kClHandoff vertices,
// the cluster writes it to the global queue as a plain list and leaves the
// rest of the traversal to k_bfs_do (same stream), which resumes at that
// level.
constexpr int kClThreads = 1024;
constexpr int kClMaxCtas = 16;
constexpr int kClCap = 1024;        // buffered vertices per CTA and parity
constexpr int kClHandoff = 32768;   // larger frontiers go to the grid kernel

__device__ __forceinline__ uint32_t cl_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
__device__ __forceinline__ uint32_t cl_size() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(r));
  return r;
}
// address of `p` (this CTA's shared memory) in CTA `rank` of the cluster
__device__ __forceinline__ uint32_t cl_map(const void *p, uint32_t rank) {
  const uint32_t a = (uint32_t)__cvta_generic_to_shared(p);
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(rank));
  return r;
}
__device__ __forceinline__ int4 cl_ld_v4(uint32_t addr) {
  int4 v;
  asm volatile("ld.shared::cluster.v4.s32 {%0, %1, %2, %3}, [%4];"
               : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
               : "r"(addr)
               : "memory");
  return v;
}
__device__ __forceinline__ void cl_st_s32(uint32_t addr, int32_t v) {
  asm volatile("st.shared::cluster.s32 [%0], %1;" ::"r"(addr), "r"(v) : "memory");
}
__device__ __forceinline__ void cl_st_u64(uint32_t addr, unsigned long long v) {
  asm volatile("st.shared::cluster.u64 [%0], %1;" ::"r"(addr), "l"(v) : "memory");
}
__device__ __forceinline__ void cl_fence() {
  asm volatile("fence.acq_rel.cluster;" ::: "memory");
}
// every thread of every CTA of the cluster; a relaxed arrival (the threads
// whose writes others must see fence first), an acquiring wait
__device__ __forceinline__ void cl_sync_relaxed() {
  asm volatile("barrier.cluster.arrive.relaxed.aligned;\n\t"
               "barrier.cluster.wait.acquire.aligned;" ::: "memory");
}
__device__ __forceinline__ void cl_sync() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\t"
               "barrier.cluster.wait.acquire.aligned;" ::: "memory");
}

struct ClSmem {
  // this CTA's part of the frontier by level parity: (vertex, row start,
  // row end, 0), so the next level reads a vertex and its row in one load
  int4 buf[2][kClCap];
  int32_t cnt[2];                  // vertices appended (past kClCap: global queue)
  unsigned long long edges[2];     // their degrees' sum
  // every CTA's cnt / edges for each parity, pushed here by that CTA
  int32_t rc[2][kClMaxCtas];
  unsigned long long re[2][kClMaxCtas];
  int32_t pref[kClMaxCtas];  // the current frontier: CTA r's entries start at pref[r]
  int32_t nb, ovf;           // buffered entries, entries in the global queue
  long long mf;              // edges leaving the frontier
};

__global__ void __launch_bounds__(kClThreads, 1) k_bfs_cluster(BfsArgs a) {
  BfsCtl *c = a.ctl;
  __shared__ ClSmem sm;
  const uint32_t rank = cl_rank(), ncta = cl_size();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int32_t max_levels = c->max_levels;
  int32_t *depth = c->depth;
  int32_t *parent = c->parent;
  const int32_t q0 = c->q_len;  // level 0: the source, in global queue 0
  const long long mf0 = c->mf;
  if (threadIdx.x < 2 * kClMaxCtas) {
    (&sm.rc[0][0])[threadIdx.x] = 0;
    (&sm.re[0][0])[threadIdx.x] = 0ull;
  }
  if (threadIdx.x == 0) {
    sm.cnt[0] = sm.cnt[1] = 0;
    sm.edges[0] = sm.edges[1] = 0ull;
  }
  cl_sync();
  // items are dealt to the CTAs 32 at a time, so a small frontier still
  // spreads over every SM of the cluster
  const int64_t first = (int64_t)warp * (32 * ncta) + rank * 32 + lane;
  const int64_t stride = (int64_t)ncta * kClThreads;
  int32_t q_last = 0;
  long long mf_last = 0;
  for (int32_t L = 0;; ++L) {
    const int p = L & 1;
    if (warp == 0) {
      // the frontier's shape from the counts every CTA pushed here
      const int32_t cr = lane < (int)ncta ? sm.rc[p][lane] : 0;
      unsigned long long er = lane < (int)ncta ? sm.re[p][lane] : 0ull;
      const int32_t b = min(cr, kClCap);
      int32_t o = max(cr - kClCap, 0), incl = b;
#pragma unroll
      for (int k = 1; k < 32; k <<= 1) {
        const int32_t t = __shfl_up_sync(0xffffffffu, incl, k);
        if (lane >= k) incl += t;
      }
      o = __reduce_add_sync(0xffffffffu, o);
#pragma unroll
      for (int k = 16; k >= 1; k >>= 1) er += __shfl_xor_sync(0xffffffffu, er, k);
      if (lane < kClMaxCtas) sm.pref[lane] = incl - b;
      if (lane == 31) sm.nb = incl;
      if (lane == 0) {
        sm.ovf = o + (L == 0 ? q0 : 0);
        sm.mf = (long long)er + (L == 0 ? mf0 : 0);
      }
    }
    if (threadIdx.x == 0) {
      // the counters this level fills were pushed to every CTA in level L - 1
      sm.cnt[p ^ 1] = 0;
      sm.edges[p ^ 1] = 0ull;
      if (rank == 0) {
        if (L >= 1 && L - 1 < kTraceLevels) {
          c->tr_dir[L - 1] = kPush;
          c->tr_q[L - 1] = q_last;
          c->tr_mf[L - 1] = mf_last;
          c->tr_t[L - 1] = globaltimer();
        }
        c->cnt3[(L + 1) % 3] = 0ull;  // the global counter of level L + 1
      }
    }
    __syncthreads();
    const int32_t nb = sm.nb, ovf = sm.ovf;
    const int32_t q = nb + ovf;
    const long long mf = sm.mf;
    const bool done = q == 0;
    const bool over = !done && L >= max_levels;
    const bool handoff = !done && !over && q > kClHandoff;
    if (done || over || handoff) {
      if (handoff) {
        // the frontier as one list: the global part stays, the CTAs' buffers
        // follow it in rank order
        int32_t *Q = queue_of(a, p);
        const int32_t at = ovf + sm.pref[rank];
        const int32_t mine = min(sm.rc[p][rank], kClCap);
        for (int32_t k = threadIdx.x; k < mine; k += kClThreads) Q[at + k] = sm.buf[p][k].x;
      }
      if (rank == 0 && threadIdx.x == 0) {
        c->level = L;
        if (handoff) {
          c->parity = p;
          c->q_len = q;
          c->mf = mf;
          c->cnt3[L % 3] = 0ull;
        } else {
          c->pull_levels = 0;
          if (over) c->error = kDevOverflow;
          c->done = 1;
        }
      }
      cl_sync();
      return;
    }
    const int32_t *Qg = queue_of(a, p);
    int32_t *Qn = queue_of(a, p ^ 1);
    unsigned long long *gctr = &c->cnt3[L % 3];
    const int64_t qr = ((int64_t)q + 31) & ~31ll;  // warp-uniform bound
    for (int64_t i = first; i < qr; i += stride) {
      int32_t u = 0, r0 = 0, r1 = 0;
      if (i < q) {
        if (i < nb) {
          uint32_t r = 0;  // the last CTA whose entries start at or before i
#pragma unroll
          for (uint32_t k = kClMaxCtas / 2; k >= 1; k >>= 1)
            if (r + k < ncta && sm.pref[r + k] <= i) r += k;
          const int4 e = cl_ld_v4(cl_map(&sm.buf[p][i - sm.pref[r]], r));
          u = e.x;
          r0 = e.y;
          r1 = e.z;
        } else {
          u = Qg[i - nb];
          if (GR_IN(u, a.n, 190)) {
            r0 = a.R[u];
            r1 = a.R[u + 1];
          }
        }
      }
      for (int32_t e0 = r0; __any_sync(0xffffffffu, e0 < r1); e0 += kTpvItems) {
        int32_t v[kTpvItems], d0[kTpvItems], d1[kTpvItems];
        uint32_t vw[kTpvItems];
        bool won[kTpvItems];
#pragma unroll
        for (int j = 0; j < kTpvItems; ++j) {
          v[j] = (e0 + j < r1 && GR_IN(e0 + j, a.m, 191)) ? a.C[e0 + j] : -1;
          if (v[j] >= 0 && !GR_IN(v[j], a.n, 192)) v[j] = -1;
        }
#pragma unroll
        for (int j = 0; j < kTpvItems; ++j) {
          vw[j] = 0xFFFFFFFFu;
          d0[j] = d1[j] = 0;
          if (v[j] >= 0) {
            vw[j] = a.visited[v[j] >> 5];
            d0[j] = a.R[v[j]];
            d1[j] = a.R[v[j] + 1];
          }
        }
        int32_t cnt = 0, deg = 0;
#pragma unroll
        for (int j = 0; j < kTpvItems; ++j) {
          won[j] = false;
          if (v[j] >= 0) {
            const uint32_t mask = 1u << (v[j] & 31);
            if (!(vw[j] & mask)) won[j] = !(atomicOr(a.visited + (v[j] >> 5), mask) & mask);
          }
          if (won[j]) {
            depth[v[j]] = L + 1;
            if (parent) parent[v[j]] = u;
            cnt += 1;
            deg += d1[j] - d0[j];
          }
        }
        // warp-level exclusive scan of the claims, one shared-memory atomic
        int32_t incl = cnt;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const int32_t t = __shfl_up_sync(0xffffffffu, incl, o);
          if (lane >= o) incl += t;
        }
        const int32_t total = __shfl_sync(0xffffffffu, incl, 31);
        if (total) {
          const int32_t dsum = __reduce_add_sync(0xffffffffu, deg);
          int32_t base = 0;
          if (lane == 0) {
            base = atomicAdd(&sm.cnt[p ^ 1], total);
            atomicAdd(&sm.edges[p ^ 1], (unsigned long long)dsum);
          }
          base = __shfl_sync(0xffffffffu, base, 0);
          // positions past the buffer go to the global queue, in the order
          // of the level's global counter
          const int32_t kfirst = max(base, kClCap);
          const int32_t ng = max(0, base + total - kfirst);
          unsigned long long g0 = 0ull;
          if (lane == 0 && ng) g0 = atomicAdd(gctr, (unsigned long long)ng);
          g0 = __shfl_sync(0xffffffffu, g0, 0);
          int32_t k = base + (incl - cnt);
#pragma unroll
          for (int j = 0; j < kTpvItems; ++j)
            if (won[j]) {
              if (k < kClCap) {
                sm.buf[p ^ 1][k] = make_int4(v[j], d0[j], d1[j], 0);
              } else {
                const long long gk = (long long)g0 + (k - kfirst);
                if (GR_IN(gk, a.n + 1, 193)) Qn[gk] = v[j];
              }
              ++k;
            }
        }
      }
    }
    q_last = q;
    mf_last = mf;
    // publish this CTA's counts in every CTA, then meet: the fences of the
    // publishing threads (after the block barrier) order the CTA's appends
    __syncthreads();
    if (threadIdx.x < ncta) {
      cl_st_s32(cl_map(&sm.rc[p ^ 1][rank], threadIdx.x), sm.cnt[p ^ 1]);
      cl_st_u64(cl_map(&sm.re[p ^ 1][rank], threadIdx.x), sm.edges[p ^ 1]);
      cl_fence();
    }
    cl_sync_relaxed();
  }
}

// ------------------------------------------------- persistent (push only)
// One cooperative grid runs every level. Per level each warp takes frontier
// vertices in turn and expands their neighbour lists lane-parallel; winners
// of the visited-bitmap claim are appended with one atomic per warp. Levels
// are separated by a sense-reversing grid barrier whose spin is bounded.
constexpr int kPersThreads = 256;
// depth[src] after an allocation-free BFS that stopped at a device-side
// limit (GR_NOALLOC_INCOMPLETE in gr.h)
constexpr int32_t kNoAllocIncomplete = -2;

__device__ __forceinline__ bool grid_barrier(BfsCtl *c, int32_t nblocks, int32_t &gen) {
  (void)nblocks;
  return grid_sync(&c->bar, &c->error, gen);
}

// level end of the persistent kernel (push only, no degree scan)
__device__ void persistent_level_end(BfsCtl *c) {
  const int32_t qn = (int32_t)(c->next_packed & 0xFFFFFFFFull);
  c->level += 1;
  c->parity ^= 1;
  c->q_prev = c->q_len;
  c->q_len = qn;
  c->next_packed = 0ull;
  if (qn == 0) {
    c->done = 1;
  } else if (c->level >= c->max_levels) {
    c->error = kDevOverflow;
    c->done = 1;
  }
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
        // the CSR is not validated by the allocation-free entry point: a
        // column outside [0, n) is skipped rather than followed
        if (e < r1 && (uint32_t)(v = a.C[e]) < (uint32_t)a.n) {
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
          if (lane == 0)
            pos = (int32_t)(atomicAdd(&c->next_packed, (unsigned long long)__popc(bal)) &
                            0xFFFFFFFFull);
          pos = __shfl_sync(0xffffffffu, pos, 0);
          const int32_t k = pos + __popc(bal & ((1u << lane) - 1u));
          if (won && GR_IN(k, a.n + 1, 150)) Qn[k] = v;
        }
      }
    }
    if (!grid_barrier(c, nblocks, gen)) break;
    if (blockIdx.x == 0 && threadIdx.x == 0) persistent_level_end(c);
    if (!grid_barrier(c, nblocks, gen)) break;
  }
  // a traversal cut short by a device-side limit (a barrier wait that ran
  // out, the level cap) marks its source, whose depth is otherwise 0
  if (blockIdx.x == 0 && threadIdx.x == 0 && *(volatile int32_t *)&c->error != kDevOk)
    depth[c->src] = kNoAllocIncomplete;
}

}  // namespace

// ---------------------------------------------------------------- host
size_t bfs_ws_bytes(const gr_graph *g) {
  const size_t n = (size_t)g->n;
  const size_t seg = (size_t)g->nwords * 32 +
                     (size_t)g->num_sms * kDoBlocksPerSm * kLvWarps * kPullWords * 32;
  return 2 * sizeof(int32_t) * (n + 1) + 2 * sizeof(int32_t) * (n + 2) +
         4 * sizeof(uint32_t) * (size_t)g->nwords + 2 * sizeof(int32_t) * seg +
         sizeof(BfsCtl);
}

gr_status bfs_ws_create(gr_graph *g, cudaStream_t s, BfsWorkspace **out) {
  std::unique_ptr<BfsWorkspace> ws(new BfsWorkspace());
  const size_t n = (size_t)g->n;
  for (int i = 0; i < 2; ++i) {
    GR_TRY(ws->q[i].alloc(sizeof(int32_t) * (n + 1), "BFS queue"));
    GR_TRY(ws->S[i].alloc(sizeof(int32_t) * (n + 2), "BFS degree scan"));
  }
  GR_TRY(ws->visited.alloc(sizeof(uint32_t) * g->nwords, "visited bitmap"));
  for (int i = 0; i < 3; ++i)
    GR_TRY(ws->fb[i].alloc(sizeof(uint32_t) * g->nwords, "frontier bitmap"));
  {
    // segment capacity for any persistent grid of num_sms .. num_sms *
    // kDoBlocksPerSm blocks (see bfs_run)
    const size_t max_blocks = (size_t)g->num_sms * kDoBlocksPerSm;
    const size_t entries = (size_t)g->nwords * 32 + max_blocks * kLvWarps * kPullWords * 32;
    GR_TRY(ws->seg_v.alloc(sizeof(int32_t) * entries, "pull segments"));
    GR_TRY(ws->seg_d.alloc(sizeof(int32_t) * entries, "pull segment degrees"));
    GR_TRY(ws->seg_cnt.alloc(sizeof(unsigned long long) * max_blocks, "pull segment counts"));
  }
  GR_TRY(ws->ctl.alloc(sizeof(BfsCtl), "BFS control"));
  GR_TRY(ws->h_ctl.alloc(sizeof(BfsCtl), "BFS control mirror"));
  GR_CUDA(cudaMemsetAsync(ws->ctl.p, 0, sizeof(BfsCtl), s));
  GR_CUDA(cudaStreamSynchronize(s));
  *out = ws.release();
  return GR_OK;
}

static BfsArgs make_args(gr_graph *g, BfsWorkspace *ws, int32_t do_bitmap) {
  BfsArgs a;
  a.R = g->row_off.as<int32_t>();
  a.C = g->col.as<int32_t>();
  a.n = g->n;
  a.nwords = g->nwords;
  a.m = g->m;
  a.iso = g->isolated_bits.as<uint32_t>();
  a.first = g->first_col.as<int32_t>();
  for (int i = 0; i < 2; ++i) {
    a.q[i] = ws->q[i].as<int32_t>();
    a.S[i] = ws->S[i].as<int32_t>();
  }
  a.visited = ws->visited.as<uint32_t>();
  for (int i = 0; i < 3; ++i) a.fb[i] = ws->fb[i].as<uint32_t>();
  a.ctl = ws->ctl.as<BfsCtl>();
  a.do_bitmap = do_bitmap;
  a.low_degree = (!do_bitmap && g->max_degree <= kLowDegreeMax) ? 1 : 0;
  a.seg_v = nullptr;
  a.seg_d = nullptr;
  a.seg_cnt = nullptr;
  a.seg_cap = 0;
  return a;
}

static int level_grid(const gr_graph *g) { return g->num_sms * kLvBlocksPerSm; }

static gr_status enqueue_level(gr_graph *g, const BfsArgs &a, cudaStream_t s,
                               cudaGraphConditionalHandle h, int use_cond) {
  k_bfs_level<<<level_grid(g), kLvThreads, 0, s>>>(a, h, use_cond);
  GR_CUDA(cudaGetLastError());
  return GR_OK;
}

static gr_status build_level_graph(gr_graph *g, BfsWorkspace *ws, int32_t do_bitmap) {
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
  gr_status st = enqueue_level(g, make_args(g, ws, do_bitmap), cs, h, 1);
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

// The one-cluster driver with the largest cluster the device co-schedules
// (16 CTAs, else 8); when none fits nothing is launched and k_bfs_do runs
// the whole traversal.
static gr_status launch_cluster_bfs(const BfsArgs &a, cudaStream_t s) {
  GR_CUDA(cudaFuncSetAttribute(k_bfs_cluster, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
  for (int ctas : {kClMaxCtas, 8}) {
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = (unsigned)ctas;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)ctas);
    cfg.blockDim = dim3(kClThreads);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    int clusters = 0;
    if (cudaOccupancyMaxActiveClusters(&clusters, k_bfs_cluster, &cfg) != cudaSuccess) {
      (void)cudaGetLastError();
      continue;
    }
    if (clusters < 1) continue;
    GR_CUDA(cudaLaunchKernelEx(&cfg, k_bfs_cluster, a));
    return GR_OK;
  }
  return GR_OK;
}

static int32_t resolve_policy(const gr_graph *g, const gr_opts &o) {
  if (o.direction == GR_DIR_PUSH) return GR_DIR_PUSH;
  if (o.direction == GR_DIR_PULL) return GR_DIR_PULL;
  if (!g->symmetric) return GR_DIR_PUSH;
  return g->tuned_direction == GR_DIR_PUSH ? GR_DIR_PUSH : GR_DIR_AUTO;
}

// mode AUTO: the tuned mode of the graph (see gr_autotune), else the
// persistent kernel (one launch, one grid barrier per level)
static int32_t resolve_mode(const gr_graph *g, const gr_opts &o, int32_t policy) {
  (void)policy;
  if (o.mode != GR_MODE_AUTO) return o.mode;
  if (g->tuned_mode != GR_MODE_AUTO) return g->tuned_mode;
  return GR_MODE_PERSISTENT;
}

gr_status bfs_check(const gr_graph *g, int32_t src, const gr_opts &o) {
  if (src < 0 || src >= g->n) return fail(GR_EINVAL, "source out of range");
  if (o.direction < GR_DIR_AUTO || o.direction > GR_DIR_PULL)
    return fail(GR_EINVAL, "unknown direction policy");
  if (o.mode < GR_MODE_AUTO || o.mode > GR_MODE_PERSISTENT)
    return fail(GR_EINVAL, "unknown mode");
  if (o.direction == GR_DIR_PULL && !g->symmetric)
    return fail(GR_EINVAL, "pull traversal needs a symmetric CSR (in-neighbours = out-neighbours)");
  if (o.alpha < 0.f || o.beta < 0.f) return fail(GR_EINVAL, "alpha/beta must be >= 0");
  return GR_OK;
}

// BFS into device outputs with an explicit workspace (no locking, no
// staging): the public gr_bfs and the query server both call this.
gr_status bfs_run(gr_graph *g, BfsWorkspace *ws, int32_t src, int32_t *depth, int32_t *parent,
                  const gr_opts &o, cudaStream_t s) {
  const int32_t policy = resolve_policy(g, o);
  const int32_t mode = resolve_mode(g, o, policy);
  const int32_t do_bitmap = policy != GR_DIR_PUSH;
  const float alpha = o.alpha > 0.f ? o.alpha : g->tuned_alpha;
  const float beta = o.beta > 0.f ? o.beta : g->tuned_beta;
  int32_t max_levels = g->n + 1;
  if (o.max_iters > 0) max_levels = std::min(max_levels, o.max_iters);
  BfsArgs a = make_args(g, ws, do_bitmap);
  k_bfs_init<<<g->num_sms * 8, 256, 0, s>>>(a, src, depth, parent, policy, alpha, beta,
                                            max_levels, (g->symmetric && do_bitmap) ? 1 : 0);
  GR_CUDA(cudaGetLastError());
  if (mode == GR_MODE_GRAPH) {
    GR_TRY(build_level_graph(g, ws, do_bitmap));
    GR_CUDA(cudaGraphLaunch(ws->exec[do_bitmap], s));
  } else if (mode == GR_MODE_PERSISTENT) {
    int per_sm = 0;
    GR_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_bfs_do, kLvThreads, 0));
    int bps = std::min(per_sm, kDoBlocksPerSm);
    const int32_t want = o.block > 0 ? o.block : g->tuned_blocks_per_sm;
    if (want > 0) bps = std::min(bps, want);
    const int blocks = std::max(1, bps) * g->num_sms;
    // per-block segments for the pull levels: a block handles at most
    // `rounds` groups of kPullWords words per warp
    const long long groups = (g->nwords + kPullWords - 1) / kPullWords;
    const long long per_round = (long long)blocks * kLvWarps;
    const long long rounds = (groups + per_round - 1) / per_round;
    a.seg_cap = (int32_t)(rounds * kLvWarps * kPullWords * 32);
    if ((size_t)blocks * a.seg_cap > ws->seg_v.bytes / sizeof(int32_t))
      return fail(GR_ECUDA, "pull segment buffer too small");
    a.seg_v = ws->seg_v.as<int32_t>();
    a.seg_d = ws->seg_d.as<int32_t>();
    a.seg_cnt = ws->seg_cnt.as<unsigned long long>();
    // low-degree graphs: the small-frontier levels in one cluster first
    if (a.low_degree) GR_TRY(launch_cluster_bfs(a, s));
    void *args[] = {&a};
    GR_CUDA(cudaLaunchCooperativeKernel((void *)k_bfs_do, blocks, kLvThreads, args, 0, s));
  } else {
    // host-driven: enqueue batches of levels, then check the done flag
    BfsCtl *h = ws->h_ctl.as<BfsCtl>();
    int32_t levels_enqueued = 0;
    int32_t batch = 4;
    for (;;) {
      for (int i = 0; i < batch; ++i) GR_TRY(enqueue_level(g, a, s, 0, 0));
      levels_enqueued += batch;
      GR_CUDA(cudaMemcpyAsync(h, ws->ctl.p, sizeof(BfsCtl), cudaMemcpyDeviceToHost, s));
      GR_CUDA(cudaStreamSynchronize(s));
      if (h->done || levels_enqueued > max_levels) break;
      batch = std::min(batch * 2, 64);
    }
  }
  return GR_OK;
}

gr_status bfs_read_ctl_error(BfsWorkspace *ws, cudaStream_t s) {
  BfsCtl h;
  // pageable destination: the copy has finished when the call returns
  GR_CUDA(cudaMemcpyAsync(&h, ws->ctl.p, sizeof(BfsCtl), cudaMemcpyDeviceToHost, s));
  if (h.error == kDevTimeout) return fail(GR_ETIMEOUT, "a device-side wait timed out");
  if (h.error == kDevOverflow) return fail(GR_ETIMEOUT, "level limit reached");
  return GR_OK;
}

}  // namespace gr

using namespace gr;

extern "C" {

gr_status gr_bfs(gr_graph *g, int32_t src, int32_t *depth, int32_t *parent,
                 const gr_opts *opts, void *stream) {
  clear_error();
  if (!g) return fail(GR_EINVAL, "graph must not be NULL");
  if (!depth) return fail(GR_EINVAL, "depth must not be NULL");
  GR_TRY(bfs_check(g, src, opts ? *opts : default_opts()));
  std::lock_guard<std::mutex> lock(g->mu);
  cudaStream_t s = (cudaStream_t)stream;
  GR_TRY(begin_call(g, s));
  if (!g->bfs) GR_TRY(bfs_ws_create(g, s, &g->bfs));
  void *d_depth, *d_parent;
  bool cp_depth, cp_parent;
  GR_TRY(resolve_output(g, 0, depth, sizeof(int32_t) * (size_t)g->n, &d_depth, &cp_depth));
  GR_TRY(resolve_output(g, 1, parent, sizeof(int32_t) * (size_t)g->n, &d_parent, &cp_parent));
  GR_TRY(bfs_run(g, g->bfs, src, (int32_t *)d_depth, (int32_t *)d_parent,
                 opts ? *opts : default_opts(), s));
  if (cp_depth)
    GR_CUDA(cudaMemcpyAsync(depth, d_depth, sizeof(int32_t) * (size_t)g->n,
                            cudaMemcpyDeviceToHost, s));
  if (cp_parent)
    GR_CUDA(cudaMemcpyAsync(parent, d_parent, sizeof(int32_t) * (size_t)g->n,
                            cudaMemcpyDeviceToHost, s));
  GR_TRY(end_call(g, s));
  return GR_OK;
}

gr_status gr_bfs_multi(gr_graph *g, int32_t k, const int32_t *srcs, int32_t *const *depth,
                       int32_t *const *parent, const gr_opts *opts, void *stream) {
  clear_error();
  if (!g) return fail(GR_EINVAL, "graph must not be NULL");
  if (k < 0) return fail(GR_EINVAL, "k must be >= 0");
  if (k == 0) return GR_OK;
  if (!srcs || !depth) return fail(GR_EINVAL, "srcs and depth must not be NULL");
  const gr_opts &o = opts ? *opts : default_opts();
  // every argument is checked before any work is enqueued
  std::vector<uint8_t> host_d(k), host_p(k);
  for (int32_t i = 0; i < k; ++i) {
    if (!depth[i]) return fail(GR_EINVAL, "depth[i] must not be NULL");
    GR_TRY(bfs_check(g, srcs[i], o));
    bool hd = false, hp = false;
    GR_TRY(output_on_host(g, depth[i], &hd));
    if (parent) GR_TRY(output_on_host(g, parent[i], &hp));
    host_d[i] = hd;
    host_p[i] = hp;
  }
  std::lock_guard<std::mutex> lock(g->mu);
  cudaStream_t s = (cudaStream_t)stream;
  GR_TRY(begin_call(g, s));
  if (!g->bfs) GR_TRY(bfs_ws_create(g, s, &g->bfs));
  if (!g->copy_stream) GR_CUDA(cudaStreamCreateWithFlags(&g->copy_stream, cudaStreamNonBlocking));
  for (int b = 0; b < 2; ++b) {
    if (!g->pipe_filled[b])
      GR_CUDA(cudaEventCreateWithFlags(&g->pipe_filled[b], cudaEventDisableTiming));
    if (!g->pipe_free[b])
      GR_CUDA(cudaEventCreateWithFlags(&g->pipe_free[b], cudaEventDisableTiming));
  }
  const size_t bytes = sizeof(int32_t) * (size_t)g->n;
  bool used[2] = {false, false};
  int last = -1;
  auto run = [&]() -> gr_status {
    int b = 0;
    for (int32_t i = 0; i < k; ++i) {
      int32_t *par = parent ? parent[i] : nullptr;
      if (!host_d[i] && !host_p[i]) {
        GR_TRY(bfs_run(g, g->bfs, srcs[i], depth[i], par, o, s));
        continue;
      }
      // staging set b is free once the copies of the search before last are done
      if (used[b]) GR_CUDA(cudaStreamWaitEvent(s, g->pipe_free[b], 0));
      DevMem &sd = g->pipe_stage[b][0], &sp = g->pipe_stage[b][1];
      if (host_d[i] && sd.bytes < bytes) GR_TRY(sd.alloc(bytes, "BFS output staging"));
      if (host_p[i] && sp.bytes < bytes) GR_TRY(sp.alloc(bytes, "BFS output staging"));
      int32_t *dd = host_d[i] ? sd.as<int32_t>() : depth[i];
      int32_t *dp = host_p[i] ? sp.as<int32_t>() : par;
      GR_TRY(bfs_run(g, g->bfs, srcs[i], dd, dp, o, s));
      GR_CUDA(cudaEventRecord(g->pipe_filled[b], s));
      GR_CUDA(cudaStreamWaitEvent(g->copy_stream, g->pipe_filled[b], 0));
      if (host_d[i])
        GR_CUDA(cudaMemcpyAsync(depth[i], dd, bytes, cudaMemcpyDeviceToHost, g->copy_stream));
      if (host_p[i])
        GR_CUDA(cudaMemcpyAsync(par, dp, bytes, cudaMemcpyDeviceToHost, g->copy_stream));
      GR_CUDA(cudaEventRecord(g->pipe_free[b], g->copy_stream));
      used[b] = true;
      last = b;
      b ^= 1;
    }
    return GR_OK;
  };
  const gr_status st = run();
  // the call's work on `stream` ends after its last copy (copies complete in
  // order on the copy stream), also when an error stopped the loop early
  if (last >= 0) {
    const cudaError_t e = cudaStreamWaitEvent(s, g->pipe_free[last], 0);
    if (st == GR_OK && e != cudaSuccess) return cuda_fail(e, "gr_bfs_multi");
  }
  if (st != GR_OK) return st;
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


gr_status gr_bfs_trace(gr_graph *g, int32_t cap, int32_t *dir, int32_t *frontier,
                       int64_t *edges, double *end_us, int32_t *levels) {
  clear_error();
  if (!g) return fail(GR_EINVAL, "graph must not be NULL");
  if (!g->bfs) return fail(GR_EINVAL, "no BFS has run on this graph");
  if (cap < 0) return fail(GR_EINVAL, "cap must be >= 0");
  std::lock_guard<std::mutex> lock(g->mu);
  GR_CUDA(cudaSetDevice(g->device));
  if (g->has_last) GR_CUDA(cudaEventSynchronize(g->last_done));
  BfsCtl h;
  GR_CUDA(cudaMemcpy(&h, g->bfs->ctl.p, sizeof(BfsCtl), cudaMemcpyDeviceToHost));
  const int32_t nl = std::min<int32_t>(h.level, kTraceLevels);
  for (int32_t i = 0; i < std::min(cap, nl); ++i) {
    if (dir) dir[i] = h.tr_dir[i];
    if (frontier) frontier[i] = h.tr_q[i];
    if (edges) edges[i] = h.tr_mf[i];
    if (end_us) end_us[i] = (double)(h.tr_t[i] - h.t_start) * 1e-3;
  }
  if (levels) *levels = nl;
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
constexpr size_t kNoAllocCtlBytes = 8192;  // BfsCtl, padded to 8 KB
constexpr size_t kNoAllocQueueBytes = sizeof(int32_t) * ((size_t)kNoAllocMaxVertices + 1);
constexpr size_t kNoAllocQueueBytesAligned = (kNoAllocQueueBytes + 255) & ~size_t(255);
constexpr size_t kNoAllocVisitedBytes = sizeof(uint32_t) * (kNoAllocMaxVertices / 32);
constexpr size_t kNoAllocScratchBytes =
    kNoAllocCtlBytes + 2 * kNoAllocQueueBytesAligned + kNoAllocVisitedBytes;
static_assert(sizeof(BfsCtl) <= kNoAllocCtlBytes, "control block does not fit its slot");

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

// device address of g_noalloc_scratch, looked up once per device context:
// a process that resets a device (cudaDeviceReset) gets a new context in
// which the array may sit elsewhere, so the cached address is keyed by the
// driver's unique id of the context it was looked up in
constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
void *g_noalloc_addr[kMaxDevices] = {};
unsigned long long g_noalloc_ctx[kMaxDevices] = {};
int g_noalloc_sms[kMaxDevices] = {};
int g_noalloc_blocks_per_sm[kMaxDevices] = {};

// Id of the calling thread's current context (0 if the driver cannot tell;
// the cached address is then kept for the life of the process).
unsigned long long current_context_id() {
  using get_current_t = int (*)(void **);
  using get_id_t = int (*)(void *, unsigned long long *);
  static get_current_t get_current = nullptr;
  static get_id_t get_id = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void *f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) ==
            cudaSuccess && q == cudaDriverEntryPointSuccess)
      get_current = (get_current_t)f;
    f = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) ==
            cudaSuccess && q == cudaDriverEntryPointSuccess)
      get_id = (get_id_t)f;
    cudaGetLastError();
  });
  void *ctx = nullptr;
  unsigned long long id = 0;
  if (!get_current || !get_id || get_current(&ctx) != 0 || !ctx || get_id(ctx, &id) != 0) return 0;
  return id;
}

gr_status noalloc_setup(int dev, void **addr, int *sms, int *per_sm) {
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  // makes the device's primary context current (no allocation)
  GR_CUDA(cudaSetDevice(dev));
  const unsigned long long ctx = current_context_id();
  if (!g_noalloc_addr[dev] || g_noalloc_ctx[dev] != ctx) {
    void *p = nullptr;
    GR_CUDA(cudaGetSymbolAddress(&p, g_noalloc_scratch));
    int nsm = 0, occ = 0;
    GR_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    GR_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_bfs_persistent,
                                                          kPersThreads, 0));
    g_noalloc_sms[dev] = nsm;
    g_noalloc_blocks_per_sm[dev] = std::max(1, std::min(occ, 4));
    g_noalloc_addr[dev] = p;
    g_noalloc_ctx[dev] = ctx;
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
