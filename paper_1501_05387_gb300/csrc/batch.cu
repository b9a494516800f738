// Multi-source traversals with 64 bitmask lanes: batched BFS and Brandes
// betweenness centrality (Sec. 5.3).
//
// Up to 64 sources advance together, one bit lane each (the multi-source BFS
// idea of Then et al., VLDB 2014). Per vertex v a 64-bit mask lm[L][v] holds
// the lanes whose frontier at level L contains v; visit[v] the lanes that
// reached v at an earlier level. One level is a pull over all vertices
// (the all-vertex frontier of the load-balanced advance, merge-path chunks,
// lanes over edges): for an edge (v, u), bits = lm[L][u] & ~visited(v) are
// the lanes in which u is a predecessor of v, and v joins lm[L+1] in those
// lanes. Every column index is read once per level; the 64 traversals share
// that read.
//
// BC (Brandes, as the paper's Sec. 5.3 describes: a forward BFS pass
// counting shortest paths sigma, then a backward pass over the BFS levels
// accumulating dependencies) keeps per vertex 64 FP64 lanes, vertex-major
// (512 bytes per vertex), so the warp that serves an edge reads the 64
// lanes of one vertex in two coalesced 256-byte loads:
//   forward   sigma[v][s] = sum of sigma[u][s] over predecessors u in lane s
//   backward  with q[w][s] = 1/sigma[w][s] + sum over children x of q[x][s]
//             (i.e. (1 + delta[w][s]) / sigma[w][s]),
//             delta[v][s] = sigma[v][s] * sum over children w of q[w][s],
//             bc[v] += delta[v][s] for every lane s that reached v at level
//             >= 1 (v is then not lane s's source).
// This is the dependency recursion delta[v] += sigma[v]/sigma[w]*(1+delta[w])
// regrouped so that each edge needs one gathered value per lane.
//
// Path counts are integers, and FP64 arithmetic is scarce on this GPU (a few
// FP64 operations per clock per SM), so the forward pass counts them exactly
// in uint64 with integer adds (exact where FP64 rounds, beyond 2^53). A batch
// whose counts pass 2^64 - 1 (an add carries out) is counted again in FP64,
// which holds counts up to about 1.8e308.
//
// The forward level loop runs in one cooperative persistent kernel
// (k_mb_do), levels separated by the bounded grid barrier, the direction of
// every level decided on the device. Each level also emits the list of the
// vertices that joined the next level (with its degree scan), so a push
// level expands exactly its frontier and nothing scans all n vertices to
// find it. A batched BFS needs no host round trip at all; BC, which keeps
// one mask array per level, stops the kernel when the next level needs an
// array not yet allocated, and the host allocates more and resumes it.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <type_traits>
#include <vector>

#include "advance.cuh"

namespace gr {

constexpr int kMbThreads = 256, kMbItems = 4;
// Batched BFS keeps the lane masks of its first kKeepLevels levels, each in
// its own array, and writes their depths in one pass at the end (full
// coalesced rows); deeper levels rotate through three arrays and write their
// depths as they are reached. On graphs of small maximum degree (meshes:
// thousands of levels, small frontiers) no level is kept.
constexpr int32_t kKeepLevels = 16;
// A batched BFS level pushes when its frontier has fewer than m / kPushDiv
// edges, and pulls over every vertex otherwise.
constexpr long long kPushDiv = 16;
// Graphs of at most this maximum degree (meshes) keep no level's masks.
constexpr int32_t kLowDegreeMaxBatch = 16;
constexpr int kMbChunk = kMbThreads * kMbItems;
// What the forward pass counts: nothing (batched BFS), path counts in uint64,
// or path counts in FP64 (a batch whose uint64 counts overflowed).
enum : int { kSigNone = 0, kSigU64 = 1, kSigF64 = 2 };


struct BatchWorkspace {
  DevMem visit, sigma, q, counter, lmp, ctl;
  DevMem cb_pull, cb_fwd;  // chunk bounds of the all-vertex pulls (fixed per graph)
  DevMem fq, fs;    // BC backward: one level's vertex list and degree scan
  DevMem fcb;       // BC backward: that list's merge-path chunk bounds
  DevMem lq[3], ls[3];  // forward: level lists (ring by level) and degree scans
  std::vector<DevMem *> lm;  // level mask arrays ("slots")
  int32_t uploaded = 0;      // slots whose pointers are in lmp
  ~BatchWorkspace() {
    for (DevMem *p : lm) delete p;
  }
};

void free_batch(BatchWorkspace *ws) { delete ws; }

GR_GUARD_REPORTER(guard_report_batch)

namespace {

// Forward state in device memory: where the level loop stands (so a
// stopped kernel can resume), the level lists' counters and the barrier.
struct MbCtl {
  GridBarrier bar;
  unsigned long long cnt3[3];  // level L+1's vertices: [31:0] count, [63:32] edges
  unsigned long long cnt_list;  // compaction of a pulled level's list
  int32_t level;   // next level to run
  int32_t push;    // its direction
  int32_t q, qe;   // its list's size and edge count
  int32_t q_prev;  // size of the list before it
  int32_t listed;       // the list of `level` exists (a push emitted it)
  int32_t prev_listed;  // the list of `level` - 1 exists
  int32_t done;
  int32_t paused;  // stopped before `level`: it needs a slot beyond cap
  int32_t error;   // kDevTimeout / kDevOverflow
  int32_t levels;  // levels holding vertices (when done)
  int32_t sig_overflow;  // a uint64 path count overflowed
};

struct MbArgs {
  const int32_t *R;
  const int32_t *C;
  int32_t n;
  long long m;
  unsigned long long all;  // mask of the lanes in use
  unsigned long long *visit;
  unsigned long long *const *lmp;  // level mask arrays
  int32_t cap;        // arrays in lmp
  int32_t keep;       // levels < keep have their own array; later ones rotate through 3
  int32_t *lq[3];     // level lists, ring by level: lq[L % 3] lists level L
  int32_t *ls[3];     // their exclusive degree scans
  void *sigma;        // [n][64] uint64 or FP64 path counts, or null (BFS)
  int32_t *depth;     // [k][n] or null (BC)
  int32_t k;
  int32_t symmetric;
  int32_t max_levels;
  MbCtl *ctl;
  // chunk bounds of the all-vertex merge paths of the pull levels (chunks of
  // kMbPullChunk items for the batched BFS, kMbChunk for BC)
  const int32_t *cb_pull;
  const int32_t *cb_fwd;
};

__device__ __forceinline__ int32_t mb_slot(const MbArgs &a, int32_t L) {
  return L < a.keep ? L : a.keep + (L - a.keep) % 3;
}

__device__ __forceinline__ unsigned long long shfl_u64(unsigned long long x, int src) {
  return __shfl_sync(0xffffffffu, x, src);
}

// Path-count arithmetic in the forward pass's type: uint64 adds record a
// carry out in `ovf`, FP64 adds cannot overflow short of infinity (caught
// when the counts are used).
template <int SK>
using CountT = typename std::conditional<SK == kSigU64, unsigned long long, double>::type;

__device__ __forceinline__ unsigned long long count_add(unsigned long long x,
                                                        unsigned long long y, bool &ovf) {
  const unsigned long long t = x + y;
  ovf |= t < x;
  return t;
}
__device__ __forceinline__ double count_add(double x, double y, bool &) { return x + y; }

__device__ __forceinline__ void count_atomic_add(unsigned long long *p, unsigned long long y,
                                                 bool &ovf) {
  const unsigned long long old = atomicAdd(p, y);
  ovf |= old + y < old;
}
__device__ __forceinline__ void count_atomic_add(double *p, double y, bool &) {
  atomicAdd(p, y);
}

// Zeroes what the forward reads first: visit, the arrays of levels 0 and 1,
// the path counts and dependencies (BC) and, when no level is kept, the
// depth output (-1: unreached; kept levels' depths are all written by the
// end-of-run pass).
__global__ void k_mb_init(MbArgs a, unsigned long long *sigma, double *q) {
  const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  unsigned long long *l0 = a.lmp[mb_slot(a, 0)], *l1 = a.lmp[mb_slot(a, 1)];
  for (int64_t v = tid; v < a.n; v += stride) {
    a.visit[v] = 0ull;
    l0[v] = 0ull;
    l1[v] = 0ull;
  }
  if (sigma) {
    for (int64_t i = tid; i < (int64_t)a.n * 64; i += stride) {
      sigma[i] = 0ull;  // 0 as uint64 and as FP64
      q[i] = 0.0;
    }
  }
  if (a.depth && a.keep == 0)
    for (int64_t i = tid; i < (int64_t)a.k * a.n; i += stride) a.depth[i] = -1;
}

// Level 0: the sources' lanes, their path counts (1) and the level list
// (each distinct source vertex once, with its degree scan). One block of 64
// threads, after k_mb_init.
struct MbSources {
  int32_t s[64];
};

__global__ void k_mb_sources(MbArgs a, MbSources srcs, int32_t sk) {
  __shared__ int32_t s_v[64], s_d[64];
  __shared__ int32_t s_cnt;
  const int s = threadIdx.x;
  if (s == 0) s_cnt = 0;
  __syncthreads();
  unsigned long long *l0 = a.lmp[mb_slot(a, 0)];
  if (s < a.k && GR_IN(srcs.s[s], a.n, 205)) {
    const int32_t v = srcs.s[s];
    if (atomicOr(l0 + v, 1ull << s) == 0ull) {
      const int32_t k = atomicAdd(&s_cnt, 1);
      s_v[k] = v;
      s_d[k] = a.R[v + 1] - a.R[v];
    }
    if (sk == kSigU64) ((unsigned long long *)a.sigma)[(int64_t)v * 64 + s] = 1ull;
    if (sk == kSigF64) ((double *)a.sigma)[(int64_t)v * 64 + s] = 1.0;
  }
  __syncthreads();
  if (s == 0) {
    const int32_t cnt = s_cnt;
    int32_t run = 0;
    for (int32_t i = 0; i < cnt; ++i) {
      a.lq[0][i] = s_v[i];
      a.ls[0][i] = run;
      run += s_d[i];
    }
    MbCtl *c = a.ctl;
    grid_barrier_reset(&c->bar);
    for (int i = 0; i < 3; ++i) c->cnt3[i] = 0ull;
    c->cnt_list = 0ull;
    c->listed = 1;
    c->prev_listed = 0;
    c->level = 0;
    c->push = 1;
    c->q = cnt;
    c->qe = run;
    c->q_prev = 0;
    c->done = cnt == 0;
    c->paused = 0;
    c->error = kDevOk;
    c->levels = cnt ? 0 : 1;
    c->sig_overflow = 0;
  }
}

// Block-local list of the vertices a push level adds to the next level,
// flushed per chunk with flush_scanned (one packed atomic per block and
// chunk); a chunk of kMbChunk items adds at most kMbChunk vertices.
constexpr int kMbPullItems = 8;
constexpr int kMbPullChunk = kMbThreads * kMbPullItems;
using MbEmitBuf = ScannedBuf<kMbChunk>;

__device__ __forceinline__ void mb_emit(MbEmitBuf &em, const MbArgs &a, int32_t v) {
  const int32_t k = atomicAdd(&em.cnt, 1);
  em.out[k] = v;
  em.deg[k] = a.R[v + 1] - a.R[v];
}

// Packed (vertices, edges) increment for a vertex that joined the next level.
__device__ __forceinline__ unsigned long long joined(const MbArgs &a, int32_t v) {
  return 1ull | ((unsigned long long)(uint32_t)(a.R[v + 1] - a.R[v]) << 32);
}

// Shared memory of the level forms (one at a time).
union MbSmem {
  struct {
    int32_t end[kMbPullChunk + 1];  // end marker of each vertex, chunk-local
    unsigned long long U[kMbPullChunk + 1];  // lanes the vertex still misses
  } pull;
  struct {
    int32_t off[kMbChunk + 1];
    unsigned long long U[kMbChunk + 1];
  } fwd;
  struct {
    int32_t off[kMbChunk + 1];
    int32_t row[kMbChunk + 1];
    unsigned long long cur[kMbChunk + 1];
    int32_t u[kMbChunk + 1];
    MbEmitBuf em;
  } push;
  MbEmitBuf list;  // compaction of a pulled level into its list
};

// Lanes of `c` at vertex v reach their depth at level L.
__device__ __forceinline__ void mb_write_depth(const MbArgs &a, int32_t v, unsigned long long c,
                                               int32_t L) {
  for (int s = 0; s < a.k; ++s)
    if (((c >> s) & 1ull) && GR_IN((int64_t)s * a.n + v, (int64_t)a.k * a.n, 204))
      a.depth[(int64_t)s * a.n + v] = L;
}

// A batched BFS pull level (no path counts): nxt[v] = OR over edges (v, u)
// of cur[u] & ~seen(v), seen(v) = visit[v] | cur[v], for every vertex v.
// Merge-based: a chunk's vertex end markers and edges form one sequence of
// kMbThreads * kMbPullItems items; each thread finds its first item's
// vertex with one search, then walks its kMbPullItems consecutive items.
// The column and lane-mask loads of all its items are issued before any is
// used, edges of vertices that already hold every lane are skipped, and the
// OR of a vertex accumulates in a register. A vertex whose edges and end
// marker all fall in one thread's items is written with a plain store (no
// other thread touches it); the others with atomicOr. The vertex loader
// folds cur into visit and, past the kept levels, writes depth L. The level
// counts the vertices whose mask goes from empty to non-empty (and their
// edges); it writes no list (a push level after it compacts one).
__device__ void mb_pull_level(const MbArgs &a, MbSmem &sm, int32_t *s_red8, int32_t L,
                              const unsigned long long *cur, unsigned long long *nxt,
                              unsigned long long *counter) {
  constexpr int ITEMS = kMbPullItems;
  constexpr int CHUNK = kMbPullChunk;
  const bool write_depth = a.depth && L >= a.keep;
  const long long total = (long long)a.n + a.R[a.n];
  const long long nchunks = (total + CHUNK - 1) / CHUNK;
  unsigned long long new_vertices = 0;
  for (long long chunk = blockIdx.x; chunk < nchunks; chunk += gridDim.x) {
    const long long d0 = chunk * CHUNK;
    const long long d1 = min(d0 + CHUNK, total);
    const int32_t i0 = a.cb_pull[chunk], i1 = a.cb_pull[chunk + 1];
    const long long j0 = d0 - i0;  // CSR position of the chunk's first edge
    const int32_t nv = (i0 <= a.n - 1) ? (min(i1, a.n - 1) - i0 + 1) : 0;
    const int32_t len = (int32_t)(d1 - d0);
    for (int32_t kk = threadIdx.x; kk < nv; kk += kMbThreads) {
      const int32_t v = i0 + kk;
      const unsigned long long c = cur[v];
      const unsigned long long seen = a.visit[v] | c;
      if (c) {
        a.visit[v] = seen;
        if (write_depth) mb_write_depth(a, v, c, L);
      }
      sm.pull.end[kk] = (int32_t)((long long)a.R[v + 1] + v - d0);
      sm.pull.U[kk] = a.all & ~seen;
    }
    __syncthreads();
    const int32_t k0 = min(len, (int32_t)threadIdx.x * ITEMS);
    const int32_t k1 = min(len, k0 + ITEMS);
    if (k0 < k1) {
      // chunk vertices whose end marker lies before k0
      int32_t lo = 0, hi = nv;
      while (lo < hi) {
        const int32_t mid = (lo + hi) >> 1;
        if (sm.pull.end[mid] < k0) lo = mid + 1;
        else hi = mid;
      }
      // classify the items: end markers (bit i of `ends`) and edges, loading
      // the column of each edge whose vertex still misses lanes
      uint32_t ends = 0u;
      int32_t u[ITEMS];
      int32_t r = lo, e = k0 - lo;  // e: chunk-local edge index
#pragma unroll
      for (int i = 0; i < ITEMS; ++i) {
        const int32_t k = k0 + i;
        u[i] = -1;
        if (k < k1 && r < nv) {
          if (sm.pull.end[r] == k) {
            ends |= 1u << i;
            ++r;
          } else {
            const long long pos = j0 + e;
            if (sm.pull.U[r] && GR_IN(pos, a.m, 202)) u[i] = (int32_t)pos;
            ++e;
          }
        }
      }
#pragma unroll
      for (int i = 0; i < ITEMS; ++i) u[i] = u[i] >= 0 ? a.C[u[i]] : -1;
      unsigned long long b[ITEMS];
#pragma unroll
      for (int i = 0; i < ITEMS; ++i) b[i] = (u[i] >= 0 && GR_IN(u[i], a.n, 203)) ? cur[u[i]] : 0ull;
      // walk: OR per vertex, written at its end marker
      r = lo;
      unsigned long long acc = 0ull;
      bool whole = false;  // the vertex's first edge lies in this thread's items
#pragma unroll
      for (int i = 0; i < ITEMS; ++i) {
        const int32_t k = k0 + i;
        if (k < k1 && r < nv) {
          if ((ends >> i) & 1u) {
            if (acc) {
              const int32_t v = i0 + r;
              if (whole) {
                nxt[v] = acc;
                new_vertices += joined(a, v);
              } else if (!atomicOr(nxt + v, acc)) {
                new_vertices += joined(a, v);
              }
            }
            acc = 0ull;
            whole = true;
            ++r;
          } else {
            acc |= b[i] & sm.pull.U[r];
          }
        }
      }
      if (acc && r < nv && !atomicOr(nxt + (i0 + r), acc))  // continues past k1
        new_vertices += joined(a, i0 + r);
    }
    __syncthreads();
  }
  for (int o = 16; o > 0; o >>= 1) new_vertices += __shfl_xor_sync(0xffffffffu, new_vertices, o);
  if ((threadIdx.x & 31) == 0 && new_vertices) atomicAdd(counter, new_vertices);
}

// A BC forward pull level: nxt[v] = OR over edges (v,u) of cur[u] &
// ~seen(v), seen(v) = visit[v] | cur[v], and the path counts of the newly
// reached lanes. The vertex loader of each chunk folds cur into visit
// (idempotent, so chunks sharing a vertex may both do it).
template <int SK>
__device__ void mb_forward_level(const MbArgs &a, MbSmem &sm, int32_t *s_red8,
                                 const unsigned long long *cur, unsigned long long *nxt,
                                 unsigned long long *counter, bool &ovf) {
  using T = CountT<SK>;
  const int lane = threadIdx.x & 31;
  const long long total = (long long)a.n + a.R[a.n];
  const long long nchunks = (total + kMbChunk - 1) / kMbChunk;
  unsigned long long new_vertices = 0;
  for (long long chunk = blockIdx.x; chunk < nchunks; chunk += gridDim.x) {
    const long long d0 = chunk * kMbChunk;
    const long long d1 = min(d0 + kMbChunk, total);
    const int32_t i0 = a.cb_fwd[chunk], i1 = a.cb_fwd[chunk + 1];
    const long long j0 = d0 - i0, j1 = d1 - i1;
    const int32_t nv = (i0 <= a.n - 1) ? (min(i1, a.n - 1) - i0 + 1) : 0;
    for (int32_t kk = threadIdx.x; kk < nv; kk += kMbThreads) {
      const int32_t v = i0 + kk;
      const unsigned long long c = cur[v];
      const unsigned long long seen = a.visit[v] | c;
      if (c) a.visit[v] = seen;
      sm.fwd.off[kk] = a.R[v];
      sm.fwd.U[kk] = a.all & ~seen;
    }
    __syncthreads();
    const int32_t ne = (int32_t)(j1 - j0);
    for (int32_t kb = 0; kb < ne; kb += kMbThreads) {
      const int32_t kk = kb + threadIdx.x;
      int32_t owner = -1, u = 0;
      unsigned long long bits = 0ull;
      if (kk < ne) {
        const int32_t e = (int32_t)(j0 + kk);
        int32_t lo = 0, hi = nv - 1;
        while (lo < hi) {
          const int32_t mid = (lo + hi + 1) >> 1;
          if (sm.fwd.off[mid] <= e) lo = mid;
          else hi = mid - 1;
        }
        owner = i0 + lo;
        if (!GR_IN(owner, a.n, 201)) owner = -1;
        const unsigned long long U = owner >= 0 ? sm.fwd.U[lo] : 0ull;
        if (U && GR_IN(e, a.m, 202)) {
          u = a.C[e];
          bits = GR_IN(u, a.n, 203) ? (cur[u] & U) : 0ull;
        }
      }
      // the warp serves the edges with bits one at a time: lane l handles
      // BFS lanes l and l + 32 of the predecessor's 64 path counts; a half
      // with no bits set is skipped by the whole warp
      T *const sigma = (T *)a.sigma;
      uint32_t act = __ballot_sync(0xffffffffu, bits != 0ull);
      int32_t cur_owner = -1;
      unsigned long long orbits = 0ull;
      T acc0 = T(0), acc1 = T(0);
      while (act) {
        const int j = __ffs(act) - 1;
        act &= act - 1u;
        const int32_t ov = __shfl_sync(0xffffffffu, owner, j);
        const int32_t uj = __shfl_sync(0xffffffffu, u, j);
        const unsigned long long bj = shfl_u64(bits, j);
        if (ov != cur_owner) {
          if (cur_owner >= 0) {
            T *sg = sigma + (int64_t)cur_owner * 64;
            if ((orbits >> lane) & 1ull) count_atomic_add(sg + lane, acc0, ovf);
            if ((orbits >> (lane + 32)) & 1ull) count_atomic_add(sg + lane + 32, acc1, ovf);
            if (lane == 0 && !atomicOr(nxt + cur_owner, orbits))
              new_vertices += joined(a, cur_owner);
          }
          cur_owner = ov;
          orbits = 0ull;
          acc0 = acc1 = T(0);
        }
        orbits |= bj;
        const T *su = sigma + (int64_t)uj * 64;
        if ((uint32_t)bj && ((bj >> lane) & 1ull)) acc0 = count_add(acc0, su[lane], ovf);
        if ((bj >> 32) && ((bj >> (lane + 32)) & 1ull))
          acc1 = count_add(acc1, su[lane + 32], ovf);
      }
      if (cur_owner >= 0) {
        T *sg = sigma + (int64_t)cur_owner * 64;
        if ((orbits >> lane) & 1ull) count_atomic_add(sg + lane, acc0, ovf);
        if ((orbits >> (lane + 32)) & 1ull) count_atomic_add(sg + lane + 32, acc1, ovf);
        if (lane == 0 && !atomicOr(nxt + cur_owner, orbits)) new_vertices += joined(a, cur_owner);
      }
    }
    __syncthreads();
  }
  for (int o = 16; o > 0; o >>= 1) new_vertices += __shfl_xor_sync(0xffffffffu, new_vertices, o);
  if (lane == 0 && new_vertices) atomicAdd(counter, new_vertices);
}

// A push level, for levels whose list has few edges (the sources' level,
// the last levels, every level of a mesh): the listed vertices send their
// lanes over their edges (merge-path chunks over the list's degree scan).
// For an edge (u, v): bits = cur[u] & ~seen(v), seen(v) = visit[v] | cur[v]
// (v may be on the list itself, its cur not yet folded into visit), and
// nxt[v] |= bits; with SIGMA (BC's forward pass) those lanes also add u's
// path counts to v's, the warp serving such edges one at a time. The
// loader folds each listed vertex's cur into visit and, past the kept
// levels, writes its depths.
template <int SK>
__device__ void mb_push_level(const MbArgs &a, MbSmem &sm, int32_t *s_red8, int32_t L,
                              const unsigned long long *cur,
                              unsigned long long *nxt, const int32_t *Q, const int32_t *S,
                              int32_t q, int32_t qe, int32_t *Qn, int32_t *Sn,
                              unsigned long long *counter, bool &ovf) {
  constexpr bool SIGMA = SK != kSigNone;
  using T = CountT<SK == kSigNone ? kSigU64 : SK>;
  const bool write_depth = a.depth && L >= a.keep;
  const int lane = threadIdx.x & 31;
  const long long total = (long long)q + qe;
  const long long nchunks = (total + kMbChunk - 1) / kMbChunk;
  // the emission buffer shares its storage with the other level forms: its
  // count starts at zero here
  if (threadIdx.x == 0) sm.push.em.cnt = 0;
  __syncthreads();
  for (long long chunk = blockIdx.x; chunk < nchunks; chunk += gridDim.x) {
    const long long d0 = chunk * kMbChunk;
    const long long d1 = min(d0 + kMbChunk, total);
    int32_t i0, i1;
    block_chunk_bounds<kMbThreads>(S, q, qe, d0, d1, kMbChunk, s_red8, &i0, &i1);
    const long long j0 = d0 - i0, j1 = d1 - i1;
    const int32_t nv = (i0 <= q - 1) ? (min(i1, q - 1) - i0 + 1) : 0;
    for (int32_t k = threadIdx.x; k < nv; k += kMbThreads) {
      const int32_t i = i0 + k;
      const int32_t u = GR_IN(i, a.n + 1, 207) ? Q[i] : 0;
      const bool ok = GR_IN(u, a.n, 208);
      const unsigned long long c = ok ? cur[u] : 0ull;
      if (c) {
        a.visit[u] |= c;
        if (write_depth) mb_write_depth(a, u, c, L);
      }
      sm.push.off[k] = S[i];
      sm.push.row[k] = ok ? a.R[u] : 0;
      sm.push.cur[k] = c;
      if (SIGMA) sm.push.u[k] = ok ? u : 0;
    }
    __syncthreads();
    const int32_t ne = (int32_t)(j1 - j0);
    for (int32_t kb = 0; kb < ne; kb += kMbThreads) {
      const int32_t k = kb + threadIdx.x;
      unsigned long long bits = 0ull;
      int32_t v = -1, u = 0;
      if (k < ne) {
        const int32_t er = (int32_t)(j0 + k);
        int32_t lo = 0, hi = nv - 1;
        while (lo < hi) {
          const int32_t mid = (lo + hi + 1) >> 1;
          if (sm.push.off[mid] <= er) lo = mid;
          else hi = mid - 1;
        }
        const long long e = (long long)sm.push.row[lo] + (er - sm.push.off[lo]);
        v = GR_IN(e, a.m, 209) ? a.C[e] : -1;
        if (v >= 0 && GR_IN(v, a.n, 210)) {
          bits = sm.push.cur[lo] & ~(a.visit[v] | cur[v]);
          if (bits && !atomicOr(nxt + v, bits)) mb_emit(sm.push.em, a, v);
          if (SIGMA) u = sm.push.u[lo];
        }
      }
      if (SIGMA) {
        T *const sigma = (T *)a.sigma;
        uint32_t act = __ballot_sync(0xffffffffu, bits != 0ull);
        while (act) {
          const int j = __ffs(act) - 1;
          act &= act - 1u;
          const int32_t vj = __shfl_sync(0xffffffffu, v, j);
          const int32_t uj = __shfl_sync(0xffffffffu, u, j);
          const unsigned long long bj = shfl_u64(bits, j);
          const T *su = sigma + (int64_t)uj * 64;
          T *sv = sigma + (int64_t)vj * 64;
          if ((bj >> lane) & 1ull) count_atomic_add(sv + lane, su[lane], ovf);
          if ((bj >> (lane + 32)) & 1ull) count_atomic_add(sv + lane + 32, su[lane + 32], ovf);
        }
      }
    }
    flush_scanned<kMbThreads>(sm.push.em, counter, Qn, Sn, (long long)a.n + 1);
  }
}

// The list of a level reached by a pull (the vertices with lanes in cur,
// with their degree scan), for the push level that expands it.
__device__ void mb_compact_list(const MbArgs &a, MbSmem &sm, const unsigned long long *cur,
                                int32_t *Q, int32_t *S, unsigned long long *counter) {
  constexpr int PER = kMbChunk / kMbThreads;
  // the list buffer shares its storage with the level forms: its count
  // starts at zero here
  if (threadIdx.x == 0) sm.list.cnt = 0;
  __syncthreads();
  for (int64_t base = (int64_t)blockIdx.x * kMbChunk; base < a.n;
       base += (int64_t)gridDim.x * kMbChunk) {  // block-uniform
#pragma unroll
    for (int j = 0; j < PER; ++j) {
      const int64_t v = base + j * kMbThreads + threadIdx.x;
      const bool take = v < a.n && cur[v] != 0ull;
      emit_scanned(sm.list, take, (int32_t)v, take ? a.R[v + 1] - a.R[v] : 0);
    }
    flush_scanned<kMbThreads>(sm.list, counter, Q, S, (long long)a.n + 1);
  }
}

// Depths of the kept levels [0, levels) from their lane masks, written once
// for every (lane, vertex), in full coalesced rows: for each lane s,
// depth[s][v] = the level L whose mask holds bit s (-1 if none). The masks
// of one vertex are disjoint, so the level of every lane follows from bit
// slices: slice j is the OR of the masks of the levels whose index has bit j
// set.
__device__ void mb_depth_pass(const MbArgs &a, int32_t levels) {
  constexpr int kSlices = 6;  // levels < 64
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t nr = ((int64_t)a.n + 31) & ~31ll;  // warp-uniform bound
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < nr; v += stride) {
    unsigned long long b[kSlices] = {0ull, 0ull, 0ull, 0ull, 0ull, 0ull}, reached = 0ull;
    if (v < a.n) {
      for (int32_t L = 0; L < levels; ++L) {
        const unsigned long long m = a.lmp[L][v];
        reached |= m;
#pragma unroll
        for (int j = 0; j < kSlices; ++j)
          if ((L >> j) & 1) b[j] |= m;
      }
    }
    for (int32_t s = 0; s < a.k; ++s) {
      int32_t d = -1;
      if ((reached >> s) & 1ull) {
        d = 0;
#pragma unroll
        for (int j = 0; j < kSlices; ++j) d |= (int32_t)((b[j] >> s) & 1ull) << j;
      }
      if (v < a.n) a.depth[(int64_t)s * a.n + v] = d;
    }
  }
}

// Blocks per SM of k_mb_do: the batched BFS at 5 (48 registers; 7.48 ms
// for 64 sources on R-MAT s23 against 8.25 ms at 6), BC at 6 (116 ms
// against 118 ms at 5).
template <int SK>
constexpr int mb_do_blocks_per_sm() { return SK == kSigNone ? 5 : 6; }

// The forward levels in one cooperative kernel. Every block runs every
// level; levels are separated by one bounded grid barrier, after which each
// block reads the level's packed counter (published with the release on
// large grids) and takes the same decisions: stop when no vertex joined,
// push when the next level's vertices have fewer than m / kPushDiv edges
// (or the graph is directed), else pull. A push level expands the list of
// its level (emitted by the push before it, or compacted from the masks
// after a pull, which writes no list). Lane-mask arrays: the one of level
// L + 2 is cleared while level L runs (all of it for a kept level, an
// array's first use in this run or when level L - 1, its last user, has no
// list; otherwise only the entries on that list). The kernel stops before a
// level whose arrays are not allocated (BC only) and records where;
// launched again, it resumes.
// Loop state of k_mb_do, the same in every block; kept in shared memory so
// that the level bodies have the registers to themselves.
struct MbLoop {
  int32_t L, push, q, qe, q_prev, listed, prev_listed;
};

template <int SK>
__global__ void __launch_bounds__(kMbThreads, mb_do_blocks_per_sm<SK>()) k_mb_do(MbArgs a) {
  MbCtl *c = a.ctl;
  __shared__ MbSmem sm;
  __shared__ int32_t s_red8[kMbThreads / 32];
  __shared__ MbLoop st;
  if (threadIdx.x == 0) {
    st.L = c->level;
    st.push = c->push;
    st.q = c->q;
    st.qe = c->qe;
    st.q_prev = c->q_prev;
    st.listed = c->listed;
    st.prev_listed = c->prev_listed;
  }
  __syncthreads();
  if (c->done) return;
  int32_t gen = 0;
  bool ovf = false;
  for (;;) {
    const int32_t L = st.L;
    if (mb_slot(a, L + 1) >= a.cap || (L + 2 < a.keep && L + 2 >= a.cap)) {
      if (blockIdx.x == 0 && threadIdx.x == 0) {
        c->level = L;
        c->push = st.push;
        c->q = st.q;
        c->qe = st.qe;
        c->q_prev = st.q_prev;
        c->listed = st.listed;
        c->prev_listed = st.prev_listed;
        c->paused = 1;
      }
      break;
    }
    if (a.depth && a.keep > 0 && L == a.keep) {
      // every kept level is complete: their depths first, then the later
      // levels' writes
      mb_depth_pass(a, a.keep);
      if (!grid_sync(&c->bar, &c->error, gen)) break;
    }
    const unsigned long long *cur = a.lmp[mb_slot(a, L)];
    unsigned long long *nxt = a.lmp[mb_slot(a, L + 1)];
    if (st.push && !st.listed) {
      mb_compact_list(a, sm, cur, a.lq[L % 3], a.ls[L % 3], &c->cnt_list);
      if (!grid_sync(&c->bar, &c->error, gen)) break;
      if (threadIdx.x == 0) st.listed = 1;
      if (blockIdx.x == 0 && threadIdx.x == 0) c->cnt_list = 0ull;  // next use: a barrier later
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) c->cnt3[(L + 2) % 3] = 0ull;
    {
      const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
      const int64_t stride = (int64_t)gridDim.x * blockDim.x;
      const int32_t s2 = mb_slot(a, L + 2);
      if (s2 < a.cap) {
        unsigned long long *clr = a.lmp[s2];
        if (L - 1 < a.keep || !st.prev_listed) {
          for (int64_t v = tid; v < a.n; v += stride) clr[v] = 0ull;
        } else {
          const int32_t *Qp = a.lq[(L + 2) % 3];  // level L - 1's list
          for (int64_t i = tid; i < st.q_prev; i += stride) {
            const int32_t v = Qp[i];
            if (GR_IN(v, a.n, 211)) clr[v] = 0ull;
          }
        }
      }
    }
    unsigned long long *counter = &c->cnt3[(L + 1) % 3];
    if (st.push) {
      mb_push_level<SK>(a, sm, s_red8, L, cur, nxt, a.lq[L % 3], a.ls[L % 3], st.q, st.qe,
                        a.lq[(L + 1) % 3], a.ls[(L + 1) % 3], counter, ovf);
    } else if (SK == kSigNone) {
      mb_pull_level(a, sm, s_red8, L, cur, nxt, counter);
    } else {
      mb_forward_level<SK == kSigNone ? kSigU64 : SK>(a, sm, s_red8, cur, nxt, counter, ovf);
    }
    unsigned long long pk = 0ull;
    if (gridDim.x > kFlatBarrierBlocks) {
      if (!grid_sync(&c->bar, &c->error, gen, counter, &pk)) break;
    } else {
      if (!grid_sync(&c->bar, &c->error, gen)) break;
      pk = *(volatile unsigned long long *)counter;
    }
    // grid_sync ends with a block barrier: every thread has read st
    const int32_t qn = (int32_t)(pk & 0xFFFFFFFFull);
    const long long en = (long long)(pk >> 32);
    const int32_t levels = L + 1;  // levels 0 .. L hold vertices
    const bool done = qn == 0;
    const bool overflow = !done && levels >= a.max_levels;
    if (done || overflow) {
      if (done && a.depth && a.keep > 0 && levels <= a.keep) mb_depth_pass(a, levels);
      if (blockIdx.x == 0 && threadIdx.x == 0) {
        c->level = levels;
        c->levels = levels;
        c->q = 0;
        if (overflow) c->error = kDevOverflow;
        c->done = 1;
      }
      break;
    }
    if (threadIdx.x == 0) {
      st.prev_listed = st.listed;
      st.listed = st.push;  // a push emitted the next level's list
      st.L = levels;
      st.q_prev = st.q;
      st.q = qn;
      st.qe = (int32_t)en;
      st.push = (!a.symmetric || en * kPushDiv < a.m) ? 1 : 0;
    }
    __syncthreads();
  }
  if (SK == kSigU64 && __any_sync(0xffffffffu, ovf) && (threadIdx.x & 31) == 0)
    atomicOr(&c->sig_overflow, 1);
}

struct BcBackArgs {
  const int32_t *R;
  const int32_t *C;
  int32_t n;
  long long m;
  const unsigned long long *lv;   // lm[L]
  const unsigned long long *lw;   // lm[L+1]
  double *q;                      // [n][64]
};

// Double-single numbers: an unevaluated sum hi + lo of two floats with
// |lo| <= ulp(hi) / 2, about 48 significant bits (Dekker's extended
// precision arithmetic; Knuth's TwoSum for exact sums, the product's error
// from one FMA). FP32 instructions issue many times faster than FP64 on this
// GPU, so BC's per-vertex finish (a reciprocal, a product and sums per lane)
// runs in this form (uint64 path counts keep every value within FP32's
// exponent range): on R-MAT s23 x 64 sources it took the finalize from
// 16.2 to 10.8 ms. The backward's per-edge sums stay in FP64: in this form
// its warp-serial loop became issue-bound (75.7 against 53.5 ms). The _rn
// intrinsics keep the compiler from contracting or reassociating the error
// terms.
struct DS {
  float hi, lo;
};

__device__ __forceinline__ DS ds_two_sum(float a, float b) {  // exact: hi + lo = a + b
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  const float err = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return {s, err};
}

__device__ __forceinline__ DS ds_fast_two_sum(float a, float b) {  // |a| >= |b|
  const float s = __fadd_rn(a, b);
  return {s, __fsub_rn(b, __fsub_rn(s, a))};
}

__device__ __forceinline__ DS ds_add(DS a, DS b) {
  DS s = ds_two_sum(a.hi, b.hi);
  const DS t = ds_two_sum(a.lo, b.lo);
  s = ds_fast_two_sum(s.hi, __fadd_rn(s.lo, t.hi));
  return ds_fast_two_sum(s.hi, __fadd_rn(s.lo, t.lo));
}

__device__ __forceinline__ DS ds_add_f(DS a, float b) {
  const DS s = ds_two_sum(a.hi, b);
  return ds_fast_two_sum(s.hi, __fadd_rn(s.lo, a.lo));
}

__device__ __forceinline__ DS ds_mul(DS a, DS b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);  // the product's rounding error, exactly
  e = __fmaf_rn(a.hi, b.lo, __fmaf_rn(a.lo, b.hi, e));
  return ds_fast_two_sum(p, e);
}

// 1 / a: the FP32 reciprocal refined by one Newton step in double-single,
// r + r (1 - a r), which squares its relative error (2^-24 -> about 2^-48).
__device__ __forceinline__ DS ds_rcp(DS a) {
  const float r = __frcp_rn(a.hi);
  const DS ar = ds_mul(a, DS{r, 0.f});
  const DS res = ds_add(DS{1.f, 0.f}, DS{-ar.hi, -ar.lo});
  return ds_add_f(ds_mul(DS{r, 0.f}, res), r);
}

// A 16-bit integer as a float without a conversion instruction: 2^23 + p
// is a float whose low mantissa bits are p.
__device__ __forceinline__ float u16_to_float(uint32_t p) {
  return __fsub_rn(__int_as_float(0x4B000000 | (int)p), 8388608.f);
}

// A uint64 path count as double-single (its four 16-bit pieces, each exact
// as a float, summed without losing more than the last of 64 bits' worth).
__device__ __forceinline__ DS ds_from_u64(unsigned long long c) {
  DS r{__fmul_rn(u16_to_float((uint32_t)(c >> 48)), 281474976710656.f), 0.f};  // 2^48
  r = ds_add_f(r, __fmul_rn(u16_to_float((uint32_t)(c >> 32) & 0xFFFFu), 4294967296.f));
  r = ds_add_f(r, __fmul_rn(u16_to_float((uint32_t)(c >> 16) & 0xFFFFu), 65536.f));
  return ds_add_f(r, u16_to_float((uint32_t)c & 0xFFFFu));
}

__device__ __forceinline__ DS ds_from_double(double x) {
  const float hi = __double2float_rn(x);
  return {hi, __double2float_rn(x - (double)hi)};
}

__device__ __forceinline__ double ds_to_double(DS a) { return (double)a.hi + (double)a.lo; }

__device__ __forceinline__ DS shfl_xor_ds(DS a, int o) {
  return {__shfl_xor_sync(0xffffffffu, a.hi, o), __shfl_xor_sync(0xffffffffu, a.lo, o)};
}

// Chunk bounds of a level list's merge path, the list's size and edge count
// read from *fpacked (its scan S[0..q) does not store S[q]): cb[c] = the
// members whose end marker S[i + 1] + i lies before c * kMbChunk,
// cb[nchunks] = q. One thread per chunk; threads past the list's chunks
// return.
__global__ void k_list_bounds(const int32_t *S, const unsigned long long *fpacked, int32_t *cb) {
  const unsigned long long fp = *fpacked;
  const int32_t q = (int32_t)(fp & 0xFFFFFFFFull);
  const int32_t qe = (int32_t)(fp >> 32);
  const long long nchunks = ((long long)q + qe + kMbChunk - 1) / kMbChunk;
  const long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (c > nchunks) return;
  if (c == nchunks) {
    cb[c] = q;
    return;
  }
  const long long d = c * kMbChunk;
  int32_t lo = 0, hi = q;  // first member whose end marker is not before d
  while (lo < hi) {
    const int32_t mid = (int32_t)(((long long)lo + hi) >> 1);
    const int32_t sv = mid + 1 == q ? qe : S[mid + 1];
    if ((long long)sv + mid < d) lo = mid + 1;
    else hi = mid;
  }
  cb[c] = lo;
}

// resident blocks per SM of the backward pass (its carveout is fitted to
// them, the rest of the shared-memory array left to L1 for the children's rows)
constexpr int kBcBackBlocksPerSm = 6;

// Backward level L: q[v][s] += q[w][s] over edges (v, w) with v in lane s's
// level L and w in its level L+1 (w's q is final: level L+1 was finished).
// Only the vertices of level L (listed with their degrees by k_mb_list) are
// visited, so the whole backward pass reads every edge about once instead of
// once per level.

__global__ void __launch_bounds__(kMbThreads) k_bc_backward(BcBackArgs a, const int32_t *Q,
                                                             const int32_t *S,
                                                             const unsigned long long *fpacked,
                                                             const int32_t *cb) {
  __shared__ int32_t s_off[kMbChunk + 1];
  __shared__ int32_t s_row[kMbChunk + 1];
  __shared__ int32_t s_v[kMbChunk + 1];
  __shared__ unsigned long long s_A[kMbChunk + 1];
  __shared__ int32_t s_red8[kMbThreads / 32];
  const int lane = threadIdx.x & 31;
  const unsigned long long fp = *fpacked;
  const int32_t q = (int32_t)(fp & 0xFFFFFFFFull);
  const int32_t qe = (int32_t)(fp >> 32);
  const long long total = (long long)q + qe;
  const long long nchunks = (total + kMbChunk - 1) / kMbChunk;
  for (long long chunk = blockIdx.x; chunk < nchunks; chunk += gridDim.x) {
    const long long d0 = chunk * kMbChunk;
    const long long d1 = min(d0 + kMbChunk, total);
    const int32_t i0 = cb[chunk], i1 = cb[chunk + 1];  // k_list_bounds
    const long long j0 = d0 - i0, j1 = d1 - i1;
    const int32_t nv = (i0 <= q - 1) ? (min(i1, q - 1) - i0 + 1) : 0;
    for (int32_t k = threadIdx.x; k < nv; k += kMbThreads) {
      const int32_t i = i0 + k;
      const int32_t v = GR_IN(i, a.n + 1, 220) ? Q[i] : 0;
      const bool ok = GR_IN(v, a.n, 221);
      s_off[k] = S[i];
      s_v[k] = ok ? v : -1;
      s_row[k] = ok ? a.R[v] : 0;
      s_A[k] = ok ? a.lv[v] : 0ull;
    }
    __syncthreads();
    const int32_t ne = (int32_t)(j1 - j0);
    for (int32_t kb = 0; kb < ne; kb += kMbThreads) {
      const int32_t k = kb + threadIdx.x;
      int32_t owner = -1, w = 0;
      unsigned long long bits = 0ull;
      if (k < ne) {
        const int32_t er = (int32_t)(j0 + k);
        int32_t lo = 0, hi = nv - 1;
        while (lo < hi) {
          const int32_t mid = (lo + hi + 1) >> 1;
          if (s_off[mid] <= er) lo = mid;
          else hi = mid - 1;
        }
        owner = s_v[lo];
        const long long e = (long long)s_row[lo] + (er - s_off[lo]);
        const unsigned long long A = s_A[lo];
        if (owner >= 0 && A && GR_IN(e, a.m, 222)) {
          w = a.C[e];
          bits = GR_IN(w, a.n, 223) ? (A & a.lw[w]) : 0ull;
        }
      }
      uint32_t act = __ballot_sync(0xffffffffu, bits != 0ull);
      int32_t cur_owner = -1;
      unsigned long long orbits = 0ull;
      double acc0 = 0.0, acc1 = 0.0;
      while (act) {
        const int j = __ffs(act) - 1;
        act &= act - 1u;
        const int32_t ov = __shfl_sync(0xffffffffu, owner, j);
        const int32_t wj = __shfl_sync(0xffffffffu, w, j);
        const unsigned long long bj = shfl_u64(bits, j);
        if (ov != cur_owner) {
          if (cur_owner >= 0) {
            double *qv = a.q + (int64_t)cur_owner * 64;
            if ((orbits >> lane) & 1ull) atomicAdd(qv + lane, acc0);
            if ((orbits >> (lane + 32)) & 1ull) atomicAdd(qv + lane + 32, acc1);
          }
          cur_owner = ov;
          orbits = 0ull;
          acc0 = acc1 = 0.0;
        }
        orbits |= bj;
        const double *qw = a.q + (int64_t)wj * 64;
        // a half with no bits set costs the warp no FP64 add
        if ((uint32_t)bj && ((bj >> lane) & 1ull)) acc0 += qw[lane];
        if ((bj >> 32) && ((bj >> (lane + 32)) & 1ull)) acc1 += qw[lane + 32];
      }
      if (cur_owner >= 0) {
        double *qv = a.q + (int64_t)cur_owner * 64;
        if ((orbits >> lane) & 1ull) atomicAdd(qv + lane, acc0);
        if ((orbits >> (lane + 32)) & 1ull) atomicAdd(qv + lane + 32, acc1);
      }
    }
    __syncthreads();
  }
}

// The vertices with lanes in `lv`, with their degree scan (block-wise
// compaction, one packed atomic per block). Vertices without edges are
// listed too (a directed graph reaches some): they have no children, but
// their dependencies still have to be finished.
__global__ void __launch_bounds__(kMbThreads) k_mb_list(const unsigned long long *lv,
                                                         const int32_t *R, int32_t n,
                                                         int32_t *Q, int32_t *S,
                                                         unsigned long long *fpacked) {
  __shared__ ScannedBuf<kMbChunk> buf;
  if (threadIdx.x == 0) buf.cnt = 0;
  __syncthreads();
  constexpr int PER = kMbChunk / kMbThreads;
  for (int64_t base = (int64_t)blockIdx.x * kMbChunk; base < n;
       base += (int64_t)gridDim.x * kMbChunk) {  // block-uniform
#pragma unroll
    for (int j = 0; j < PER; ++j) {
      const int64_t v = base + j * kMbThreads + threadIdx.x;
      int32_t d = 0;
      bool take = false;
      if (v < n && lv[v]) {
        d = R[v + 1] - R[v];
        take = true;
      }
      emit_scanned(buf, take, (int32_t)v, d);
    }
    flush_scanned<kMbThreads>(buf, fpacked, Q, S, (long long)n + 1);
  }
}

// Finish level L: delta[v][s] = sigma[v][s] * q[v][s] (q holds the child
// sum), bc[v] += delta over the lanes of lm[L][v], then q[v][s] becomes
// 1/sigma + child sum for level L-1. The vertices of level L come listed by
// k_mb_list (Q[0..q), q in fpacked; a vertex of a level >= 1 has an edge).
// One warp per vertex, lanes over s.
template <int SK>
__global__ void k_bc_finalize(const unsigned long long *lv, const int32_t *Q,
                              const unsigned long long *fpacked, const void *sigma_p,
                              double *q, double *bc, int32_t n, int32_t *overflow) {
  const int64_t gw = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int lane = threadIdx.x & 31;
  const CountT<SK> *sigma = (const CountT<SK> *)sigma_p;
  const int32_t nq = (int32_t)(*fpacked & 0xFFFFFFFFull);
  for (int64_t i = gw; i < nq; i += nw) {
    const int32_t v0 = Q[i];
    if (!GR_IN(v0, n, 230)) continue;
    const int64_t v = v0;
    const unsigned long long A = lv[v];
    if (!A) continue;
    if (SK == kSigU64) {
      // double-single: delta = sigma * (child sum), q = 1/sigma + child sum
      DS part{0.f, 0.f};
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int s = lane + 32 * h;
        if ((uint32_t)(A >> (32 * h)) == 0u) continue;  // warp-uniform
        if ((A >> s) & 1ull) {
          const DS child = ds_from_double(q[v * 64 + s]);
          const unsigned long long c = (unsigned long long)sigma[v * 64 + s];
          if (c == 0ull) *overflow = 1;  // a reached lane has at least one path
          const DS sg = ds_from_u64(c);
          part = ds_add(part, ds_mul(sg, child));
          q[v * 64 + s] = ds_to_double(ds_add(ds_rcp(sg), child));
        }
      }
      for (int o = 16; o > 0; o >>= 1) part = ds_add(part, shfl_xor_ds(part, o));
      if (lane == 0) bc[v] += ds_to_double(part);
      continue;
    }
    double part = 0.0;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int s = lane + 32 * h;
      if ((uint32_t)(A >> (32 * h)) == 0u) continue;  // warp-uniform
      if ((A >> s) & 1ull) {
        const double child = q[v * 64 + s];
        double sg;
        if (SK == kSigU64) {
          const unsigned long long c = (unsigned long long)sigma[v * 64 + s];
          if (c == 0ull) *overflow = 1;  // a reached lane has at least one path
          sg = (double)c;
        } else {
          sg = (double)sigma[v * 64 + s];
          if (!isfinite(sg) || sg <= 0.0) *overflow = 1;
        }
        part = fma(sg, child, part);
        q[v * 64 + s] = 1.0 / sg + child;
      }
    }
    for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
    if (lane == 0) bc[v] += part;
  }
}

__global__ void k_fill_f64(double *x, int64_t n, double val) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    x[i] = val;
}

// Before k_mb_do runs again after it stopped for more level arrays: a fresh
// barrier (its generation restarts with every launch).
__global__ void k_mb_resume(MbCtl *c) {
  grid_barrier_reset(&c->bar);
  c->paused = 0;
}

}  // namespace

// Levels of a batched BFS kept in their own mask arrays on this graph.
static int32_t bfs_keep_levels(const gr_graph *g) {
  return g->max_degree <= kLowDegreeMaxBatch ? 0 : kKeepLevels;
}

size_t batch_ws_bytes(const gr_graph *g) {
  // visit masks, the level arrays of a batched BFS, the level lists
  const size_t n = (size_t)g->n;
  return sizeof(unsigned long long) * n * (1 + bfs_keep_levels(g) + 3) +
         3 * sizeof(int32_t) * (2 * n + 3) + sizeof(MbCtl) + 4096;
}

gr_status batch_ws_create(gr_graph *g, BatchWorkspace **out) {
  std::unique_ptr<BatchWorkspace> ws(new BatchWorkspace());
  GR_TRY(ws->visit.alloc(sizeof(unsigned long long) * (size_t)g->n, "lane visit masks"));
  GR_TRY(ws->counter.alloc(sizeof(unsigned long long) * 4, "batch counters"));
  GR_TRY(ws->ctl.alloc(sizeof(MbCtl), "batch control"));
  {
    // the pull levels' merge paths over all vertices are the same on every
    // level: their chunk bounds are found once
    const int32_t *R = g->row_off.as<int32_t>();
    const int32_t cp = merge_chunks(g->n, g->m, kMbPullChunk);
    const int32_t cf = merge_chunks(g->n, g->m, kMbChunk);
    GR_TRY(ws->cb_pull.alloc(sizeof(int32_t) * ((size_t)cp + 1), "batch pull chunk bounds"));
    GR_TRY(ws->cb_fwd.alloc(sizeof(int32_t) * ((size_t)cf + 1), "BC pull chunk bounds"));
    k_chunk_bounds<<<(cp + 256) / 256, 256>>>(R, g->n, kMbPullChunk, cp, ws->cb_pull.as<int32_t>());
    k_chunk_bounds<<<(cf + 256) / 256, 256>>>(R, g->n, kMbChunk, cf, ws->cb_fwd.as<int32_t>());
    GR_CUDA(cudaGetLastError());
    GR_CUDA(cudaStreamSynchronize(0));
  }
  for (int i = 0; i < 3; ++i) {
    GR_TRY(ws->lq[i].alloc(sizeof(int32_t) * ((size_t)g->n + 1), "batch level list"));
    GR_TRY(ws->ls[i].alloc(sizeof(int32_t) * ((size_t)g->n + 2), "batch level list scan"));
  }
  *out = ws.release();
  return GR_OK;
}

// Most merge-path chunks a BC level list can have (n vertices, m edges).
static long long bc_list_max_chunks(const gr_graph *g) {
  return ((long long)g->n + g->m) / kMbChunk + 1;
}

static gr_status ensure_batch_ws(gr_graph *g, BatchWorkspace **slot, bool need_bc) {
  if (!*slot) GR_TRY(batch_ws_create(g, slot));
  BatchWorkspace *ws = *slot;
  if (need_bc && !ws->sigma.p) {
    GR_TRY(ws->sigma.alloc(sizeof(double) * 64 * (size_t)g->n, "BC path counts"));
    GR_TRY(ws->q.alloc(sizeof(double) * 64 * (size_t)g->n, "BC dependencies"));
  }
  if (need_bc && !ws->fq.p) {
    GR_TRY(ws->fq.alloc(sizeof(int32_t) * ((size_t)g->n + 1), "BC level list"));
    GR_TRY(ws->fs.alloc(sizeof(int32_t) * ((size_t)g->n + 2), "BC level list scan"));
    GR_TRY(ws->fcb.alloc(sizeof(int32_t) * (size_t)(bc_list_max_chunks(g) + 1),
                         "BC level list chunk bounds"));
  }
  return GR_OK;
}

// At least `slots` level mask arrays, their device pointers in lmp. New
// arrays are zeroed on `s` (the forward clears the arrays it reuses itself).
static gr_status ensure_slots(gr_graph *g, BatchWorkspace *ws, int32_t slots, cudaStream_t s) {
  const size_t bytes = sizeof(unsigned long long) * (size_t)g->n;
  if ((int32_t)ws->lm.size() < slots) {
    // the old table may still be read by enqueued work
    GR_CUDA(cudaStreamSynchronize(s));
    while ((int32_t)ws->lm.size() < slots) {
      std::unique_ptr<DevMem> m(new DevMem());
      GR_TRY(m->alloc(bytes, "level lane masks"));
      GR_CUDA(cudaMemsetAsync(m->p, 0, bytes, s));
      ws->lm.push_back(m.release());
    }
  }
  if (ws->uploaded < slots || !ws->lmp.p) {
    const int32_t cap = (int32_t)ws->lm.size();
    std::vector<unsigned long long *> ptrs(cap);
    for (int32_t i = 0; i < cap; ++i) ptrs[i] = ws->lm[i]->as<unsigned long long>();
    if (ws->lmp.bytes < sizeof(void *) * (size_t)cap) {
      GR_CUDA(cudaStreamSynchronize(s));
      GR_TRY(ws->lmp.alloc(sizeof(void *) * (size_t)std::max<int32_t>(cap, 64), "level mask table"));
    }
    // pageable source: staged before the call returns, copied in stream order
    GR_CUDA(cudaMemcpyAsync(ws->lmp.p, ptrs.data(), sizeof(void *) * (size_t)cap,
                            cudaMemcpyHostToDevice, s));
    ws->uploaded = cap;
  }
  return GR_OK;
}

static MbArgs mb_args(gr_graph *g, BatchWorkspace *ws, int32_t k, int32_t *depth, int32_t keep,
                      int32_t max_levels, bool with_sigma) {
  MbArgs a;
  std::memset(&a, 0, sizeof(a));
  a.R = g->row_off.as<int32_t>();
  a.C = g->col.as<int32_t>();
  a.n = g->n;
  a.m = g->m;
  a.all = k == 64 ? ~0ull : ((1ull << k) - 1ull);
  a.visit = ws->visit.as<unsigned long long>();
  a.lmp = (unsigned long long *const *)ws->lmp.p;
  a.cap = (int32_t)ws->lm.size();
  a.keep = keep;
  for (int i = 0; i < 3; ++i) {
    a.lq[i] = ws->lq[i].as<int32_t>();
    a.ls[i] = ws->ls[i].as<int32_t>();
  }
  a.sigma = with_sigma ? ws->sigma.p : nullptr;
  a.depth = depth;
  a.k = k;
  a.symmetric = g->symmetric ? 1 : 0;
  a.max_levels = max_levels;
  a.ctl = ws->ctl.as<MbCtl>();
  a.cb_pull = ws->cb_pull.as<int32_t>();
  a.cb_fwd = ws->cb_fwd.as<int32_t>();
  return a;
}

static gr_status mb_launch(gr_graph *g, const MbArgs &a, int sk, cudaStream_t s) {
  void *kern = sk == kSigU64   ? (void *)k_mb_do<kSigU64>
               : sk == kSigF64 ? (void *)k_mb_do<kSigF64>
                               : (void *)k_mb_do<kSigNone>;
  const int want = sk == kSigNone ? mb_do_blocks_per_sm<kSigNone>() : mb_do_blocks_per_sm<kSigU64>();
  int per_sm = 1;
  GR_TRY(fit_carveout(kern, kMbThreads, want, g->device, &per_sm));
  const int blocks = per_sm * g->num_sms;
  MbArgs arg = a;
  void *args[] = {&arg};
  GR_CUDA(cudaLaunchCooperativeKernel(kern, blocks, kMbThreads, args, 0, s));
  return GR_OK;
}

// Forward levels of one batch of k <= 64 sources (device-driven), counting
// paths as `sk` says. A batched BFS (depth != null) has every array it can
// need before it starts and never synchronises; BC (levels_out != null)
// keeps every level's array, so the kernel may stop for more and is
// resumed, and the call synchronises to report the level count and
// whether a uint64 path count overflowed.
static gr_status run_forward(gr_graph *g, BatchWorkspace *ws, const int32_t *h_srcs, int32_t k,
                             int32_t *depth, int sk, cudaStream_t s, int32_t max_levels,
                             int32_t *levels_out = nullptr, bool *overflowed = nullptr) {
  const bool with_sigma = sk != kSigNone;
  const int32_t keep = with_sigma ? INT32_MAX : bfs_keep_levels(g);
  GR_TRY(ensure_slots(g, ws, with_sigma ? std::max<int32_t>(16, (int32_t)ws->lm.size())
                                        : keep + 3, s));
  MbArgs a = mb_args(g, ws, k, depth, keep, max_levels, with_sigma);
  const int grid = g->num_sms * 8;
  k_mb_init<<<grid, 256, 0, s>>>(a, with_sigma ? ws->sigma.as<unsigned long long>() : nullptr,
                                 with_sigma ? ws->q.as<double>() : nullptr);
  MbSources src;  // by value: no host-to-device copy
  for (int32_t i = 0; i < 64; ++i) src.s[i] = i < k ? h_srcs[i] : 0;
  k_mb_sources<<<1, 64, 0, s>>>(a, src, sk);
  GR_CUDA(cudaGetLastError());
  GR_TRY(mb_launch(g, a, sk, s));
  if (!levels_out) return GR_OK;
  for (;;) {
    MbCtl h;
    GR_CUDA(cudaMemcpyAsync(&h, ws->ctl.p, sizeof(MbCtl), cudaMemcpyDeviceToHost, s));
    GR_CUDA(cudaStreamSynchronize(s));
    if (h.error == kDevTimeout) return fail(GR_ETIMEOUT, "a device-side wait timed out");
    if (h.error == kDevOverflow) return fail(GR_ETIMEOUT, "level limit reached");
    if (h.done) {
      *levels_out = h.levels;
      if (overflowed) *overflowed = h.sig_overflow != 0;
      return GR_OK;
    }
    if (!h.paused) return fail(GR_ECUDA, "batched forward stopped without a reason");
    // the next levels need more arrays: double them and resume
    GR_TRY(ensure_slots(g, ws, 2 * (int32_t)ws->lm.size(), s));
    a = mb_args(g, ws, k, depth, keep, max_levels, with_sigma);
    k_mb_resume<<<1, 1, 0, s>>>(a.ctl);
    GR_CUDA(cudaGetLastError());
    GR_TRY(mb_launch(g, a, sk, s));
  }
}

gr_status batch_read_ctl_error(BatchWorkspace *ws, cudaStream_t s) {
  MbCtl h;
  // pageable destination: the copy has finished when the call returns
  GR_CUDA(cudaMemcpyAsync(&h, ws->ctl.p, sizeof(MbCtl), cudaMemcpyDeviceToHost, s));
  if (h.error == kDevTimeout) return fail(GR_ETIMEOUT, "a device-side wait timed out");
  if (h.error == kDevOverflow) return fail(GR_ETIMEOUT, "level limit reached");
  if (!h.done) return fail(GR_ECUDA, "batched BFS did not finish");
  return GR_OK;
}

// Batched BFS into a device depth array [k][n] with an explicit workspace.
gr_status bfs_batch_run(gr_graph *g, BatchWorkspace *ws, const int32_t *h_srcs, int32_t k,
                        int32_t *depth, int32_t max_levels, cudaStream_t s) {
  return run_forward(g, ws, h_srcs, k, depth, kSigNone, s, max_levels);
}

}  // namespace gr

using namespace gr;

extern "C" {

gr_status gr_bfs_batch(gr_graph *g, const int32_t *srcs, int32_t k, int32_t *depth,
                       const gr_opts *opts, void *stream) {
  clear_error();
  if (!g) return fail(GR_EINVAL, "graph must not be NULL");
  if (k < 1 || k > 64) return fail(GR_EINVAL, "k must be in [1, 64]");
  if (!srcs || !depth) return fail(GR_EINVAL, "srcs/depth must not be NULL");
  for (int32_t i = 0; i < k; ++i)
    if (srcs[i] < 0 || srcs[i] >= g->n) return fail(GR_EINVAL, "source out of range");
  const gr_opts &o = opts ? *opts : default_opts();
  std::lock_guard<std::mutex> lock(g->mu);
  cudaStream_t s = (cudaStream_t)stream;
  GR_TRY(begin_call(g, s));
  GR_TRY(ensure_batch_ws(g, &g->batch, false));
  void *d_depth;
  bool cp;
  const size_t bytes = sizeof(int32_t) * (size_t)k * (size_t)g->n;
  GR_TRY(resolve_output(g, 0, depth, bytes, &d_depth, &cp));
  const int32_t max_levels = o.max_iters > 0 ? o.max_iters : g->n + 1;
  GR_TRY(bfs_batch_run(g, g->batch, srcs, k, (int32_t *)d_depth, max_levels, s));
  if (cp) GR_CUDA(cudaMemcpyAsync(depth, d_depth, bytes, cudaMemcpyDeviceToHost, s));
  GR_TRY(end_call(g, s));
  return GR_OK;
}

gr_status gr_bfs_batch_stats(gr_graph *g, int32_t *levels) {
  clear_error();
  if (!g) return fail(GR_EINVAL, "graph must not be NULL");
  if (!g->batch) return fail(GR_EINVAL, "no batched traversal has run on this graph");
  std::lock_guard<std::mutex> lock(g->mu);
  GR_CUDA(cudaSetDevice(g->device));
  if (g->has_last) GR_CUDA(cudaEventSynchronize(g->last_done));
  MbCtl h;
  GR_CUDA(cudaMemcpy(&h, g->batch->ctl.p, sizeof(MbCtl), cudaMemcpyDeviceToHost));
  if (h.error == kDevTimeout) return fail(GR_ETIMEOUT, "a device-side wait timed out");
  if (h.error == kDevOverflow) return fail(GR_ETIMEOUT, "level limit reached");
  if (levels) *levels = h.levels;
  return GR_OK;
}

gr_status gr_bc(gr_graph *g, const int32_t *srcs, int32_t k, double *bc, const gr_opts *opts,
                void *stream) {
  clear_error();
  if (!g) return fail(GR_EINVAL, "graph must not be NULL");
  if (k < 0) return fail(GR_EINVAL, "k must be >= 0");
  if ((k > 0 && !srcs) || !bc) return fail(GR_EINVAL, "srcs/bc must not be NULL");
  for (int32_t i = 0; i < k; ++i)
    if (srcs[i] < 0 || srcs[i] >= g->n) return fail(GR_EINVAL, "source out of range");
  const gr_opts &o = opts ? *opts : default_opts();
  std::lock_guard<std::mutex> lock(g->mu);
  cudaStream_t s = (cudaStream_t)stream;
  GR_TRY(begin_call(g, s));
  GR_TRY(ensure_batch_ws(g, &g->batch, true));
  void *d_bc;
  bool cp;
  GR_TRY(resolve_output(g, 0, bc, sizeof(double) * (size_t)g->n, &d_bc, &cp));
  const int grid = g->num_sms * 8;
  k_fill_f64<<<grid, 256, 0, s>>>((double *)d_bc, g->n, 0.0);
  BatchWorkspace *ws = g->batch;
  int32_t *overflow = (int32_t *)(ws->counter.as<unsigned long long>() + 1);
  GR_CUDA(cudaMemsetAsync(overflow, 0, sizeof(int32_t), s));
  const int32_t max_levels = o.max_iters > 0 ? o.max_iters : g->n + 1;
  for (int32_t b = 0; b < k; b += 64) {
    const int32_t kb = std::min<int32_t>(64, k - b);
    int32_t levels = 0;
    // exact uint64 path counts; a batch whose counts overflow them is
    // counted again in FP64
    int sk = kSigU64;
    bool overflowed = false;
    GR_TRY(run_forward(g, ws, srcs + b, kb, nullptr, sk, s, max_levels, &levels, &overflowed));
    if (overflowed) {
      sk = kSigF64;
      GR_TRY(run_forward(g, ws, srcs + b, kb, nullptr, sk, s, max_levels, &levels));
    }
    // backward over levels levels-2 .. 1 (level levels-1 has no children;
    // level 0 holds the sources, which take no credit)
    BcBackArgs ba;
    ba.R = g->row_off.as<int32_t>();
    ba.C = g->col.as<int32_t>();
    ba.n = g->n;
    ba.m = g->m;
    ba.q = ws->q.as<double>();
    unsigned long long *fpacked = ws->counter.as<unsigned long long>() + 2;
    int32_t *fq = ws->fq.as<int32_t>(), *fs = ws->fs.as<int32_t>();
    const int list_bound_blocks = (int)((bc_list_max_chunks(g) + 1 + 255) / 256);
    int back_per_sm = 1;
    GR_TRY(fit_carveout(k_bc_backward, kMbThreads, kBcBackBlocksPerSm, g->device, &back_per_sm));
    for (int32_t L = levels - 1; L >= 1; --L) {
      // the vertices of level L (in any lane) with their degree scan
      ba.lv = ws->lm[L]->as<unsigned long long>();
      GR_CUDA(cudaMemsetAsync(fpacked, 0, sizeof(unsigned long long), s));
      k_mb_list<<<grid, kMbThreads, 0, s>>>(ba.lv, ba.R, g->n, fq, fs, fpacked);
      if (L + 1 < levels) {
        ba.lw = ws->lm[L + 1]->as<unsigned long long>();
        k_list_bounds<<<list_bound_blocks, 256, 0, s>>>(fs, fpacked, ws->fcb.as<int32_t>());
        k_bc_backward<<<g->num_sms * back_per_sm, kMbThreads, 0, s>>>(ba, fq, fs, fpacked,
                                                                       ws->fcb.as<int32_t>());
      }
      if (sk == kSigU64)
        k_bc_finalize<kSigU64><<<grid, 256, 0, s>>>(ba.lv, fq, fpacked, ws->sigma.p,
                                                    ws->q.as<double>(), (double *)d_bc, g->n,
                                                    overflow);
      else
        k_bc_finalize<kSigF64><<<grid, 256, 0, s>>>(ba.lv, fq, fpacked, ws->sigma.p,
                                                    ws->q.as<double>(), (double *)d_bc, g->n,
                                                    overflow);
      GR_CUDA(cudaGetLastError());
    }
  }
  if (cp) GR_CUDA(cudaMemcpyAsync(bc, d_bc, sizeof(double) * (size_t)g->n,
                                  cudaMemcpyDeviceToHost, s));
  int32_t h_over = 0;
  GR_CUDA(cudaMemcpyAsync(&h_over, overflow, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  GR_CUDA(cudaStreamSynchronize(s));
  GR_TRY(end_call(g, s));
  if (h_over)
    return fail(GR_EINVAL, "shortest-path counts overflow FP64 on this graph (BC undefined)");
  return GR_OK;
}

}  // extern "C"
