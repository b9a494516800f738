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
// The level loop is host-driven (one small read-back per level) because BC
// keeps one mask array per level and allocates them as levels appear.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <type_traits>
#include <vector>

#include "advance.cuh"

namespace gr {

constexpr int kMbThreads = 256, kMbItems = 4;
// Batched BFS keeps the lane masks of its first kKeepLevels levels and
// writes their depths in one pass (k_mb_depth); deeper levels write depths
// as they are reached.
constexpr int32_t kKeepLevels = 64;
// A batched BFS level pushes when its frontier has fewer than m / kPushDiv
// edges, and pulls over every vertex otherwise.
constexpr long long kPushDiv = 16;
constexpr int kMbChunk = kMbThreads * kMbItems;
// What the forward pass counts: nothing (batched BFS), path counts in uint64,
// or path counts in FP64 (a batch whose uint64 counts overflowed).
enum : int { kSigNone = 0, kSigU64 = 1, kSigF64 = 2 };

struct BatchWorkspace {
  DevMem visit, sigma, q, counter, srcs, lmp;
  DevMem fq, fs;  // frontier list and degree scan of the push levels
  std::vector<DevMem *> lm;  // lm[L]: lane masks of level L
  ~BatchWorkspace() {
    for (DevMem *p : lm) delete p;
  }
};

void free_batch(BatchWorkspace *ws) { delete ws; }

GR_GUARD_REPORTER(guard_report_batch)

namespace {

struct MbArgs {
  const int32_t *R;
  const int32_t *C;
  int32_t n;
  long long m;
  unsigned long long all;  // mask of the lanes in use
  unsigned long long *visit;
  const unsigned long long *cur;  // lm[L]
  unsigned long long *nxt;        // lm[L+1], zero on entry
  void *sigma;                    // [n][64] uint64 or FP64 path counts, or null (BFS)
  int32_t *sig_overflow;          // set when a uint64 path count overflows
  int32_t *depth;                 // [k][n] or null (BC)
  int32_t k;
  int32_t level;
  unsigned long long *count;      // [31:0] vertices that joined lm[L+1], [63:32] their edges
};

// Packed (vertices, edges) increment for a vertex that joined the next level.
__device__ __forceinline__ unsigned long long joined(const MbArgs &a, int32_t v) {
  return 1ull | ((unsigned long long)(uint32_t)(a.R[v + 1] - a.R[v]) << 32);
}

__device__ __forceinline__ unsigned long long shfl_u64(unsigned long long x, int src) {
  return __shfl_sync(0xffffffffu, x, src);
}

__device__ __forceinline__ unsigned long long shfl_down_u64(unsigned long long x, int o) {
  return __shfl_down_sync(0xffffffffu, x, o);
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

__global__ void k_mb_init(unsigned long long *visit, unsigned long long *lm0,
                          unsigned long long *sigma, double *q, int32_t n) {
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n;
       v += (int64_t)gridDim.x * blockDim.x) {
    visit[v] = 0ull;
    lm0[v] = 0ull;
  }
  if (sigma) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < (int64_t)n * 64;
         i += (int64_t)gridDim.x * blockDim.x) {
      sigma[i] = 0ull;  // 0 as uint64 and as FP64
      q[i] = 0.0;
    }
  }
}

__global__ void k_mb_sources(const int32_t *srcs, int32_t k, unsigned long long *lm0,
                             void *sigma, int32_t sk, int32_t n_vertices) {
  const int s = threadIdx.x;
  if (s < k && GR_IN(srcs[s], n_vertices, 205)) {
    const int32_t v = srcs[s];
    atomicOr(lm0 + v, 1ull << s);
    if (sk == kSigU64) ((unsigned long long *)sigma)[(int64_t)v * 64 + s] = 1ull;
    if (sk == kSigF64) ((double *)sigma)[(int64_t)v * 64 + s] = 1.0;
  }
}

// One batched BFS pull level (no path counts): lm[L+1][v] = OR over edges
// (v, u) of lm[L][u] & ~seen(v), seen(v) = visit[v] | lm[L][v]. Merge-based:
// a chunk's vertex end markers and edges form one sequence of
// kMbThreads * kMbPullItems items; each thread finds its first item's
// vertex with one search, then walks its kMbPullItems consecutive items.
// The column and lane-mask loads of all its items are issued before any is
// used, edges of vertices that already hold every lane are skipped, and the
// OR of a vertex accumulates in a register. A vertex whose edges and end
// marker all fall in one thread's items is written with a plain store (no
// other thread touches it); the others with atomicOr. The vertex loader
// folds lm[L] into visit and, past the kept levels, writes depth L.
constexpr int kMbPullItems = 8, kMbPullBlocksPerSm = 6;
__global__ void __launch_bounds__(kMbThreads, kMbPullBlocksPerSm) k_mb_pull(MbArgs a) {
  constexpr int ITEMS = kMbPullItems;
  constexpr int CHUNK = kMbThreads * ITEMS;
  __shared__ int32_t s_end[CHUNK + 1];  // end marker of each vertex, chunk-local
  __shared__ unsigned long long s_U[CHUNK + 1];  // lanes the vertex still misses
  __shared__ int32_t s_red8[kMbThreads / 32];
  const int lane = threadIdx.x & 31;
  const long long total = (long long)a.n + a.R[a.n];
  const long long nchunks = (total + CHUNK - 1) / CHUNK;
  unsigned long long new_vertices = 0;
  for (long long chunk = blockIdx.x; chunk < nchunks; chunk += gridDim.x) {
    const long long d0 = chunk * CHUNK;
    const long long d1 = min(d0 + CHUNK, total);
    int32_t i0, i1;
    block_chunk_bounds<kMbThreads>(a.R, a.n, a.R[a.n], d0, d1, CHUNK, s_red8, &i0, &i1);
    const long long j0 = d0 - i0;  // CSR position of the chunk's first edge
    const int32_t nv = (i0 <= a.n - 1) ? (min(i1, a.n - 1) - i0 + 1) : 0;
    const int32_t len = (int32_t)(d1 - d0);
    for (int32_t kk = threadIdx.x; kk < nv; kk += kMbThreads) {
      const int32_t v = i0 + kk;
      const unsigned long long c = a.cur[v];
      const unsigned long long seen = a.visit[v] | c;
      if (c) {
        a.visit[v] = seen;
        if (a.depth) {
          for (int s = 0; s < a.k; ++s)
            if (((c >> s) & 1ull) && GR_IN((int64_t)s * a.n + v, (int64_t)a.k * a.n, 204))
              a.depth[(int64_t)s * a.n + v] = a.level;
        }
      }
      s_end[kk] = (int32_t)((long long)a.R[v + 1] + v - d0);
      s_U[kk] = a.all & ~seen;
    }
    __syncthreads();
    const int32_t k0 = min(len, (int32_t)threadIdx.x * ITEMS);
    const int32_t k1 = min(len, k0 + ITEMS);
    if (k0 < k1) {
      // chunk vertices whose end marker lies before k0
      int32_t lo = 0, hi = nv;
      while (lo < hi) {
        const int32_t mid = (lo + hi) >> 1;
        if (s_end[mid] < k0) lo = mid + 1;
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
          if (s_end[r] == k) {
            ends |= 1u << i;
            ++r;
          } else {
            const long long pos = j0 + e;
            if (s_U[r] && GR_IN(pos, a.m, 202)) u[i] = (int32_t)pos;
            ++e;
          }
        }
      }
#pragma unroll
      for (int i = 0; i < ITEMS; ++i) u[i] = u[i] >= 0 ? a.C[u[i]] : -1;
      unsigned long long b[ITEMS];
#pragma unroll
      for (int i = 0; i < ITEMS; ++i) b[i] = (u[i] >= 0 && GR_IN(u[i], a.n, 203)) ? a.cur[u[i]] : 0ull;
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
                a.nxt[v] = acc;
                new_vertices += joined(a, v);
              } else if (!atomicOr(a.nxt + v, acc)) {
                new_vertices += joined(a, v);
              }
            }
            acc = 0ull;
            whole = true;
            ++r;
          } else {
            acc |= b[i] & s_U[r];
          }
        }
      }
      if (acc && r < nv && !atomicOr(a.nxt + (i0 + r), acc))  // continues past k1
        new_vertices += joined(a, i0 + r);
    }
    __syncthreads();
  }
  for (int o = 16; o > 0; o >>= 1) new_vertices += __shfl_xor_sync(0xffffffffu, new_vertices, o);
  if (lane == 0 && new_vertices) atomicAdd(a.count, new_vertices);
}

// One BC forward pull level: lm[L+1][v] = OR over edges (v,u) of
// lm[L][u] & ~seen(v), seen(v) = visit[v] | lm[L][v], and the path counts of
// the newly reached lanes. The vertex loader of each chunk folds lm[L] into
// visit (idempotent, so chunks sharing a vertex may both do it).
template <int SK>
__global__ void __launch_bounds__(kMbThreads) k_mb_forward(MbArgs a) {
  static_assert(SK != kSigNone, "batched BFS pulls with k_mb_pull");
  using T = CountT<SK>;
  bool ovf = false;
  __shared__ int32_t s_off[kMbChunk + 1];
  __shared__ unsigned long long s_U[kMbChunk + 1];
  __shared__ int32_t s_red8[kMbThreads / 32];
  const int lane = threadIdx.x & 31;
  const long long total = (long long)a.n + a.R[a.n];
  const long long nchunks = (total + kMbChunk - 1) / kMbChunk;
  unsigned long long new_vertices = 0;
  for (long long chunk = blockIdx.x; chunk < nchunks; chunk += gridDim.x) {
    const long long d0 = chunk * kMbChunk;
    const long long d1 = min(d0 + kMbChunk, total);
    int32_t i0, i1;
    block_chunk_bounds<kMbThreads>(a.R, a.n, a.R[a.n], d0, d1, kMbChunk, s_red8, &i0, &i1);
    const long long j0 = d0 - i0, j1 = d1 - i1;
    const int32_t nv = (i0 <= a.n - 1) ? (min(i1, a.n - 1) - i0 + 1) : 0;
    for (int32_t kk = threadIdx.x; kk < nv; kk += kMbThreads) {
      const int32_t v = i0 + kk;
      const unsigned long long c = a.cur[v];
      const unsigned long long seen = a.visit[v] | c;
      if (c) {
        a.visit[v] = seen;
        if (a.depth) {
          for (int s = 0; s < a.k; ++s)
            if (((c >> s) & 1ull) && GR_IN((int64_t)s * a.n + v, (int64_t)a.k * a.n, 204))
            a.depth[(int64_t)s * a.n + v] = a.level;
        }
      }
      s_off[kk] = a.R[v];
      s_U[kk] = a.all & ~seen;
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
          if (s_off[mid] <= e) lo = mid;
          else hi = mid - 1;
        }
        owner = i0 + lo;
        if (!GR_IN(owner, a.n, 201)) owner = -1;
        const unsigned long long U = owner >= 0 ? s_U[lo] : 0ull;
        if (U && GR_IN(e, a.m, 202)) {
          u = a.C[e];
          bits = GR_IN(u, a.n, 203) ? (a.cur[u] & U) : 0ull;
        }
      }
      {
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
              if (lane == 0) {
                const unsigned long long old = atomicOr(a.nxt + cur_owner, orbits);
                if (!old) new_vertices += joined(a, cur_owner);
              }
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
          if (lane == 0) {
            const unsigned long long old = atomicOr(a.nxt + cur_owner, orbits);
            if (!old) new_vertices += joined(a, cur_owner);
          }
        }
      }
    }
    __syncthreads();
  }
  // new_vertices counts runs whose atomicOr found an empty mask: exactly the
  // vertices that joined lm[L+1] (and their edges)
  for (int o = 16; o > 0; o >>= 1) new_vertices += __shfl_xor_sync(0xffffffffu, new_vertices, o);
  if (lane == 0 && new_vertices) atomicAdd(a.count, new_vertices);
  if (SK == kSigU64 && __any_sync(0xffffffffu, ovf) && lane == 0) atomicOr(a.sig_overflow, 1);
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

// Backward level L: q[v][s] += q[w][s] over edges (v, w) with v in lane s's
// level L and w in its level L+1 (w's q is final: level L+1 was finished).
// Only the vertices of level L (listed with their degrees by k_mb_list) are
// visited, so the whole backward pass reads every edge about once instead of
// once per level.
__global__ void __launch_bounds__(kMbThreads) k_bc_backward(BcBackArgs a, const int32_t *Q,
                                                             const int32_t *S,
                                                             const unsigned long long *fpacked) {
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
    int32_t i0, i1;
    block_chunk_bounds<kMbThreads>(S, q, qe, d0, d1, kMbChunk, s_red8, &i0, &i1);
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

// Push form of a batched BFS level, for frontiers with few edges (the
// sources' level and the last levels): instead of every vertex pulling from
// all its neighbours, the frontier's vertices push their lanes.
// k_mb_compact lists the frontier (vertices with lanes in lm[L]) with its
// degree scan, folds lm[L] into visit (the pull's vertex loader does that)
// and, past the kept levels, writes the level's depths; k_mb_push sends, over
// every edge (u, v) of the frontier, u's lanes that v has not seen to v's
// mask in lm[L+1] (merge-path chunks over the listed vertices' edges).
__global__ void __launch_bounds__(kMbThreads) k_mb_compact(MbArgs a, int32_t *Q, int32_t *S,
                                                            unsigned long long *fpacked) {
  __shared__ ScannedBuf<kMbChunk> buf;
  if (threadIdx.x == 0) buf.cnt = 0;
  __syncthreads();
  constexpr int PER = kMbChunk / kMbThreads;
  for (int64_t base = (int64_t)blockIdx.x * kMbChunk; base < a.n;
       base += (int64_t)gridDim.x * kMbChunk) {  // block-uniform
#pragma unroll
    for (int j = 0; j < PER; ++j) {
      const int64_t v = base + j * kMbThreads + threadIdx.x;
      int32_t d = 0;
      bool take = false;
      if (v < a.n) {
        const unsigned long long c = a.cur[v];
        if (c) {
          a.visit[v] |= c;
          if (a.depth) {
            for (int s = 0; s < a.k; ++s)
              if (((c >> s) & 1ull) && GR_IN((int64_t)s * a.n + v, (int64_t)a.k * a.n, 206))
                a.depth[(int64_t)s * a.n + v] = a.level;
          }
          d = a.R[v + 1] - a.R[v];
          take = d > 0;
        }
      }
      emit_scanned(buf, take, (int32_t)v, d);
    }
    flush_scanned<kMbThreads>(buf, fpacked, Q, S, (long long)a.n + 1);
  }
}

__global__ void k_mb_close(const unsigned long long *fpacked, int32_t *S) {
  const unsigned long long p = *fpacked;
  S[(int32_t)(p & 0xFFFFFFFFull)] = (int32_t)(p >> 32);
}

// With SIGMA (BC's forward pass) the lanes newly sent to v also add u's path
// counts to v's: the warp serves such edges one at a time, lane l adding
// lanes l and l + 32.
template <int SK>
__global__ void __launch_bounds__(kMbThreads) k_mb_push(MbArgs a, const int32_t *Q,
                                                         const int32_t *S,
                                                         const unsigned long long *fpacked) {
  constexpr bool SIGMA = SK != kSigNone;
  using T = CountT<SK>;
  bool ovf = false;
  __shared__ int32_t s_off[kMbChunk + 1];
  __shared__ int32_t s_row[kMbChunk + 1];
  __shared__ unsigned long long s_cur[kMbChunk + 1];
  __shared__ int32_t s_u[SIGMA ? kMbChunk + 1 : 1];
  __shared__ int32_t s_red8[kMbThreads / 32];
  const int lane = threadIdx.x & 31;
  const unsigned long long fp = *fpacked;
  const int32_t q = (int32_t)(fp & 0xFFFFFFFFull);
  const int32_t qe = (int32_t)(fp >> 32);
  const long long total = (long long)q + qe;
  const long long nchunks = (total + kMbChunk - 1) / kMbChunk;
  unsigned long long added = 0;
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
      s_off[k] = (i == q) ? qe : S[i];
      s_row[k] = ok ? a.R[u] : 0;
      s_cur[k] = ok ? a.cur[u] : 0ull;
      if (SIGMA) s_u[k] = ok ? u : 0;
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
          if (s_off[mid] <= er) lo = mid;
          else hi = mid - 1;
        }
        const long long e = (long long)s_row[lo] + (er - s_off[lo]);
        v = GR_IN(e, a.m, 209) ? a.C[e] : -1;
        if (v >= 0 && GR_IN(v, a.n, 210)) {
          bits = s_cur[lo] & ~a.visit[v];
          if (bits) {
            const unsigned long long old = atomicOr(a.nxt + v, bits);
            if (!old) added += joined(a, v);
          }
          if (SIGMA) u = s_u[lo];
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
    __syncthreads();
  }
  for (int o = 16; o > 0; o >>= 1) added += __shfl_xor_sync(0xffffffffu, added, o);
  if (lane == 0 && added) atomicAdd(a.count, added);
  if (SK == kSigU64 && __any_sync(0xffffffffu, ovf) && lane == 0) atomicOr(a.sig_overflow, 1);
}

// Depths of a batched BFS from its per-level lane masks, written once, in
// full coalesced rows: for each lane s, depth[s][v] = the level L whose mask
// lm[L][v] holds bit s (-1 if none). The masks of one vertex are disjoint,
// so the level of every lane follows from six bit slices: slice j is the OR
// of the masks of the levels whose index has bit j set.
__global__ void k_mb_depth(const unsigned long long *const *lm, int32_t levels, int32_t n,
                           int32_t k, int32_t *depth) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t nr = ((int64_t)n + 31) & ~31ll;  // warp-uniform bound
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < nr; v += stride) {
    unsigned long long b[6] = {0ull, 0ull, 0ull, 0ull, 0ull, 0ull}, reached = 0ull;
    if (v < n) {
      for (int32_t L = 0; L < levels; ++L) {
        const unsigned long long m = lm[L][v];
        reached |= m;
#pragma unroll
        for (int j = 0; j < 6; ++j)
          if ((L >> j) & 1) b[j] |= m;
      }
    }
    for (int32_t s = 0; s < k; ++s) {
      int32_t d = -1;
      if ((reached >> s) & 1ull) {
        d = 0;
#pragma unroll
        for (int j = 0; j < 6; ++j) d |= (int32_t)((b[j] >> s) & 1ull) << j;
      }
      if (v < n) depth[(int64_t)s * n + v] = d;
    }
  }
}

__global__ void k_fill_f64(double *x, int64_t n, double val) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    x[i] = val;
}

}  // namespace

size_t batch_ws_bytes(const gr_graph *g) {
  // visit masks, the level masks of a typical traversal, the push frontier
  return 12 * sizeof(unsigned long long) * (size_t)g->n + 512;
}

gr_status batch_ws_create(gr_graph *g, BatchWorkspace **out) {
  std::unique_ptr<BatchWorkspace> ws(new BatchWorkspace());
  GR_TRY(ws->lmp.alloc(sizeof(unsigned long long *) * kKeepLevels, "level mask table"));
  GR_TRY(ws->visit.alloc(sizeof(unsigned long long) * (size_t)g->n, "lane visit masks"));
  GR_TRY(ws->counter.alloc(sizeof(unsigned long long) * 4, "batch counters"));
  GR_TRY(ws->srcs.alloc(sizeof(int32_t) * 64, "batch sources"));
  *out = ws.release();
  return GR_OK;
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
  }
  return GR_OK;
}

// level masks, allocated as levels appear (zeroed before use)
static gr_status level_mask(gr_graph *g, BatchWorkspace *ws, size_t L, cudaStream_t s,
                            unsigned long long **out) {
  while (ws->lm.size() <= L) {
    std::unique_ptr<DevMem> m(new DevMem());
    GR_TRY(m->alloc(sizeof(unsigned long long) * (size_t)g->n, "level lane masks"));
    ws->lm.push_back(m.release());
  }
  GR_CUDA(cudaMemsetAsync(ws->lm[L]->p, 0, sizeof(unsigned long long) * (size_t)g->n, s));
  *out = ws->lm[L]->as<unsigned long long>();
  return GR_OK;
}

// Forward levels of one batch of k <= 64 sources, counting paths as `sk`
// says. Returns the number of levels holding vertices (the sources' level
// included); with kSigU64, *overflowed tells whether a count passed 2^64 - 1.
static gr_status run_forward(gr_graph *g, BatchWorkspace *ws, const int32_t *h_srcs, int32_t k,
                             int32_t *depth, int sk, cudaStream_t s,
                             int32_t max_levels, int32_t *levels_out,
                             bool *overflowed = nullptr) {
  const bool with_sigma = sk != kSigNone;
  const int grid = g->num_sms * 8;
  unsigned long long *lm0;
  GR_TRY(level_mask(g, ws, 0, s, &lm0));
  int32_t *sig_overflow = (int32_t *)(ws->counter.as<unsigned long long>() + 3);
  if (with_sigma) GR_CUDA(cudaMemsetAsync(sig_overflow, 0, sizeof(int32_t), s));
  k_mb_init<<<grid, 256, 0, s>>>(ws->visit.as<unsigned long long>(), lm0,
                                 with_sigma ? ws->sigma.as<unsigned long long>() : nullptr,
                                 with_sigma ? ws->q.as<double>() : nullptr, g->n);
  GR_CUDA(cudaMemcpyAsync(ws->srcs.p, h_srcs, sizeof(int32_t) * k, cudaMemcpyHostToDevice, s));
  k_mb_sources<<<1, 64, 0, s>>>(ws->srcs.as<int32_t>(), k, lm0,
                                with_sigma ? ws->sigma.p : nullptr, sk, g->n);
  GR_CUDA(cudaGetLastError());
  MbArgs a;
  a.R = g->row_off.as<int32_t>();
  a.C = g->col.as<int32_t>();
  a.n = g->n;
  a.m = g->m;
  a.all = k == 64 ? ~0ull : ((1ull << k) - 1ull);
  a.visit = ws->visit.as<unsigned long long>();
  a.sigma = with_sigma ? ws->sigma.p : nullptr;
  a.sig_overflow = sig_overflow;
  a.depth = depth;
  a.k = k;
  a.count = ws->counter.as<unsigned long long>();
  int32_t L = 0;
  // BC keeps every level's masks for the backward pass; BFS keeps those of
  // its first kKeepLevels levels (their depths are written in one pass) and
  // then alternates two arrays, writing depths level by level
  auto slot = [&](int32_t lvl) {
    if (with_sigma || lvl < kKeepLevels) return (size_t)lvl;
    return (size_t)(kKeepLevels + ((lvl - kKeepLevels) & 1));
  };
  bool depth_pass_done = false;
  // level 0 (the sources) pushes; later levels choose by frontier edges
  bool push = true;
  unsigned long long *fpacked = ws->counter.as<unsigned long long>() + 2;
  if (!ws->fq.p) {
    GR_TRY(ws->fq.alloc(sizeof(int32_t) * ((size_t)g->n + 1), "batch push frontier"));
    GR_TRY(ws->fs.alloc(sizeof(int32_t) * ((size_t)g->n + 2), "batch push frontier scan"));
  }
  auto depth_pass = [&](int32_t levels) -> gr_status {
    std::vector<unsigned long long *> ptrs(kKeepLevels, nullptr);
    for (int32_t i = 0; i < levels; ++i) ptrs[i] = ws->lm[i]->as<unsigned long long>();
    GR_CUDA(cudaMemcpyAsync(ws->lmp.p, ptrs.data(), sizeof(unsigned long long *) * kKeepLevels,
                            cudaMemcpyHostToDevice, s));
    k_mb_depth<<<grid, 256, 0, s>>>((const unsigned long long *const *)ws->lmp.p, levels, g->n,
                                    k, depth);
    GR_CUDA(cudaGetLastError());
    depth_pass_done = true;
    return GR_OK;
  };
  for (;;) {
    if (depth && L == kKeepLevels) GR_TRY(depth_pass(kKeepLevels));
    unsigned long long *nxt;
    GR_TRY(level_mask(g, ws, slot(L + 1), s, &nxt));
    a.cur = ws->lm[slot(L)]->as<unsigned long long>();
    a.nxt = nxt;
    a.level = L;
    a.depth = (depth && L >= kKeepLevels) ? depth : nullptr;
    GR_CUDA(cudaMemsetAsync(a.count, 0, sizeof(unsigned long long), s));
    if (push) {
      int32_t *fq = ws->fq.as<int32_t>(), *fs = ws->fs.as<int32_t>();
      GR_CUDA(cudaMemsetAsync(fpacked, 0, sizeof(unsigned long long), s));
      k_mb_compact<<<grid, kMbThreads, 0, s>>>(a, fq, fs, fpacked);
      k_mb_close<<<1, 1, 0, s>>>(fpacked, fs);
      if (sk == kSigU64)
        k_mb_push<kSigU64><<<g->num_sms * 8, kMbThreads, 0, s>>>(a, fq, fs, fpacked);
      else if (sk == kSigF64)
        k_mb_push<kSigF64><<<g->num_sms * 8, kMbThreads, 0, s>>>(a, fq, fs, fpacked);
      else
        k_mb_push<kSigNone><<<g->num_sms * 8, kMbThreads, 0, s>>>(a, fq, fs, fpacked);
    } else if (sk == kSigU64) {
      k_mb_forward<kSigU64><<<g->num_sms * 4, kMbThreads, 0, s>>>(a);
    } else if (sk == kSigF64) {
      k_mb_forward<kSigF64><<<g->num_sms * 4, kMbThreads, 0, s>>>(a);
    } else {
      k_mb_pull<<<g->num_sms * kMbPullBlocksPerSm, kMbThreads, 0, s>>>(a);
    }
    GR_CUDA(cudaGetLastError());
    unsigned long long cnt = 0;
    GR_CUDA(cudaMemcpyAsync(&cnt, a.count, sizeof(cnt), cudaMemcpyDeviceToHost, s));
    GR_CUDA(cudaStreamSynchronize(s));
    ++L;
    const uint32_t joined_vertices = (uint32_t)(cnt & 0xFFFFFFFFull);
    const long long joined_edges = (long long)(cnt >> 32);
    if (joined_vertices == 0) break;  // level L is empty; levels 0..L-1 hold vertices
    if (L >= max_levels) return fail(GR_ETIMEOUT, "level limit reached");
    // a pull reads v's row as v's predecessors: only a symmetric CSR has them
    // there, so a directed graph pushes on every level
    push = !g->symmetric || joined_edges * kPushDiv < g->m;
  }
  if (depth && !depth_pass_done) GR_TRY(depth_pass(L));
  *levels_out = L;
  if (overflowed) {
    *overflowed = false;
    if (sk == kSigU64) {
      int32_t h = 0;
      GR_CUDA(cudaMemcpyAsync(&h, sig_overflow, sizeof(h), cudaMemcpyDeviceToHost, s));
      GR_CUDA(cudaStreamSynchronize(s));
      *overflowed = h != 0;
    }
  }
  return GR_OK;
}

// Batched BFS into a device depth array [k][n] with an explicit workspace.
gr_status bfs_batch_run(gr_graph *g, BatchWorkspace *ws, const int32_t *h_srcs, int32_t k,
                        int32_t *depth, int32_t max_levels, cudaStream_t s) {
  int32_t levels = 0;  // every depth entry is written by run_forward
  return run_forward(g, ws, h_srcs, k, depth, kSigNone, s, max_levels, &levels);
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
    for (int32_t L = levels - 1; L >= 1; --L) {
      // the vertices of level L (in any lane) with their degree scan
      ba.lv = ws->lm[L]->as<unsigned long long>();
      GR_CUDA(cudaMemsetAsync(fpacked, 0, sizeof(unsigned long long), s));
      k_mb_list<<<grid, kMbThreads, 0, s>>>(ba.lv, ba.R, g->n, fq, fs, fpacked);
      if (L + 1 < levels) {
        ba.lw = ws->lm[L + 1]->as<unsigned long long>();
        k_bc_backward<<<g->num_sms * 4, kMbThreads, 0, s>>>(ba, fq, fs, fpacked);
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
