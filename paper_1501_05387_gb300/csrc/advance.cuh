// Generic frontier operators shared by the primitives.
//
// The paper's advance step (Sec. 4.1) expands a vertex frontier into the
// neighbours of its vertices; its load-balanced form (Sec. 4.4) first scans
// the frontier's degrees ("scanned edge offset queue") and then hands every
// block an equal share of work, finding each edge's owner by a sorted
// search. Per-edge work is a functor inlined into the kernel, the paper's
// kernel fusion of compute into advance/filter (Sec. 4.3).
//
// Here the equal shares are merge-path chunks: the frontier's vertex ends
// and its edge ranks form one merged sequence, and each chunk takes a fixed
// number of its items, so a chunk never holds more vertices or more edges
// than its size whatever the degree mix (zero-degree vertices included).
#pragma once

#include <algorithm>

#include "gr_internal.cuh"

namespace gr {

// ------------------------------------------------------------- advance
// Block-cooperative merge-path search: the count c in [lo, hi] of
// positions i whose end marker S[i+1] + i lies before diagonal d (markers
// are strictly increasing in i). Each round every thread probes one
// position and the block counts the probes before d, shrinking the range by
// a factor of THREADS, so c takes ceil(log_THREADS(hi - lo)) + 1 rounds of
// independent loads instead of log2(hi - lo) dependent ones. s_q stands in
// for S[q] (pass S[q] when it is stored). Block-uniform call; s_red holds
// THREADS / 32 ints.
template <int THREADS>
__device__ int32_t block_merge_search(const int32_t *S, int32_t q, int32_t s_q, long long d,
                                      int32_t lo, int32_t hi, int32_t *s_red) {
  constexpr int WARPS = THREADS / 32;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (;;) {
    const int32_t len = hi - lo;
    if (len <= 0) return lo;
    const int32_t step = len <= THREADS ? 1 : (len + THREADS - 1) / THREADS;
    const long long p = (long long)lo + (long long)threadIdx.x * step;
    bool pred = false;
    if (p < hi) {
      const int32_t pi = (int32_t)p;
      const int32_t sv = (pi + 1 == q) ? s_q : S[pi + 1];
      pred = (long long)sv + pi < d;
    }
    const uint32_t b = __ballot_sync(0xffffffffu, pred);
    if (lane == 0) s_red[wid] = __popc(b);
    __syncthreads();
    int32_t k = 0;
#pragma unroll
    for (int w = 0; w < WARPS; ++w) k += s_red[w];
    __syncthreads();
    if (step == 1) return lo + k;
    if (k == 0) return lo;
    const int32_t nlo = lo + (k - 1) * step + 1;
    const int32_t nhi = (int32_t)min((long long)hi, (long long)lo + (long long)k * step);
    lo = nlo;
    hi = nhi;
  }
}

// Both ends of a chunk [d0, d1) (d1 - d0 <= chunk): i0 over the whole
// frontier, then i1 within i0 + chunk. The path starts at vertex 0 and ends
// at vertex q, so the first and the last chunk skip that search (d0 and d1
// are the same for the whole block).
template <int THREADS>
__device__ __forceinline__ void block_chunk_bounds(const int32_t *S, int32_t q, int32_t s_q,
                                                   long long d0, long long d1, int32_t chunk,
                                                   int32_t *s_red, int32_t *i0, int32_t *i1) {
  *i0 = d0 <= 0 ? 0 : block_merge_search<THREADS>(S, q, s_q, d0, 0, q, s_red);
  *i1 = d1 >= (long long)q + s_q
            ? q
            : block_merge_search<THREADS>(S, q, s_q, d1, *i0, min(q, *i0 + chunk), s_red);
}

// Append `v` to one of two block-local output buffers selected per thread
// (code 1 -> buffer 0, code 2 -> buffer 1), warp-aggregated.
__device__ __forceinline__ void warp_append(int code, int32_t v, int32_t *buf0,
                                            int32_t *cnt0, int32_t *buf1, int32_t *cnt1) {
  const int lane = threadIdx.x & 31;
  const uint32_t lt = (1u << lane) - 1u;
  const uint32_t b0 = __ballot_sync(0xffffffffu, code == 1);
  const uint32_t b1 = __ballot_sync(0xffffffffu, code == 2);
  if (b0) {
    const int leader = __ffs(b0) - 1;
    int32_t pos = 0;
    if (lane == leader) pos = atomicAdd(cnt0, __popc(b0));
    pos = __shfl_sync(0xffffffffu, pos, leader);
    if (code == 1) buf0[pos + __popc(b0 & lt)] = v;
  }
  if (b1) {
    const int leader = __ffs(b1) - 1;
    int32_t pos = 0;
    if (lane == leader) pos = atomicAdd(cnt1, __popc(b1));
    pos = __shfl_sync(0xffffffffu, pos, leader);
    if (code == 2) buf1[pos + __popc(b1 & lt)] = v;
  }
}

// Load-balanced advance over frontier Q[0..q) with scanned degrees S[0..q].
// For every edge e = (u, v) of a frontier vertex, f(u, v, e) runs once and
// returns 0 (drop), 1 (append v to out0) or 2 (append v to out1, only when
// NOUT == 2); with NOUT == 0 nothing is appended and the output arguments
// are not used. Column loads are coalesced: consecutive threads take
// consecutive edge ranks. Outputs are compacted per chunk in shared memory
// and appended to the global queues with one atomic per chunk and queue.
// Q == nullptr means the all-vertex frontier (Q[i] = i, S = R, q = n).
template <int THREADS, int ITEMS, int NOUT, class F>
__device__ void lb_advance(const int32_t *R, const int32_t *C, const int32_t *Q, int32_t q,
                           const int32_t *S, F &f, int32_t *out0, int32_t *len0,
                           int32_t *out1, int32_t *len1) {
  constexpr int CHUNK = THREADS * ITEMS;
  const long long total = (long long)q + S[q];
  const long long nchunks = (total + CHUNK - 1) / CHUNK;
  __shared__ int32_t s_off[CHUNK + 1];
  __shared__ int32_t s_u[CHUNK + 1];
  __shared__ int32_t s_row[CHUNK + 1];
  __shared__ int32_t s_out0[NOUT > 0 ? CHUNK : 1];
  __shared__ int32_t s_out1[NOUT == 2 ? CHUNK : 1];
  __shared__ int32_t s_red8[THREADS / 32];
  __shared__ int32_t s_cnt[2], s_base[2];
  for (long long chunk = blockIdx.x; chunk < nchunks; chunk += gridDim.x) {
    const long long d0 = chunk * CHUNK;
    const long long d1 = min(d0 + CHUNK, total);
    if (threadIdx.x < 2) s_cnt[threadIdx.x] = 0;
    int32_t i0, i1;
    block_chunk_bounds<THREADS>(S, q, S[q], d0, d1, CHUNK, s_red8, &i0, &i1);
    const long long j0 = d0 - i0, j1 = d1 - i1;
    const int32_t nv = (i0 <= q - 1) ? (min(i1, q - 1) - i0 + 1) : 0;
    for (int32_t k = threadIdx.x; k < nv; k += THREADS) {
      const int32_t i = i0 + k;
      const int32_t u = Q ? Q[i] : i;
      s_off[k] = S[i];
      s_u[k] = u;
      s_row[k] = Q ? R[u] : S[i];
    }
    __syncthreads();
    const int32_t ne = (int32_t)(j1 - j0);
    for (int32_t kb = 0; kb < ne; kb += THREADS) {
      const int32_t k = kb + threadIdx.x;
      int code = 0;
      int32_t v = 0;
      if (k < ne) {
        const int32_t er = (int32_t)(j0 + k);
        int32_t lo = 0, hi = nv - 1;
        while (lo < hi) {
          const int32_t mid = (lo + hi + 1) >> 1;
          if (s_off[mid] <= er) lo = mid;
          else hi = mid - 1;
        }
        const int32_t e = s_row[lo] + (er - s_off[lo]);
        v = C[e];
        code = f(s_u[lo], v, e);
        if (NOUT < 2 && code == 2) code = 0;
        if (NOUT == 0) code = 0;
      }
      if constexpr (NOUT > 0) warp_append(code, v, s_out0, &s_cnt[0], s_out1, &s_cnt[1]);
    }
    __syncthreads();
    if constexpr (NOUT > 0) {
      if (threadIdx.x < NOUT) {
        const int32_t cnt = s_cnt[threadIdx.x];
        s_base[threadIdx.x] = cnt ? atomicAdd(threadIdx.x ? len1 : len0, cnt) : 0;
      }
      __syncthreads();
      for (int32_t k = threadIdx.x; k < s_cnt[0]; k += THREADS) out0[s_base[0] + k] = s_out0[k];
      if (NOUT == 2)
        for (int32_t k = threadIdx.x; k < s_cnt[1]; k += THREADS) out1[s_base[1] + k] = s_out1[k];
      __syncthreads();
    }
  }
}

}  // namespace gr

namespace gr {

// --------------------------------------------------- neighbourhood reduce
// Gather-reduce over neighbourhoods (the operator the paper proposes in
// Sec. 7 for reductions over neighbour lists): for each vertex v of a set,
// acc[v] = OP over the entries e = (v, u) of v's row of g(u, e).
//
// The set is either a vertex range [v0, v0 + q) (Q == nullptr; S = R + v0,
// so S[i] is the CSR position of vertex v0 + i's row) or a frontier list
// Q[0..q) with its exclusive degree scan S (S[0] = 0, S[q] = its entries).
// Merge-based form: the vertices' end markers and their entries form one
// merged sequence split into equal chunks (as in lb_advance). A block
// stages its chunk's end markers and the gathered values g(C[e], e) of its
// entries in shared memory (coalesced column loads for a range, all gathers
// of the chunk in flight at once); then each thread takes ITEMS consecutive
// items of the chunk, finds its start with one search in shared memory and
// walks them in order, combining values and closing a vertex at each end
// marker. A vertex whose entries lie inside one thread's items is written
// with a plain store; the pieces of a vertex split between threads or chunks
// are combined with OP's atomic. acc[v] must hold OP's identity beforehand
// for every vertex of the set, and a frontier must not repeat a vertex.
template <class T>
struct ReduceSum {
  static __device__ __forceinline__ T identity() { return T(0); }
  static __device__ __forceinline__ T op(T a, T b) { return a + b; }
  static __device__ __forceinline__ void atomic(T *p, T v) { atomicAdd(p, v); }
};
struct ReduceMinI32 {
  static __device__ __forceinline__ int32_t identity() { return INT32_MAX; }
  static __device__ __forceinline__ int32_t op(int32_t a, int32_t b) { return min(a, b); }
  static __device__ __forceinline__ void atomic(int32_t *p, int32_t v) { atomicMin(p, v); }
};
struct ReduceMaxI32 {
  static __device__ __forceinline__ int32_t identity() { return INT32_MIN; }
  static __device__ __forceinline__ int32_t op(int32_t a, int32_t b) { return max(a, b); }
  static __device__ __forceinline__ void atomic(int32_t *p, int32_t v) { atomicMax(p, v); }
};

// cb (vertex ranges only; may be null): the chunk bounds precomputed by
// k_chunk_bounds for this range and chunk size, cb[c] = the members whose
// end marker lies before chunk c, so a chunk needs no search.
template <int THREADS, int ITEMS, class T, class OP, bool FRONTIER, class G>
__device__ void lb_gather_reduce(const int32_t *R, const int32_t *C, const int32_t *Q,
                                 const int32_t *S, int32_t q, int32_t v0, G &g, T *acc,
                                 const int32_t *cb = nullptr) {
  constexpr int CHUNK = THREADS * ITEMS;
  // diagonals are absolute: d + S[0] (the path starts at S[0], the first
  // entry's CSR position for a range, 0 for a frontier)
  const int32_t s0 = S[0];
  const long long total = (long long)q + (S[q] - s0);
  const long long nchunks = (total + CHUNK - 1) / CHUNK;
  __shared__ int32_t s_end[CHUNK + 1];  // end marker of each vertex, chunk-local
  __shared__ T s_val[CHUNK];
  __shared__ int32_t s_off[FRONTIER ? CHUNK + 1 : 1];  // frontier: the vertices' scan values
  __shared__ int32_t s_row[FRONTIER ? CHUNK + 1 : 1];  // frontier: their row starts
  __shared__ int32_t s_red8[THREADS / 32];
  (void)s_off;
  (void)s_row;
  for (long long chunk = blockIdx.x; chunk < nchunks; chunk += gridDim.x) {
    const long long d0 = chunk * CHUNK + s0;
    const long long d1 = min(chunk * CHUNK + CHUNK, total) + s0;
    int32_t i0, i1;
    if (!FRONTIER && cb) {
      i0 = cb[chunk];
      i1 = cb[chunk + 1];
    } else {
      block_chunk_bounds<THREADS>(S, q, S[q], d0, d1, CHUNK, s_red8, &i0, &i1);
    }
    const long long j0 = d0 - i0, j1 = d1 - i1;  // entries [j0, j1) (scan positions)
    const int32_t nv = (i0 <= q - 1) ? (min(i1, q - 1) - i0 + 1) : 0;
    const int32_t ne = (int32_t)(j1 - j0);
    const int32_t len = (int32_t)(d1 - d0);
    for (int32_t k = threadIdx.x; k < nv; k += THREADS) {
      s_end[k] = (int32_t)((long long)S[i0 + k + 1] + i0 + k - d0);
      if (FRONTIER) {
        s_off[k] = S[i0 + k];
        s_row[k] = R[Q[i0 + k]];
      }
    }
    if (FRONTIER) __syncthreads();
    {
      // all column loads of the thread first, then all gathers: ITEMS
      // independent gathers in flight per thread
      int32_t col[ITEMS], pos[ITEMS];
#pragma unroll
      for (int i = 0; i < ITEMS; ++i) {
        const int32_t k = threadIdx.x + i * THREADS;
        pos[i] = 0;
        if (k < ne) {
          if (FRONTIER) {
            const int32_t er = (int32_t)(j0 + k);  // rank in the frontier's entries
            int32_t lo = 0, hi = nv - 1;
            while (lo < hi) {
              const int32_t mid = (lo + hi + 1) >> 1;
              if (s_off[mid] <= er) lo = mid;
              else hi = mid - 1;
            }
            pos[i] = s_row[lo] + (er - s_off[lo]);
          } else {
            pos[i] = (int32_t)(j0 + k);
          }
        }
        col[i] = k < ne ? C[pos[i]] : 0;
      }
#pragma unroll
      for (int i = 0; i < ITEMS; ++i) {
        const int32_t k = threadIdx.x + i * THREADS;
        if (k < ne) s_val[k] = g(col[i], pos[i]);
      }
    }
    __syncthreads();
    // this thread's items [k0, k1) of the chunk
    const int32_t k0 = min(len, (int32_t)threadIdx.x * ITEMS);
    const int32_t k1 = min(len, k0 + ITEMS);
    if (k0 < k1) {
      // vertices whose end marker lies before k0
      int32_t lo = 0, hi = nv;
      while (lo < hi) {
        const int32_t mid = (lo + hi) >> 1;
        if (s_end[mid] < k0) lo = mid + 1;
        else hi = mid;
      }
      int32_t r = lo;
      int32_t e = k0 - r;   // chunk-local entry index
      T red = OP::identity();
      bool first = true;    // the current vertex may have entries before k0
      for (int32_t k = k0; k < k1; ++k) {
        if (r < nv && s_end[r] == k) {  // end marker of set member i0 + r
          const int32_t v = FRONTIER ? Q[i0 + r] : v0 + i0 + r;
          if (red != OP::identity()) {
            if (first) OP::atomic(acc + v, red);
            else acc[v] = red;
          }
          red = OP::identity();
          first = false;
          ++r;
        } else {
          red = OP::op(red, s_val[e]);
          ++e;
        }
      }
      if (red != OP::identity() && r < nv)  // continues past k1
        OP::atomic(acc + (FRONTIER ? Q[i0 + r] : v0 + i0 + r), red);
    }
    __syncthreads();
  }
}

// All vertices, summed (PageRank's gather): acc[v] += sum of g over v's row.
template <int THREADS, int ITEMS, class T, class G>
__device__ __forceinline__ void lb_neighbor_reduce(const int32_t *R, const int32_t *C, int32_t n,
                                                   G &g, T *acc, const int32_t *cb = nullptr) {
  lb_gather_reduce<THREADS, ITEMS, T, ReduceSum<T>, false>(R, C, nullptr, R, n, 0, g, acc, cb);
}

// Chunk bounds of the merge path over a vertex range (S = R + v0, q
// members, entries S[0] .. S[q]) in chunks of `chunk` items:
// cb[c] = the number of members whose end marker S[i+1] + i lies before
// c * chunk + S[0] (the path's absolute diagonal), c in [0, chunks), and
// cb[chunks] = q. One thread per chunk, a binary search each.
static __global__ void k_chunk_bounds(const int32_t *S, int32_t q, int32_t chunk,
                                      int32_t chunks, int32_t *cb) {
  const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (c > chunks) return;
  if (c == chunks) {
    cb[c] = q;
    return;
  }
  const long long d = c * (long long)chunk + S[0];
  int32_t lo = 0, hi = q;  // first member whose end marker is not before d
  while (lo < hi) {
    const int32_t mid = (int32_t)(((long long)lo + hi) >> 1);
    if ((long long)S[mid + 1] + mid < d) lo = mid + 1;
    else hi = mid;
  }
  cb[c] = lo;
}

// Sets kernel f's shared-memory carveout to the smallest share of the SM's
// unified L1/shared-memory array that holds `blocks` resident blocks of it,
// leaving the rest to the L1 cache (the gather-reduce's random reads of
// neighbour values hit there), and reports the resident blocks per SM that
// the occupancy calculator then allows for `threads`-thread blocks.
template <class K>
static gr_status fit_carveout(K f, int threads, int blocks, int device, int *per_sm) {
  cudaFuncAttributes fa;
  GR_CUDA(cudaFuncGetAttributes(&fa, f));
  int max_sm = 0, reserved = 0;
  GR_CUDA(cudaDeviceGetAttribute(&max_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, device));
  GR_CUDA(cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, device));
  const long long need = (long long)blocks * ((long long)fa.sharedSizeBytes + reserved);
  const int pct = max_sm > 0 ? (int)std::min<long long>(100, (need * 100 + max_sm - 1) / max_sm)
                             : (int)cudaSharedmemCarveoutDefault;
  GR_CUDA(cudaFuncSetAttribute(f, cudaFuncAttributePreferredSharedMemoryCarveout, pct));
  GR_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, f, threads, 0));
  if (*per_sm < 1) *per_sm = 1;
  if (*per_sm > blocks) *per_sm = blocks;
  return GR_OK;
}

// Chunks of the merge path over q members whose entries span S[0] .. S[q].
__host__ __device__ __forceinline__ int32_t merge_chunks(int32_t q, long long entries,
                                                         int32_t chunk) {
  return (int32_t)(((long long)q + entries + chunk - 1) / chunk);
}

}  // namespace gr

namespace gr {

// ------------------------------------------- scanned frontier emission
// A block-local buffer of newly produced frontier vertices and their
// degrees. flush_scanned writes it to a queue Qn together with the queue's
// exclusive degree scan Sn (the scanned edge offsets the next advance
// needs), reserving both ranges with one atomicAdd on a packed counter
// ([31:0] vertices, [63:32] edges), so queue order and scan order agree and
// no separate scan pass is needed.
template <int CAP>
struct ScannedBuf {
  int32_t out[CAP];
  int32_t deg[CAP];
  int32_t cnt;
  int32_t vbase, ebase;
  uint32_t red[33];
};

template <int CAP>
__device__ __forceinline__ void emit_scanned(ScannedBuf<CAP> &b, bool take, int32_t v,
                                             int32_t d) {
  const int lane = threadIdx.x & 31;
  const uint32_t bal = __ballot_sync(0xffffffffu, take);
  if (!bal) return;
  const int leader = __ffs(bal) - 1;
  int32_t pos = 0;
  if (lane == leader) pos = atomicAdd(&b.cnt, __popc(bal));
  pos = __shfl_sync(0xffffffffu, pos, leader);
  if (take) {
    const int32_t k = pos + __popc(bal & ((1u << lane) - 1u));
    b.out[k] = v;
    b.deg[k] = d;
  }
}

// Block-uniform call; leaves b.cnt = 0.
template <int THREADS, int CAP>
__device__ void flush_scanned(ScannedBuf<CAP> &b, unsigned long long *packed, int32_t *Qn,
                              int32_t *Sn, long long cap = (1ll << 62)) {
  static_assert(CAP % THREADS == 0, "buffer must split evenly over the block");
  constexpr int PER = CAP / THREADS;
  __syncthreads();
  const int32_t cnt = b.cnt;
  if (cnt) {
    const int32_t k0 = threadIdx.x * PER;
    uint32_t local = 0;
#pragma unroll
    for (int j = 0; j < PER; ++j)
      if (k0 + j < cnt) local += (uint32_t)b.deg[k0 + j];
    uint32_t total;
    uint32_t run = block_excl_sum(local, b.red, &total);
    if (threadIdx.x == 0) {
      const unsigned long long old =
          atomicAdd(packed, ((unsigned long long)total << 32) | (unsigned long long)cnt);
      b.vbase = (int32_t)(old & 0xFFFFFFFFull);
      b.ebase = (int32_t)(old >> 32);
    }
    __syncthreads();
    const int32_t vb = b.vbase, eb = b.ebase;
#pragma unroll
    for (int j = 0; j < PER; ++j) {
      const int32_t k = k0 + j;
      if (k < cnt) {
        if (GR_IN(vb + k, cap, 501)) {
          Qn[vb + k] = b.out[k];
          Sn[vb + k] = eb + (int32_t)run;
        }
        run += (uint32_t)b.deg[k];
      }
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) b.cnt = 0;
  __syncthreads();
}

// A plain block-local append buffer (no degrees), flushed with one
// atomicAdd on a length counter.
template <int CAP>
struct AppendBuf {
  int32_t out[CAP];
  int32_t cnt;
  int32_t base;
};

template <int CAP>
__device__ __forceinline__ void emit_plain(AppendBuf<CAP> &b, bool take, int32_t v) {
  const int lane = threadIdx.x & 31;
  const uint32_t bal = __ballot_sync(0xffffffffu, take);
  if (!bal) return;
  const int leader = __ffs(bal) - 1;
  int32_t pos = 0;
  if (lane == leader) pos = atomicAdd(&b.cnt, __popc(bal));
  pos = __shfl_sync(0xffffffffu, pos, leader);
  if (take) b.out[pos + __popc(bal & ((1u << lane) - 1u))] = v;
}

template <int THREADS, int CAP>
__device__ void flush_plain(AppendBuf<CAP> &b, int32_t *len, int32_t *Q,
                            long long cap = (1ll << 62)) {
  __syncthreads();
  const int32_t cnt = b.cnt;
  if (threadIdx.x == 0 && cnt) b.base = atomicAdd(len, cnt);
  __syncthreads();
  for (int32_t k = threadIdx.x; k < cnt; k += THREADS)
    if (GR_IN((long long)b.base + k, cap, 502)) Q[b.base + k] = b.out[k];
  __syncthreads();
  if (threadIdx.x == 0) b.cnt = 0;
  __syncthreads();
}

}  // namespace gr

namespace gr {

// ------------------------------------------------------------ grid barrier
// Barrier of the persistent (cooperative) kernels. Blocks arrive at one of
// kBarrierGroups group counters; a group's last arriver clears it and
// arrives at the root; the root's last arriver releases everyone by bumping
// the generation (grids of at most kFlatBarrierBlocks blocks arrive at the
// root directly). Every counter sits on its own 128-byte line so that the
// waiters' polling does not slow the arrivals. The wait is bounded: after
// kSpinLimit polls the block records kDevTimeout in *error and returns
// false (callers then leave their loop; the other blocks time out too).
constexpr int kBarrierGroups = 16;
constexpr int kFlatBarrierBlocks = 256;  // grids up to this size use a one-level barrier

struct alignas(128) BarrierLine {
  int32_t v;
};

// A value the releasing block publishes with the release: two 64-bit words,
// each [63:32] the barrier's generation and [31:0] one half of the value, so a
// waiter that sees both tags equal to the generation it waits for holds the
// value without another round trip (each word is read atomically).
struct alignas(128) PayloadLine {
  unsigned long long w[2];
};

struct GridBarrier {
  BarrierLine group[kBarrierGroups];
  BarrierLine root;
  BarrierLine gen;
  PayloadLine pay;
};

__device__ __forceinline__ void grid_barrier_reset(GridBarrier *b) {
  for (int i = 0; i < kBarrierGroups; ++i) b->group[i].v = 0;
  b->root.v = 0;
  b->gen.v = 0;
  b->pay.w[0] = 0ull;
  b->pay.w[1] = 0ull;
}

// `gen` is the block's private count of barriers passed (starts at 0).
// With pay_src, the releasing block reads *pay_src (a 64-bit value every
// block finished writing before it arrived) and publishes it with the
// release; every block receives it in *pay_out.
__device__ __forceinline__ bool grid_sync(GridBarrier *b, int32_t *error, int32_t &gen,
                                          const unsigned long long *pay_src = nullptr,
                                          unsigned long long *pay_out = nullptr) {
  __syncthreads();
  bool ok = true;
  __shared__ int32_t s_ok;
  __shared__ unsigned long long s_pay;
  if (threadIdx.x == 0) {
    __threadfence();
    const int32_t nblocks = gridDim.x;
    const int32_t my_gen = gen;
    bool release = false;
    if (nblocks <= kFlatBarrierBlocks) {
      // small grids: every block arrives at the root directly (one atomic
      // round trip less than the two-level form)
      if (atomicAdd(&b->root.v, 1) == nblocks - 1) {
        b->root.v = 0;
        __threadfence();
        release = true;
      }
    } else {
      const int32_t grp = blockIdx.x % kBarrierGroups;
      const int32_t members = (nblocks - grp + kBarrierGroups - 1) / kBarrierGroups;
      const int32_t groups = min(nblocks, kBarrierGroups);
      if (atomicAdd(&b->group[grp].v, 1) == members - 1) {
        b->group[grp].v = 0;
        __threadfence();
        if (atomicAdd(&b->root.v, 1) == groups - 1) {
          b->root.v = 0;
          __threadfence();
          release = true;
        }
      }
    }
    const unsigned long long tag = (unsigned long long)(uint32_t)(my_gen + 1) << 32;
    if (release) {
      if (pay_src) {
        const unsigned long long v = *(const volatile unsigned long long *)pay_src;
        s_pay = v;
        volatile unsigned long long *pw = b->pay.w;
        pw[0] = tag | (v & 0xFFFFFFFFull);
        pw[1] = tag | (v >> 32);
        __threadfence();
      }
      atomicExch(&b->gen.v, my_gen + 1);
    } else {
      int64_t spins = 0;
      unsigned ns = 32;
      for (;;) {
        if (pay_src) {
          const volatile unsigned long long *pw = b->pay.w;
          const unsigned long long w0 = pw[0], w1 = pw[1];
          if ((w0 & ~0xFFFFFFFFull) == tag && (w1 & ~0xFFFFFFFFull) == tag) {
            s_pay = (w0 & 0xFFFFFFFFull) | (w1 << 32);
            break;
          }
        } else if (*(volatile int32_t *)&b->gen.v != my_gen) {
          break;
        }
        if (++spins > kSpinLimit) {
          atomicExch(error, kDevTimeout);
          ok = false;
          break;
        }
        __nanosleep(ns);
        ns = ns < 256 ? ns * 2 : 256;
      }
    }
    __threadfence();
    s_ok = ok;
  }
  gen += 1;
  __syncthreads();
  if (pay_out) *pay_out = s_pay;
  return s_ok != 0;
}

}  // namespace gr
