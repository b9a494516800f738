// Single-source shortest paths with a near/far frontier split (Alg. 1,
// Sec. 4.5 "Priority queue", Sec. 5.2).
//
// Alg. 1 initialises labels to infinity and label[root] = 0, then loops
// advance (UpdateLabel = atomicMin relaxation), filter (RemoveRedundant, an
// output-queue stamp per vertex) and the priority-queue split until the
// frontier is empty. Here one iteration of the device-side loop is ONE
// kernel, k_sssp_iter, in one of three modes chosen on the device:
//
//   relax  load-balanced advance over the near frontier (merge-path chunks
//          over its vertex ends and edge ranks, Sec. 4.4); per edge
//          new = dist[u] + w(e), atomicMin on dist[v]; an improved v joins
//          the next near frontier if new < T (deduplicated by a
//          per-iteration stamp, the RemoveRedundant filter) and the far pile
//          otherwise (deduplicated by a per-phase stamp)
//   pull   the relaxation in pull form (direction-optimising SSSP, which
//          the paper names for future work in Sec. 4.5 and Sec. 7), for
//          near frontiers holding most of the edges on a symmetric graph:
//          every vertex takes the minimum of dist[u] + w(e) over its
//          in-edges (= its row) and keeps it if lower, so no atomic is
//          needed except for vertices whose row is split between threads;
//          the improved vertices go to near / far exactly as in relax
//   split  only when the near frontier is empty: the far pile is split by
//          the raised threshold into near and far; entries whose distance
//          fell below the old threshold were already expanded and are
//          dropped
//
// New near vertices are emitted with their degree scan (one packed atomic
// per block), so no scan pass separates two iterations. The last block of
// an iteration swaps the buffers, raises T (jumping to the bucket of the
// smallest far distance when the next bucket would be empty) and ends the
// loop when both piles are empty.
//
// T starts at delta and grows by delta per phase (delta = UINT32_MAX: one
// bucket, i.e. plain frontier relaxation). Distances do not depend on delta.
// An optional last pass fills pred[v] with the smallest u that has an edge
// (u, v) with dist[u] + w = dist[v].
//
// Batched form (gr_sssp_batch): k sources run as ONE search over k disjoint
// copies of the graph. Vertex id l*n + v stands for vertex v in copy
// (lane) l: its row is row v of the CSR, its neighbours are l*n + C[e], and
// dist / stamps / queues are indexed by the lane-major id. Copy l holds
// only source l, and no edge joins two copies, so each lane's distances are
// exactly those of a search from its own source; the lanes share the
// threshold T and the device-side loop, so k high-diameter searches cost
// about as many iterations as one.
#include <algorithm>
#include <climits>
#include <cstring>

#include "advance.cuh"

namespace gr {

enum : int32_t { kSsspRelax = 0, kSsspSplit = 1, kSsspPull = 2 };

struct SsspCtl {
  uint32_t *dist;
  int32_t *pred;
  int32_t src;
  int32_t mode;          // kSsspRelax / kSsspSplit / kSsspPull for the current iteration
  int32_t near_parity;   // which near buffer holds the current frontier
  int32_t far_parity;    // which far buffer holds the current pile
  int32_t near_len;
  int32_t far_len;        // atomic (relax appends to the current pile)
  int32_t far_next_len;   // atomic (split output)
  int32_t done;
  int32_t error;
  int32_t iter;           // iteration id, also the near-frontier stamp
  int32_t far_epoch;      // far-pile stamp
  int32_t max_iters;
  int32_t phases;         // number of splits
  int32_t pad_;
  uint32_t far_min;       // lower bound of far-pile distances (atomicMin)
  uint32_t far_min_next;  // min distance of entries kept by a split
  unsigned long long near_next_packed;  // [31:0] next near size, [63:32] its edges
  // iteration-kernel blocks finished so far in this run; the block whose
  // arrival makes it a multiple of the grid size ends the iteration
  unsigned long long arrivals;
  unsigned long long T;   // near criterion: dist < T
  unsigned long long T_old;
  unsigned long long delta;
  long long near_edges;   // edges of the current near frontier
  long long relaxations;  // edges expanded (statistics)
  // a relaxation whose near frontier has at least this many edges runs in
  // pull form (LLONG_MAX: never; pull needs a symmetric CSR and one lane)
  long long pull_min_edges;
  int32_t pulls;          // relaxations run in pull form (statistics)
  int32_t pad2_;
  // persistent kernel: counter rings and grid barrier
  unsigned long long ring_near[3];
  int32_t ring_far[3];
  uint32_t ring_fmin[3];
  GridBarrier bar;
};

struct SsspArgs {
  const int32_t *R;
  const int32_t *C;
  const uint32_t *W;
  int32_t n;
  int32_t nv;  // vertex ids in use: lanes * n (lane-major copies of the graph)
  long long m;
  int32_t *nearq[2];
  int32_t *nearS[2];
  int32_t *farq[2];
  int32_t *stamp;
  int32_t *far_stamp;
  SsspCtl *ctl;
  int32_t low_degree;  // graph of small maximum degree: per-thread relaxation
  const int32_t *cb;   // chunk bounds of the pull relaxation's all-vertex merge path
  int32_t *qcb;        // room for the chunk bounds of a dense near frontier (or null)
};

constexpr int kSsspThreads = 256, kSsspItems = 4;
constexpr int kSsspChunk = kSsspThreads * kSsspItems;
constexpr int kSsspBlocksPerSm = 5;
// Largest maximum degree for which relaxation takes one frontier vertex per
// thread (mesh-like graphs), and the neighbours a thread loads at once.
constexpr int32_t kSsspLowDegreeMax = 16;
constexpr int kSsspTpvItems = 4;
// A persistent relaxation first finds every chunk's bounds in one pass once
// its frontier has at least this many chunks per block.
constexpr int kSsspBoundsChunksPerBlock = 4;
// Most sources one batched run takes.
constexpr int32_t kSsspMaxLanes = 64;

struct SsspWorkspace {
  int32_t lanes = 1;  // copies of the graph the buffers hold (batched form)
  DevMem nearq[2], nearS[2], farq[2], stamp, far_stamp, ctl;
  DevMem cb;  // chunk bounds of the pull relaxation (single search; fixed per graph)
  DevMem qcb;  // chunk bounds of a dense near frontier (persistent driver)
  cudaGraphExec_t exec = nullptr;
  cudaGraph_t graph = nullptr;
  ~SsspWorkspace() {
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
  }
};

void free_sssp(SsspWorkspace *ws) { delete ws; }

GR_GUARD_REPORTER(guard_report_sssp)

namespace {

__device__ __forceinline__ int32_t *pick(int32_t *const *a, int p) { return p ? a[1] : a[0]; }

// First id of the graph copy that lane-major id x lies in (0 for one lane).
__device__ __forceinline__ int32_t lane_base(int32_t x, int32_t n) {
  return x >= n ? x - x % n : 0;
}

// Sources of one run: lane l starts at vertex s[l] (id l*n + s[l]).
struct SsspSources {
  int32_t k;
  int32_t s[kSsspMaxLanes];
};

__global__ void k_sssp_init(SsspArgs a, SsspSources src, uint32_t *dist, int32_t *pred,
                            unsigned long long delta, int32_t max_iters,
                            long long pull_min_edges) {
  const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t v = tid; v < a.nv; v += stride) {
    const int32_t x = (int32_t)v;
    const int32_t base = lane_base(x, a.n);
    dist[v] = x - base == src.s[base ? base / a.n : 0] ? 0u : 0xFFFFFFFFu;
    a.stamp[v] = -1;
    a.far_stamp[v] = -1;
  }
  if (tid == 0) {
    SsspCtl *c = a.ctl;
    // the initial near frontier: every lane's source with its degree scan
    int32_t edges = 0;
    for (int32_t l = 0; l < src.k; ++l) {
      const int32_t u = src.s[l];
      a.nearq[0][l] = l * a.n + u;
      a.nearS[0][l] = edges;
      edges += a.R[u + 1] - a.R[u];
    }
    a.nearS[0][src.k] = edges;
    c->dist = dist;
    c->pred = pred;
    c->src = src.s[0];
    c->mode = kSsspRelax;
    c->near_parity = 0;
    c->far_parity = 0;
    c->near_len = src.k;
    c->far_len = 0;
    c->far_next_len = 0;
    c->done = 0;
    c->error = kDevOk;
    c->iter = 0;
    c->far_epoch = 0;
    c->max_iters = max_iters;
    c->phases = 0;
    c->arrivals = 0ull;
    c->far_min = 0xFFFFFFFFu;
    c->far_min_next = 0xFFFFFFFFu;
    c->near_next_packed = 0ull;
    c->delta = delta;
    c->T = delta;
    c->T_old = 0;
    c->near_edges = edges;
    c->relaxations = 0;
    c->pull_min_edges = pull_min_edges;
    c->pulls = 0;
    for (int i = 0; i < 3; ++i) {
      c->ring_near[i] = 0ull;
      c->ring_far[i] = 0;
      c->ring_fmin[i] = 0xFFFFFFFFu;
    }
    grid_barrier_reset(&c->bar);
  }
}

struct SsspSmem {
  int32_t off[kSsspChunk + 1];
  uint32_t du[kSsspChunk + 1];
  int32_t row[kSsspChunk + 1];
  int32_t base[kSsspChunk + 1];  // first id of the vertex's graph copy
  ScannedBuf<kSsspChunk> nearb;
  AppendBuf<kSsspChunk> farb;
  int32_t i[2];
  int32_t sred[kSsspThreads / 32];
  int32_t last;
};

// The state one iteration reads and the counters it fills; the graph-mode
// kernel takes them from the control block, the persistent kernel from
// block-private copies and a ring of counters.
struct SsspStep {
  int32_t near_parity, far_parity;
  int32_t q;              // near frontier size
  int32_t q_edges;        // its edges (S[q])
  int32_t far_len;        // current far pile size (split input)
  unsigned long long T, T_old;
  int32_t iter, far_epoch;
  unsigned long long *near_ctr;  // packed (vertices, edges) of the next near frontier
  int32_t *far_ctr;              // far appends (relax) or far-next size (split)
  int32_t *far_dest;             // where far appends land (pile start + base)
  long long far_cap;             // entries available at far_dest
  uint32_t *fmin;                // min distance sent to the far pile
};

// The merge-path chunk bounds of a near frontier (q members, exclusive
// degree scan S[0..q), s_q entries in all: S[q] itself is not stored),
// grid-stride: cb[c] = the members whose end marker S[i + 1] + i lies before
// c * kSsspChunk, cb[nchunks] = q.
__device__ void frontier_chunk_bounds(const int32_t *S, int32_t q, int32_t s_q,
                                      long long nchunks, int32_t *cb) {
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c <= nchunks;
       c += (long long)gridDim.x * blockDim.x) {
    if (c == nchunks) {
      cb[c] = q;
      continue;
    }
    const long long d = c * kSsspChunk;
    int32_t lo = 0, hi = q;  // first member whose end marker is not before d
    while (lo < hi) {
      const int32_t mid = (int32_t)(((long long)lo + hi) >> 1);
      const int32_t sv = mid + 1 == q ? s_q : S[mid + 1];
      if ((long long)sv + mid < d) lo = mid + 1;
      else hi = mid;
    }
    cb[c] = lo;
  }
}

// qcb (may be null): the frontier's chunk bounds, computed for this
// iteration by frontier_chunk_bounds, so a chunk needs no search.
__device__ void relax_body(const SsspArgs &a, uint32_t *dist, SsspSmem &sm, const SsspStep &st,
                           const int32_t *qcb = nullptr) {
  const int32_t np = st.near_parity;
  const int32_t *Q = pick(a.nearq, np);
  const int32_t *S = pick(a.nearS, np);
  int32_t *Qn = pick(a.nearq, np ^ 1);
  int32_t *Sn = pick(a.nearS, np ^ 1);
  const int32_t q = st.q;
  const unsigned long long T = st.T;
  const int32_t iter = st.iter, epoch = st.far_epoch;
  const long long total = (long long)q + st.q_edges;
  const long long nchunks = (total + kSsspChunk - 1) / kSsspChunk;
  for (long long chunk = blockIdx.x; chunk < nchunks; chunk += gridDim.x) {
    const long long d0 = chunk * kSsspChunk;
    const long long d1 = min(d0 + kSsspChunk, total);
    int32_t i0, i1;
    if (qcb) {
      i0 = qcb[chunk];
      i1 = qcb[chunk + 1];
    } else {
      block_chunk_bounds<kSsspThreads>(S, q, st.q_edges, d0, d1, kSsspChunk, sm.sred, &i0, &i1);
    }
    const long long j0 = d0 - i0, j1 = d1 - i1;
    const int32_t nv = (i0 <= q - 1) ? (min(i1, q - 1) - i0 + 1) : 0;
    // per chunk vertex: its scan offset, its row start and its distance (read
    // once here instead of once per edge)
    for (int32_t k = threadIdx.x; k < nv; k += kSsspThreads) {
      const int32_t i = i0 + k;
      const int32_t u0 = GR_IN(i, a.nv + 1, 301) ? Q[i] : 0;
      const int32_t u = GR_IN(u0, a.nv, 303) ? u0 : 0;
      const int32_t ub = lane_base(u, a.n);
      sm.off[k] = GR_IN(i, a.nv + 2, 302) ? S[i] : 0;
      sm.row[k] = a.R[u - ub];
      sm.base[k] = ub;
      sm.du[k] = dist[u];
    }
    __syncthreads();
    // each thread takes kSsspItems edges (ranks tid, tid + T, ...) and issues
    // each step's loads (heads and weights, head distances, atomicMin, stamps,
    // degrees) for all of them before using any, so the latency chains of the
    // items overlap
    const int32_t ne = (int32_t)(j1 - j0);  // <= kSsspChunk: one pass
    int32_t e[kSsspItems], v[kSsspItems], vl[kSsspItems], vb[kSsspItems], code[kSsspItems],
        dv[kSsspItems];
    uint32_t wt[kSsspItems], du[kSsspItems], nd[kSsspItems], cur[kSsspItems];
#pragma unroll
    for (int j = 0; j < kSsspItems; ++j) {
      const int32_t k = j * kSsspThreads + threadIdx.x;
      e[j] = -1;
      vb[j] = 0;
      du[j] = 0xFFFFFFFFu;
      if (k < ne) {
        const int32_t er = (int32_t)(j0 + k);
        int32_t lo = 0, hi = nv - 1;
        while (lo < hi) {
          const int32_t mid = (lo + hi + 1) >> 1;
          if (sm.off[mid] <= er) lo = mid;
          else hi = mid - 1;
        }
        const int32_t ee = sm.row[lo] + (er - sm.off[lo]);
        if (GR_IN(ee, a.m, 304)) {
          e[j] = ee;
          vb[j] = sm.base[lo];
          du[j] = sm.du[lo];
        }
      }
    }
#pragma unroll
    for (int j = 0; j < kSsspItems; ++j) {
      vl[j] = e[j] >= 0 ? a.C[e[j]] : -1;
      wt[j] = e[j] >= 0 ? a.W[e[j]] : 0u;
    }
#pragma unroll
    for (int j = 0; j < kSsspItems; ++j) {
      nd[j] = 0xFFFFFFFFu;  // not representable below 0xFFFFFFFF: no improvement
      if (vl[j] >= 0 && !GR_IN(vl[j], a.n, 305)) vl[j] = -1;
      v[j] = vl[j] >= 0 ? vb[j] + vl[j] : -1;  // the neighbour in the same copy
      if (v[j] >= 0) {
        const unsigned long long t = (unsigned long long)du[j] + wt[j];
        if (t < 0xFFFFFFFFull) nd[j] = (uint32_t)t;
      }
    }
#pragma unroll
    for (int j = 0; j < kSsspItems; ++j)
      cur[j] = nd[j] != 0xFFFFFFFFu ? dist[v[j]] : 0u;  // plain-load cull
#pragma unroll
    for (int j = 0; j < kSsspItems; ++j) {
      const bool try_it = nd[j] < cur[j];
      cur[j] = try_it ? atomicMin(dist + v[j], nd[j]) : 0u;
      if (!try_it) nd[j] = 0xFFFFFFFFu;
    }
#pragma unroll
    for (int j = 0; j < kSsspItems; ++j) {
      code[j] = 0;
      if (nd[j] < cur[j]) {  // this thread lowered dist[v]
        if (nd[j] < T) {
          code[j] = atomicExch(a.stamp + v[j], iter) != iter ? 1 : 0;
        } else {
          atomicMin(st.fmin, nd[j]);
          code[j] = atomicExch(a.far_stamp + v[j], epoch) != epoch ? 2 : 0;
        }
      }
    }
#pragma unroll
    for (int j = 0; j < kSsspItems; ++j)
      dv[j] = code[j] == 1 ? a.R[vl[j] + 1] - a.R[vl[j]] : 0;
#pragma unroll
    for (int j = 0; j < kSsspItems; ++j) {
      emit_scanned(sm.nearb, code[j] == 1, v[j], dv[j]);
      emit_plain(sm.farb, code[j] == 2, v[j]);
    }
    flush_scanned<kSsspThreads>(sm.nearb, st.near_ctr, Qn, Sn, a.nv + 1);
    flush_plain<kSsspThreads>(sm.farb, st.far_ctr, st.far_dest, st.far_cap);
  }
}

// Relaxation for graphs of small maximum degree (meshes): one thread per
// near-frontier vertex relaxes its whole neighbour list (the per-thread
// expansion of Sec. 4.4, balanced when every degree is small), so no
// merge-path search is needed. Each candidate's row offsets are loaded with
// its distance, so a vertex entering the near frontier brings its degree (for
// the frontier's edge count) without an extra round trip. Near and far
// entries are appended with one atomic per warp each.
__device__ void relax_body_thread(const SsspArgs &a, uint32_t *dist, const SsspStep &st) {
  const int32_t *Q = pick(a.nearq, st.near_parity);
  int32_t *Qn = pick(a.nearq, st.near_parity ^ 1);
  const int32_t q = st.q;
  const unsigned long long T = st.T;
  const int32_t iter = st.iter, epoch = st.far_epoch;
  const int lane = threadIdx.x & 31;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t qr = ((int64_t)q + 31) & ~31ll;  // warp-uniform bound
  uint32_t local_min = 0xFFFFFFFFu;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < qr; i += stride) {
    int32_t u = 0, ub = 0, r0 = 0, r1 = 0;
    uint32_t du = 0xFFFFFFFFu;
    if (i < q && GR_IN(i, a.nv + 1, 320)) {
      u = Q[i];
      if (GR_IN(u, a.nv, 321)) {
        ub = lane_base(u, a.n);
        r0 = a.R[u - ub];
        r1 = a.R[u - ub + 1];
        du = dist[u];
      }
    }
    for (int32_t e0 = r0; __any_sync(0xffffffffu, e0 < r1); e0 += kSsspTpvItems) {
      int32_t v[kSsspTpvItems], d0[kSsspTpvItems], d1[kSsspTpvItems];
      uint32_t w[kSsspTpvItems], dv[kSsspTpvItems];
      int code[kSsspTpvItems];
#pragma unroll
      for (int j = 0; j < kSsspTpvItems; ++j) {
        const int32_t e = e0 + j;
        v[j] = -1;
        w[j] = 0u;
        if (e < r1 && GR_IN(e, a.m, 322)) {
          v[j] = a.C[e];
          w[j] = a.W[e];
          if (!GR_IN(v[j], a.n, 323)) v[j] = -1;
        }
      }
#pragma unroll
      for (int j = 0; j < kSsspTpvItems; ++j) {
        dv[j] = 0u;
        d0[j] = d1[j] = 0;
        if (v[j] >= 0) {
          d0[j] = a.R[v[j]];
          d1[j] = a.R[v[j] + 1];
          v[j] += ub;  // from here on: the neighbour's id in u's copy
          dv[j] = dist[v[j]];
        }
      }
      uint32_t ncnt = 0, ndeg = 0, fcnt = 0;
#pragma unroll
      for (int j = 0; j < kSsspTpvItems; ++j) {
        code[j] = 0;
        if (v[j] < 0) continue;
        const unsigned long long nd = (unsigned long long)du + w[j];
        if (nd >= 0xFFFFFFFFull) continue;  // not representable: no improvement
        const uint32_t nd32 = (uint32_t)nd;
        if (nd32 >= dv[j]) continue;  // plain-load cull
        const uint32_t old = atomicMin(dist + v[j], nd32);
        if (nd32 >= old) continue;
        if (nd < T) {
          if (atomicExch(a.stamp + v[j], iter) != iter) {
            code[j] = 1;
            ncnt += 1;
            ndeg += (uint32_t)(d1[j] - d0[j]);
          }
        } else {
          local_min = min(local_min, nd32);
          if (atomicExch(a.far_stamp + v[j], epoch) != epoch) {
            code[j] = 2;
            fcnt += 1;
          }
        }
      }
      // near: warp scan of (edges, vertices), one packed atomic
      const unsigned long long nmine = ((unsigned long long)ndeg << 32) | ncnt;
      unsigned long long nincl = nmine;
      uint32_t fincl = fcnt;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long t = __shfl_up_sync(0xffffffffu, nincl, o);
        const uint32_t tf = __shfl_up_sync(0xffffffffu, fincl, o);
        if (lane >= o) {
          nincl += t;
          fincl += tf;
        }
      }
      const unsigned long long ntot = __shfl_sync(0xffffffffu, nincl, 31);
      const uint32_t ftot = __shfl_sync(0xffffffffu, fincl, 31);
      unsigned long long nbase = 0;
      int32_t fbase = 0;
      if (lane == 0) {
        if (ntot) nbase = atomicAdd(st.near_ctr, ntot);
        if (ftot) fbase = atomicAdd(st.far_ctr, (int32_t)ftot);
      }
      nbase = __shfl_sync(0xffffffffu, nbase, 0);
      fbase = __shfl_sync(0xffffffffu, fbase, 0);
      int32_t kn = (int32_t)((nbase + (nincl - nmine)) & 0xFFFFFFFFull);
      long long kf = (long long)fbase + (fincl - fcnt);
#pragma unroll
      for (int j = 0; j < kSsspTpvItems; ++j) {
        if (code[j] == 1) {
          if (GR_IN(kn, a.nv + 1, 324)) Qn[kn] = v[j];
          ++kn;
        } else if (code[j] == 2) {
          if (GR_IN(kf, st.far_cap, 325)) st.far_dest[kf] = v[j];
          ++kf;
        }
      }
    }
  }
  for (int o = 16; o > 0; o >>= 1) local_min = min(local_min, __shfl_xor_sync(0xffffffffu, local_min, o));
  if (lane == 0 && local_min != 0xFFFFFFFFu) atomicMin(st.fmin, local_min);
}

// Pull form of one relaxation: for every vertex v (one graph copy), the
// smallest dist[u] + w(e) over the entries e = (v, u) of its row, which on a
// symmetric CSR are its in-edges, replaces dist[v] if smaller. Merge-based
// like the neighbourhood gather-reduce: a chunk's vertex end markers and its
// edges form one sequence; the block gathers dist[C[e]] + W[e] of the
// chunk's edges into shared memory (coalesced column and weight loads, the
// distance gathers of the chunk in flight at once), then each thread walks
// kSsspItems consecutive items, taking the minimum per vertex. A vertex
// whose row lies inside one thread's items is lowered with a plain store
// (nobody else writes it in this iteration); the pieces of a split row use
// atomicMin. A lowered vertex joins the next near frontier (below T) or the
// far pile, deduplicated by the same stamps as in relax.
__device__ void pull_relax_body(const SsspArgs &a, uint32_t *dist, SsspSmem &sm,
                                const SsspStep &st) {
  constexpr int ITEMS = kSsspItems;
  constexpr int CHUNK = kSsspChunk;
  int32_t *Qn = pick(a.nearq, st.near_parity ^ 1);
  int32_t *Sn = pick(a.nearS, st.near_parity ^ 1);
  const unsigned long long T = st.T;
  const int32_t iter = st.iter, epoch = st.far_epoch;
  int32_t *s_end = sm.off;  // end marker of each chunk vertex, chunk-local
  uint32_t *s_val = sm.du;  // dist[u] + w(e) of each chunk edge
  uint32_t local_min = 0xFFFFFFFFu;
  const long long total = (long long)a.n + a.m;
  const long long nchunks = (total + CHUNK - 1) / CHUNK;
  for (long long chunk = blockIdx.x; chunk < nchunks; chunk += gridDim.x) {
    const long long d0 = chunk * CHUNK;
    const long long d1 = min(d0 + CHUNK, total);
    const int32_t i0 = a.cb[chunk], i1 = a.cb[chunk + 1];
    const long long j0 = d0 - i0, j1 = d1 - i1;
    const int32_t nv = (i0 <= a.n - 1) ? (min(i1, a.n - 1) - i0 + 1) : 0;
    const int32_t ne = (int32_t)(j1 - j0);
    const int32_t len = (int32_t)(d1 - d0);
    for (int32_t k = threadIdx.x; k < nv; k += kSsspThreads)
      s_end[k] = (int32_t)((long long)a.R[i0 + k + 1] + i0 + k - d0);
    {
      int32_t col[ITEMS];
      uint32_t wt[ITEMS];
#pragma unroll
      for (int i = 0; i < ITEMS; ++i) {
        const int32_t k = threadIdx.x + i * kSsspThreads;
        col[i] = -1;
        wt[i] = 0u;
        if (k < ne && GR_IN(j0 + k, a.m, 330)) {
          col[i] = a.C[j0 + k];
          wt[i] = a.W[j0 + k];
          if (!GR_IN(col[i], a.n, 331)) col[i] = -1;
        }
      }
#pragma unroll
      for (int i = 0; i < ITEMS; ++i) {
        const int32_t k = threadIdx.x + i * kSsspThreads;
        if (k < ne) {
          uint32_t val = 0xFFFFFFFFu;
          if (col[i] >= 0) {
            const unsigned long long t = (unsigned long long)dist[col[i]] + wt[i];
            if (t < 0xFFFFFFFFull) val = (uint32_t)t;
          }
          s_val[k] = val;
        }
      }
    }
    __syncthreads();
    // this thread's items [k0, k1) of the chunk: item i closes at most one
    // vertex (slot i), and slot ITEMS holds the vertex continuing past k1
    int32_t cv[ITEMS + 1];
    uint32_t cd[ITEMS + 1];
    bool cw[ITEMS + 1];  // whole: the vertex's row lies in this thread's items
#pragma unroll
    for (int j = 0; j <= ITEMS; ++j) {
      cv[j] = -1;
      cd[j] = 0xFFFFFFFFu;
      cw[j] = false;
    }
    const int32_t k0 = min(len, (int32_t)threadIdx.x * ITEMS);
    const int32_t k1 = min(len, k0 + ITEMS);
    if (k0 < k1) {
      int32_t lo = 0, hi = nv;
      while (lo < hi) {
        const int32_t mid = (lo + hi) >> 1;
        if (s_end[mid] < k0) lo = mid + 1;
        else hi = mid;
      }
      int32_t r = lo, e = k0 - r;
      uint32_t best = 0xFFFFFFFFu;
      bool first = true;  // the current vertex may have entries before k0
#pragma unroll
      for (int i = 0; i < ITEMS; ++i) {
        const int32_t k = k0 + i;
        if (k < k1) {
          if (r < nv && s_end[r] == k) {  // end marker of vertex i0 + r
            cv[i] = i0 + r;
            cd[i] = best;
            cw[i] = !first;
            best = 0xFFFFFFFFu;
            first = false;
            ++r;
          } else {
            best = min(best, s_val[e]);
            ++e;
          }
        }
      }
      if (r < nv && best != 0xFFFFFFFFu) {  // continues past k1
        cv[ITEMS] = i0 + r;
        cd[ITEMS] = best;
        cw[ITEMS] = false;
      }
    }
    // lower, classify and emit (warp-uniform emission calls)
#pragma unroll
    for (int j = 0; j <= ITEMS; ++j) {
      int code = 0;
      int32_t dvg = 0;
      const int32_t v = cv[j];
      const uint32_t nd = cd[j];
      if (v >= 0 && nd != 0xFFFFFFFFu) {
        bool lowered;
        if (cw[j]) {
          lowered = nd < dist[v];
          if (lowered) dist[v] = nd;
        } else {
          lowered = nd < atomicMin(dist + v, nd);
        }
        if (lowered) {
          if ((unsigned long long)nd < T) {
            if (atomicExch(a.stamp + v, iter) != iter) {
              code = 1;
              dvg = a.R[v + 1] - a.R[v];
            }
          } else {
            local_min = min(local_min, nd);
            code = atomicExch(a.far_stamp + v, epoch) != epoch ? 2 : 0;
          }
        }
      }
      emit_scanned(sm.nearb, code == 1, v, dvg);
      emit_plain(sm.farb, code == 2, v);
    }
    flush_scanned<kSsspThreads>(sm.nearb, st.near_ctr, Qn, Sn, a.nv + 1);
    flush_plain<kSsspThreads>(sm.farb, st.far_ctr, st.far_dest, st.far_cap);
  }
  for (int o = 16; o > 0; o >>= 1) local_min = min(local_min, __shfl_xor_sync(0xffffffffu, local_min, o));
  if ((threadIdx.x & 31) == 0 && local_min != 0xFFFFFFFFu) atomicMin(st.fmin, local_min);
}

__device__ void split_body(const SsspArgs &a, const uint32_t *dist, SsspSmem &sm,
                           const SsspStep &st) {
  const int32_t *F = pick(a.farq, st.far_parity);
  const int32_t np = st.near_parity;
  int32_t *Qn = pick(a.nearq, np ^ 1);
  int32_t *Sn = pick(a.nearS, np ^ 1);
  const int32_t len = st.far_len;
  const unsigned long long T = st.T, T_old = st.T_old;
  const int32_t iter = st.iter, epoch = st.far_epoch + 1;
  uint32_t local_min = 0xFFFFFFFFu;
  const long long per_round = (long long)gridDim.x * kSsspThreads;
  const long long rounds = (len + per_round - 1) / per_round;
  for (long long r = 0; r < rounds; ++r) {
    const long long i = (r * gridDim.x + blockIdx.x) * kSsspThreads + threadIdx.x;
    int code = 0;
    int32_t v = 0, dv = 0;
    if (i < len && GR_IN(i, a.nv + 1, 310) && GR_IN(F[i], a.nv, 311)) {
      v = F[i];
      const uint32_t d = dist[v];
      if ((unsigned long long)d < T_old) {
        code = 0;  // stale: improved below the old threshold and expanded
      } else if ((unsigned long long)d < T) {
        if (atomicExch(a.stamp + v, iter) != iter) {
          code = 1;
          const int32_t vl = v - lane_base(v, a.n);
          dv = a.R[vl + 1] - a.R[vl];
        }
      } else {
        local_min = min(local_min, d);
        code = atomicExch(a.far_stamp + v, epoch) != epoch ? 2 : 0;
      }
    }
    emit_scanned(sm.nearb, code == 1, v, dv);
    emit_plain(sm.farb, code == 2, v);
    if ((r + 1) % (kSsspChunk / kSsspThreads) == 0 || r == rounds - 1) {
      flush_scanned<kSsspThreads>(sm.nearb, st.near_ctr, Qn, Sn, a.nv + 1);
      flush_plain<kSsspThreads>(sm.farb, st.far_ctr, st.far_dest, st.far_cap);
    }
  }
  for (int o = 16; o > 0; o >>= 1) local_min = min(local_min, __shfl_xor_sync(0xffffffffu, local_min, o));
  if ((threadIdx.x & 31) == 0 && local_min != 0xFFFFFFFFu) atomicMin(st.fmin, local_min);
}

template <bool LOW>
__device__ void relax_mode(const SsspArgs &a, SsspCtl *c, SsspSmem &sm) {
  SsspStep st;
  st.near_parity = c->near_parity;
  st.far_parity = c->far_parity;
  st.q = c->near_len;
  st.q_edges = (int32_t)c->near_edges;
  st.far_len = c->far_len;
  st.T = c->T;
  st.T_old = c->T_old;
  st.iter = c->iter;
  st.far_epoch = c->far_epoch;
  st.near_ctr = &c->near_next_packed;
  st.far_ctr = &c->far_len;  // absolute positions in the current pile
  st.far_dest = pick(a.farq, c->far_parity);
  st.far_cap = (long long)a.nv + 1;
  st.fmin = &c->far_min;
  if (!LOW && c->mode == kSsspPull) pull_relax_body(a, c->dist, sm, st);
  else if (LOW) relax_body_thread(a, c->dist, st);
  else relax_body(a, c->dist, sm, st);
}

__device__ void split_mode(const SsspArgs &a, SsspCtl *c, SsspSmem &sm) {
  SsspStep st;
  st.near_parity = c->near_parity;
  st.far_parity = c->far_parity;
  st.q = c->near_len;
  st.q_edges = (int32_t)c->near_edges;
  st.far_len = c->far_len;
  st.T = c->T;
  st.T_old = c->T_old;
  st.iter = c->iter;
  st.far_epoch = c->far_epoch;
  st.near_ctr = &c->near_next_packed;
  st.far_ctr = &c->far_next_len;
  st.far_dest = pick(a.farq, c->far_parity ^ 1);
  st.far_cap = (long long)a.nv + 1;
  st.fmin = &c->far_min_next;
  split_body(a, c->dist, sm, st);
}

__device__ __forceinline__ unsigned long long bucket_end(uint32_t d, unsigned long long delta) {
  return ((unsigned long long)d / delta + 1ull) * delta;
}

// Run by the last block of an iteration.
__device__ void sssp_end(const SsspArgs &a, SsspCtl *c) {
  if (c->error) {
    c->done = 1;
    return;
  }
  // counters the other blocks filled with atomics: read past L1
  const unsigned long long packed = *(volatile unsigned long long *)&c->near_next_packed;
  const int32_t qn = (int32_t)(packed & 0xFFFFFFFFull);
  const long long en = (long long)(packed >> 32);
  if (c->mode != kSsspSplit) {
    c->relaxations += c->mode == kSsspPull ? a.m : c->near_edges;
    c->pulls += c->mode == kSsspPull;
    c->far_len = *(volatile int32_t *)&c->far_len;
    c->far_min = *(volatile uint32_t *)&c->far_min;
  } else {
    c->far_len = *(volatile int32_t *)&c->far_next_len;
    c->far_parity ^= 1;
    c->far_epoch += 1;
    c->far_min = *(volatile uint32_t *)&c->far_min_next;
    c->phases += 1;
  }
  c->near_len = qn;
  c->near_edges = en;
  c->near_parity ^= 1;
  pick(a.nearS, c->near_parity)[qn] = (int32_t)en;
  c->near_next_packed = 0ull;
  c->far_next_len = 0;
  c->far_min_next = 0xFFFFFFFFu;
  c->iter += 1;
  if (c->near_len > 0) {
    c->mode = c->near_edges >= c->pull_min_edges ? kSsspPull : kSsspRelax;
  } else if (c->far_len > 0) {
    c->mode = kSsspSplit;
    c->T_old = c->T;
    const unsigned long long t = c->T + c->delta;
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

// LOW: per-thread relaxation (graphs of small maximum degree)
template <bool LOW>
__global__ void __launch_bounds__(kSsspThreads, kSsspBlocksPerSm)
    k_sssp_iter(SsspArgs a, cudaGraphConditionalHandle h, int32_t use_cond) {
  SsspCtl *c = a.ctl;
  if (*(volatile int32_t *)&c->done) {
    // an iteration kernel after the run ended (host-driven batches enqueue a
    // few extra): every block leaves; inside a graph the loop condition is
    // cleared here too, so the while loop cannot outlive the run
    if (use_cond && blockIdx.x == 0 && threadIdx.x == 0) cudaGraphSetConditional(h, 0u);
    return;
  }
  __shared__ SsspSmem sm;
  if (threadIdx.x == 0) {
    sm.nearb.cnt = 0;
    sm.farb.cnt = 0;
  }
  __syncthreads();
  if (c->mode != kSsspSplit) relax_mode<LOW>(a, c, sm);
  else split_mode(a, c, sm);
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    const unsigned long long old = atomicAdd(&c->arrivals, 1ull);
    sm.last = (old + 1ull) % gridDim.x == 0ull;
  }
  __syncthreads();
  if (sm.last && threadIdx.x == 0) {
    __threadfence();
    sssp_end(a, c);
    if (use_cond) cudaGraphSetConditional(h, c->done ? 0u : 1u);
  }
}

// Persistent form: the whole SSSP in one cooperative kernel, one grid
// barrier per iteration. After the barrier every block reads the
// iteration's counters and recomputes the same next state in registers; the
// counters form rings of three (the one an iteration fills, the one just
// read, the one block 0 clears for the next iteration).
template <bool LOW>
__global__ void __launch_bounds__(kSsspThreads, kSsspBlocksPerSm) k_sssp_do(SsspArgs a) {
  SsspCtl *c = a.ctl;
  __shared__ SsspSmem sm;
  if (threadIdx.x == 0) {
    sm.nearb.cnt = 0;
    sm.farb.cnt = 0;
  }
  __syncthreads();
  uint32_t *dist = c->dist;
  const unsigned long long delta = c->delta;
  const int32_t max_iters = c->max_iters;
  int32_t mode = kSsspRelax, near_parity = 0, far_parity = 0, near_len = c->near_len, far_len = 0;
  long long near_edges = c->near_edges, relaxations = 0;
  const long long pull_min_edges = c->pull_min_edges;
  int32_t iter = 0, far_epoch = 0, phases = 0, gen = 0, pulls = 0;
  uint32_t far_min = 0xFFFFFFFFu;
  unsigned long long T = delta, T_old = 0;
  for (;;) {
    const int32_t slot = iter % 3, clear = (iter + 1) % 3;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      c->ring_near[clear] = 0ull;
      c->ring_far[clear] = 0;
      c->ring_fmin[clear] = 0xFFFFFFFFu;
    }
    SsspStep st;
    st.near_parity = near_parity;
    st.far_parity = far_parity;
    st.q = near_len;
    st.q_edges = (int32_t)near_edges;
    st.far_len = far_len;
    st.T = T;
    st.T_old = T_old;
    st.iter = iter;
    st.far_epoch = far_epoch;
    st.near_ctr = &c->ring_near[slot];
    st.far_ctr = &c->ring_far[slot];
    st.fmin = &c->ring_fmin[slot];
    if (mode != kSsspSplit) {
      st.far_dest = pick(a.farq, far_parity) + far_len;  // appended after the pile
      st.far_cap = (long long)a.nv + 1 - far_len;
      if (!LOW && mode == kSsspPull) {
        pull_relax_body(a, dist, sm, st);
      } else if (LOW) {
        relax_body_thread(a, dist, st);
      } else {
        // a dense frontier's chunk bounds in one grid-wide pass (every block
        // then starts its chunks without a search)
        const long long nchunks = ((long long)near_len + near_edges + kSsspChunk - 1) / kSsspChunk;
        const bool bounds = a.qcb && nchunks >= (long long)kSsspBoundsChunksPerBlock * gridDim.x;
        if (bounds) {
          frontier_chunk_bounds(pick(a.nearS, near_parity), near_len, (int32_t)near_edges,
                                nchunks, a.qcb);
          if (!grid_sync(&c->bar, &c->error, gen)) break;
        }
        relax_body(a, dist, sm, st, bounds ? a.qcb : nullptr);
      }
    } else {
      st.far_dest = pick(a.farq, far_parity ^ 1);
      st.far_cap = (long long)a.nv + 1;
      split_body(a, dist, sm, st);
    }
    if (!grid_sync(&c->bar, &c->error, gen)) break;  // a wait gave up: error is set
    const unsigned long long pk = *(volatile unsigned long long *)&c->ring_near[slot];
    const int32_t fcnt = *(volatile int32_t *)&c->ring_far[slot];
    const uint32_t fmin = *(volatile uint32_t *)&c->ring_fmin[slot];
    if (mode != kSsspSplit) {
      relaxations += mode == kSsspPull ? a.m : near_edges;
      pulls += mode == kSsspPull;
      far_len += fcnt;
      far_min = min(far_min, fmin);
    } else {
      far_len = fcnt;
      far_parity ^= 1;
      far_epoch += 1;
      far_min = fmin;
      phases += 1;
    }
    near_len = (int32_t)(pk & 0xFFFFFFFFull);
    near_edges = (long long)(pk >> 32);
    near_parity ^= 1;
    iter += 1;
    bool done = false, overflow = false;
    if (near_len > 0) {
      mode = near_edges >= pull_min_edges ? kSsspPull : kSsspRelax;
    } else if (far_len > 0) {
      mode = kSsspSplit;
      T_old = T;
      const unsigned long long t = T + delta;
      const unsigned long long j = bucket_end(far_min, delta);
      T = t > j ? t : j;
    } else {
      done = true;
    }
    if (!done && iter >= max_iters) overflow = true;
    if (done || overflow) {
      if (blockIdx.x == 0 && threadIdx.x == 0) {
        c->iter = iter;
        c->phases = phases;
        c->relaxations = relaxations;
        c->pulls = pulls;
        if (overflow) c->error = kDevOverflow;
        c->done = 1;
      }
      break;
    }
  }
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

size_t sssp_ws_bytes(const gr_graph *g, int32_t lanes) {
  const size_t n = (size_t)g->n * (size_t)std::max(lanes, 1);
  const size_t qcb = g->max_degree > kSsspLowDegreeMax
                         ? sizeof(int32_t) * ((n + (size_t)std::max(lanes, 1) * (size_t)g->m) /
                                                  kSsspChunk + 3)
                         : 0;
  return 4 * sizeof(int32_t) * (n + 1) + 2 * sizeof(int32_t) * (n + 2) +
         2 * sizeof(int32_t) * n + sizeof(SsspCtl) + qcb;
}

int32_t sssp_batch_max_lanes(const gr_graph *g) {
  // lane-major ids and queue positions (up to lanes * n + 1), and a
  // frontier's edge count (up to lanes * m), are int32
  long long k = kSsspMaxLanes;
  k = std::min<long long>(k, (INT32_MAX - 2) / std::max<int32_t>(g->n, 1));
  if (g->m > 0) k = std::min<long long>(k, INT32_MAX / g->m);
  return (int32_t)std::max<long long>(k, 1);
}

gr_status sssp_ws_create(gr_graph *g, cudaStream_t s, SsspWorkspace **out, int32_t lanes) {
  if (lanes < 1 || lanes > sssp_batch_max_lanes(g))
    return fail(GR_EINVAL, "SSSP workspace: lane count out of range for this graph");
  std::unique_ptr<SsspWorkspace> ws(new SsspWorkspace());
  ws->lanes = lanes;
  const size_t n = (size_t)g->n * (size_t)lanes;
  for (int i = 0; i < 2; ++i) {
    GR_TRY(ws->nearq[i].alloc(sizeof(int32_t) * (n + 1), "SSSP near queue"));
    GR_TRY(ws->nearS[i].alloc(sizeof(int32_t) * (n + 2), "SSSP near degree scan"));
    GR_TRY(ws->farq[i].alloc(sizeof(int32_t) * (n + 1), "SSSP far pile"));
  }
  GR_TRY(ws->stamp.alloc(sizeof(int32_t) * n, "SSSP near stamps"));
  GR_TRY(ws->far_stamp.alloc(sizeof(int32_t) * n, "SSSP far stamps"));
  GR_TRY(ws->ctl.alloc(sizeof(SsspCtl), "SSSP control"));
  if (g->max_degree > kSsspLowDegreeMax) {
    // a frontier holds at most n vertices of each lane and their edges
    const long long chunks = ((long long)n + (long long)lanes * g->m) / kSsspChunk + 2;
    GR_TRY(ws->qcb.alloc(sizeof(int32_t) * ((size_t)chunks + 1), "SSSP frontier chunk bounds"));
  }
  if (lanes == 1) {
    // the pull relaxation's merge path over all vertices never changes
    const int32_t chunks = merge_chunks(g->n, g->m, kSsspChunk);
    GR_TRY(ws->cb.alloc(sizeof(int32_t) * ((size_t)chunks + 1), "SSSP pull chunk bounds"));
    k_chunk_bounds<<<(chunks + 256) / 256, 256, 0, s>>>(g->row_off.as<int32_t>(), g->n,
                                                         kSsspChunk, chunks, ws->cb.as<int32_t>());
    GR_CUDA(cudaGetLastError());
  }
  GR_CUDA(cudaMemsetAsync(ws->ctl.p, 0, sizeof(SsspCtl), s));
  GR_CUDA(cudaStreamSynchronize(s));
  *out = ws.release();
  return GR_OK;
}

static SsspArgs sssp_args(gr_graph *g, SsspWorkspace *ws, int32_t lanes = 1) {
  SsspArgs a;
  a.R = g->row_off.as<int32_t>();
  a.C = g->col.as<int32_t>();
  a.W = g->w.as<uint32_t>();
  a.n = g->n;
  a.nv = g->n * lanes;
  a.m = g->m;
  for (int i = 0; i < 2; ++i) {
    a.nearq[i] = ws->nearq[i].as<int32_t>();
    a.nearS[i] = ws->nearS[i].as<int32_t>();
    a.farq[i] = ws->farq[i].as<int32_t>();
  }
  a.stamp = ws->stamp.as<int32_t>();
  a.far_stamp = ws->far_stamp.as<int32_t>();
  a.ctl = ws->ctl.as<SsspCtl>();
  a.low_degree = g->max_degree <= kSsspLowDegreeMax ? 1 : 0;
  a.cb = ws->cb.as<int32_t>();  // null for batched workspaces, which never pull
  a.qcb = ws->qcb.as<int32_t>();  // null on low-degree graphs
  return a;
}

// Smallest near-frontier edge count at which a relaxation pulls. Pull reads
// every row once where push reads the frontier's rows (and pays atomics and
// its per-chunk chain), so it pays only where the frontier covers most of
// the graph: at m / opts->alpha edges, else at m / the graph's tuned alpha
// (0: never, the default until gr_autotune finds pulling faster); GR_DIR_PUSH
// never pulls, GR_DIR_PULL pulls every relaxation. Only a symmetric CSR
// (rows = in-neighbours) and a single search can pull.
static long long sssp_pull_min_edges(const gr_graph *g, const gr_opts &o, int32_t lanes) {
  if (!g->symmetric || lanes != 1 || g->max_degree <= kSsspLowDegreeMax || g->m == 0 ||
      o.direction == GR_DIR_PUSH)
    return LLONG_MAX;
  if (o.direction == GR_DIR_PULL) return 1;
  const double div = o.alpha > 0.f ? (double)o.alpha : (double)g->tuned_sssp_alpha;
  if (div <= 0.0) return LLONG_MAX;
  return std::max<long long>(1, (long long)((double)g->m / div));
}

static gr_status sssp_enqueue_iter(gr_graph *g, const SsspArgs &a, cudaStream_t s,
                                   cudaGraphConditionalHandle h, int use_cond) {
  if (a.low_degree)
    k_sssp_iter<true><<<g->num_sms * kSsspBlocksPerSm, kSsspThreads, 0, s>>>(a, h, use_cond);
  else
    k_sssp_iter<false><<<g->num_sms * kSsspBlocksPerSm, kSsspThreads, 0, s>>>(a, h, use_cond);
  GR_CUDA(cudaGetLastError());
  return GR_OK;
}

static gr_status build_sssp_graph(gr_graph *g, SsspWorkspace *ws) {
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
  gr_status st = sssp_enqueue_iter(g, sssp_args(g, ws), cs, h, 1);
  cudaGraph_t captured;
  cudaError_t e = cudaStreamEndCapture(cs, &captured);
  cudaStreamDestroy(cs);
  if (st != GR_OK) return st;
  GR_CUDA(e);
  GR_CUDA(cudaGraphInstantiate(&ws->exec, graph, 0));
  ws->graph = graph;
  return GR_OK;
}

gr_status sssp_read_ctl_error(SsspWorkspace *ws, cudaStream_t s) {
  SsspCtl h;
  // pageable destination: the copy has finished when the call returns
  GR_CUDA(cudaMemcpyAsync(&h, ws->ctl.p, sizeof(SsspCtl), cudaMemcpyDeviceToHost, s));
  if (h.error == kDevTimeout) return fail(GR_ETIMEOUT, "a device-side wait timed out");
  if (h.error == kDevOverflow) return fail(GR_ETIMEOUT, "iteration limit reached");
  return GR_OK;
}

gr_status sssp_check(const gr_graph *g, int32_t src, const gr_opts &o) {
  if (!g->has_weights) return fail(GR_EINVAL, "SSSP needs edge weights (w was NULL at creation)");
  if (src < 0 || src >= g->n) return fail(GR_EINVAL, "source out of range");
  if (o.mode < GR_MODE_AUTO || o.mode > GR_MODE_PERSISTENT)
    return fail(GR_EINVAL, "unknown mode");
  if (o.direction < GR_DIR_AUTO || o.direction > GR_DIR_PULL)
    return fail(GR_EINVAL, "unknown direction policy");
  if (o.direction == GR_DIR_PULL && !g->symmetric)
    return fail(GR_EINVAL, "pull relaxation needs a symmetric CSR (in-neighbours = out-neighbours)");
  if (o.alpha < 0.f) return fail(GR_EINVAL, "alpha must be >= 0");
  return GR_OK;
}

// Runs the device-side loop of an initialised search with the given driver.
static gr_status sssp_drive(gr_graph *g, SsspWorkspace *ws, SsspArgs a, int32_t mode,
                            const gr_opts &o, int32_t max_iters, cudaStream_t s) {
  if (mode == GR_MODE_PERSISTENT) {
    void *kern = a.low_degree ? (void *)k_sssp_do<true> : (void *)k_sssp_do<false>;
    const int32_t want = o.block > 0 ? o.block : g->tuned_sssp_blocks_per_sm;
    // the carveout fitted to the blocks that run leaves the rest to L1
    int bps = 1;
    GR_TRY(fit_carveout(kern, kSsspThreads, want > 0 ? std::min(want, kSsspBlocksPerSm)
                                                      : kSsspBlocksPerSm,
                        g->device, &bps));
    void *args[] = {&a};
    GR_CUDA(cudaLaunchCooperativeKernel(kern, std::max(1, bps) * g->num_sms,
                                        kSsspThreads, args, 0, s));
  } else if (mode == GR_MODE_LAUNCH) {
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
    GR_TRY(build_sssp_graph(g, ws));
    GR_CUDA(cudaGraphLaunch(ws->exec, s));
  }
  return GR_OK;
}

static unsigned long long sssp_delta_of(const gr_graph *g, const gr_opts &o) {
  return o.delta == UINT32_MAX ? (1ull << 40) : (o.delta ? o.delta : g->sssp_delta);
}

static int32_t sssp_max_iters_of(const gr_graph *g, const gr_opts &o) {
  return o.max_iters > 0 ? o.max_iters
                         : (int32_t)std::min<long long>(INT32_MAX, 8ll * g->n + 1024);
}

// SSSP into device outputs with an explicit workspace (no locking, no
// staging): the public gr_sssp and the query server both call this.
gr_status sssp_run(gr_graph *g, SsspWorkspace *ws, int32_t src, uint32_t *dist, int32_t *pred,
                   const gr_opts &o, cudaStream_t s) {
  const unsigned long long delta = sssp_delta_of(g, o);
  const int32_t max_iters = sssp_max_iters_of(g, o);
  SsspArgs a = sssp_args(g, ws);
  SsspSources one;
  one.k = 1;
  one.s[0] = src;
  k_sssp_init<<<g->num_sms * 8, 256, 0, s>>>(a, one, dist, pred, delta, max_iters,
                                             sssp_pull_min_edges(g, o, 1));
  GR_CUDA(cudaGetLastError());
  const int32_t mode = o.mode != GR_MODE_AUTO ? o.mode : g->tuned_sssp_mode;
  GR_TRY(sssp_drive(g, ws, a, mode, o, max_iters, s));
  if (pred) {
    const int grid = g->num_sms * 8;
    k_sssp_pred_init<<<grid, 256, 0, s>>>(pred, g->n);
    k_sssp_pred<<<grid, 256, 0, s>>>(a.R, a.C, a.W, dist, pred, g->n, src);
    k_sssp_pred_fin<<<grid, 256, 0, s>>>(pred, g->n, src);
    GR_CUDA(cudaGetLastError());
  }
  return GR_OK;
}

// k searches as one over k copies of the graph into dist[k][n] (device).
// The CUDA-graph driver holds one-lane arguments, so every driver but the
// persistent kernel becomes the host-driven loop here.
gr_status sssp_batch_run(gr_graph *g, SsspWorkspace *ws, const int32_t *h_srcs, int32_t k,
                         uint32_t *dist, const gr_opts &o, cudaStream_t s) {
  if (k < 1 || k > ws->lanes) return fail(GR_EINVAL, "batched SSSP: k exceeds the workspace");
  const unsigned long long delta = sssp_delta_of(g, o);
  const int32_t max_iters = sssp_max_iters_of(g, o);
  SsspArgs a = sssp_args(g, ws, k);
  SsspSources srcs;
  srcs.k = k;
  for (int32_t l = 0; l < kSsspMaxLanes; ++l) srcs.s[l] = l < k ? h_srcs[l] : 0;
  k_sssp_init<<<g->num_sms * 8, 256, 0, s>>>(a, srcs, dist, nullptr, delta, max_iters,
                                             LLONG_MAX);
  GR_CUDA(cudaGetLastError());
  int32_t mode = o.mode != GR_MODE_AUTO ? o.mode : g->tuned_sssp_mode;
  if (mode != GR_MODE_PERSISTENT) mode = GR_MODE_LAUNCH;
  gr_opts ob = o;
  // k lanes carry k times the frontier of one search per iteration: where
  // the single search was tuned to one block per SM, two do better (16
  // sources on the 4096^2 mesh: 282 ms at 2 blocks per SM, 321 at 1, 297 at
  // 3, 335 at 5)
  if (k > 1 && ob.block == 0 && g->tuned_sssp_blocks_per_sm == 1) ob.block = 2;
  return sssp_drive(g, ws, a, mode, ob, max_iters, s);
}

}  // namespace gr

using namespace gr;

extern "C" {

gr_status gr_sssp(gr_graph *g, int32_t src, uint32_t *dist, int32_t *pred,
                  const gr_opts *opts, void *stream) {
  clear_error();
  if (!g) return fail(GR_EINVAL, "graph must not be NULL");
  if (!dist) return fail(GR_EINVAL, "dist must not be NULL");
  const gr_opts &o = opts ? *opts : default_opts();
  GR_TRY(sssp_check(g, src, o));
  std::lock_guard<std::mutex> lock(g->mu);
  cudaStream_t s = (cudaStream_t)stream;
  GR_TRY(begin_call(g, s));
  if (!g->sssp) GR_TRY(sssp_ws_create(g, s, &g->sssp));
  void *d_dist, *d_pred;
  bool cp_dist, cp_pred;
  GR_TRY(resolve_output(g, 0, dist, sizeof(uint32_t) * (size_t)g->n, &d_dist, &cp_dist));
  GR_TRY(resolve_output(g, 1, pred, sizeof(int32_t) * (size_t)g->n, &d_pred, &cp_pred));
  GR_TRY(sssp_run(g, g->sssp, src, (uint32_t *)d_dist, (int32_t *)d_pred, o, s));
  if (cp_dist)
    GR_CUDA(cudaMemcpyAsync(dist, d_dist, sizeof(uint32_t) * (size_t)g->n,
                            cudaMemcpyDeviceToHost, s));
  if (cp_pred)
    GR_CUDA(cudaMemcpyAsync(pred, d_pred, sizeof(int32_t) * (size_t)g->n,
                            cudaMemcpyDeviceToHost, s));
  GR_TRY(end_call(g, s));
  return GR_OK;
}

gr_status gr_sssp_batch(gr_graph *g, const int32_t *srcs, int32_t k, uint32_t *dist,
                        const gr_opts *opts, void *stream) {
  clear_error();
  if (!g) return fail(GR_EINVAL, "graph must not be NULL");
  if (!srcs || !dist) return fail(GR_EINVAL, "srcs/dist must not be NULL");
  const int32_t kmax = sssp_batch_max_lanes(g);
  if (k < 1 || k > kmax)
    return fail(GR_EINVAL, "k must be in [1, " + std::to_string(kmax) +
                               "] (64, and k*n and k*m must fit in int32)");
  const gr_opts &o = opts ? *opts : default_opts();
  for (int32_t i = 0; i < k; ++i) GR_TRY(sssp_check(g, srcs[i], o));
  std::lock_guard<std::mutex> lock(g->mu);
  cudaStream_t s = (cudaStream_t)stream;
  GR_TRY(begin_call(g, s));
  if (g->sssp_batch && g->sssp_batch->lanes < k) {
    // the old buffers may still be in use by enqueued work
    GR_CUDA(cudaStreamSynchronize(s));
    free_sssp(g->sssp_batch);
    g->sssp_batch = nullptr;
  }
  if (!g->sssp_batch) GR_TRY(sssp_ws_create(g, s, &g->sssp_batch, k));
  void *d_dist;
  bool cp;
  const size_t bytes = sizeof(uint32_t) * (size_t)k * (size_t)g->n;
  GR_TRY(resolve_output(g, 0, dist, bytes, &d_dist, &cp));
  GR_TRY(sssp_batch_run(g, g->sssp_batch, srcs, k, (uint32_t *)d_dist, o, s));
  if (cp) GR_CUDA(cudaMemcpyAsync(dist, d_dist, bytes, cudaMemcpyDeviceToHost, s));
  GR_TRY(end_call(g, s));
  return GR_OK;
}

gr_status gr_sssp_batch_stats(gr_graph *g, int32_t *iterations, int32_t *phases,
                              int64_t *relaxations) {
  clear_error();
  if (!g) return fail(GR_EINVAL, "graph must not be NULL");
  if (!g->sssp_batch) return fail(GR_EINVAL, "no batched SSSP has run on this graph");
  std::lock_guard<std::mutex> lock(g->mu);
  GR_CUDA(cudaSetDevice(g->device));
  if (g->has_last) GR_CUDA(cudaEventSynchronize(g->last_done));
  SsspCtl h;
  GR_CUDA(cudaMemcpy(&h, g->sssp_batch->ctl.p, sizeof(h), cudaMemcpyDeviceToHost));
  if (h.error == kDevTimeout) return fail(GR_ETIMEOUT, "a device-side wait timed out");
  if (h.error == kDevOverflow) return fail(GR_ETIMEOUT, "iteration limit reached");
  if (iterations) *iterations = h.iter;
  if (phases) *phases = h.phases;
  if (relaxations) *relaxations = h.relaxations;
  return GR_OK;
}

gr_status gr_sssp_pull_stats(gr_graph *g, int32_t *pulls) {
  clear_error();
  if (!g) return fail(GR_EINVAL, "graph must not be NULL");
  if (!g->sssp) return fail(GR_EINVAL, "no SSSP has run on this graph");
  std::lock_guard<std::mutex> lock(g->mu);
  GR_CUDA(cudaSetDevice(g->device));
  if (g->has_last) GR_CUDA(cudaEventSynchronize(g->last_done));
  SsspCtl h;
  GR_CUDA(cudaMemcpy(&h, g->sssp->ctl.p, sizeof(h), cudaMemcpyDeviceToHost));
  if (pulls) *pulls = h.pulls;
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
