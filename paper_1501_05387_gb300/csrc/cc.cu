// Connected components by hooking and pointer jumping (Sec. 5.4).
//
// The paper runs hooking as a filter over an edge frontier (every edge tries
// to give the smaller component id of its ends to the other end; edges whose
// ends already agree are filtered out) until no id changes, then pointer
// jumping as a filter over vertices until every vertex points at its root.
//
// Hooking here links roots only, larger root under smaller (atomicCAS on the
// larger root's own entry, so a root is re-pointed only while it is still a
// root). A CAS that loses a race retries with the roots it now finds, so
// each edge is settled in one visit: the paper's "repeat until no id
// changes" happens per edge instead of per sweep, and a single sweep over
// the CSR's edges (the all-vertex frontier of the load-balanced advance)
// leaves one tree per component. Finding a root halves the path it walks.
// Pointer jumping then points every vertex at its root. Because a root is
// only ever hooked under a smaller id, the root of each component is its
// smallest vertex id, which is the canonical label.
//
// Symmetric graphs store each undirected edge twice, so most edges need no
// visit at all: the sampling form of the hooking sweep first hooks every
// vertex to its first kCcSample neighbours and compresses, which on graphs
// with one giant component already places most vertices in it; the
// component that most of a fixed sample of vertices lies in is then
// skipped, and only the vertices outside it hook all their edges (an edge
// between two vertices of that component needs no visit, one leaving it is
// visited from its other end). Labels are the same as with a full sweep:
// hooking under the smaller root makes every root its component's smallest
// id whatever the order. For a directed CSR every arc hooks in one sweep,
// giving weakly connected components (an arc is not visible from its head).
#include <algorithm>
#include <vector>

#include "advance.cuh"

namespace gr {

constexpr int kCcThreads = 256, kCcItems = 8;
constexpr int kCcSample = 2;    // neighbours per vertex hooked before the skip
constexpr int kCcPicks = 1024;  // vertices whose roots choose the skipped component
constexpr int kCcFrontierCap = 1024;

struct CcWorkspace {
  DevMem counter;  // [0] components, [1] scratch; [2..3] packed frontier counter
  DevMem q, sc, picks;
};

void free_cc(CcWorkspace *ws) { delete ws; }

GR_GUARD_REPORTER(guard_report_cc)

namespace {

__global__ void k_cc_init(int32_t *label, int32_t n) {
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n;
       v += (int64_t)gridDim.x * blockDim.x)
    label[v] = (int32_t)v;
}

// root of x with path halving (pointers only ever decrease)
__device__ __forceinline__ int32_t find_root(int32_t *label, int32_t x);

// Join the trees of u and v: the larger root is re-pointed to the smaller
// one with a CAS, retried from the current roots if another thread moved
// the root first.
__device__ __forceinline__ void hook(int32_t *label, int32_t u, int32_t v);

__device__ __forceinline__ int32_t find_root(int32_t *label, int32_t x) {
  int32_t p = label[x];
  while (p != x) {
    const int32_t gp = label[p];
    if (gp != p) label[x] = gp;  // halving: benign race, gp is an ancestor
    x = p;
    p = gp;
  }
  return x;
}

__device__ __forceinline__ void hook(int32_t *label, int32_t u, int32_t v) {
  int32_t a = find_root(label, u);
  int32_t b = find_root(label, v);
  while (a != b) {
    const int32_t hi = max(a, b), lo = min(a, b);
    const int32_t prev = atomicCAS(label + hi, hi, lo);
    if (prev == hi) break;  // hooked
    // hi stopped being a root: continue from the roots as they are now
    a = find_root(label, prev);
    b = find_root(label, lo);
  }
}

struct HookF {
  int32_t *label;
  int32_t only_lower;  // symmetric graph: hook each undirected edge once
  int32_t n;
  __device__ __forceinline__ int operator()(int32_t u, int32_t v, int32_t) const {
    if (!GR_IN(u, n, 401) || !GR_IN(v, n, 402)) return 0;
    if (only_lower && v >= u) return 0;
    hook(label, u, v);
    return 0;  // edge settled: filtered out of the edge frontier
  }
};

// Each vertex hooks to its first kCcSample neighbours.
__global__ void k_cc_sample(const int32_t *R, const int32_t *C, int32_t n, int32_t *label) {
  for (int64_t vv = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; vv < n;
       vv += (int64_t)gridDim.x * blockDim.x) {
    const int32_t v = (int32_t)vv;
    const int32_t r0 = R[v], r1 = min(R[v + 1], r0 + kCcSample);
    for (int32_t e = r0; e < r1; ++e) {
      const int32_t u = C[e];
      if (GR_IN(u, n, 403)) hook(label, v, u);
    }
  }
}

// Roots (labels after compression) of kCcPicks vertices spread over the ids
// by a multiplicative hash.
__global__ void k_cc_pick(const int32_t *label, int32_t n, int32_t *picks) {
  const int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < kCcPicks) picks[i] = label[(int32_t)(((unsigned long long)i * 2654435761ull) % n)];
}

// The vertices outside component `skip` that have edges, with their
// degrees (an exclusive scan, emitted block by block with one packed atomic):
// the frontier whose edges the last hooking pass visits.
__global__ void __launch_bounds__(kCcThreads) k_cc_rest_frontier(const int32_t *R,
                                                                  const int32_t *label, int32_t n,
                                                                  int32_t skip, int32_t *Q,
                                                                  int32_t *S,
                                                                  unsigned long long *packed) {
  __shared__ ScannedBuf<kCcFrontierCap> buf;
  if (threadIdx.x == 0) buf.cnt = 0;
  __syncthreads();
  constexpr int PER = kCcFrontierCap / kCcThreads;
  for (int64_t base = (int64_t)blockIdx.x * kCcFrontierCap; base < n;
       base += (int64_t)gridDim.x * kCcFrontierCap) {  // block-uniform
#pragma unroll
    for (int j = 0; j < PER; ++j) {
      const int64_t v = base + j * kCcThreads + threadIdx.x;
      int32_t d = 0;
      bool take = false;
      if (v < n) {
        d = R[v + 1] - R[v];
        take = d > 0 && label[v] != skip;
      }
      emit_scanned(buf, take, (int32_t)v, d);
    }
    flush_scanned<kCcThreads>(buf, packed, Q, S, (long long)n + 1);
  }
}

// S[q] = the frontier's edge total (the advance reads it as the scan's end).
__global__ void k_cc_close(const unsigned long long *packed, int32_t *S) {
  const unsigned long long p = *packed;
  S[(int32_t)(p & 0xFFFFFFFFull)] = (int32_t)(p >> 32);
}

// Hook every edge of the frontier Q (size and scan from k_cc_rest_frontier).
__global__ void __launch_bounds__(kCcThreads) k_cc_hook_rest(const int32_t *R, const int32_t *C,
                                                              int32_t n, int32_t *label,
                                                              const int32_t *Q, const int32_t *S,
                                                              const unsigned long long *packed) {
  HookF f{label, 0, n};
  const int32_t q = (int32_t)(*packed & 0xFFFFFFFFull);
  lb_advance<kCcThreads, kCcItems, 0>(R, C, Q, q, S, f, nullptr, nullptr, nullptr, nullptr);
}

__global__ void __launch_bounds__(kCcThreads) k_cc_hook(const int32_t *R, const int32_t *C,
                                                         int32_t n, int32_t *label,
                                                         int32_t only_lower) {
  HookF f{label, only_lower, n};
  // every edge is settled in its visit: the edge frontier it would filter
  // into stays empty, so the advance appends nothing
  lb_advance<kCcThreads, kCcItems, 0>(R, C, nullptr, n, R, f, nullptr, nullptr, nullptr,
                                      nullptr);
}

__global__ void k_cc_jump(int32_t *label, int32_t n, int32_t *num_roots) {
  int32_t roots = 0;
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n;
       v += (int64_t)gridDim.x * blockDim.x) {
    int32_t r = label[v];
    while (label[r] != r) r = label[r];
    label[v] = r;
    roots += r == v;
  }
  for (int o = 16; o > 0; o >>= 1) roots += __shfl_xor_sync(0xffffffffu, roots, o);
  if ((threadIdx.x & 31) == 0 && roots) atomicAdd(num_roots, roots);
}

}  // namespace

size_t cc_ws_bytes(const gr_graph *g) {
  return sizeof(int32_t) * 4 + sizeof(int32_t) * (2 * (size_t)g->n + 3) +
         sizeof(int32_t) * kCcPicks;
}

gr_status cc_ws_create(gr_graph *g, CcWorkspace **out) {
  std::unique_ptr<CcWorkspace> ws(new CcWorkspace());
  GR_TRY(ws->counter.alloc(sizeof(int32_t) * 4, "CC counters"));
  if (g->symmetric) {
    GR_TRY(ws->q.alloc(sizeof(int32_t) * ((size_t)g->n + 1), "CC frontier"));
    GR_TRY(ws->sc.alloc(sizeof(int32_t) * ((size_t)g->n + 2), "CC frontier degree scan"));
    GR_TRY(ws->picks.alloc(sizeof(int32_t) * kCcPicks, "CC root sample"));
  }
  *out = ws.release();
  return GR_OK;
}

// CC into a device label array with an explicit workspace; the component
// count is left in the workspace counter (cc_count reads it).
gr_status cc_run(gr_graph *g, CcWorkspace *ws, int32_t *label, cudaStream_t s) {
  int32_t *cnt = ws->counter.as<int32_t>();
  const int grid = g->num_sms * 8;
  const int32_t *R = g->row_off.as<int32_t>(), *C = g->col.as<int32_t>();
  GR_CUDA(cudaMemsetAsync(cnt, 0, sizeof(int32_t) * 4, s));
  k_cc_init<<<grid, 256, 0, s>>>(label, g->n);
  if (!g->symmetric) {
    k_cc_hook<<<g->num_sms * 4, kCcThreads, 0, s>>>(R, C, g->n, label, 0);
  } else {
    k_cc_sample<<<grid, 256, 0, s>>>(R, C, g->n, label);
    k_cc_jump<<<grid, 256, 0, s>>>(label, g->n, cnt + 1);  // compress (count unused)
    k_cc_pick<<<(kCcPicks + 255) / 256, 256, 0, s>>>(label, g->n, ws->picks.as<int32_t>());
    GR_CUDA(cudaGetLastError());
    std::vector<int32_t> picks(kCcPicks);
    GR_CUDA(cudaMemcpyAsync(picks.data(), ws->picks.p, sizeof(int32_t) * kCcPicks,
                            cudaMemcpyDeviceToHost, s));
    GR_CUDA(cudaStreamSynchronize(s));
    std::sort(picks.begin(), picks.end());
    int32_t skip = picks[0], best = 0;
    for (size_t i = 0; i < picks.size();) {
      size_t j = i;
      while (j < picks.size() && picks[j] == picks[i]) ++j;
      if ((int32_t)(j - i) > best) {
        best = (int32_t)(j - i);
        skip = picks[i];
      }
      i = j;
    }
    unsigned long long *packed = ws->counter.as<unsigned long long>() + 1;
    int32_t *Q = ws->q.as<int32_t>(), *S = ws->sc.as<int32_t>();
    k_cc_rest_frontier<<<grid, kCcThreads, 0, s>>>(R, label, g->n, skip, Q, S, packed);
    k_cc_close<<<1, 1, 0, s>>>(packed, S);
    k_cc_hook_rest<<<g->num_sms * 4, kCcThreads, 0, s>>>(R, C, g->n, label, Q, S, packed);
  }
  k_cc_jump<<<grid, 256, 0, s>>>(label, g->n, cnt);
  GR_CUDA(cudaGetLastError());
  return GR_OK;
}

}  // namespace gr

using namespace gr;

extern "C" {

gr_status gr_cc(gr_graph *g, int32_t *label, int32_t *num_components, const gr_opts *opts,
                void *stream) {
  clear_error();
  (void)opts;
  if (!g) return fail(GR_EINVAL, "graph must not be NULL");
  if (!label) return fail(GR_EINVAL, "label must not be NULL");
  std::lock_guard<std::mutex> lock(g->mu);
  cudaStream_t s = (cudaStream_t)stream;
  GR_TRY(begin_call(g, s));
  if (!g->cc) GR_TRY(cc_ws_create(g, &g->cc));
  void *d_label;
  bool cp_label;
  GR_TRY(resolve_output(g, 0, label, sizeof(int32_t) * (size_t)g->n, &d_label, &cp_label));
  GR_TRY(cc_run(g, g->cc, (int32_t *)d_label, s));
  if (cp_label)
    GR_CUDA(cudaMemcpyAsync(label, d_label, sizeof(int32_t) * (size_t)g->n,
                            cudaMemcpyDeviceToHost, s));
  if (num_components) {
    int32_t h = 0;
    GR_CUDA(cudaMemcpyAsync(&h, g->cc->counter.p, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    GR_CUDA(cudaStreamSynchronize(s));
    *num_components = h;
  }
  GR_TRY(end_call(g, s));
  return GR_OK;
}

}  // extern "C"
