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
// Symmetric graphs store each undirected edge twice; only the (u, v) with
// u > v copy hooks. For a directed CSR every arc hooks, giving weakly
// connected components.
#include <algorithm>

#include "advance.cuh"

namespace gr {

constexpr int kCcThreads = 256, kCcItems = 8;

struct CcWorkspace {
  DevMem counter;
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

struct HookF {
  int32_t *label;
  int32_t only_lower;  // symmetric graph: hook each undirected edge once
  int32_t n;
  __device__ __forceinline__ int operator()(int32_t u, int32_t v, int32_t) const {
    if (!GR_IN(u, n, 401) || !GR_IN(v, n, 402)) return 0;
    if (only_lower && v >= u) return 0;
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
    return 0;  // edge settled: filtered out of the edge frontier
  }
};

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

size_t cc_ws_bytes(const gr_graph *) { return sizeof(int32_t) * 4; }

gr_status cc_ws_create(gr_graph *, CcWorkspace **out) {
  std::unique_ptr<CcWorkspace> ws(new CcWorkspace());
  GR_TRY(ws->counter.alloc(sizeof(int32_t) * 4, "CC counters"));
  *out = ws.release();
  return GR_OK;
}

// CC into a device label array with an explicit workspace; the component
// count is left in the workspace counter (cc_count reads it).
gr_status cc_run(gr_graph *g, CcWorkspace *ws, int32_t *label, cudaStream_t s) {
  int32_t *cnt = ws->counter.as<int32_t>();
  const int grid = g->num_sms * 8;
  GR_CUDA(cudaMemsetAsync(cnt, 0, sizeof(int32_t), s));
  k_cc_init<<<grid, 256, 0, s>>>(label, g->n);
  k_cc_hook<<<g->num_sms * 4, kCcThreads, 0, s>>>(g->row_off.as<int32_t>(),
                                                  g->col.as<int32_t>(), g->n, label,
                                                  g->symmetric ? 1 : 0);
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
