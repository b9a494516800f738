// Internal definitions shared by the library's translation units: the graph
// object, error reporting, scratch buffers and warp/block primitives.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <memory>
#include <mutex>
#include <string>
#include <vector>

#include "gr.h"

namespace gr {

// ------------------------------------------------------------ errors
void set_error(const std::string &msg);
void clear_error();
gr_status fail(gr_status st, const std::string &msg);
gr_status cuda_fail(cudaError_t e, const char *what);

#define GR_CUDA(call)                                   \
  do {                                                  \
    cudaError_t e_ = (call);                            \
    if (e_ != cudaSuccess) return ::gr::cuda_fail(e_, #call); \
  } while (0)

#define GR_TRY(expr)                        \
  do {                                      \
    gr_status s_ = (expr);                  \
    if (s_ != GR_OK) return s_;             \
  } while (0)

// Host-side allocation-failure injection (gr_diag_fail_alloc): when >= 0,
// the number of device allocations still allowed to succeed.
extern std::atomic<int64_t> g_fail_alloc_after;

// Device-side error codes written into control blocks.
enum : int32_t { kDevOk = 0, kDevTimeout = 1, kDevOverflow = 2 };

// Iteration limit of every device-side spin wait; after it the waiting
// thread records kDevTimeout and leaves the wait.
constexpr int64_t kSpinLimit = 1ll << 24;

// ------------------------------------------------------------ buffers
// Owning device allocation (cudaMalloc/cudaFree), move-only.
struct DevMem {
  void *p = nullptr;
  size_t bytes = 0;
  DevMem() = default;
  DevMem(const DevMem &) = delete;
  DevMem &operator=(const DevMem &) = delete;
  ~DevMem() { reset(); }
  void reset() {
    if (p) cudaFree(p);
    p = nullptr;
    bytes = 0;
  }
  gr_status alloc(size_t nbytes, const char *what);
  template <class T>
  T *as() const { return (T *)p; }
};

struct PinnedMem {
  void *p = nullptr;
  ~PinnedMem() {
    if (p) cudaFreeHost(p);
  }
  gr_status alloc(size_t nbytes, const char *what);
  template <class T>
  T *as() const { return (T *)p; }
};

struct BfsWorkspace;
struct SsspWorkspace;
struct CcWorkspace;
struct PrWorkspace;
struct BatchWorkspace;
struct RankWorkspace;

}  // namespace gr

// The opaque handle of the C ABI.
struct gr_graph {
  int device = 0;
  int num_sms = 0;
  int32_t n = 0;
  int64_t m = 0;
  int32_t nwords = 0;  // ceil(n / 32): words of one vertex bitmap
  gr::DevMem row_off, col, w;
  gr::DevMem isolated_bits;  // bit v set iff deg(v) == 0
  gr::DevMem first_col;      // first neighbour of v (C[R[v]]), -1 if deg(v) == 0
  gr::DevMem degree;         // int32 deg(v), used by PageRank
  int32_t max_degree = 0;
  int32_t num_isolated = 0;
  bool symmetric = false;
  bool rows_sorted = false;
  bool has_weights = false;
  uint32_t sssp_delta = 1;    // tuned near/far bucket width
  float tuned_alpha = 14.f;   // push -> pull threshold (see gr_autotune)
  float tuned_beta = 24.f;    // pull -> push threshold
  int32_t tuned_mode = GR_MODE_AUTO;
  int32_t tuned_direction = GR_DIR_AUTO;  // GR_DIR_PUSH: never pull
  int32_t tuned_blocks_per_sm = 0;  // persistent BFS grid (0: all resident)
  int32_t tuned_sssp_mode = GR_MODE_GRAPH;
  int32_t tuned_sssp_blocks_per_sm = 0;
  // SSSP relaxations pull once the near frontier has m / alpha edges (0:
  // never; set by gr_autotune)
  float tuned_sssp_alpha = 0.f;
  double tuned_bfs_ms = 0.0, tuned_sssp_ms = 0.0;  // measured by gr_autotune
  double mean_weight = 0.0;

  std::mutex mu;  // serialises host-side enqueueing on this graph
  cudaEvent_t last_done = nullptr;
  cudaStream_t last_stream = nullptr;
  bool has_last = false;

  // lazily created scratch, one per primitive (freed by destroy_workspaces)
  gr::BfsWorkspace *bfs = nullptr;
  gr::SsspWorkspace *sssp = nullptr;
  gr::SsspWorkspace *sssp_batch = nullptr;  // gr_sssp_batch (lane-major copies)
  gr::CcWorkspace *cc = nullptr;
  gr::PrWorkspace *pr = nullptr;
  gr::BatchWorkspace *batch = nullptr;
  gr::RankWorkspace *rank = nullptr;  // gr_neighbor_reduce, gr_hits, gr_salsa, gr_ppr

  gr::DevMem stage[2];  // device staging for host output pointers

  // gr_bfs_multi: a copy stream for host outputs, two staging sets (depth,
  // parent) that alternate between searches, and per set the events "the
  // search filled it" and "its copies finished"
  cudaStream_t copy_stream = nullptr;
  gr::DevMem pipe_stage[2][2];
  cudaEvent_t pipe_filled[2] = {nullptr, nullptr};
  cudaEvent_t pipe_free[2] = {nullptr, nullptr};

  ~gr_graph();
};

namespace gr {

// Begin/end of a call that uses the graph's scratch on `s`: orders the call
// after the previous call on the graph when that ran on another stream.
gr_status begin_call(gr_graph *g, cudaStream_t s);
gr_status end_call(gr_graph *g, cudaStream_t s);

// Whether an output pointer is host memory (NULL counts as device); fails
// for device memory of another device.
gr_status output_on_host(const gr_graph *g, const void *user, bool *host);

// Output pointer handling: returns a device pointer to write to. If `user`
// is host memory, a staging buffer of `bytes` is used and *needs_copy set.
gr_status resolve_output(gr_graph *g, int slot, void *user, size_t bytes,
                         void **dev, bool *needs_copy);

const gr_opts &default_opts();

// Internal primitive entry points with explicit workspaces (device outputs,
// no locking, no staging); used by the C ABI wrappers and the server.
gr_status bfs_ws_create(gr_graph *g, cudaStream_t s, BfsWorkspace **out);
size_t bfs_ws_bytes(const gr_graph *g);
gr_status bfs_check(const gr_graph *g, int32_t src, const gr_opts &o);
gr_status bfs_run(gr_graph *g, BfsWorkspace *ws, int32_t src, int32_t *depth, int32_t *parent,
                  const gr_opts &o, cudaStream_t s);
gr_status bfs_read_ctl_error(BfsWorkspace *ws, cudaStream_t s);
// lanes > 1: buffers for that many lane-major copies (sssp_batch_run)
gr_status sssp_ws_create(gr_graph *g, cudaStream_t s, SsspWorkspace **out, int32_t lanes = 1);
size_t sssp_ws_bytes(const gr_graph *g, int32_t lanes = 1);
// most sources one batched SSSP run on this graph may take
int32_t sssp_batch_max_lanes(const gr_graph *g);
// k searches (k <= the workspace's lanes) into dist[k][n] on the device
gr_status sssp_batch_run(gr_graph *g, SsspWorkspace *ws, const int32_t *h_srcs, int32_t k,
                         uint32_t *dist, const gr_opts &o, cudaStream_t s);
gr_status sssp_check(const gr_graph *g, int32_t src, const gr_opts &o);
// GR_ETIMEOUT when the last SSSP on ws stopped at a device-side limit
gr_status sssp_read_ctl_error(SsspWorkspace *ws, cudaStream_t s);
gr_status sssp_run(gr_graph *g, SsspWorkspace *ws, int32_t src, uint32_t *dist, int32_t *pred,
                   const gr_opts &o, cudaStream_t s);
gr_status cc_ws_create(gr_graph *g, CcWorkspace **out);
size_t cc_ws_bytes(const gr_graph *g);
gr_status cc_run(gr_graph *g, CcWorkspace *ws, int32_t *label, cudaStream_t s);
gr_status batch_ws_create(gr_graph *g, BatchWorkspace **out);
size_t batch_ws_bytes(const gr_graph *g);
gr_status bfs_batch_run(gr_graph *g, BatchWorkspace *ws, const int32_t *h_srcs, int32_t k,
                        int32_t *depth, int32_t max_levels, cudaStream_t s);
// GR_ETIMEOUT when the last batched BFS on ws stopped at a device-side limit
gr_status batch_read_ctl_error(BatchWorkspace *ws, cudaStream_t s);

// Degree-statistics prior of the tuned settings (set at graph creation).
void tune_prior(gr_graph *g);

// Per-primitive scratch release, defined next to each primitive.
void free_bfs(BfsWorkspace *);
void free_sssp(SsspWorkspace *);
void free_cc(CcWorkspace *);
void free_pr(PrWorkspace *);
void free_batch(BatchWorkspace *);
void free_rank(RankWorkspace *);

// ------------------------------------------------------ bounds guards
// In a GR_CHECKED build every data-dependent index of the kernels is checked
// before use: an index outside its buffer records (site, index, bound) in a
// per-translation-unit record and the access is skipped; gr_diag_guard
// reports the first record. Normal builds compile the checks away.
struct GuardRec {
  int32_t hit;
  int32_t site;
  long long idx;
  long long bound;
};

#ifdef GR_CHECKED
namespace {
__device__ GuardRec g_guard_rec;
__device__ __noinline__ void gr_guard_fail(int site, long long idx, long long bound) {
  if (atomicCAS(&g_guard_rec.hit, 0, 1) == 0) {
    g_guard_rec.site = site;
    g_guard_rec.idx = idx;
    g_guard_rec.bound = bound;
  }
}
}  // namespace
#define GR_IN(idx, bound, site)                                                  \
  ((((long long)(idx)) >= 0 && ((long long)(idx)) < ((long long)(bound)))        \
       ? true                                                                    \
       : (gr_guard_fail((site), (long long)(idx), (long long)(bound)), false))
#define GR_GUARD_REPORTER(name)                                                  \
  gr_status name(GuardRec *out) {                                                \
    GR_CUDA(cudaMemcpyFromSymbol(out, g_guard_rec, sizeof(GuardRec)));           \
    return GR_OK;                                                                \
  }
#else
#define GR_IN(idx, bound, site) true
#define GR_GUARD_REPORTER(name)                                                  \
  gr_status name(GuardRec *out) {                                                \
    out->hit = 0;                                                                \
    return GR_OK;                                                                \
  }
#endif

// one reporter per translation unit with guarded kernels
gr_status guard_report_bfs(GuardRec *);
gr_status guard_report_batch(GuardRec *);
gr_status guard_report_sssp(GuardRec *);
gr_status guard_report_cc(GuardRec *);
gr_status guard_report_pr(GuardRec *);

// ------------------------------------------------------ device helpers
__device__ __forceinline__ int lane_id() { return threadIdx.x & 31; }

template <class T>
__device__ __forceinline__ T warp_incl_sum(T v) {
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    T t = __shfl_up_sync(0xffffffffu, v, o);
    if (lane_id() >= o) v += t;
  }
  return v;
}

template <class T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Block-wide exclusive sum; `smem` holds >= 33 elements. Returns the
// exclusive prefix of this thread and writes the block total to *total.
template <class T>
__device__ __forceinline__ T block_excl_sum(T v, T *smem, T *total) {
  const int lane = lane_id(), wid = threadIdx.x >> 5;
  const int nw = (blockDim.x + 31) >> 5;
  T incl = warp_incl_sum(v);
  if (lane == 31) smem[wid] = incl;
  __syncthreads();
  if (wid == 0) {
    T x = lane < nw ? smem[lane] : T(0);
    T xi = warp_incl_sum(x);
    if (lane < nw) smem[lane] = xi - x;
    if (lane == nw - 1) smem[32] = xi;
  }
  __syncthreads();
  T res = smem[wid] + incl - v;
  *total = smem[32];
  __syncthreads();
  return res;
}

template <class T>
__device__ __forceinline__ T block_sum(T v, T *smem) {
  T total;
  block_excl_sum(v, smem, &total);
  return total;
}

__device__ __forceinline__ bool test_bit(const uint32_t *bits, int32_t v) {
  return (bits[v >> 5] >> (v & 31)) & 1u;
}

}  // namespace gr
