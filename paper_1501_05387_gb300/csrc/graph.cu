// Graph object of the C ABI: CSR validation and upload (Sec. 3: CSR with
// row offsets R and column indices C, SOA per-vertex data), per-graph
// derived data, error reporting and call ordering.
#include <cstdio>
#include <algorithm>
#include <cstring>

#include "gr_internal.cuh"

namespace gr {

namespace {
thread_local std::string t_err;
}

void set_error(const std::string &msg) { t_err = msg; }
void clear_error() { t_err.clear(); }

gr_status fail(gr_status st, const std::string &msg) {
  set_error(msg);
  return st;
}

gr_status cuda_fail(cudaError_t e, const char *what) {
  std::string msg = std::string(what) + ": " + cudaGetErrorName(e) + " (" +
                    cudaGetErrorString(e) + ")";
  set_error(msg);
  return e == cudaErrorMemoryAllocation ? GR_ENOMEM : GR_ECUDA;
}

gr_status DevMem::alloc(size_t nbytes, const char *what) {
  reset();
  if (nbytes == 0) nbytes = 16;
  for (int64_t left = g_fail_alloc_after.load(); left >= 0;
       left = g_fail_alloc_after.load()) {
    if (left == 0)
      return fail(GR_ENOMEM, std::string("device allocation for ") + what +
                                 " refused (injected failure)");
    if (g_fail_alloc_after.compare_exchange_weak(left, left - 1)) break;
  }
  cudaError_t e = cudaMalloc(&p, nbytes);
  if (e != cudaSuccess) {
    p = nullptr;
    cudaGetLastError();
    return fail(e == cudaErrorMemoryAllocation ? GR_ENOMEM : GR_ECUDA,
                std::string("device allocation of ") + std::to_string(nbytes) +
                    " bytes for " + what + " failed: " + cudaGetErrorString(e));
  }
  bytes = nbytes;
  return GR_OK;
}

gr_status PinnedMem::alloc(size_t nbytes, const char *what) {
  if (p) cudaFreeHost(p);
  p = nullptr;
  cudaError_t e = cudaMallocHost(&p, nbytes);
  if (e != cudaSuccess) {
    p = nullptr;
    cudaGetLastError();
    return fail(GR_ENOMEM, std::string("pinned allocation for ") + what +
                               " failed: " + cudaGetErrorString(e));
  }
  return GR_OK;
}

const gr_opts &default_opts() {
  static const gr_opts o = {GR_DIR_AUTO, GR_MODE_AUTO, 0, 0, 0.f, 0.f, 0u, 0};
  return o;
}

gr_status begin_call(gr_graph *g, cudaStream_t s) {
  GR_CUDA(cudaSetDevice(g->device));
  if (g->has_last && g->last_stream != s)
    GR_CUDA(cudaStreamWaitEvent(s, g->last_done, 0));
  return GR_OK;
}

gr_status end_call(gr_graph *g, cudaStream_t s) {
  GR_CUDA(cudaEventRecord(g->last_done, s));
  g->last_stream = s;
  g->has_last = true;
  return GR_OK;
}

gr_status output_on_host(const gr_graph *g, const void *user, bool *host) {
  *host = false;
  if (!user) return GR_OK;
  cudaPointerAttributes attr;
  cudaError_t e = cudaPointerGetAttributes(&attr, user);
  if (e != cudaSuccess) {
    cudaGetLastError();
    attr.type = cudaMemoryTypeUnregistered;
  }
  if (attr.type == cudaMemoryTypeDevice || attr.type == cudaMemoryTypeManaged) {
    if (attr.type == cudaMemoryTypeDevice && attr.device != g->device)
      return fail(GR_EINVAL, "output pointer is on another device");
    return GR_OK;
  }
  *host = true;  // page-locked or pageable host memory
  return GR_OK;
}

gr_status resolve_output(gr_graph *g, int slot, void *user, size_t bytes,
                         void **dev, bool *needs_copy) {
  *needs_copy = false;
  *dev = user;
  bool host = false;
  GR_TRY(output_on_host(g, user, &host));
  if (!host) return GR_OK;
  // host memory: write to staging, copy at the end
  DevMem &st = g->stage[slot];
  if (st.bytes < bytes) GR_TRY(st.alloc(bytes, "output staging"));
  *dev = st.p;
  *needs_copy = true;
  return GR_OK;
}

// ------------------------------------------------------- device checks
namespace {

__global__ void k_validate_csr(const int32_t *R, const int32_t *C, int32_t n,
                               int64_t m, int32_t *bad) {
  int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t v = tid; v < n; v += stride) {
    if (R[v] > R[v + 1] || R[v] < 0) atomicOr(bad, 1);
  }
  if (tid == 0 && (R[0] != 0 || (int64_t)R[n] != m)) atomicOr(bad, 2);
  for (int64_t e = tid; e < m; e += stride) {
    int32_t c = C[e];
    if (c < 0 || c >= n) atomicOr(bad, 4);
  }
}

// first neighbour of every vertex, stored densely: the bottom-up (pull)
// BFS level tests it first and reads it with coalesced loads
__global__ void k_first_col(const int32_t *R, const int32_t *C, int32_t n, int32_t *first) {
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n;
       v += (int64_t)gridDim.x * blockDim.x) {
    const int32_t r0 = R[v];
    first[v] = R[v + 1] > r0 ? C[r0] : -1;
  }
}

// degree statistics + isolated-vertex bitmap, one warp per 32 vertices
__global__ void k_graph_stats(const int32_t *R, int32_t n, int32_t nwords,
                              uint32_t *iso_bits, int32_t *deg_out,
                              int32_t *max_deg, int32_t *num_iso) {
  int64_t gw = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  int lane = threadIdx.x & 31;
  int32_t local_max = 0, local_iso = 0;
  for (int64_t w = gw; w < nwords; w += nwarps) {
    int64_t v = w * 32 + lane;
    int32_t d = 0;
    bool iso = false;
    if (v < n) {
      d = R[v + 1] - R[v];
      deg_out[v] = d;
      iso = d == 0;
    }
    uint32_t b = __ballot_sync(0xffffffffu, iso);
    if (lane == 0) {
      iso_bits[w] = b;
      local_iso += __popc(b);
    }
    local_max = max(local_max, d);
  }
  for (int o = 16; o > 0; o >>= 1)
    local_max = max(local_max, __shfl_xor_sync(0xffffffffu, local_max, o));
  if (lane == 0) {
    atomicMax(max_deg, local_max);
    if (local_iso) atomicAdd(num_iso, local_iso);
  }
}

// rows_sorted: every row's columns are non-decreasing (one warp per row)
__global__ void k_rows_sorted(const int32_t *R, const int32_t *C, int32_t n,
                              int32_t *unsorted) {
  int64_t gw = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  int lane = threadIdx.x & 31;
  for (int64_t v = gw; v < n; v += nwarps) {
    bool bad = false;
    for (int32_t e = R[v] + 1 + lane; e < R[v + 1]; e += 32)
      bad |= C[e - 1] > C[e];
    if (__any_sync(0xffffffffu, bad) && lane == 0) *unsorted = 1;
  }
}

// symmetric: for each entry (u, v) the row of v contains u (binary search;
// rows sorted). One warp per row u, lanes over its entries.
__global__ void k_symmetric(const int32_t *R, const int32_t *C, int32_t n,
                            int32_t *asym) {
  int64_t gw = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  int lane = threadIdx.x & 31;
  for (int64_t uu = gw; uu < n; uu += nwarps) {
    int32_t u = (int32_t)uu;
    bool bad = false;
    for (int32_t e = R[u] + lane; e < R[u + 1]; e += 32) {
      int32_t v = C[e];
      int32_t a = R[v], b = R[v + 1], end = b;
      while (a < b) {
        int32_t mid = a + (b - a) / 2;
        if (C[mid] < u) a = mid + 1; else b = mid;
      }
      bad |= (a >= end || C[a] != u);
    }
    if (__any_sync(0xffffffffu, bad) && lane == 0) *asym = 1;
  }
}

__global__ void k_weight_sum(const uint32_t *W, int64_t m, unsigned long long *sum) {
  unsigned long long local = 0;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < m;
       e += (int64_t)gridDim.x * blockDim.x)
    local += W[e];
  for (int o = 16; o > 0; o >>= 1) local += __shfl_xor_sync(0xffffffffu, local, o);
  if ((threadIdx.x & 31) == 0 && local) atomicAdd(sum, local);
}

}  // namespace

gr_status validate_host_csr(int32_t n, int64_t m, const int32_t *R,
                            const int32_t *C) {
  if (R[0] != 0) return fail(GR_EINVAL, "row_off[0] must be 0");
  for (int64_t v = 0; v < n; ++v)
    if (R[v + 1] < R[v])
      return fail(GR_EINVAL, "row_off must be non-decreasing (at vertex " +
                                 std::to_string(v) + ")");
  if ((int64_t)R[n] != m) return fail(GR_EINVAL, "row_off[n] must equal m");
  for (int64_t e = 0; e < m; ++e)
    if (C[e] < 0 || C[e] >= n)
      return fail(GR_EINVAL, "column index out of range at entry " +
                                 std::to_string(e));
  return GR_OK;
}

}  // namespace gr

gr_graph::~gr_graph() {
  if (last_done) cudaEventDestroy(last_done);
  for (int i = 0; i < 2; ++i) {
    if (pipe_filled[i]) cudaEventDestroy(pipe_filled[i]);
    if (pipe_free[i]) cudaEventDestroy(pipe_free[i]);
  }
  if (copy_stream) cudaStreamDestroy(copy_stream);
}

using namespace gr;

namespace gr {
static void destroy_workspaces(gr_graph *g) {
  free_bfs(g->bfs);
  g->bfs = nullptr;
  free_sssp(g->sssp);
  g->sssp = nullptr;
  free_sssp(g->sssp_batch);
  g->sssp_batch = nullptr;
  free_cc(g->cc);
  g->cc = nullptr;
  free_pr(g->pr);
  g->pr = nullptr;
  free_batch(g->batch);
  g->batch = nullptr;
  free_rank(g->rank);
  g->rank = nullptr;
}
}  // namespace gr

extern "C" {

const char *gr_last_error(void) { return gr::t_err.c_str(); }

gr_status gr_graph_create(int32_t n, int64_t m, const int32_t *row_off,
                          const int32_t *col, const uint32_t *w,
                          int inputs_on_device, void *stream, gr_graph **out) {
  clear_error();
  if (!out) return fail(GR_EINVAL, "out must not be NULL");
  *out = nullptr;
  if (n < 1) return fail(GR_EINVAL, "n must be >= 1");
  if (m < 0 || m > INT32_MAX)
    return fail(GR_EINVAL, "m must be in [0, INT32_MAX] (int32 offsets)");
  if (n == INT32_MAX) return fail(GR_EINVAL, "n must be < INT32_MAX");
  if (!row_off || (m > 0 && !col)) return fail(GR_EINVAL, "row_off/col must not be NULL");
  if (!inputs_on_device) GR_TRY(validate_host_csr(n, m, row_off, col));

  cudaStream_t s = (cudaStream_t)stream;
  std::unique_ptr<gr_graph> g(new gr_graph());
  GR_CUDA(cudaGetDevice(&g->device));
  cudaDeviceProp prop;
  GR_CUDA(cudaGetDeviceProperties(&prop, g->device));
  g->num_sms = prop.multiProcessorCount;
  g->n = n;
  g->m = m;
  g->nwords = (n + 31) / 32;
  g->has_weights = w != nullptr;
  GR_CUDA(cudaEventCreateWithFlags(&g->last_done, cudaEventDisableTiming));

  GR_TRY(g->row_off.alloc(sizeof(int32_t) * ((size_t)n + 1), "row offsets"));
  GR_TRY(g->col.alloc(sizeof(int32_t) * (size_t)m, "column indices"));
  if (w) GR_TRY(g->w.alloc(sizeof(uint32_t) * (size_t)m, "weights"));
  cudaMemcpyKind kind = inputs_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  GR_CUDA(cudaMemcpyAsync(g->row_off.p, row_off, sizeof(int32_t) * ((size_t)n + 1), kind, s));
  if (m) GR_CUDA(cudaMemcpyAsync(g->col.p, col, sizeof(int32_t) * (size_t)m, kind, s));
  if (w && m) GR_CUDA(cudaMemcpyAsync(g->w.p, w, sizeof(uint32_t) * (size_t)m, kind, s));

  DevMem flags;
  GR_TRY(flags.alloc(sizeof(int32_t) * 8, "flags"));
  GR_CUDA(cudaMemsetAsync(flags.p, 0, sizeof(int32_t) * 8, s));
  int32_t *f = flags.as<int32_t>();
  int grid = g->num_sms * 4;
  if (inputs_on_device) {
    k_validate_csr<<<grid, 256, 0, s>>>(g->row_off.as<int32_t>(), g->col.as<int32_t>(),
                                        n, m, f + 0);
    GR_CUDA(cudaGetLastError());
  }
  int32_t hf[8];
  GR_CUDA(cudaMemcpyAsync(hf, f, sizeof(hf), cudaMemcpyDeviceToHost, s));
  GR_CUDA(cudaStreamSynchronize(s));
  if (hf[0]) return fail(GR_EINVAL, "invalid CSR (device check flags " + std::to_string(hf[0]) + ")");

  GR_TRY(g->isolated_bits.alloc(sizeof(uint32_t) * (size_t)g->nwords, "isolated bitmap"));
  GR_TRY(g->degree.alloc(sizeof(int32_t) * (size_t)n, "degrees"));
  k_graph_stats<<<grid, 256, 0, s>>>(g->row_off.as<int32_t>(), n, g->nwords,
                                     g->isolated_bits.as<uint32_t>(),
                                     g->degree.as<int32_t>(), f + 1, f + 2);
  GR_CUDA(cudaGetLastError());
  k_rows_sorted<<<grid, 256, 0, s>>>(g->row_off.as<int32_t>(), g->col.as<int32_t>(), n, f + 3);
  GR_CUDA(cudaGetLastError());
  GR_TRY(g->first_col.alloc(sizeof(int32_t) * (size_t)n, "first neighbours"));
  k_first_col<<<grid, 256, 0, s>>>(g->row_off.as<int32_t>(), g->col.as<int32_t>(), n,
                                   g->first_col.as<int32_t>());
  GR_CUDA(cudaGetLastError());
  GR_CUDA(cudaMemcpyAsync(hf, f, sizeof(hf), cudaMemcpyDeviceToHost, s));
  GR_CUDA(cudaStreamSynchronize(s));
  g->max_degree = hf[1];
  g->num_isolated = hf[2];
  g->rows_sorted = hf[3] == 0;
  g->symmetric = false;
  if (g->rows_sorted) {
    k_symmetric<<<grid * 2, 256, 0, s>>>(g->row_off.as<int32_t>(), g->col.as<int32_t>(),
                                          n, f + 4);
    GR_CUDA(cudaGetLastError());
    GR_CUDA(cudaMemcpyAsync(hf, f, sizeof(hf), cudaMemcpyDeviceToHost, s));
    GR_CUDA(cudaStreamSynchronize(s));
    g->symmetric = hf[4] == 0;
  }
  if (w && m) {
    GR_CUDA(cudaMemsetAsync(flags.p, 0, sizeof(unsigned long long), s));
    k_weight_sum<<<grid, 256, 0, s>>>(g->w.as<uint32_t>(), m,
                                      (unsigned long long *)flags.p);
    GR_CUDA(cudaGetLastError());
    unsigned long long wsum = 0;
    GR_CUDA(cudaMemcpyAsync(&wsum, flags.p, sizeof(wsum), cudaMemcpyDeviceToHost, s));
    GR_CUDA(cudaStreamSynchronize(s));
    g->mean_weight = (double)wsum / (double)m;
    // near/far bucket width: a few mean edge weights keeps the near
    // frontier wide enough to fill the GPU
    double d = 2.0 * g->mean_weight;
    g->sssp_delta = (uint32_t)std::max(1.0, std::min(d, 4.0e9));
  }
  tune_prior(g.get());
  *out = g.release();
  return GR_OK;
}

gr_status gr_graph_destroy(gr_graph *g) {
  clear_error();
  if (!g) return GR_OK;
  cudaSetDevice(g->device);
  cudaDeviceSynchronize();
  destroy_workspaces(g);
  delete g;
  return GR_OK;
}

gr_status gr_graph_info(const gr_graph *g, int32_t *n, int64_t *m,
                        int32_t *max_degree, int32_t *num_isolated,
                        int32_t *symmetric, int32_t *has_weights) {
  clear_error();
  if (!g) return fail(GR_EINVAL, "graph must not be NULL");
  if (n) *n = g->n;
  if (m) *m = g->m;
  if (max_degree) *max_degree = g->max_degree;
  if (num_isolated) *num_isolated = g->num_isolated;
  if (symmetric) *symmetric = g->symmetric ? 1 : 0;
  if (has_weights) *has_weights = g->has_weights ? 1 : 0;
  return GR_OK;
}

}  // extern "C"
