// Diagnostics for failure handling, exercised without faulting the GPU:
//   * gr_diag_wait_timeout runs the library's bounded spin wait against a
//     flag that nothing sets, with a caller-chosen limit, and reports the
//     timeout status the kernel records (the context stays usable);
//   * gr_diag_fail_alloc makes the library's device allocations fail on
//     the host side, so that callers' GR_ENOMEM paths can be tested.
#include "gr_internal.cuh"

namespace gr {

std::atomic<int64_t> g_fail_alloc_after{-1};

namespace {

// Spin on *flag (never set) up to `limit` polls; record the outcome.
__global__ void k_wait_flag(const volatile int32_t *flag, int64_t limit, int32_t *status) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  int64_t spins = 0;
  while (*flag == 0) {
    if (++spins > limit) {
      *status = kDevTimeout;
      return;
    }
    __nanosleep(64);
  }
  *status = kDevOk;
}

}  // namespace
}  // namespace gr

using namespace gr;

extern "C" {

gr_status gr_diag_wait_timeout(int64_t spin_limit, void *stream) {
  clear_error();
  if (spin_limit < 0 || spin_limit > kSpinLimit)
    return fail(GR_EINVAL, "spin_limit must be in [0, 2^24]");
  cudaStream_t s = (cudaStream_t)stream;
  DevMem buf;
  GR_TRY(buf.alloc(2 * sizeof(int32_t), "diagnostic flags"));
  GR_CUDA(cudaMemsetAsync(buf.p, 0, 2 * sizeof(int32_t), s));
  int32_t *f = buf.as<int32_t>();
  k_wait_flag<<<1, 32, 0, s>>>(f, spin_limit, f + 1);
  GR_CUDA(cudaGetLastError());
  int32_t st = -1;
  GR_CUDA(cudaMemcpyAsync(&st, f + 1, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  GR_CUDA(cudaStreamSynchronize(s));
  if (st == kDevTimeout) return fail(GR_ETIMEOUT, "device wait gave up after its limit");
  return GR_OK;
}

gr_status gr_diag_guard(int32_t *site, int64_t *index, int64_t *bound) {
  clear_error();
  gr_status (*reporters[])(GuardRec *) = {guard_report_bfs, guard_report_batch,
                                          guard_report_sssp, guard_report_cc, guard_report_pr};
  if (site) *site = 0;
  for (auto rep : reporters) {
    GuardRec r;
    GR_TRY(rep(&r));
    if (r.hit) {
      if (site) *site = r.site;
      if (index) *index = r.idx;
      if (bound) *bound = r.bound;
      break;
    }
  }
  return GR_OK;
}

gr_status gr_diag_fail_alloc(int64_t after) {
  clear_error();
  g_fail_alloc_after.store(after < 0 ? -1 : after);
  return GR_OK;
}

}  // extern "C"
