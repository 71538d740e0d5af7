// pr_norms_noalloc: the norms of the initial guess computed without any device allocation.
//
// Who needs it: code that must not call cudaMalloc/cudaFree. Examples are work issued while a CUDA graph
// is being captured (allocation calls are not capturable and fail or invalidate the capture), paths
// where the implicit synchronisation of cudaFree is not acceptable, and applications whose device memory
// is already reserved in full by their own caching allocator or fixed budget. Such callers pass their own
// input and output buffers, and the library's scratch lives in a fixed array in the module's device
// memory instead.
#include "pr_internal.h"

#include <mutex>

namespace {

constexpr int kMaxDevices = 64;

// Column and row abs-sums, PR_NORMS_NOALLOC_MAX_N doubles each. Every device that loads the library keeps
// this array (2 x 65536 x 8 bytes = 1 MiB) until the process exits. All calls on a device share it.
__device__ __align__(256) double g_norm_scratch[2 * PR_NORMS_NOALLOC_MAX_N];

std::mutex g_mu;
double* g_scratch_addr[kMaxDevices] = {};  // device address of g_norm_scratch, per device

// In host code g_norm_scratch names a host-side stand-in, not device memory, so the kernels get the
// address that cudaGetSymbolAddress reports for the current device (looked up once per device).
cudaError_t scratch_for_current_device(double** out) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_norm_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_addr[dev] = static_cast<double*>(p);
  }
  *out = g_scratch_addr[dev];
  return cudaSuccess;
}

}  // namespace

extern "C" pr_status pr_norms_noalloc(const double* A, int64_t n, double* out, void* stream) {
  if (!A || !out) {
    pr::set_handleless_error("pr_norms_noalloc: A or out is NULL");
    return PR_EINVAL;
  }
  if (n < 1 || n > PR_NORMS_NOALLOC_MAX_N) {
    pr::set_handleless_error("pr_norms_noalloc: n must be in [1, PR_NORMS_NOALLOC_MAX_N = 65536]");
    return PR_EINVAL;
  }
  double* scratch = nullptr;
  if (scratch_for_current_device(&scratch) != cudaSuccess) {
    pr::set_handleless_error("pr_norms_noalloc: cudaGetSymbolAddress of the scratch array failed");
    return PR_ECUDA;
  }
  // Each call writes every scratch element it reads (the n column sums and n row sums) before reading
  // it, so nothing has to be cleared between calls; overlapping calls on one device would race.
  if (pr::abs_norms(A, (int)n, scratch, out, (cudaStream_t)stream) != cudaSuccess) {
    pr::set_handleless_error("pr_norms_noalloc: kernel launch failed");
    return PR_ECUDA;
  }
  return PR_OK;
}
