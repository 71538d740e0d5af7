// pr_selftest_wait: the failure path of the library's bounded device waits, exercised on purpose.
//
// Every wait in the tcgen05 kernels goes through ptx::mbar_wait, which gives up after a fixed limit,
// records a code in a device error word and returns false; the kernel then stops its work and the host
// reports PR_ETIMEOUT with the CUDA context intact. A wait that runs out needs a barrier that nothing
// completes. This kernel sets one up (an mbarrier expecting one arrival that never comes), waits on it
// with the same helper and returns: no trap, no fault, no endless loop.
#include "pr_internal.h"
#include "tc_ptx.h"

#include <string>

namespace {

__global__ void k_wait_selftest(int* err, unsigned long long* elapsed_ns) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x != 0) return;
  const uint32_t b = pr::ptx::smem_u32(&bar);
  pr::ptx::mbar_init(b, 1);
  pr::ptx::fence_barrier_init();
  const uint64_t t0 = pr::ptx::globaltimer();
  const bool done = pr::ptx::mbar_wait(b, 0, err, 99);  // nothing arrives: runs out after the limit
  *elapsed_ns = pr::ptx::globaltimer() - t0;
  if (done) atomicCAS(err, 0, -1);  // the phase completed although nothing arrived: report it
}

}  // namespace

extern "C" {

pr_status pr_selftest_wait(void* stream, double* waited_s) {
  cudaStream_t s = (cudaStream_t)stream;
  int* err = nullptr;
  unsigned long long* el = nullptr;
  int word = 0;
  unsigned long long ns = 0;
  cudaError_t e = cudaMalloc((void**)&err, sizeof(int));
  if (e == cudaSuccess) e = cudaMalloc((void**)&el, sizeof(unsigned long long));
  if (e == cudaSuccess) e = cudaMemsetAsync(err, 0, sizeof(int), s);
  if (e == cudaSuccess) {
    k_wait_selftest<<<1, 32, 0, s>>>(err, el);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(&word, err, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&ns, el, sizeof(ns), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (err) cudaFree(err);
  if (el) cudaFree(el);
  if (e != cudaSuccess) {
    pr::set_handleless_error((std::string("pr_selftest_wait: ") + cudaGetErrorName(e)).c_str());
    return e == cudaErrorMemoryAllocation ? PR_ENOMEM : PR_ECUDA;
  }
  if (waited_s) *waited_s = (double)ns * 1e-9;
  if (word == 99) {
    pr::set_handleless_error("pr_selftest_wait: the bounded wait expired (expected)");
    return PR_ETIMEOUT;
  }
  pr::set_handleless_error("pr_selftest_wait: the wait did not run out");
  return PR_ECUDA;
}

}  // extern "C"
