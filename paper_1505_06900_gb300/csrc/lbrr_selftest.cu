// Self-test of the bounded waits used by the kernels that hand work over
// with mbarriers: one block waits on an mbarrier that nothing arrives on,
// with the same try-wait loop as those kernels, and records the expiry in
// *status like them. Nothing is in flight, so the block simply returns.
#include "lbrr_launch.h"
#include "lbrr_tc.cuh"

namespace lbrr {

namespace {

__global__ void __launch_bounds__(32) wait_selftest_kernel(uint32_t iterations, int *status) {
  __shared__ uint64_t mbar;
  const uint32_t a = tc::smem_u32(&mbar);
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(a) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  __syncthreads();
  const bool ok = tc::mbar_wait(a, 0, iterations);  // phase 0 never completes
  if (__syncthreads_or(!ok) && threadIdx.x == 0) atomicExch(status, 1);
}

}  // namespace

cudaError_t launch_wait_selftest(unsigned iterations, int *status, cudaStream_t st) {
  wait_selftest_kernel<<<1, 32, 0, st>>>(iterations, status);
  return cudaGetLastError();
}

}  // namespace lbrr
