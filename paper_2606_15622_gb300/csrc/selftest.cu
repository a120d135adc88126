// selftest.cu -- self-test of the bounded mbarrier wait that every consumer
// of a bulk copy in this library uses (tma.cuh): one CTA initialises an
// mbarrier that nothing completes and waits on its first phase with a short
// limit; the wait must give up and say so instead of spinning.
#include <cstdint>

#include "tma.cuh"

namespace fpc {

__global__ void wait_timeout_kernel(uint64_t limit_ns, int32_t *status, uint64_t *waited_ns) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) mbar_init(&bar, 1);
  __syncthreads();
  if (threadIdx.x == 0) {
    const uint64_t t0 = global_timer_ns();
    const bool completed = mbar_wait_bounded(&bar, 0, limit_ns);
    *waited_ns = global_timer_ns() - t0;
    *status = completed ? 1 : 0;
  }
}

void launch_wait_timeout(uint64_t limit_ns, int32_t *status, uint64_t *waited_ns, cudaStream_t st) {
  wait_timeout_kernel<<<1, 32, 0, st>>>(limit_ns, status, waited_ns);
}

}  // namespace fpc
