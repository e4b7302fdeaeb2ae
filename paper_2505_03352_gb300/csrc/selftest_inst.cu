// Self-test of the device-side timeout path: one block waits, with the
// contraction kernels' bounded mbarrier wait, on a barrier nothing arrives
// at; the wait gives up after `cycles` SM clock cycles, the block records
// the timeout in the error flag and returns.
#include "epsc_contract_tma.cuh"
#include "epsc_launch.h"

namespace epsc {

__global__ void __launch_bounds__(NTHREADS) selftest_timeout_kernel(const __grid_constant__ SelftestArgs a) {
  __shared__ uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);   // one arrival completes phase 0; none comes
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  __syncthreads();
  if (threadIdx.x == 0 && !mbar_wait_bounded(&bar, 0u, a.cycles)) atomicOr(a.err, ERRFLAG_TIMEOUT);
}

const void *selftest_timeout_entry() { return (const void *)&selftest_timeout_kernel; }

}  // namespace epsc
