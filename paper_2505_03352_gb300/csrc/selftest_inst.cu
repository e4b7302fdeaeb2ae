// Self-tests of the device-side error paths.  Timeout: one block waits,
// with the contraction kernels' bounded mbarrier wait, on a barrier nothing
// arrives at; the wait gives up after `cycles` SM clock cycles, the block
// records the timeout in the error flag and returns.
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

// Debug-bounds builds: one thread runs a bounds check that fails (element n
// of a buffer of n elements) and touches no memory, so the host then reads
// EPS_ERR_DEVICE_BOUNDS.  In release builds the check compiles away.
__global__ void __launch_bounds__(NTHREADS) selftest_bounds_kernel(const __grid_constant__ SelftestArgs a) {
  if (threadIdx.x == 0) {
    [[maybe_unused]] const size_t n = 16;   // unused where the check compiles away
    if (!EPSC_IN_BOUNDS(n, 1, n, a.err)) return;
  }
}

const void *selftest_bounds_entry() { return (const void *)&selftest_bounds_kernel; }

}  // namespace epsc
