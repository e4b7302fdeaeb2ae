// Instantiations of the batched adjoint scatter on wide tiles (TA x 64
// subpixels), the second tile shape the batched calls' autotuner chooses
// from: element-wise staging for radius classes 1 .. 12, bulk-copy staging
// for 3 .. 12, both boundary rules.
#include "epsc_bwd.cuh"
#include "epsc_launch.h"

namespace epsc {

constexpr int TB_WIDE = 64;
static_assert(BwdSmem<MAX_RP1, TB_WIDE>::BYTES <= 200 * 1024, "wide scatter tile shared memory");

#define EPSC_WIDE_PAIR(KERNEL, R)                                                        \
  {clamp ? (const void *)&KERNEL<R, EPS_BC_CLAMP, TB_WIDE>                               \
         : (const void *)&KERNEL<R, EPS_BC_PERIODIC, TB_WIDE>,                           \
   BwdSmem<R, TB_WIDE>::BYTES}

KernelEntry bwd_batched_wide_entry(int rp1, int bc) {
  const bool clamp = bc == EPS_BC_CLAMP;
  switch (rp1) {
#define EPSC_CASE(R) \
  case R:            \
    return EPSC_WIDE_PAIR(bwd_batched_kernel, R);
    EPSC_CASE(1) EPSC_CASE(2) EPSC_CASE(3) EPSC_CASE(4) EPSC_CASE(5) EPSC_CASE(6)
    EPSC_CASE(7) EPSC_CASE(8) EPSC_CASE(9) EPSC_CASE(10) EPSC_CASE(11) EPSC_CASE(12)
#undef EPSC_CASE
    default: return {nullptr, 0};
  }
}

KernelEntry bwd_tma_batched_wide_entry(int rp1, int bc) {
  const bool clamp = bc == EPS_BC_CLAMP;
  switch (rp1) {
#define EPSC_CASE(R) \
  case R:            \
    return EPSC_WIDE_PAIR(bwd_tma_batched_kernel, R);
    EPSC_CASE(3) EPSC_CASE(4) EPSC_CASE(5) EPSC_CASE(6) EPSC_CASE(7) EPSC_CASE(8)
    EPSC_CASE(9) EPSC_CASE(10) EPSC_CASE(11) EPSC_CASE(12)
#undef EPSC_CASE
    default: return {nullptr, 0};
  }
}

#undef EPSC_WIDE_PAIR

}  // namespace epsc
