// Explicit instantiations of the adjoint scatter with bulk-copy staging,
// single-region and batched, radius classes 3 .. 12 (smaller classes keep
// the element-wise gather), both boundary rules.
#include "epsc_bwd.cuh"
#include "epsc_launch.h"

namespace epsc {

KernelEntry bwd_tma_entry(int rp1, int bc) {
  const bool clamp = bc == EPS_BC_CLAMP;
  switch (rp1) {
#define EPSC_BWD_TMA_CASE(R)                                                             \
  case R:                                                                              \
    return {clamp ? (const void *)&bwd_tma_kernel<R, EPS_BC_CLAMP>                     \
                  : (const void *)&bwd_tma_kernel<R, EPS_BC_PERIODIC>,                 \
            BwdSmem<R>::BYTES};
    EPSC_BWD_TMA_CASE(3) EPSC_BWD_TMA_CASE(4) EPSC_BWD_TMA_CASE(5) EPSC_BWD_TMA_CASE(6)
    EPSC_BWD_TMA_CASE(7) EPSC_BWD_TMA_CASE(8) EPSC_BWD_TMA_CASE(9) EPSC_BWD_TMA_CASE(10)
    EPSC_BWD_TMA_CASE(11) EPSC_BWD_TMA_CASE(12)
#undef EPSC_BWD_TMA_CASE
    default: return {nullptr, 0};
  }
}

KernelEntry bwd_tma_batched_entry(int rp1, int bc) {
  const bool clamp = bc == EPS_BC_CLAMP;
  switch (rp1) {
#define EPSC_BWD_TMA_BATCH_CASE(R)                                                       \
  case R:                                                                              \
    return {clamp ? (const void *)&bwd_tma_batched_kernel<R, EPS_BC_CLAMP>             \
                  : (const void *)&bwd_tma_batched_kernel<R, EPS_BC_PERIODIC>,         \
            BwdSmem<R>::BYTES};
    EPSC_BWD_TMA_BATCH_CASE(3) EPSC_BWD_TMA_BATCH_CASE(4) EPSC_BWD_TMA_BATCH_CASE(5)
    EPSC_BWD_TMA_BATCH_CASE(6) EPSC_BWD_TMA_BATCH_CASE(7) EPSC_BWD_TMA_BATCH_CASE(8)
    EPSC_BWD_TMA_BATCH_CASE(9) EPSC_BWD_TMA_BATCH_CASE(10) EPSC_BWD_TMA_BATCH_CASE(11)
    EPSC_BWD_TMA_BATCH_CASE(12)
#undef EPSC_BWD_TMA_BATCH_CASE
    default: return {nullptr, 0};
  }
}

}  // namespace epsc
