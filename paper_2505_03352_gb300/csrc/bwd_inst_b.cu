// Explicit instantiations of the adjoint scatter kernels for RP1 = 7 .. 12, both
// boundary rules, single-region and batched.
#include "epsc_bwd.cuh"
#include "epsc_launch.h"

namespace epsc {

KernelEntry bwd_entry_b(int rp1, int bc, bool batched) {
  const bool clamp = bc == EPS_BC_CLAMP;
  switch (rp1) {
    case 7:
      if (batched)
        return {clamp ? (const void *)&bwd_batched_kernel<7, EPS_BC_CLAMP> : (const void *)&bwd_batched_kernel<7, EPS_BC_PERIODIC>, BwdSmem<7>::BYTES};
      return {clamp ? (const void *)&bwd_kernel<7, EPS_BC_CLAMP> : (const void *)&bwd_kernel<7, EPS_BC_PERIODIC>, BwdSmem<7>::BYTES};
    case 8:
      if (batched)
        return {clamp ? (const void *)&bwd_batched_kernel<8, EPS_BC_CLAMP> : (const void *)&bwd_batched_kernel<8, EPS_BC_PERIODIC>, BwdSmem<8>::BYTES};
      return {clamp ? (const void *)&bwd_kernel<8, EPS_BC_CLAMP> : (const void *)&bwd_kernel<8, EPS_BC_PERIODIC>, BwdSmem<8>::BYTES};
    case 9:
      if (batched)
        return {clamp ? (const void *)&bwd_batched_kernel<9, EPS_BC_CLAMP> : (const void *)&bwd_batched_kernel<9, EPS_BC_PERIODIC>, BwdSmem<9>::BYTES};
      return {clamp ? (const void *)&bwd_kernel<9, EPS_BC_CLAMP> : (const void *)&bwd_kernel<9, EPS_BC_PERIODIC>, BwdSmem<9>::BYTES};
    case 10:
      if (batched)
        return {clamp ? (const void *)&bwd_batched_kernel<10, EPS_BC_CLAMP> : (const void *)&bwd_batched_kernel<10, EPS_BC_PERIODIC>, BwdSmem<10>::BYTES};
      return {clamp ? (const void *)&bwd_kernel<10, EPS_BC_CLAMP> : (const void *)&bwd_kernel<10, EPS_BC_PERIODIC>, BwdSmem<10>::BYTES};
    case 11:
      if (batched)
        return {clamp ? (const void *)&bwd_batched_kernel<11, EPS_BC_CLAMP> : (const void *)&bwd_batched_kernel<11, EPS_BC_PERIODIC>, BwdSmem<11>::BYTES};
      return {clamp ? (const void *)&bwd_kernel<11, EPS_BC_CLAMP> : (const void *)&bwd_kernel<11, EPS_BC_PERIODIC>, BwdSmem<11>::BYTES};
    case 12:
      if (batched)
        return {clamp ? (const void *)&bwd_batched_kernel<12, EPS_BC_CLAMP> : (const void *)&bwd_batched_kernel<12, EPS_BC_PERIODIC>, BwdSmem<12>::BYTES};
      return {clamp ? (const void *)&bwd_kernel<12, EPS_BC_CLAMP> : (const void *)&bwd_kernel<12, EPS_BC_PERIODIC>, BwdSmem<12>::BYTES};
    default: return {nullptr, 0};
  }
}

}  // namespace epsc
