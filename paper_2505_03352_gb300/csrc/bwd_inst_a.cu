// Explicit instantiations of the adjoint scatter kernels for RP1 = 1 .. 6, both
// boundary rules, single-region and batched.
#include "epsc_bwd.cuh"
#include "epsc_launch.h"

namespace epsc {

KernelEntry bwd_entry_a(int rp1, int bc, bool batched) {
  const bool clamp = bc == EPS_BC_CLAMP;
  switch (rp1) {
    case 1:
      if (batched)
        return {clamp ? (const void *)&bwd_batched_kernel<1, EPS_BC_CLAMP> : (const void *)&bwd_batched_kernel<1, EPS_BC_PERIODIC>, BwdSmem<1>::BYTES};
      return {clamp ? (const void *)&bwd_kernel<1, EPS_BC_CLAMP> : (const void *)&bwd_kernel<1, EPS_BC_PERIODIC>, BwdSmem<1>::BYTES};
    case 2:
      if (batched)
        return {clamp ? (const void *)&bwd_batched_kernel<2, EPS_BC_CLAMP> : (const void *)&bwd_batched_kernel<2, EPS_BC_PERIODIC>, BwdSmem<2>::BYTES};
      return {clamp ? (const void *)&bwd_kernel<2, EPS_BC_CLAMP> : (const void *)&bwd_kernel<2, EPS_BC_PERIODIC>, BwdSmem<2>::BYTES};
    case 3:
      if (batched)
        return {clamp ? (const void *)&bwd_batched_kernel<3, EPS_BC_CLAMP> : (const void *)&bwd_batched_kernel<3, EPS_BC_PERIODIC>, BwdSmem<3>::BYTES};
      return {clamp ? (const void *)&bwd_kernel<3, EPS_BC_CLAMP> : (const void *)&bwd_kernel<3, EPS_BC_PERIODIC>, BwdSmem<3>::BYTES};
    case 4:
      if (batched)
        return {clamp ? (const void *)&bwd_batched_kernel<4, EPS_BC_CLAMP> : (const void *)&bwd_batched_kernel<4, EPS_BC_PERIODIC>, BwdSmem<4>::BYTES};
      return {clamp ? (const void *)&bwd_kernel<4, EPS_BC_CLAMP> : (const void *)&bwd_kernel<4, EPS_BC_PERIODIC>, BwdSmem<4>::BYTES};
    case 5:
      if (batched)
        return {clamp ? (const void *)&bwd_batched_kernel<5, EPS_BC_CLAMP> : (const void *)&bwd_batched_kernel<5, EPS_BC_PERIODIC>, BwdSmem<5>::BYTES};
      return {clamp ? (const void *)&bwd_kernel<5, EPS_BC_CLAMP> : (const void *)&bwd_kernel<5, EPS_BC_PERIODIC>, BwdSmem<5>::BYTES};
    case 6:
      if (batched)
        return {clamp ? (const void *)&bwd_batched_kernel<6, EPS_BC_CLAMP> : (const void *)&bwd_batched_kernel<6, EPS_BC_PERIODIC>, BwdSmem<6>::BYTES};
      return {clamp ? (const void *)&bwd_kernel<6, EPS_BC_CLAMP> : (const void *)&bwd_kernel<6, EPS_BC_PERIODIC>, BwdSmem<6>::BYTES};
    default: return {nullptr, 0};
  }
}

}  // namespace epsc
