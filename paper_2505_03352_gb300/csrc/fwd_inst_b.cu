// Explicit instantiations of the forward (stencil) kernels for RP1 = 7 .. 12, both
// boundary rules, single-region and batched.
#include "epsc_fwd.cuh"
#include "epsc_launch.h"

namespace epsc {

KernelEntry fwd_entry_b(int rp1, int bc, bool batched) {
  const bool clamp = bc == EPS_BC_CLAMP;
  switch (rp1) {
    case 7:
      if (batched)
        return {clamp ? (const void *)&fwd_batched_kernel<7, EPS_BC_CLAMP> : (const void *)&fwd_batched_kernel<7, EPS_BC_PERIODIC>, FwdSmem<7>::BYTES};
      return {clamp ? (const void *)&fwd_kernel<7, EPS_BC_CLAMP> : (const void *)&fwd_kernel<7, EPS_BC_PERIODIC>, FwdSmem<7>::BYTES};
    case 8:
      if (batched)
        return {clamp ? (const void *)&fwd_batched_kernel<8, EPS_BC_CLAMP> : (const void *)&fwd_batched_kernel<8, EPS_BC_PERIODIC>, FwdSmem<8>::BYTES};
      return {clamp ? (const void *)&fwd_kernel<8, EPS_BC_CLAMP> : (const void *)&fwd_kernel<8, EPS_BC_PERIODIC>, FwdSmem<8>::BYTES};
    case 9:
      if (batched)
        return {clamp ? (const void *)&fwd_batched_kernel<9, EPS_BC_CLAMP> : (const void *)&fwd_batched_kernel<9, EPS_BC_PERIODIC>, FwdSmem<9>::BYTES};
      return {clamp ? (const void *)&fwd_kernel<9, EPS_BC_CLAMP> : (const void *)&fwd_kernel<9, EPS_BC_PERIODIC>, FwdSmem<9>::BYTES};
    case 10:
      if (batched)
        return {clamp ? (const void *)&fwd_batched_kernel<10, EPS_BC_CLAMP> : (const void *)&fwd_batched_kernel<10, EPS_BC_PERIODIC>, FwdSmem<10>::BYTES};
      return {clamp ? (const void *)&fwd_kernel<10, EPS_BC_CLAMP> : (const void *)&fwd_kernel<10, EPS_BC_PERIODIC>, FwdSmem<10>::BYTES};
    case 11:
      if (batched)
        return {clamp ? (const void *)&fwd_batched_kernel<11, EPS_BC_CLAMP> : (const void *)&fwd_batched_kernel<11, EPS_BC_PERIODIC>, FwdSmem<11>::BYTES};
      return {clamp ? (const void *)&fwd_kernel<11, EPS_BC_CLAMP> : (const void *)&fwd_kernel<11, EPS_BC_PERIODIC>, FwdSmem<11>::BYTES};
    case 12:
      if (batched)
        return {clamp ? (const void *)&fwd_batched_kernel<12, EPS_BC_CLAMP> : (const void *)&fwd_batched_kernel<12, EPS_BC_PERIODIC>, FwdSmem<12>::BYTES};
      return {clamp ? (const void *)&fwd_kernel<12, EPS_BC_CLAMP> : (const void *)&fwd_kernel<12, EPS_BC_PERIODIC>, FwdSmem<12>::BYTES};
    default: return {nullptr, 0};
  }
}

}  // namespace epsc
