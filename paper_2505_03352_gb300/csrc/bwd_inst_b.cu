// Explicit instantiations of the adjoint scatter kernel for RP1 = 7 .. 12.
#include "epsc_bwd.cuh"
#include "epsc_launch.h"

namespace epsc {

KernelEntry bwd_entry_b(int rp1) {
  switch (rp1) {
    case 7: return {(const void *)&bwd_kernel<7>, BwdSmem<7>::BYTES};
    case 8: return {(const void *)&bwd_kernel<8>, BwdSmem<8>::BYTES};
    case 9: return {(const void *)&bwd_kernel<9>, BwdSmem<9>::BYTES};
    case 10: return {(const void *)&bwd_kernel<10>, BwdSmem<10>::BYTES};
    case 11: return {(const void *)&bwd_kernel<11>, BwdSmem<11>::BYTES};
    case 12: return {(const void *)&bwd_kernel<12>, BwdSmem<12>::BYTES};
    default: return {nullptr, 0};
  }
}

}  // namespace epsc
