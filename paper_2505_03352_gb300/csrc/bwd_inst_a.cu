// Explicit instantiations of the adjoint scatter kernel for RP1 = 1 .. 6.
#include "epsc_bwd.cuh"
#include "epsc_launch.h"

namespace epsc {

KernelEntry bwd_entry_a(int rp1) {
  switch (rp1) {
    case 1: return {(const void *)&bwd_kernel<1>, BwdSmem<1>::BYTES};
    case 2: return {(const void *)&bwd_kernel<2>, BwdSmem<2>::BYTES};
    case 3: return {(const void *)&bwd_kernel<3>, BwdSmem<3>::BYTES};
    case 4: return {(const void *)&bwd_kernel<4>, BwdSmem<4>::BYTES};
    case 5: return {(const void *)&bwd_kernel<5>, BwdSmem<5>::BYTES};
    case 6: return {(const void *)&bwd_kernel<6>, BwdSmem<6>::BYTES};
    default: return {nullptr, 0};
  }
}

}  // namespace epsc
