// Explicit instantiations of the forward kernel for RP1 = 1 .. 6.
#include "epsc_fwd.cuh"
#include "epsc_launch.h"

namespace epsc {

KernelEntry fwd_entry_a(int rp1) {
  switch (rp1) {
    case 1: return {(const void *)&fwd_kernel<1>, FwdSmem<1>::BYTES};
    case 2: return {(const void *)&fwd_kernel<2>, FwdSmem<2>::BYTES};
    case 3: return {(const void *)&fwd_kernel<3>, FwdSmem<3>::BYTES};
    case 4: return {(const void *)&fwd_kernel<4>, FwdSmem<4>::BYTES};
    case 5: return {(const void *)&fwd_kernel<5>, FwdSmem<5>::BYTES};
    case 6: return {(const void *)&fwd_kernel<6>, FwdSmem<6>::BYTES};
    default: return {nullptr, 0};
  }
}

}  // namespace epsc
