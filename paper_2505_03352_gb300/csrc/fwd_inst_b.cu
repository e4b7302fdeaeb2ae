// Explicit instantiations of the forward kernel for RP1 = 7 .. 12.
#include "epsc_fwd.cuh"
#include "epsc_launch.h"

namespace epsc {

KernelEntry fwd_entry_b(int rp1) {
  switch (rp1) {
    case 7: return {(const void *)&fwd_kernel<7>, FwdSmem<7>::BYTES};
    case 8: return {(const void *)&fwd_kernel<8>, FwdSmem<8>::BYTES};
    case 9: return {(const void *)&fwd_kernel<9>, FwdSmem<9>::BYTES};
    case 10: return {(const void *)&fwd_kernel<10>, FwdSmem<10>::BYTES};
    case 11: return {(const void *)&fwd_kernel<11>, FwdSmem<11>::BYTES};
    case 12: return {(const void *)&fwd_kernel<12>, FwdSmem<12>::BYTES};
    default: return {nullptr, 0};
  }
}

}  // namespace epsc
