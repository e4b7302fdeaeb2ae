// Explicit instantiations of the subpixel-map kernels for RP1 = 1 .. 6, both
// boundary rules, all four kinds.
#include "epsc_morph.cuh"
#include "epsc_launch.h"

namespace epsc {

template <int RP1>
static KernelEntry map_pick(int bc, int kind) {
  const bool clamp = bc == EPS_BC_CLAMP;
  const void *fn = nullptr;
  switch (kind) {
    case MAP_FRONT:
      fn = clamp ? (const void *)&map_kernel<RP1, EPS_BC_CLAMP, MAP_FRONT> : (const void *)&map_kernel<RP1, EPS_BC_PERIODIC, MAP_FRONT>;
      break;
    case MAP_LSE:
      fn = clamp ? (const void *)&map_kernel<RP1, EPS_BC_CLAMP, MAP_LSE> : (const void *)&map_kernel<RP1, EPS_BC_PERIODIC, MAP_LSE>;
      break;
    case MAP_LSE_T:
      fn = clamp ? (const void *)&map_kernel<RP1, EPS_BC_CLAMP, MAP_LSE_T> : (const void *)&map_kernel<RP1, EPS_BC_PERIODIC, MAP_LSE_T>;
      break;
    case MAP_FRONT_T:
      fn = clamp ? (const void *)&map_kernel<RP1, EPS_BC_CLAMP, MAP_FRONT_T> : (const void *)&map_kernel<RP1, EPS_BC_PERIODIC, MAP_FRONT_T>;
      break;
    default:
      return {nullptr, 0};
  }
  return {fn, MapSmem<RP1>::BYTES};
}

KernelEntry map_entry_a(int rp1, int bc, int kind) {
  switch (rp1) {
    case 1: return map_pick<1>(bc, kind);
    case 2: return map_pick<2>(bc, kind);
    case 3: return map_pick<3>(bc, kind);
    case 4: return map_pick<4>(bc, kind);
    case 5: return map_pick<5>(bc, kind);
    case 6: return map_pick<6>(bc, kind);
  }
  return {nullptr, 0};
}

}  // namespace epsc
