// Explicit instantiations of the subpixel-map kernels for RP1 = 7 .. 12, both
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

KernelEntry map_entry_b(int rp1, int bc, int kind) {
  switch (rp1) {
    case 7: return map_pick<7>(bc, kind);
    case 8: return map_pick<8>(bc, kind);
    case 9: return map_pick<9>(bc, kind);
    case 10: return map_pick<10>(bc, kind);
    case 11: return map_pick<11>(bc, kind);
    case 12: return map_pick<12>(bc, kind);
  }
  return {nullptr, 0};
}

}  // namespace epsc
