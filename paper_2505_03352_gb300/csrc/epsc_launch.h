// Host-side launch table of the templated kernels (one entry per RP1).
#pragma once

#include <cuda_runtime.h>

#include "epsc_common.cuh"

namespace epsc {

struct KernelEntry {
  const void *fn;     // kernel function pointer
  size_t smem;        // dynamic shared memory bytes
};

// Defined in the instantiation units (RP1 1..6 in *_a, 7..12 in *_b);
// return {nullptr, 0} outside their range.
KernelEntry fwd_entry_a(int rp1, int bc, bool batched);
KernelEntry fwd_entry_b(int rp1, int bc, bool batched);
KernelEntry bwd_entry_a(int rp1, int bc, bool batched);
KernelEntry bwd_entry_b(int rp1, int bc, bool batched);
// Single-region scatter staging interior tiles through bulk tensor copies
// (radius classes 3 .. 12; {nullptr, 0} otherwise).
KernelEntry bwd_tma_entry(int rp1, int bc);
// The batched scatter of one radius group with bulk-copy staging (radius
// classes 3 .. 12; {nullptr, 0} otherwise).
KernelEntry bwd_tma_batched_entry(int rp1, int bc);
// The batched scatter on wide tiles (TA x 64 subpixels): element-wise
// staging (radius classes 1 .. 12) and bulk-copy staging (3 .. 12).
KernelEntry bwd_batched_wide_entry(int rp1, int bc);
KernelEntry bwd_tma_batched_wide_entry(int rp1, int bc);

// Contraction kernel with 4 or 8 lanes per column.
const void *contract_entry(int lanes);
// Contraction over many regions in one launch.
const void *contract_batched_entry();
// Contraction kernel fed by bulk tensor copies (complex64 fields), with room
// for at least n_lambda wavelengths' tensor maps.
const void *contract_tma_entry(int n_lambda);
// Contraction over many regions fed by bulk tensor copies, with room for at
// least nmaps tensor maps (2 per region and wavelength).
const void *contract_tma_batch_entry(int nmaps);
// Column sums of a real cotangent over the support planes, by bulk copies.
const void *contract_tma_real_entry();
// One block that waits (bounded) on a barrier nothing arrives at.
struct SelftestArgs {
  int *err;
  long long cycles;
};
const void *selftest_timeout_entry();
// One thread whose bounds check fails (debug-bounds builds; no memory access).
const void *selftest_bounds_entry();

// Reduced-precision field path.
const void *pack_amax_entry();
const void *pack_entry();
const void *pack_finish_entry();
const void *contract_packed_entry();
const void *contract_packed_bulk_entry();

// Seeds of Eq. 1 (factor * W), any number of regions.
const void *seeds_entry();

// Mixed-radius batched stencil / scatter (one persistent launch per phase).
const void *fwd_multi_entry(int bc);
const void *bwd_multi_entry(int bc);

// Subpixel-map kernels of the morphology path (kind: MapKind).
KernelEntry map_entry_a(int rp1, int bc, int kind);
KernelEntry map_entry_b(int rp1, int bc, int kind);

inline KernelEntry map_entry(int rp1, int bc, int kind) {
  return rp1 <= 6 ? map_entry_a(rp1, bc, kind) : map_entry_b(rp1, bc, kind);
}

inline KernelEntry fwd_entry(int rp1, int bc, bool batched = false) {
  return rp1 <= 6 ? fwd_entry_a(rp1, bc, batched) : fwd_entry_b(rp1, bc, batched);
}
inline KernelEntry bwd_entry(int rp1, int bc, bool batched = false) {
  return rp1 <= 6 ? bwd_entry_a(rp1, bc, batched) : bwd_entry_b(rp1, bc, batched);
}

}  // namespace epsc
