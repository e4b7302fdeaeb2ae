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
KernelEntry fwd_entry_a(int rp1);
KernelEntry fwd_entry_b(int rp1);
KernelEntry bwd_entry_a(int rp1);
KernelEntry bwd_entry_b(int rp1);

inline KernelEntry fwd_entry(int rp1) { return rp1 <= 6 ? fwd_entry_a(rp1) : fwd_entry_b(rp1); }
inline KernelEntry bwd_entry(int rp1) { return rp1 <= 6 ? bwd_entry_a(rp1) : bwd_entry_b(rp1); }

}  // namespace epsc
