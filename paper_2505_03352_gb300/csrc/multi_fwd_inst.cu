// Instantiation of the mixed-radius batched stencil kernel (both boundary rules).
#include "epsc_launch.h"
#include "epsc_multi.cuh"

namespace epsc {

const void *fwd_multi_entry(int bc) {
  return bc == EPS_BC_CLAMP ? (const void *)&fwd_multi_kernel<EPS_BC_CLAMP>
                            : (const void *)&fwd_multi_kernel<EPS_BC_PERIODIC>;
}

}  // namespace epsc
