// Instantiation of the bulk-copy contraction of a real cotangent.
#include "epsc_contract_tma_real.cuh"
#include "epsc_launch.h"

namespace epsc {

const void *contract_tma_real_entry() {
  return (const void *)&contract_tma_real_kernel<TMA_REAL_NSTAGE>;
}

}  // namespace epsc
