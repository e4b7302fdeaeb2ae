// Instantiations of the Eq. 1 contraction kernel (4 lanes per column with
// 32-byte sector loads, or 8 lanes per column with 16-byte loads).
#include "epsc_contract.cuh"
#include "epsc_contract_tma.cuh"
#include "epsc_launch.h"

namespace epsc {

const void *contract_entry(int lanes) {
  return lanes == 4 ? (const void *)&contract_kernel<4> : (const void *)&contract_kernel<8>;
}

const void *contract_batched_entry() { return (const void *)&contract_batched_kernel<0>; }

const void *contract_tma_entry(int n_lambda) {
  if (n_lambda <= 1) return (const void *)&contract_tma_kernel<TMA_NSTAGE, 2>;
  if (n_lambda <= 2) return (const void *)&contract_tma_kernel<TMA_NSTAGE, 4>;
  if (n_lambda <= 4) return (const void *)&contract_tma_kernel<TMA_NSTAGE, 8>;
  if (n_lambda <= 8) return (const void *)&contract_tma_kernel<TMA_NSTAGE, 16>;
  return (const void *)&contract_tma_kernel<TMA_NSTAGE, EPS_MAX_LAMBDA * 2>;
}

}  // namespace epsc
