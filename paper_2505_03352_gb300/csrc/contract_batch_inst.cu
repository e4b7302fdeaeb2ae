// Instantiations of the batched TMA contraction, by tensor-map capacity.
#include "epsc_contract_tma_batch.cuh"
#include "epsc_launch.h"

namespace epsc {

const void *contract_tma_batch_entry(int nmaps) {
  if (nmaps <= 32) return (const void *)&contract_tma_batch_kernel<TMA_NSTAGE, 32>;
  if (nmaps <= 64) return (const void *)&contract_tma_batch_kernel<TMA_NSTAGE, 64>;
  if (nmaps <= 128) return (const void *)&contract_tma_batch_kernel<TMA_NSTAGE, 128>;
  return (const void *)&contract_tma_batch_kernel<TMA_NSTAGE, TMA_BATCH_MAX_MAPS>;
}

}  // namespace epsc
