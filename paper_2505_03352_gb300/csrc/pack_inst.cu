// Kernels of the reduced-precision field path (packing and contraction).
#define EPSC_PACK_KERNELS
#include "epsc_launch.h"
#include "epsc_pack.cuh"

namespace epsc {

const void *pack_amax_entry() { return (const void *)&pack_amax_kernel; }
const void *pack_entry() { return (const void *)&pack_kernel; }
const void *pack_finish_entry() { return (const void *)&pack_finish_kernel; }
const void *contract_packed_entry() { return (const void *)&contract_packed_kernel; }
const void *contract_packed_bulk_entry() { return (const void *)&contract_packed_bulk_kernel; }

}  // namespace epsc
