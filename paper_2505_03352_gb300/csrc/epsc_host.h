// Host-side helpers shared by the library's translation units (defined in
// abi.cu).  Not part of the C ABI.
#pragma once

#include <cuda_runtime.h>

#include "epschain.h"

namespace epsc_host {

// Validate `prob` as every entry point does and return the conic filter of
// Eq. 2: weights in a dense (2 rp1 - 1)^2 box, row-major (w holds
// MAX_BOX^2 floats), and rp1 = ceil(radius) (at least 1).
eps_status_t conic_filter(const eps_problem_t *prob, float *w, int *rp1);

// The argument checks eps_vjp makes before its first launch (an empty
// problem passes).
eps_status_t check_vjp_args(const eps_problem_t *prob, const float *C, int32_t n_lambda,
                            int32_t field_type, const void *const *EF, const void *const *EA,
                            const float *field_scales, float scale, const float *dJdC,
                            const float *eps_out, const void *ws, size_t ws_bytes);

// Launch one of the library's kernels (one by-value argument struct, 256
// threads per block), with per-kernel timing while profiling is on.
eps_status_t launch_kernel(const char *name, const void *fn, dim3 grid, size_t smem, void *args,
                           cudaStream_t s, bool pdl);

// Count one kernel launch made outside launch_kernel (eps_launch_count).
void note_launch();

// Byte offset, inside an eps_vjp / eps_vjp_real workspace for `prob`, of
// the per-subpixel factor (beta/2)(eps_core - eps_clad) rho (1 - rho)
// [mx][my] that the stencil pass writes, and the workspace size.
eps_status_t subpixel_factor_offset(const eps_problem_t *prob, size_t *offset, size_t *ws_needed);

// Byte offset of the base chain's workspace inside an eps_vjp_morph
// workspace, and the morphology workspace size.
eps_status_t morph_base_offset(const eps_problem_t *prob, const eps_morph_t *morph, size_t *offset,
                               size_t *ws_needed);

// Multiprocessor count of the current device.
eps_status_t sm_count_current(int *n);

// Device address of the library's error flag on the current device (the
// flag eps_sync_status reads), for kernels that record timeouts or debug
// bounds failures.
eps_status_t error_flag(int **flag);

}  // namespace epsc_host
