// Adjoint seeds of Eq. 1: seed = W * factor per Yee column.
//
// The stencil kernel writes, per column, the factors of the seeds that are
// linear in the column's Eq. 1 sums (dJ/dA_x, dJ/dH_x, dJ/dg of U_x per
// W_x; the same per W_y; dJ/dH_z per W_zf); dJ/dA_z is W_zi itself.  This
// kernel runs once both the contraction and the stencil have completed
// (ordinary stream order) and turns the factors into seeds in place, over
// all regions of a call (one region for the single-region calls).
#include "epsc_launch.h"

namespace epsc {

__global__ void __launch_bounds__(NTHREADS) seeds_kernel(const __grid_constant__ SeedsArgs a) {
  // the scatter kernel queued behind may begin launching; it waits for this
  // grid before it reads the seeds
  griddep_launch_dependents();
  for (long c = (long)blockIdx.x * NTHREADS + threadIdx.x; c < a.ncol; c += (long)gridDim.x * NTHREADS) {
    int k = 0;
    while (k + 1 < a.n && c >= a.r[k + 1].col_start) ++k;
    const SeedsRegion &rg = a.r[k];
    const long j = c - rg.col_start, p = rg.ncol;
    if (!EPSC_IN_BOUNDS(j, 1, p, a.err)) continue;
    const float Wx = __ldg(rg.W + j), Wy = __ldg(rg.W + p + j);
    const float Wzi = __ldg(rg.W + 2 * p + j), Wzf = __ldg(rg.W + 3 * p + j);
    float *s = rg.seeds + j;
    s[S_DAX * p] *= Wx;
    s[S_DHX * p] *= Wx;
    s[S_GXX * p] *= Wx;
    s[S_GYX * p] *= Wx;
    s[S_DAY * p] *= Wy;
    s[S_DHY * p] *= Wy;
    s[S_GXY * p] *= Wy;
    s[S_GYY * p] *= Wy;
    s[S_DAZ * p] = Wzi;
    s[S_DHZ * p] *= Wzf;
  }
}

const void *seeds_entry() { return (const void *)&seeds_kernel; }

}  // namespace epsc
