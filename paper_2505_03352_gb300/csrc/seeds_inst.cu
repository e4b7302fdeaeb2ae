// Adjoint seeds of Eq. 1: seed = W * factor per Yee column.
//
// The stencil kernel writes, per column, the factors of the seeds that are
// linear in the column's Eq. 1 sums (dJ/dA_x, dJ/dH_x, dJ/dg of U_x per
// W_x; the same per W_y; dJ/dH_z per W_zf); dJ/dA_z is W_zi itself.  This
// kernel runs once both the contraction and the stencil have completed
// (ordinary stream order) and turns the factors into seeds in place, over
// all regions of a call (one region for the single-region calls), or over
// one band of columns of a single region (pipelined calls: it then waits
// only for that band's contraction).  When the
// Eq. 1 surrogate is requested (single-region calls) it also adds
// sum over columns of eps_col . W to *S, from the per-column eps values the
// stencil left in epsc.
#include "epsc_launch.h"

namespace epsc {

__device__ __forceinline__ float4 mul4(float4 v, float4 w) {
  return make_float4(v.x * w.x, v.y * w.y, v.z * w.z, v.w * w.w);
}

// sum of the four products (FP32: a handful of terms per thread; the block
// and grid sums that follow run in FP64)
__device__ __forceinline__ float dot4(float4 v, float4 w) {
  return fmaf(v.x, w.x, v.y * w.y) + fmaf(v.z, w.z, v.w * w.w);
}

__global__ void __launch_bounds__(NTHREADS) seeds_kernel(const __grid_constant__ SeedsArgs a) {
  // the scatter kernel queued behind may begin launching; it waits for this
  // grid before it reads the seeds
  griddep_launch_dependents();
  const bool band = a.band_hi > 0;
  if (a.n == 1 && (a.r[0].ncol & 3) == 0 && (a.band_lo & 3) == 0 && (a.band_hi & 3) == 0) {
    // one region whose maps are whole float4 rows (the workspace sections are
    // 256-byte aligned): four columns per thread, 16-byte accesses, the same
    // products element by element
    const SeedsRegion &rg = a.r[0];
    const long p4 = rg.ncol >> 2;
    const long q0 = band ? a.band_lo >> 2 : 0, q1 = band ? a.band_hi >> 2 : p4;
    const float4 *W = reinterpret_cast<const float4 *>(rg.W);
    const float4 *E = reinterpret_cast<const float4 *>(a.epsc);
    float4 *s = reinterpret_cast<float4 *>(rg.seeds);
    double sum = 0.0;
    for (long q = q0 + (long)blockIdx.x * NTHREADS + threadIdx.x; q < q1; q += (long)gridDim.x * NTHREADS) {
      const float4 Wx = __ldg(W + q), Wy = __ldg(W + p4 + q);
      const float4 Wzi = __ldg(W + 2 * p4 + q), Wzf = __ldg(W + 3 * p4 + q);
      // every factor is loaded before the first store: the planes share one
      // base pointer, so loads after a store would wait for it
      const float4 fax = s[S_DAX * p4 + q], fhx = s[S_DHX * p4 + q];
      const float4 gxx = s[S_GXX * p4 + q], gyx = s[S_GYX * p4 + q];
      const float4 fay = s[S_DAY * p4 + q], fhy = s[S_DHY * p4 + q];
      const float4 gxy = s[S_GXY * p4 + q], gyy = s[S_GYY * p4 + q];
      const float4 fhz = s[S_DHZ * p4 + q];
      if (a.S) sum += dot4(__ldg(E + q), Wx) + dot4(__ldg(E + p4 + q), Wy) +
                      dot4(__ldg(E + 2 * p4 + q), Wzi) + dot4(__ldg(E + 3 * p4 + q), Wzf);
      s[S_DAX * p4 + q] = mul4(fax, Wx);
      s[S_DHX * p4 + q] = mul4(fhx, Wx);
      s[S_GXX * p4 + q] = mul4(gxx, Wx);
      s[S_GYX * p4 + q] = mul4(gyx, Wx);
      s[S_DAY * p4 + q] = mul4(fay, Wy);
      s[S_DHY * p4 + q] = mul4(fhy, Wy);
      s[S_GXY * p4 + q] = mul4(gxy, Wy);
      s[S_GYY * p4 + q] = mul4(gyy, Wy);
      s[S_DAZ * p4 + q] = Wzi;
      s[S_DHZ * p4 + q] = mul4(fhz, Wzf);
    }
    if (a.S) block_add_to(a.S, sum);   // uniform over the grid
    return;
  }
  double sum = 0.0;
  const long c0 = band ? a.band_lo : 0, c1 = band ? a.band_hi : a.ncol;
  for (long c = c0 + (long)blockIdx.x * NTHREADS + threadIdx.x; c < c1; c += (long)gridDim.x * NTHREADS) {
    int k = 0;
    while (k + 1 < a.n && c >= a.r[k + 1].col_start) ++k;
    const SeedsRegion &rg = a.r[k];
    const long j = c - rg.col_start, p = rg.ncol;
    if (!EPSC_IN_BOUNDS(j, 1, p, a.err)) continue;
    const float Wx = __ldg(rg.W + j), Wy = __ldg(rg.W + p + j);
    const float Wzi = __ldg(rg.W + 2 * p + j), Wzf = __ldg(rg.W + 3 * p + j);
    float *s = rg.seeds + j;
    const float fax = s[S_DAX * p], fhx = s[S_DHX * p], gxx = s[S_GXX * p], gyx = s[S_GYX * p];
    const float fay = s[S_DAY * p], fhy = s[S_DHY * p], gxy = s[S_GXY * p], gyy = s[S_GYY * p];
    const float fhz = s[S_DHZ * p];
    s[S_DAX * p] = fax * Wx;
    s[S_DHX * p] = fhx * Wx;
    s[S_GXX * p] = gxx * Wx;
    s[S_GYX * p] = gyx * Wx;
    s[S_DAY * p] = fay * Wy;
    s[S_DHY * p] = fhy * Wy;
    s[S_GXY * p] = gxy * Wy;
    s[S_GYY * p] = gyy * Wy;
    s[S_DAZ * p] = Wzi;
    s[S_DHZ * p] = fhz * Wzf;
    if (a.S && a.n == 1) {
      const float *e = a.epsc + j;
      sum += fmaf(e[0], Wx, e[p] * Wy) + fmaf(e[2 * p], Wzi, e[3 * p] * Wzf);
    }
  }
  if (a.S) block_add_to(a.S, sum);
}

const void *seeds_entry() { return (const void *)&seeds_kernel; }

}  // namespace epsc
