// Coarse control variables (Eq. 2 with the basis shifted to the nodes of a
// rectangular grid spanning the design region) and the transpose.
//
//   Phi[a, b] = sum_{i, j} c[i, j] B((x_a - X_i) / h_x) B((y_b - Y_j) / h_y)
//   B(t) = max(0, 1 - |t|),  X_i = i h_x,  h_x = mx / (ncx - 1),  x_a = a + 1/2
//
// With the hat basis each subpixel sees the two nodes around it per axis:
// i0 = floor(x_a / h_x) (clamped to ncx - 2) and i0 + 1 with weights 1 - t
// and t, t = x_a / h_x - i0.  The transpose gives each node the weighted
// sum of the subpixel gradient over its support, |x_a - X_i| < h_x: one block
// per node, fixed-order reductions (deterministic).
#pragma once

#include "epsc_common.cuh"

namespace epsc {

struct CoarseArgs {
  int mx, my, ncx, ncy;
  const float *c;     // [ncx][ncy]
  float *phi;         // [mx][my]
  const float *g;     // [mx][my]  (transpose)
  float *dc;          // [ncx][ncy] (transpose)
  int *err;           // error flag (debug bounds checks)
};

// Subpixel a's centre in node units is s = (a + 1/2) / h = (2a + 1)(nc - 1) / (2m):
// a ratio of integers.  The node index and the hat weights are taken from
// the exact integer numerator, so each weight is one rounded division
// (the projection downstream amplifies errors of Phi by up to beta/2).
__device__ __forceinline__ void hat_pair(int a, int m, int nc, int &i0, float &t) {
  const long num = (long)(2 * a + 1) * (nc - 1), den = 2L * m;
  i0 = min((int)(num / den), nc - 2);
  t = (float)(num - (long)i0 * den) / (float)den;
}

// hat((x_a - X_i) / h) = max(0, 1 - |num - i den| / den)
__device__ __forceinline__ float hat_w(int a, int i, int m, int nc) {
  const long num = (long)(2 * a + 1) * (nc - 1), den = 2L * m;
  const long d = num - (long)i * den;
  const long ad = d < 0 ? -d : d;
  return ad >= den ? 0.f : (float)(den - ad) / (float)den;
}

__global__ void __launch_bounds__(NTHREADS) coarse_expand_kernel(const __grid_constant__ CoarseArgs a) {
  griddep_launch_dependents();
  griddep_wait();
  const long n = (long)a.mx * a.my;
  for (long k = (long)blockIdx.x * NTHREADS + threadIdx.x; k < n; k += (long)gridDim.x * NTHREADS) {
    const int xa = (int)(k / a.my), yb = (int)(k - (long)xa * a.my);
    int i0, j0;
    float tx, ty;
    hat_pair(xa, a.mx, a.ncx, i0, tx);
    hat_pair(yb, a.my, a.ncy, j0, ty);
    // nodes (i0, j0) .. (i0 + 1, j0 + 1)
    if (!EPSC_IN_BOUNDS((size_t)i0 * a.ncy + j0, (size_t)a.ncy + 2, (size_t)a.ncx * a.ncy, a.err))
      continue;
    const float *c0 = a.c + (size_t)i0 * a.ncy + j0;
    const float *c1 = c0 + a.ncy;
    const float lo = fmaf(ty, __ldg(c0 + 1), (1.f - ty) * __ldg(c0));
    const float hi = fmaf(ty, __ldg(c1 + 1), (1.f - ty) * __ldg(c1));
    a.phi[k] = fmaf(tx, hi, (1.f - tx) * lo);
  }
}

// one block per node: warp w takes rows a_lo + w, a_lo + w + 8, ..., lanes
// take columns; per-lane, per-warp and per-block sums in a fixed order
__global__ void __launch_bounds__(NTHREADS) coarse_transpose_kernel(const __grid_constant__ CoarseArgs a) {
  __shared__ float s_part[NTHREADS / 32];
  griddep_launch_dependents();
  griddep_wait();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const long node = blockIdx.x;
  const int i = (int)(node / a.ncy), j = (int)(node - (long)i * a.ncy);
  // subpixels whose centre lies within one spacing of the node:
  // |(2a + 1)(nc - 1) - 2 i m| < 2m
  const long dx = 2L * a.mx, dy = 2L * a.my;
  const int a_lo = max(0, (int)((2L * i * a.mx - dx) / (2L * (a.ncx - 1))) - 1);
  const int a_hi = min(a.mx - 1, (int)((2L * i * a.mx + dx) / (2L * (a.ncx - 1))) + 1);
  const int b_lo = max(0, (int)((2L * j * a.my - dy) / (2L * (a.ncy - 1))) - 1);
  const int b_hi = min(a.my - 1, (int)((2L * j * a.my + dy) / (2L * (a.ncy - 1))) + 1);
  float acc = 0.f;
  for (int xa = a_lo + warp; xa <= a_hi; xa += NTHREADS / 32) {
    const float wx = hat_w(xa, i, a.mx, a.ncx);
    if (wx == 0.f) continue;
    if (!EPSC_IN_BOUNDS((size_t)xa * a.my + b_lo, b_hi - b_lo + 1, (size_t)a.mx * a.my, a.err))
      continue;
    const float *row = a.g + (size_t)xa * a.my;
    float racc = 0.f;
    for (int yb = b_lo + lane; yb <= b_hi; yb += 32) racc = fmaf(hat_w(yb, j, a.my, a.ncy), __ldg(row + yb), racc);
    acc = fmaf(wx, racc, acc);
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
  if (lane == 0) s_part[warp] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    float t = 0.f;
    for (int w = 0; w < NTHREADS / 32; ++w) t += s_part[w];
    a.dc[node] = t;
  }
}

}  // namespace epsc
