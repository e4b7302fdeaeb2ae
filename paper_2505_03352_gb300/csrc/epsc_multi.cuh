// Batched stencil and scatter over regions of different filter radius in
// one persistent launch each.
//
// The conic weights of every radius class RP1 = 1 .. MAX_RP1 present in the
// launch sit back to back in the kernel parameters (class RP1 at offset
// woff(RP1), a dense (2 RP1 - 1)^2 box); each block walks its tiles b,
// b + gridDim.x, ... of the launch's tile list (regions in the host's
// cost order) and dispatches on the tile's region class to the stencil or
// scatter tile of that radius, whose weight indices stay compile-time
// constants.  A launch holds at most one radius per class (the host splits
// the rare batches that mix two radii of one class into several launches).
#pragma once

#include "epsc_bwd.cuh"
#include "epsc_fwd.cuh"

namespace epsc {

__host__ __device__ constexpr int woff(int rp1) {
  int s = 0;
  for (int r = 1; r < rp1; ++r) s += (2 * r - 1) * (2 * r - 1);
  return s;
}
constexpr int W_ALL = woff(MAX_RP1 + 1);
template <int RP1>
constexpr int WOFF = woff(RP1);

// Weight view of one radius class: `w` points at its box in the parameters;
// `err` is the launch's error flag (debug bounds checks).
template <int RP1>
struct WView {
  const float *w;
  int *err;
};

struct FwdMultiArgs {
  int n;
  int tile_start[EPS_MAX_BATCH + 1];
  int tiles_j[EPS_MAX_BATCH];
  int rp1[EPS_MAX_BATCH];
  FwdRegion r[EPS_MAX_BATCH];
  int *err;
  float w[W_ALL];
};

struct BwdMultiArgs {
  int n;
  int tile_start[EPS_MAX_BATCH + 1];
  int tiles_j[EPS_MAX_BATCH];
  int rp1[EPS_MAX_BATCH];
  BwdRegion r[EPS_MAX_BATCH];
  int *err;
  float w[W_ALL];
};

// kernel parameters are limited to 32764 bytes
static_assert(sizeof(FwdMultiArgs) <= 32764, "FwdMultiArgs too large for kernel parameters");
static_assert(sizeof(BwdMultiArgs) <= 32764, "BwdMultiArgs too large for kernel parameters");

#define EPSC_MULTI_CASES(F) \
  F(1) F(2) F(3) F(4) F(5) F(6) F(7) F(8) F(9) F(10) F(11) F(12)

template <int BC>
__global__ void __launch_bounds__(NTHREADS, 3) fwd_multi_kernel(const __grid_constant__ FwdMultiArgs a) {
  const int total = a.tile_start[a.n];
  for (int b = blockIdx.x; b < total; b += gridDim.x) {
    int k, t;
    batch_tile(a, b, k, t);
    const int tj = a.tiles_j[k], ti = t / tj;
    const int i0 = ti * TI, j0 = (t - ti * tj) * TJ;
    switch (a.rp1[k]) {
#define EPSC_FWD_CASE(R) \
  case R:                \
    fwd_tile<R, BC>(WView<R>{a.w + WOFF<R>, a.err}, a.r[k], i0, j0); \
    break;
      EPSC_MULTI_CASES(EPSC_FWD_CASE)
#undef EPSC_FWD_CASE
    }
    __syncthreads();   // the next tile reuses shared memory (bulk stores have drained)
  }
}

template <int BC>
__global__ void __launch_bounds__(NTHREADS, 3) bwd_multi_kernel(const __grid_constant__ BwdMultiArgs a) {
  const int total = a.tile_start[a.n];
  for (int b = blockIdx.x; b < total; b += gridDim.x) {
    int k, t;
    batch_tile(a, b, k, t);
    const int tj = a.tiles_j[k], ti = t / tj;
    const int a0 = ti * TA, b0 = (t - ti * tj) * TB;
    switch (a.rp1[k]) {
#define EPSC_BWD_CASE(R) \
  case R:                \
    bwd_tile<R, BC>(WView<R>{a.w + WOFF<R>, a.err}, a.r[k], a0, b0); \
    break;
      EPSC_MULTI_CASES(EPSC_BWD_CASE)
#undef EPSC_BWD_CASE
    }
    __syncthreads();   // the next tile reuses shared memory
  }
}

}  // namespace epsc
