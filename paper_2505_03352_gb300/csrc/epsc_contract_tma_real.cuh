// Column sums of a real cotangent G [3][nx][ny][nz] (float32) over the
// J-support planes, through bulk tensor copies: the contraction of the
// vector-Jacobian product for an arbitrary G (Sec. 3), which the autograd
// backward pass runs.  Per Yee column:
//   W_x  = sum G_x over planes k0+1 .. k0+nk,   W_y likewise,
//   W_zi = sum G_z over planes k0+1 .. k0+nk-1, W_zf = G_z(k0) + G_z(k0+nk).
// G is viewed as a 3-D tensor (component, column, nz floats); one copy moves
// the 32-byte sectors holding planes k0 .. k0+nk of TMA_REAL_BY consecutive
// columns of all three components.  Blocks walk chunks through an
// NSTAGE-deep ring (thread 0 keeps the copies in flight, one
// transaction-counted mbarrier per stage); eight lanes per column sum their
// planes, a shuffle reduction finishes the column, and the block takes a
// chunk's columns in passes of 32 (a window is only 16-32 floats, so wide
// chunks keep the per-chunk barrier cost small against the bytes moved).
// Every wait is bounded: on a timeout the block records
// EPS_ERR_DEVICE_TIMEOUT, waits (bounded) for its own copies and returns.
#pragma once

#include "epsc_contract_tma.cuh"

namespace epsc {

constexpr int TMA_REAL_NSTAGE = 4;
constexpr int TMA_REAL_BY = 128;      // columns per chunk (box rows)
constexpr int TMA_REAL_BX_MAX = 32;   // support window per column, floats (ring <= 197 KB)

struct __align__(128) ContractTmaRealArgs {
  float *W;                 // [4][nx][ny]
  int *err;
  int nx, ny, k0, nk;
  int x0, bx;               // support window in floats (multiples of 8)
  CUtensorMap map;          // G
};

// dynamic shared memory: NSTAGE stages of 3 * TMA_REAL_BY * bx floats, plus 128
// bytes of slack to align the ring to 128 bytes
template <int NSTAGE>
__global__ void __launch_bounds__(NTHREADS) contract_tma_real_kernel(const __grid_constant__ ContractTmaRealArgs a) {
  extern __shared__ float smem_raw[];
  __shared__ uint64_t full[NSTAGE];
  __shared__ int s_abort;
  float *smem = reinterpret_cast<float *>((reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~uintptr_t(127));

  const int tid = threadIdx.x;
  const long ncol = (long)a.nx * a.ny;
  const int nchunks = (int)((ncol + TMA_REAL_BY - 1) / TMA_REAL_BY);
  const int bx = a.bx;
  const int stage_floats = 3 * TMA_REAL_BY * bx;
  const unsigned stage_bytes = (unsigned)stage_floats * 4u;
  const int total = blockIdx.x < nchunks ? (nchunks - 1 - blockIdx.x) / gridDim.x + 1 : 0;

  // the stencil kernel queued behind this grid may start its own blocks now
  griddep_launch_dependents();

  if (tid == 0) {
    for (int s = 0; s < NSTAGE; ++s) mbar_init(&full[s], 1);
    s_abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  __syncthreads();

  auto issue = [&](int j) {
    const int s = j % NSTAGE;
    const int chunk = blockIdx.x + j * gridDim.x;
    mbar_arrive_expect_tx(&full[s], stage_bytes);
    tma_load_3d(smem + (size_t)s * stage_floats, &a.map, a.x0, chunk * TMA_REAL_BY, 0, &full[s]);
  };
  if (tid == 0)
    for (int j = 0; j < min(NSTAGE, total); ++j) issue(j);

  const int row = tid >> 3, gl = tid & 7;   // column of a 32-column pass, lane in the column
  const int klo = a.k0, khi = a.k0 + a.nk;
  int consumed = 0;
  for (int i = 0; i < total; ++i) {
    const int s = i % NSTAGE;
    if (tid == 0 && !mbar_wait_bounded(&full[s], (unsigned)((i / NSTAGE) & 1))) s_abort = 1;
    __syncthreads();
    if (s_abort) break;
    const float *st = smem + (size_t)s * stage_floats;
#pragma unroll
    for (int pass = 0; pass < TMA_REAL_BY / 32; ++pass) {
      const int r = pass * 32 + row;
      float w0 = 0.f, w1 = 0.f, w2 = 0.f, w3 = 0.f;
      for (int f = gl; f < bx; f += 8) {
        const int k = a.x0 + f;
        const float gx = st[(0 * TMA_REAL_BY + r) * bx + f];
        const float gy = st[(1 * TMA_REAL_BY + r) * bx + f];
        const float gz = st[(2 * TMA_REAL_BY + r) * bx + f];
        const bool xy = k >= klo + 1 && k <= khi;
        w0 += xy ? gx : 0.f;
        w1 += xy ? gy : 0.f;
        w2 += (k >= klo + 1 && k <= khi - 1) ? gz : 0.f;
        w3 += (k == klo || k == khi) ? gz : 0.f;
      }
#pragma unroll
      for (int off = 4; off > 0; off >>= 1) {
        w0 += __shfl_xor_sync(0xffffffffu, w0, off);
        w1 += __shfl_xor_sync(0xffffffffu, w1, off);
        w2 += __shfl_xor_sync(0xffffffffu, w2, off);
        w3 += __shfl_xor_sync(0xffffffffu, w3, off);
      }
      const long col = (long)(blockIdx.x + i * gridDim.x) * TMA_REAL_BY + r;
      if (gl == 0 && col < ncol) {
        a.W[0 * ncol + col] = w0;
        a.W[1 * ncol + col] = w1;
        a.W[2 * ncol + col] = w2;
        a.W[3 * ncol + col] = w3;
      }
    }
    consumed = i + 1;
    __syncthreads();   // stage s fully read
    if (tid == 0 && i + NSTAGE < total) issue(i + NSTAGE);
  }

  if (s_abort) {
    // record the timeout, then let every copy this block issued land before
    // its shared memory is released (each wait bounded again)
    if (tid == 0) {
      atomicOr(a.err, ERRFLAG_TIMEOUT);
      const int issued = min(total, consumed + NSTAGE);
      for (int j = consumed; j < issued; ++j)
        mbar_wait_bounded(&full[j % NSTAGE], (unsigned)((j / NSTAGE) & 1));
    }
    __syncthreads();
  }
}

}  // namespace epsc
