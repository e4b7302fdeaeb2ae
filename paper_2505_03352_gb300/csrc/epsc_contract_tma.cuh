// Eq. 1 field contraction with TMA (complex64 fields).
//
// Each field array [3][nx][ny][nz] (complex64) is viewed as a 3-D tensor
// (component, Yee column, 2*nz floats).  One bulk tensor copy moves, for
// all three components, the J-support window of BY consecutive columns --
// the 32-byte sectors that hold planes k0 .. k0+nk -- into shared memory,
// skipping the cladding planes between columns.  A launch covers the columns
// [col_lo, col_hi) (all of them, or one band of a pipelined call); a
// chunk that runs past col_hi reads its last columns but writes no W for
// them.  A block processes (chunk, wavelength)
// items through an NSTAGE-deep ring: thread 0 keeps NSTAGE - 1 items in
// flight (one mbarrier per stage, transaction-counted), all threads consume
// from shared memory (eight lanes per column, 16 bytes each), and after the
// last wavelength of a chunk the eight lanes reduce and write the four
// column sums W_x, W_y, W_zi, W_zf.
//
// Every wait is bounded: if a stage does not complete within about a
// second the block records EPS_ERR_DEVICE_TIMEOUT in the error flag, waits
// (bounded again) for its other copies and returns.
#pragma once

#include <cuda.h>

#include "epsc_common.cuh"

namespace epsc {

constexpr int TMA_BY = 32;        // columns per box
constexpr int TMA_NSTAGE = 2; // ring depth
constexpr int TMA_BX_MAX = 64;    // floats per box row (support window)

// The tensor maps come last: the kernel is instantiated for 2, 4, 8, 16 or
// 2 EPS_MAX_LAMBDA maps and takes only its own count; the host fills the
// full-size struct and the launch copies the kernel's parameter bytes, a
// common prefix (smaller parameter blocks launch faster).
template <int NMAPS>
struct __align__(128) ContractTmaArgsN {
  float *W;                                // [4][nx][ny]
  int *err;
  int nx, ny, k0, nk, nlambda;
  int x0;                                  // first float of the window in a column
  int bx;                                  // window width in floats (multiple of 8)
  long col_lo, col_hi;                     // the launch's columns [col_lo, col_hi)
  float fs[EPS_MAX_LAMBDA][3];
  CUtensorMap maps[NMAPS];                 // [wavelength][field F/A]
};
using ContractTmaArgs = ContractTmaArgsN<EPS_MAX_LAMBDA * 2>;

__device__ __forceinline__ unsigned smem_addr(const void *p) {
  return (unsigned)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_addr(bar)), "r"(count)
               : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_addr(bar)),
               "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n"
      " mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, 20000;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait on a phase of an mbarrier: `limit` SM clock cycles (by
// default 2^31, about one second).  Each try suspends the thread for up to
// 20 us (hint) instead of spinning.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, unsigned parity,
                                                  long long limit = 1ll << 31) {
  const long long t0 = clock64();
  while (!mbar_try_wait(bar, parity)) {
    if (clock64() - t0 > limit) return false;
  }
  return true;
}

__device__ __forceinline__ void tma_load_3d(void *dst, const CUtensorMap *map, int x, int y, int z,
                                            uint64_t *bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4}], [%5];\n" ::"r"(smem_addr(dst)),
      "l"(map), "r"(x), "r"(y), "r"(z), "r"(smem_addr(bar))
      : "memory");
}

// dynamic shared memory: NSTAGE stages of 6 * TMA_BY * bx floats, plus
// 128 bytes of slack to align the ring to 128 bytes
template <int NSTAGE, int NMAPS>
__global__ void __launch_bounds__(NTHREADS) contract_tma_kernel(const __grid_constant__ ContractTmaArgsN<NMAPS> a) {
  extern __shared__ float smem_raw[];
  __shared__ uint64_t full[NSTAGE];
  __shared__ int s_abort;
  float *smem = reinterpret_cast<float *>((reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~uintptr_t(127));

  const int tid = threadIdx.x;
  const long ncol = (long)a.nx * a.ny;       // W plane stride
  const long col_lo = a.col_lo;
  const int nchunks = (int)((a.col_hi - col_lo + TMA_BY - 1) / TMA_BY);
  const int nl = a.nlambda;
  const int bx = a.bx;
  const int stage_floats = 6 * TMA_BY * bx;
  const unsigned stage_bytes = (unsigned)stage_floats * 4u;
  // items of this block: chunk c_b = blockIdx.x + q * gridDim.x, wavelength l
  const int my_chunks = blockIdx.x < nchunks ? (nchunks - 1 - blockIdx.x) / gridDim.x + 1 : 0;
  const int total = my_chunks * nl;

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
    const int chunk = blockIdx.x + (j / nl) * gridDim.x;
    const int l = j % nl;
    float *dst = smem + (size_t)s * stage_floats;
    mbar_arrive_expect_tx(&full[s], stage_bytes);
    const int c0 = (int)(col_lo + (long)chunk * TMA_BY);
    tma_load_3d(dst, &a.maps[l * 2 + 0], a.x0, c0, 0, &full[s]);
    tma_load_3d(dst + 3 * TMA_BY * bx, &a.maps[l * 2 + 1], a.x0, c0, 0, &full[s]);
  };

  if (tid == 0)
    for (int j = 0; j < min(NSTAGE, total); ++j) issue(j);

  // consumer mapping: 8 lanes per column, 32 columns per item
  const int row = tid >> 3, gl = tid & 7;
  const int klo = a.k0, khi = a.k0 + a.nk;
  const int nf4 = bx >> 2;
  float acc0 = 0.f, acc1 = 0.f, acc2 = 0.f, acc3 = 0.f;
  int consumed = 0;

  for (int i = 0; i < total; ++i) {
    const int s = i % NSTAGE;
    const unsigned parity = (unsigned)((i / NSTAGE) & 1);
    // one thread waits for the stage (bounded); the others sleep in the barrier
    if (tid == 0 && !mbar_wait_bounded(&full[s], parity)) s_abort = 1;
    __syncthreads();
    if (s_abort) break;
    const int l = i % nl;
    const float *st = smem + (size_t)s * stage_floats;
    const float sx = a.fs[l][0], sy = a.fs[l][1], sz = a.fs[l][2];
    for (int f4 = gl; f4 < nf4; f4 += 8) {
      const int k = (a.x0 >> 1) + 2 * f4;   // planes k and k + 1
      float4 fe[3], ae[3];
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        fe[c] = *reinterpret_cast<const float4 *>(st + (c * TMA_BY + row) * bx + 4 * f4);
        ae[c] = *reinterpret_cast<const float4 *>(st + ((3 + c) * TMA_BY + row) * bx + 4 * f4);
      }
      const bool xy0 = k >= klo + 1 && k <= khi, xy1 = k + 1 >= klo + 1 && k + 1 <= khi;
      const bool zi0 = k >= klo + 1 && k <= khi - 1, zi1 = k + 1 >= klo + 1 && k + 1 <= khi - 1;
      const bool zf0 = k == klo || k == khi, zf1 = k + 1 == klo || k + 1 == khi;
      float r0[3], r1[3];
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        r0[c] = fmaf(fe[c].x, ae[c].x, -fe[c].y * ae[c].y);
        r1[c] = fmaf(fe[c].z, ae[c].z, -fe[c].w * ae[c].w);
      }
      acc0 = fmaf(sx, (xy0 ? r0[0] : 0.f) + (xy1 ? r1[0] : 0.f), acc0);
      acc1 = fmaf(sy, (xy0 ? r0[1] : 0.f) + (xy1 ? r1[1] : 0.f), acc1);
      acc2 = fmaf(sz, (zi0 ? r0[2] : 0.f) + (zi1 ? r1[2] : 0.f), acc2);
      acc3 = fmaf(sz, (zf0 ? r0[2] : 0.f) + (zf1 ? r1[2] : 0.f), acc3);
    }
    if (l == nl - 1) {
#pragma unroll
      for (int off = 4; off > 0; off >>= 1) {
        acc0 += __shfl_xor_sync(0xffffffffu, acc0, off);
        acc1 += __shfl_xor_sync(0xffffffffu, acc1, off);
        acc2 += __shfl_xor_sync(0xffffffffu, acc2, off);
        acc3 += __shfl_xor_sync(0xffffffffu, acc3, off);
      }
      const long col = col_lo + (long)(blockIdx.x + (i / nl) * gridDim.x) * TMA_BY + row;
      if (gl == 0 && col < a.col_hi) {
        a.W[0 * ncol + col] = acc0;
        a.W[1 * ncol + col] = acc1;
        a.W[2 * ncol + col] = acc2;
        a.W[3 * ncol + col] = acc3;
      }
      acc0 = acc1 = acc2 = acc3 = 0.f;
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
