// Eq. 1 field contraction with TMA over many design regions in one launch.
//
// The regions' chunks (TMA_BY consecutive Yee columns each) form one index
// space: region k owns chunks [chunk_start, chunk_start + its chunk count),
// and each region has its own pair of tensor maps per wavelength (its
// fields' shapes differ).  Blocks walk (chunk, wavelength) items through
// the same NSTAGE ring as the single-region kernel, with the same consumer
// mapping (eight lanes per column, 16 bytes each, the same lane order and
// the same shuffle reduction), so every column's four sums are bitwise
// those a single-region call computes.  The ring's stages are sized for the
// widest support window of the batch; a region with a narrower window
// fills part of a stage.
//
// Every wait is bounded exactly as in the single-region kernel: on a
// timeout the block records EPS_ERR_DEVICE_TIMEOUT, waits (bounded) for
// its own copies in flight and returns.
#pragma once

#include "epsc_contract_tma.cuh"

namespace epsc {

// Tensor maps one launch can carry in its parameters (2 per region and
// wavelength); larger batches use the register-load contraction.
constexpr int TMA_BATCH_MAX_MAPS = 192;

struct ContractTmaBatchRegion {
  float *W;                                // [4][nx][ny] of this region
  long ncol;                               // nx ny
  int chunk_start;                         // first chunk in the launch's chunk space
  int k0, nk;                              // slab planes
  int x0, bx;                              // support window in floats (bx a multiple of 8)
  int map0;                                // maps[map0 + 2 l + f], f = 0 (E_F) or 1 (E_A)
  float fs[EPS_MAX_BATCH_LAMBDA][3];
};

// The tensor maps come last, as in the single-region arguments: the kernel
// is instantiated for a few map counts and the launch copies only its
// prefix of the host's full-size struct.
template <int NMAPS>
struct __align__(128) ContractTmaBatchArgsN {
  int n, nlambda, nchunks, stage_floats;   // stage_floats: 6 TMA_BY max(bx)
  int *err;
  ContractTmaBatchRegion r[EPS_MAX_BATCH];
  CUtensorMap maps[NMAPS];
};
using ContractTmaBatchArgs = ContractTmaBatchArgsN<TMA_BATCH_MAX_MAPS>;
static_assert(sizeof(ContractTmaBatchArgs) <= 32764, "kernel parameter space");

// Region of a chunk: the last region whose first chunk is at or before it.
template <class Args>
__device__ __forceinline__ int batch_region_of(const Args &a, int chunk) {
  int lo = 0, hi = a.n - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (a.r[mid].chunk_start <= chunk) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// dynamic shared memory: NSTAGE stages of stage_floats floats, plus 128
// bytes of slack to align the ring to 128 bytes
template <int NSTAGE, int NMAPS>
__global__ void __launch_bounds__(NTHREADS) contract_tma_batch_kernel(const __grid_constant__ ContractTmaBatchArgsN<NMAPS> a) {
  extern __shared__ float smem_raw[];
  __shared__ uint64_t full[NSTAGE];
  __shared__ int s_abort;
  float *smem = reinterpret_cast<float *>((reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~uintptr_t(127));

  const int tid = threadIdx.x;
  const int nl = a.nlambda;
  const int nchunks = a.nchunks;
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
    const ContractTmaBatchRegion &rg = a.r[batch_region_of(a, chunk)];
    float *dst = smem + (size_t)s * a.stage_floats;
    mbar_arrive_expect_tx(&full[s], (unsigned)(6 * TMA_BY * rg.bx) * 4u);
    const int y = (chunk - rg.chunk_start) * TMA_BY;
    tma_load_3d(dst, &a.maps[rg.map0 + 2 * l + 0], rg.x0, y, 0, &full[s]);
    tma_load_3d(dst + 3 * TMA_BY * rg.bx, &a.maps[rg.map0 + 2 * l + 1], rg.x0, y, 0, &full[s]);
  };

  if (tid == 0)
    for (int j = 0; j < min(NSTAGE, total); ++j) issue(j);

  // consumer mapping: 8 lanes per column, 32 columns per item
  const int row = tid >> 3, gl = tid & 7;
  float acc0 = 0.f, acc1 = 0.f, acc2 = 0.f, acc3 = 0.f;
  int consumed = 0;

  for (int i = 0; i < total; ++i) {
    const int s = i % NSTAGE;
    const unsigned parity = (unsigned)((i / NSTAGE) & 1);
    // one thread waits for the stage (bounded); the others sleep in the barrier
    if (tid == 0 && !mbar_wait_bounded(&full[s], parity)) s_abort = 1;
    __syncthreads();
    if (s_abort) break;
    const int chunk = blockIdx.x + (i / nl) * gridDim.x;
    const int l = i % nl;
    const ContractTmaBatchRegion &rg = a.r[batch_region_of(a, chunk)];
    const int bx = rg.bx;
    const float *st = smem + (size_t)s * a.stage_floats;
    const float sx = rg.fs[l][0], sy = rg.fs[l][1], sz = rg.fs[l][2];
    const int klo = rg.k0, khi = rg.k0 + rg.nk;
    const int nf4 = bx >> 2;
    for (int f4 = gl; f4 < nf4; f4 += 8) {
      const int k = (rg.x0 >> 1) + 2 * f4;   // planes k and k + 1
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
      const long col = (long)(chunk - rg.chunk_start) * TMA_BY + row;
      if (gl == 0 && col < rg.ncol) {
        rg.W[0 * rg.ncol + col] = acc0;
        rg.W[1 * rg.ncol + col] = acc1;
        rg.W[2 * rg.ncol + col] = acc2;
        rg.W[3 * rg.ncol + col] = acc3;
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
