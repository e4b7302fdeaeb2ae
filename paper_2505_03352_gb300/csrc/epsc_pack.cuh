// Reduced-precision field storage for the Eq. 1 contraction.
//
// Packed field buffer (one per wavelength and per forward/adjoint field):
//   bytes [0, 16)   float scale[3] (one per component) and one float of pad
//   bytes [16, ...) [3][nx][ny][NP] elements, each an (re, im) pair of bf16
//                   or fp16 (4 bytes), holding planes k0 .. k0 + NP - 1 of
//                   the component divided by its scale; NP = nk + 1 rounded
//                   up to a multiple of 4 (planes past nz are zero).
// So a packed field holds exactly the J-support planes, contiguous per
// column, and decodes as value = scale[c] * stored.  The scale of a
// component is max(|re|, |im|) over its support planes divided by the
// format's target magnitude (1 for bf16, 2^14 for fp16), or 1 if that max
// is 0.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "epsc_common.cuh"
#include "epsc_contract_tma.cuh"

namespace epsc {

constexpr float BF16_TARGET = 1.0f;
constexpr float F16_TARGET = 16384.0f;

struct PackArgs {
  int nx, ny, nz, k0, nk, np;   // np: packed planes per column (multiple of 4)
  int type;                     // EPS_FIELD_BF16X2_SCALED or EPS_FIELD_F16X2_SCALED
  const float2 *src;            // complex64 [3][nx][ny][nz]
  unsigned char *dst;           // packed buffer
  int *err;                     // error flag (debug bounds checks)
};

struct ContractPackedArgs {
  int nx, ny, k0, nk, np, nlambda, type;
  const unsigned char *EF[EPS_MAX_LAMBDA];
  const unsigned char *EA[EPS_MAX_LAMBDA];
  float fs[EPS_MAX_LAMBDA][3];   // scale * extra caller factors
  float *W;                      // [4][nx][ny]
  int *err;                      // error flag (debug bounds checks)
  int nstage;                    // bulk-copy ring depth (contract_packed_bulk_kernel)
  long col_lo, col_hi;           // contract_packed_bulk_kernel: the launch's columns
};

// Bulk-copy form of the packed contraction: PK_BY columns per chunk, one
// thread per (column, component) of a chunk.  Wide chunks make each bulk
// copy one long contiguous run (4.5 KB per component at nk = 11).  Measured
// at the 3000 x 3000, eight-wavelength BF16 call: with two blocks per SM,
// 128 columns stream the packed planes in 0.90 ms where 64 or 32 take 1.28
// or 2.26 ms (a fixed cost per ring item, whatever the ring depth), and 256
// columns at one block per SM 1.26 ms; the whole call at 96 columns and
// three blocks per SM 1.140 ms, against 1.165-1.171 ms at 128 and two (80
// columns and three blocks 1.204, 64 and four 1.176, 64 and five 1.245,
// 96 with three stages and two blocks 1.382).
constexpr int PK_BY = 96;
constexpr int PK_THREADS = 3 * PK_BY;
constexpr int PK_MAX_STAGE = 8;

// The kernels below are compiled in one translation unit only.
#ifdef EPSC_PACK_KERNELS

// max |re|, |im| over the support planes of each component, into the
// header (as float bits, non-negative floats order like their bit patterns)
__global__ void __launch_bounds__(NTHREADS) pack_amax_kernel(const __grid_constant__ PackArgs a) {
  const long ncol = (long)a.nx * a.ny;
  unsigned *hdr = reinterpret_cast<unsigned *>(a.dst);
  const int c = blockIdx.y;
  float m = 0.f;
  const long total = ncol * (a.nk + 1);
  for (long t = (long)blockIdx.x * NTHREADS + threadIdx.x; t < total; t += (long)gridDim.x * NTHREADS) {
    const long col = t / (a.nk + 1);
    const int k = a.k0 + (int)(t - col * (a.nk + 1));
    const size_t si = ((size_t)c * ncol + col) * a.nz + k;
    if (!EPSC_IN_BOUNDS(si, 1, (size_t)3 * ncol * a.nz, a.err)) continue;
    const float2 v = a.src[si];
    m = fmaxf(m, fmaxf(fabsf(v.x), fabsf(v.y)));
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, off));
  if ((threadIdx.x & 31) == 0 && m > 0.f) atomicMax(hdr + c, __float_as_uint(m));
}

// convert the header maxima to scales, then write the packed planes
__global__ void __launch_bounds__(NTHREADS) pack_kernel(const __grid_constant__ PackArgs a) {
  const long ncol = (long)a.nx * a.ny;
  const float *hdr = reinterpret_cast<const float *>(a.dst);
  const float target = a.type == EPS_FIELD_BF16X2_SCALED ? BF16_TARGET : F16_TARGET;
  const long total = 3 * ncol * a.np;
  unsigned *out = reinterpret_cast<unsigned *>(a.dst + 16);
  for (long t = (long)blockIdx.x * NTHREADS + threadIdx.x; t < total; t += (long)gridDim.x * NTHREADS) {
    const long cc = t / a.np;               // component * ncol + column
    const int kk = (int)(t - cc * a.np);
    const int c = (int)(cc / ncol);
    const float amax = hdr[c];
    const float inv = amax > 0.f ? target / amax : 1.f;
    const int k = a.k0 + kk;
    float2 v = make_float2(0.f, 0.f);
    if (kk <= a.nk && k < a.nz && EPSC_IN_BOUNDS((size_t)cc * a.nz + k, 1, (size_t)3 * ncol * a.nz, a.err))
      v = a.src[(size_t)cc * a.nz + k];
    unsigned bits;
    if (a.type == EPS_FIELD_BF16X2_SCALED) {
      const __nv_bfloat162 h = __floats2bfloat162_rn(v.x * inv, v.y * inv);
      bits = *reinterpret_cast<const unsigned *>(&h);
    } else {
      const __half2 h = __floats2half2_rn(v.x * inv, v.y * inv);
      bits = *reinterpret_cast<const unsigned *>(&h);
    }
    out[t] = bits;
  }
}

// header maxima -> scales (one thread per component), after pack_kernel
__global__ void pack_finish_kernel(unsigned char *dst, int type) {
  float *hdr = reinterpret_cast<float *>(dst);
  const int c = threadIdx.x;
  if (c < 3) {
    const float target = type == EPS_FIELD_BF16X2_SCALED ? BF16_TARGET : F16_TARGET;
    const float amax = hdr[c];
    hdr[c] = amax > 0.f ? amax / target : 1.f;
  }
}

__device__ __forceinline__ float2 unpack2(unsigned bits, int type) {
  if (type == EPS_FIELD_BF16X2_SCALED) {
    __nv_bfloat162 h = *reinterpret_cast<const __nv_bfloat162 *>(&bits);
    return __bfloat1622float2(h);
  }
  __half2 h = *reinterpret_cast<const __half2 *>(&bits);
  return __half22float2(h);
}

// Contraction over packed fields: one thread per column and wavelength
// pass, 16-byte loads of four packed planes at a time, FP32 accumulation.
__global__ void __launch_bounds__(NTHREADS) contract_packed_kernel(const __grid_constant__ ContractPackedArgs a) {
  griddep_launch_dependents();
  const long ncol = (long)a.nx * a.ny;
  const int nq = a.np >> 2;   // uint4 per column and component
  for (long col = (long)blockIdx.x * NTHREADS + threadIdx.x; col < ncol; col += (long)gridDim.x * NTHREADS) {
    float wx = 0.f, wy = 0.f, wzi = 0.f, wzf = 0.f;
    for (int l = 0; l < a.nlambda; ++l) {
      const float *hf = reinterpret_cast<const float *>(a.EF[l]);
      const float *ha = reinterpret_cast<const float *>(a.EA[l]);
      const uint4 *pf = reinterpret_cast<const uint4 *>(a.EF[l] + 16);
      const uint4 *pa = reinterpret_cast<const uint4 *>(a.EA[l] + 16);
      float sums[4] = {0.f, 0.f, 0.f, 0.f};   // x, y, z interior, z faces (unscaled)
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const size_t base = ((size_t)c * ncol + col) * nq;
        if (!EPSC_IN_BOUNDS(base, nq, (size_t)3 * ncol * nq, a.err)) continue;
        float s_in = 0.f, s_face = 0.f;
#pragma unroll 4
        for (int q = 0; q < nq; ++q) {   // unrolled: more loads in flight per thread
          const uint4 f = __ldg(pf + base + q);
          const uint4 e = __ldg(pa + base + q);
          const unsigned fb[4] = {f.x, f.y, f.z, f.w};
          const unsigned eb[4] = {e.x, e.y, e.z, e.w};
#pragma unroll
          for (int t = 0; t < 4; ++t) {
            const int kk = 4 * q + t;   // packed plane kk is plane k0 + kk
            const float2 x = unpack2(fb[t], a.type);
            const float2 y = unpack2(eb[t], a.type);
            const float re = fmaf(x.x, y.x, -x.y * y.y);
            const bool in = c < 2 ? (kk >= 1 && kk <= a.nk) : (kk >= 1 && kk <= a.nk - 1);
            const bool face = c == 2 && (kk == 0 || kk == a.nk);
            s_in += in ? re : 0.f;
            s_face += face ? re : 0.f;
          }
        }
        const float sc = __ldg(hf + c) * __ldg(ha + c) * a.fs[l][c];
        if (c < 2) {
          sums[c] = __fmul_rn(s_in, sc);
        } else {
          sums[2] = __fmul_rn(s_in, sc);
          sums[3] = __fmul_rn(s_face, sc);
        }
      }
      // a rounded product, then a rounded sum: one fixed order whatever the
      // compiler could fuse
      wx = __fadd_rn(wx, sums[0]);
      wy = __fadd_rn(wy, sums[1]);
      wzi = __fadd_rn(wzi, sums[2]);
      wzf = __fadd_rn(wzf, sums[3]);
    }
    a.W[0 * ncol + col] = wx;
    a.W[1 * ncol + col] = wy;
    a.W[2 * ncol + col] = wzi;
    a.W[3 * ncol + col] = wzf;
  }
}

// Untiled bulk copy of `bytes` contiguous bytes global -> shared, completing
// on mbarrier `bar` (both addresses 16-byte aligned, bytes a multiple of 16).
__device__ __forceinline__ void bulk_load(void *dst, const void *src, unsigned bytes,
                                          uint64_t *bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::
          "r"(smem_addr(dst)), "l"(src), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}

// Contraction over packed fields through untiled bulk copies.  The packed
// planes of a component are 4 np bytes per column, contiguous, so the
// component's part of a chunk of PK_BY columns is one contiguous run: an
// item (chunk, wavelength) is six copies (E_F and E_A, three components)
// into one stage of an nstage-deep shared-memory ring.  Thread 0 keeps
// nstage - 1 items in flight ahead of the consumers; every thread waits on
// the stage's barrier itself (bounded), thread t takes column t % PK_BY and
// component t / PK_BY of the chunk (consecutive threads read 16-byte words
// 48 bytes apart: no bank conflicts), and one block barrier per item frees
// the stage for the next copy.  The arithmetic per column and component is
// contract_packed_kernel's, in the same order, so W is bitwise the same.
// Few blocks per SM (the ring is in shared memory, not in registers) leave
// SM slots to the stencil launched behind this grid.
__global__ void __launch_bounds__(PK_THREADS) contract_packed_bulk_kernel(
    const __grid_constant__ ContractPackedArgs a) {
  extern __shared__ unsigned char pk_raw[];
  __shared__ uint64_t full[PK_MAX_STAGE];
  __shared__ int s_abort;
  unsigned char *ring =
      reinterpret_cast<unsigned char *>((reinterpret_cast<uintptr_t>(pk_raw) + 127) & ~uintptr_t(127));
  const int tid = threadIdx.x;
  const long ncol = (long)a.nx * a.ny;       // component and W plane stride
  const long col_lo = a.col_lo, col_hi = a.col_hi;
  const long nchunks = (col_hi - col_lo + PK_BY - 1) / PK_BY;
  const int nl = a.nlambda, ns = a.nstage;
  const unsigned colb = (unsigned)a.np * 4u;                 // bytes per column and component
  const unsigned stage_bytes = 6u * PK_BY * colb;
  const long my_chunks = blockIdx.x < nchunks ? (nchunks - 1 - blockIdx.x) / gridDim.x + 1 : 0;
  const long total = my_chunks * nl;

  griddep_launch_dependents();
  if (tid == 0) {
    for (int s = 0; s < ns; ++s) mbar_init(&full[s], 1);
    s_abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  __syncthreads();

  auto issue = [&](long j) {
    const int s = (int)(j % ns);
    const long chunk = blockIdx.x + (j / nl) * gridDim.x;
    const int l = (int)(j % nl);
    const long col0 = col_lo + chunk * PK_BY;
    const unsigned n = (unsigned)min((long)PK_BY, col_hi - col0);
    unsigned char *dst = ring + (size_t)s * stage_bytes;
    mbar_arrive_expect_tx(&full[s], 6u * n * colb);
#pragma unroll
    for (int f = 0; f < 2; ++f) {
      const unsigned char *base = (f == 0 ? a.EF[l] : a.EA[l]) + 16;
#pragma unroll
      for (int c = 0; c < 3; ++c)
        bulk_load(dst + (f * 3 + c) * PK_BY * colb, base + ((size_t)c * ncol + col0) * colb,
                  n * colb, &full[s]);
    }
  };
  if (tid == 0)
    for (long j = 0; j < min((long)ns, total); ++j) issue(j);

  const int c = tid / PK_BY, col = tid - c * PK_BY;
  const int nq = a.np >> 2;
  float acc_in = 0.f, acc_face = 0.f;
  long consumed = 0;
  for (long i = 0; i < total; ++i) {
    const int s = (int)(i % ns);
    const bool ok = mbar_wait_bounded(&full[s], (unsigned)((i / ns) & 1));
    if (!ok) s_abort = 1;
    const int l = (int)(i % nl);
    if (ok) {
      const uint4 *pf = reinterpret_cast<const uint4 *>(ring + (size_t)s * stage_bytes +
                                                        (c * PK_BY + col) * colb);
      const uint4 *pa = reinterpret_cast<const uint4 *>(ring + (size_t)s * stage_bytes +
                                                        ((3 + c) * PK_BY + col) * colb);
      float s_in = 0.f, s_face = 0.f;
      for (int q = 0; q < nq; ++q) {
        const uint4 f = pf[q];
        const uint4 e = pa[q];
        const unsigned fb[4] = {f.x, f.y, f.z, f.w};
        const unsigned eb[4] = {e.x, e.y, e.z, e.w};
#pragma unroll
        for (int t = 0; t < 4; ++t) {
          const int kk = 4 * q + t;   // packed plane kk is plane k0 + kk
          const float2 x = unpack2(fb[t], a.type);
          const float2 y = unpack2(eb[t], a.type);
          const float re = fmaf(x.x, y.x, -x.y * y.y);
          const bool in = c < 2 ? (kk >= 1 && kk <= a.nk) : (kk >= 1 && kk <= a.nk - 1);
          const bool face = c == 2 && (kk == 0 || kk == a.nk);
          s_in += in ? re : 0.f;
          s_face += face ? re : 0.f;
        }
      }
      const float sc = __ldg(reinterpret_cast<const float *>(a.EF[l]) + c) *
                       __ldg(reinterpret_cast<const float *>(a.EA[l]) + c) * a.fs[l][c];
      // a rounded product, then a rounded sum, per wavelength
      acc_in = __fadd_rn(acc_in, __fmul_rn(s_in, sc));
      if (c == 2) acc_face = __fadd_rn(acc_face, __fmul_rn(s_face, sc));
      if (l == nl - 1) {
        const long gcol = col_lo + (blockIdx.x + (i / nl) * gridDim.x) * PK_BY + col;
        if (gcol < col_hi) {
          a.W[(size_t)c * ncol + gcol] = acc_in;
          if (c == 2) a.W[3 * (size_t)ncol + gcol] = acc_face;
        }
        acc_in = acc_face = 0.f;
      }
    }
    __syncthreads();   // stage s fully read (and every thread's timeout flag visible)
    if (s_abort) break;
    consumed = i + 1;
    if (tid == 0 && i + ns < total) issue(i + ns);
  }

  if (s_abort) {
    // record the timeout, then let every copy this block issued land before
    // its shared memory is released (each wait bounded again)
    if (tid == 0) {
      atomicOr(a.err, ERRFLAG_TIMEOUT);
      const long issued = min(total, consumed + ns);
      for (long j = consumed; j < issued; ++j)
        mbar_wait_bounded(&full[j % ns], (unsigned)((j / ns) & 1));
    }
    __syncthreads();
  }
}

#endif  // EPSC_PACK_KERNELS

}  // namespace epsc
