// Eq. 1 field contraction: per Yee column, the sums over the J-support
// planes of scale * s_F s_A * Re(E_F E_A) (unconjugated, summed over the
// wavelengths), one map each for
//   W_x  (Ex planes k0+1 .. k0+nk), W_y (Ey, same planes),
//   W_zi (Ez planes k0+1 .. k0+nk-1), W_zf (Ez face planes k0 and k0+nk),
// written as float32 [4][nx][ny].  Pure streaming: no stencil, so the
// kernel runs at high occupancy with many loads in flight per thread.
//
// Fast path (complex64, nz % 4 == 0, 32-byte aligned fields): four lanes
// per column, each reading one 32-byte sector (four complex planes) of
// every component of E_F and E_A with a 256-bit load.  Generic path: eight
// lanes per column reading 16-byte pieces.  Plane classification uses
// selects, so whatever the caller keeps outside the support planes never
// enters the sums.
#pragma once

#include "epsc_common.cuh"

namespace epsc {

struct ContractArgs {
  int nx, ny, nz, k0, nk;
  int nlambda;
  int mode;               // MODE_C64 or MODE_REAL
  const float *EF[EPS_MAX_LAMBDA];
  const float *EA[EPS_MAX_LAMBDA];
  float fs[EPS_MAX_LAMBDA][3];   // scale * s_F * s_A per wavelength and component
  const float *G;                // MODE_REAL cotangent
  float *W;                      // [4][nx][ny]
  int *err;                      // error flag (debug bounds checks)
};

struct F8 {
  float v[8];
};

__device__ __forceinline__ F8 ld_sector(const float *p) {
  F8 r;
  asm volatile(
      "ld.global.nc.L1::no_allocate.v8.f32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
      : "=f"(r.v[0]), "=f"(r.v[1]), "=f"(r.v[2]), "=f"(r.v[3]), "=f"(r.v[4]), "=f"(r.v[5]),
        "=f"(r.v[6]), "=f"(r.v[7])
      : "l"(p));
  return r;
}

__device__ __forceinline__ float4 ld_piece(const float *p) {
  float4 v;
  asm volatile("ld.global.nc.L1::no_allocate.v4.f32 {%0,%1,%2,%3}, [%4];"
               : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
               : "l"(p));
  return v;
}

// Lanes per column L (4: 32-byte sectors of 4 complex planes; 8: 16-byte
// pieces of 2 planes).  Each lane group handles UNR columns per iteration.
template <int L>
__global__ void __launch_bounds__(NTHREADS) contract_kernel(const __grid_constant__ ContractArgs a) {
  constexpr int PL = L == 4 ? 4 : 2;            // complex planes per lane piece
  constexpr int UNR = 2;
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  const int gl = lane & (L - 1);                // lane within the column group
  const int gw = lane / L;                      // column group within the warp
  constexpr int GPW = 32 / L;                   // column groups per warp
  const long ncol = (long)a.nx * a.ny;
  const int klo = a.k0, khi = a.k0 + a.nk;
  const int p_lo = klo / PL;                    // first piece touching plane k0
  const int p_hi = khi / PL;
  const size_t cstride = (size_t)ncol * a.nz * 2;   // floats per component
  // the stencil kernel queued behind this grid may start its own blocks now
  griddep_launch_dependents();

  // The loop bound is uniform across the warp (shuffles below need every
  // lane); each group owns columns base .. base + UNR - 1.
  float acc[UNR][4];
  const long warp_step = (long)gridDim.x * (NTHREADS / 32) * GPW * UNR;
  for (long wbase = ((long)blockIdx.x * (NTHREADS / 32) + warp) * GPW * UNR; wbase < ncol;
       wbase += warp_step) {
    const long base = wbase + (long)gw * UNR;
#pragma unroll
    for (int u = 0; u < UNR; ++u)
#pragma unroll
      for (int q = 0; q < 4; ++q) acc[u][q] = 0.f;
    if (a.mode == MODE_C64) {
      for (int l = 0; l < a.nlambda; ++l) {
        const float *ef = a.EF[l];
        const float *ea = a.EA[l];
        const float sx = a.fs[l][0], sy = a.fs[l][1], sz = a.fs[l][2];
        for (int pc = p_lo + gl; pc <= p_hi; pc += L) {
          const int k = pc * PL;   // first plane of this piece
#pragma unroll
          for (int u = 0; u < UNR; ++u) {
            const long col = base + u;
            if (col >= ncol) break;
            const size_t off = (size_t)col * a.nz * 2 + (size_t)k * 2;
            if (!EPSC_IN_BOUNDS(off, 2 * PL, cstride, a.err)) continue;
            float re[3][PL];
            if (L == 4) {
              F8 f[3], e[3];
#pragma unroll
              for (int c = 0; c < 3; ++c) {
                f[c] = ld_sector(ef + c * cstride + off);
                e[c] = ld_sector(ea + c * cstride + off);
              }
#pragma unroll
              for (int c = 0; c < 3; ++c)
#pragma unroll
                for (int t = 0; t < PL; ++t)
                  re[c][t] = fmaf(f[c].v[2 * t], e[c].v[2 * t], -f[c].v[2 * t + 1] * e[c].v[2 * t + 1]);
            } else {
              float4 f[3], e[3];
#pragma unroll
              for (int c = 0; c < 3; ++c) {
                f[c] = ld_piece(ef + c * cstride + off);
                e[c] = ld_piece(ea + c * cstride + off);
              }
#pragma unroll
              for (int c = 0; c < 3; ++c) {
                re[c][0] = fmaf(f[c].x, e[c].x, -f[c].y * e[c].y);
                re[c][PL - 1] = fmaf(f[c].z, e[c].z, -f[c].w * e[c].w);
              }
            }
            float sxy = 0.f, syy = 0.f, szi = 0.f, szf = 0.f;
#pragma unroll
            for (int t = 0; t < PL; ++t) {
              const int kk = k + t;
              const bool in_xy = kk >= klo + 1 && kk <= khi;
              const bool in_zi = kk >= klo + 1 && kk <= khi - 1;
              const bool in_zf = kk == klo || kk == khi;
              sxy += in_xy ? re[0][t] : 0.f;
              syy += in_xy ? re[1][t] : 0.f;
              szi += in_zi ? re[2][t] : 0.f;
              szf += in_zf ? re[2][t] : 0.f;
            }
            acc[u][0] = fmaf(sx, sxy, acc[u][0]);
            acc[u][1] = fmaf(sy, syy, acc[u][1]);
            acc[u][2] = fmaf(sz, szi, acc[u][2]);
            acc[u][3] = fmaf(sz, szf, acc[u][3]);
          }
        }
      }
    } else {
      // real cotangent G [3][nx][ny][nz]: lanes stride over the planes
      const size_t gs = (size_t)ncol * a.nz;
#pragma unroll
      for (int u = 0; u < UNR; ++u) {
        const long col = base + u;
        if (col >= ncol) break;
        const float *gc = a.G + (size_t)col * a.nz;
        for (int k = klo + gl; k <= khi; k += L) {
          if (!EPSC_IN_BOUNDS((size_t)col * a.nz + k, 1, gs, a.err)) continue;
          const float gx = __ldg(gc + k), gy = __ldg(gc + gs + k), gz = __ldg(gc + 2 * gs + k);
          const bool in_xy = k >= klo + 1;
          acc[u][0] += in_xy ? gx : 0.f;
          acc[u][1] += in_xy ? gy : 0.f;
          acc[u][2] += (k >= klo + 1 && k <= khi - 1) ? gz : 0.f;
          acc[u][3] += (k == klo || k == khi) ? gz : 0.f;
        }
      }
    }
#pragma unroll
    for (int u = 0; u < UNR; ++u) {
#pragma unroll
      for (int q = 0; q < 4; ++q) {
#pragma unroll
        for (int off = L / 2; off > 0; off >>= 1)
          acc[u][q] += __shfl_xor_sync(0xffffffffu, acc[u][q], off);
      }
      const long col = base + u;
      if (gl == 0 && col < ncol) {
#pragma unroll
        for (int q = 0; q < 4; ++q) a.W[(size_t)q * ncol + col] = acc[u][q];
      }
    }
  }
}

// ---- batched contraction: many regions in one launch -------------------

struct ContractBatchRegion {
  long col_start;                         // first column in the launch's column space
  int nz, k0, nk, nlambda;
  float *W;                               // [4][nx][ny] of this region
  const float *EF[EPS_MAX_BATCH_LAMBDA];
  const float *EA[EPS_MAX_BATCH_LAMBDA];
  float fs[EPS_MAX_BATCH_LAMBDA][3];
};

struct ContractBatchArgs {
  int n;
  long ncol;                              // total columns over all regions
  int *err;                               // error flag (debug bounds checks)
  ContractBatchRegion r[EPS_MAX_BATCH];
};

// Eight lanes per column, 16-byte pieces (any even nz, 16-byte aligned
// fields); the columns of all regions form one index space.
template <int V>
__global__ void __launch_bounds__(NTHREADS) contract_batched_kernel(const __grid_constant__ ContractBatchArgs a) {
  constexpr int L = 8, GPW = 32 / L;
  griddep_launch_dependents();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int gl = lane & (L - 1), gw = lane / L;
  const long step = (long)gridDim.x * (NTHREADS / 32) * GPW;
  for (long wbase = ((long)blockIdx.x * (NTHREADS / 32) + warp) * GPW; wbase < a.ncol; wbase += step) {
    const long col = wbase + gw;
    float acc[4] = {0.f, 0.f, 0.f, 0.f};
    int k = 0;
    if (col < a.ncol) {
      while (k + 1 < a.n && col >= a.r[k + 1].col_start) ++k;
      const ContractBatchRegion &rg = a.r[k];
      const long lc = col - rg.col_start;
      const long ncr = (k + 1 < a.n ? a.r[k + 1].col_start : a.ncol) - rg.col_start;
      const size_t cstride = (size_t)ncr * rg.nz * 2;
      const int klo = rg.k0, khi = rg.k0 + rg.nk;
      for (int l = 0; l < rg.nlambda; ++l) {
        const float *ef = rg.EF[l];
        const float *ea = rg.EA[l];
        for (int pc = (klo >> 1) + gl; pc <= (khi >> 1); pc += L) {
          const size_t off = (size_t)lc * rg.nz * 2 + (size_t)pc * 4;
          if (!EPSC_IN_BOUNDS(off, 4, cstride, a.err)) continue;
          float re0[3], re1[3];
#pragma unroll
          for (int c = 0; c < 3; ++c) {
            const float4 f = ld_piece(ef + c * cstride + off);
            const float4 e = ld_piece(ea + c * cstride + off);
            re0[c] = fmaf(f.x, e.x, -f.y * e.y);
            re1[c] = fmaf(f.z, e.z, -f.w * e.w);
          }
          const int kk = 2 * pc;
          const bool xy0 = kk >= klo + 1 && kk <= khi, xy1 = kk + 1 >= klo + 1 && kk + 1 <= khi;
          const bool zi0 = kk >= klo + 1 && kk <= khi - 1, zi1 = kk + 1 >= klo + 1 && kk + 1 <= khi - 1;
          const bool zf0 = kk == klo || kk == khi, zf1 = kk + 1 == klo || kk + 1 == khi;
          acc[0] = fmaf(rg.fs[l][0], (xy0 ? re0[0] : 0.f) + (xy1 ? re1[0] : 0.f), acc[0]);
          acc[1] = fmaf(rg.fs[l][1], (xy0 ? re0[1] : 0.f) + (xy1 ? re1[1] : 0.f), acc[1]);
          acc[2] = fmaf(rg.fs[l][2], (zi0 ? re0[2] : 0.f) + (zi1 ? re1[2] : 0.f), acc[2]);
          acc[3] = fmaf(rg.fs[l][2], (zf0 ? re0[2] : 0.f) + (zf1 ? re1[2] : 0.f), acc[3]);
        }
      }
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
#pragma unroll
      for (int off = L / 2; off > 0; off >>= 1) acc[q] += __shfl_xor_sync(0xffffffffu, acc[q], off);
    }
    if (gl == 0 && col < a.ncol) {
      const ContractBatchRegion &rg = a.r[k];
      const long lc = col - rg.col_start;
      const long ncr = (k + 1 < a.n ? a.r[k + 1].col_start : a.ncol) - rg.col_start;
#pragma unroll
      for (int q = 0; q < 4; ++q) rg.W[(size_t)q * ncr + lc] = acc[q];
    }
  }
}

}  // namespace epsc
