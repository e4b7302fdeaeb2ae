// Forward chain + Eq. 1 contraction + adjoint seeds, one 8 x 32 tile of Yee
// columns per block.
//
// Stages (all in shared memory except the field reads and the outputs):
//   1. C tile with a halo of R + 3 subpixels, boundary rule applied on load.
//   2. u = K * C (Eq. 2) on the (2 TI + 5) x (2 TJ + 5) subpixel region the
//      dual cells and the Sobel halo touch, then rho (Eq. 6), eps = mix(rho)
//      and 1/eps.
//   3. Dual-cell means (Eq. 8): A_c, H_c for the tile's cells, U_x, U_y for
//      the tile plus a one-cell halo; Sobel gradients and normal weights.
//   4. Eq. 7 per column; eps_hat written for every z plane.
//   5. (VJP) W = sum over the slab planes of scale * Re(E_F E_A) (Eq. 1), or
//      of a real cotangent G; only the J-support planes are read.
//   6. (VJP) per-column seeds dJ/dA_c, dJ/dH_c, dJ/dg and the tile's u are
//      written to the workspace for the scatter kernel.
#pragma once

#include "epsc_common.cuh"

namespace epsc {

template <int RP1>
struct FwdSmem {
  static constexpr int R = RP1 - 1;
  static constexpr int CA = UA + 2 * R;
  static constexpr int CB = UB + 2 * R;
  static constexpr int HP = TJ + 2;              // pitch of the halo cell maps
  static constexpr int HN = (TI + 2) * HP;
  static constexpr int OFF_C = 0;
  static constexpr int OFF_U = OFF_C + CA * CB;
  static constexpr int OFF_E = OFF_U + UA * UB;
  static constexpr int OFF_IE = OFF_E + UA * UB;
  static constexpr int OFF_UX = OFF_IE + UA * UB;
  static constexpr int OFF_UY = OFF_UX + HN;
  static constexpr int OFF_W = OFF_UY + HN;      // 4 x NTHREADS contraction sums
  static constexpr int OFF_EPS = OFF_W + 4 * NTHREADS;   // 6 x NTHREADS column values
  static constexpr int TOTAL = OFF_EPS + 6 * NTHREADS;
  static constexpr size_t BYTES = sizeof(float) * TOTAL;
};

__device__ __forceinline__ float4 ld_stream(const float4 *p) {
  float4 v;
  asm volatile("ld.global.nc.L1::no_allocate.v4.f32 {%0,%1,%2,%3}, [%4];"
               : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
               : "l"(p));
  return v;
}

// value of eps_hat component `comp` on plane k given the column's Eq. 7 values
__device__ __forceinline__ float plane_value(int comp, int k, int k0, int nk, float exy, float ezi,
                                             float ezf, float clad) {
  if (comp < 2) return (k >= k0 + 1 && k <= k0 + nk) ? exy : clad;
  if (k >= k0 + 1 && k <= k0 + nk - 1) return ezi;
  if (k == k0 || k == k0 + nk) return ezf;
  return clad;
}

template <int RP1>
__global__ void __launch_bounds__(NTHREADS) fwd_kernel(const __grid_constant__ FwdArgs a) {
  using S = FwdSmem<RP1>;
  constexpr int R = S::R;
  constexpr int CB = S::CB;
  extern __shared__ float smem[];
  float *sC = smem + S::OFF_C;
  float *su = smem + S::OFF_U;
  float *se = smem + S::OFF_E;
  float *sie = smem + S::OFF_IE;
  float *sUx = smem + S::OFF_UX;
  float *sUy = smem + S::OFF_UY;
  float *sW = smem + S::OFF_W;
  float *sE = smem + S::OFF_EPS;

  const Geometry &g = a.g;
  const int tid = threadIdx.x;
  const int j0 = blockIdx.x * TJ;
  const int i0 = blockIdx.y * TI;
  const int ua0 = 2 * i0 - 3;
  const int ub0 = 2 * j0 - 3;
  const int ca0 = ua0 - R;
  const int cb0 = ub0 - R;

  // ---- 1. control tile with halo --------------------------------------
  for (int idx = tid; idx < S::CA * CB; idx += NTHREADS) {
    const int r = idx / CB;
    const int c = idx - r * CB;
    const int ga = bc_map(ca0 + r, g.mx, g.bc);
    const int gb = bc_map(cb0 + c, g.my, g.bc);
    sC[idx] = __ldg(a.C + (size_t)ga * g.my + gb);
  }
  __syncthreads();

  // ---- 2. filtered density, projection, mixing -------------------------
  constexpr int NSTRIP = UA / NA_F;
  for (int item = tid; item < NSTRIP * UB; item += NTHREADS) {
    const int s = item / UB;
    const int col = item - s * UB;
    const int r0 = s * NA_F;
    float hi[NA_F], lo[NA_F];
    strip_stencil<RP1, NA_F, true>(sC + r0 * CB + col, CB, a, hi, lo);
#pragma unroll
    for (int k = 0; k < NA_F; ++k) {
      const int o = (r0 + k) * UB + col;
      const float x = g.beta * ((hi[k] - g.eta) + lo[k]);
      const float rho = fmaf(0.5f, tanhf(x), 0.5f);
      const float e = fmaf(rho, g.deps, g.eps_clad);
      su[o] = hi[k] + lo[k];
      se[o] = e;
      sie[o] = 1.0f / e;
    }
  }
  __syncthreads();

  // edge replicate: subpixels outside the region take the edge subpixel's values
  if (g.bc == EPS_BC_CLAMP && (ua0 < 0 || ub0 < 0 || ua0 + UA > g.mx || ub0 + UB > g.my)) {
    for (int idx = tid; idx < UA * UB; idx += NTHREADS) {
      const int r = idx / UB;
      const int c = idx - r * UB;
      const int ga = ua0 + r, gb = ub0 + c;
      const int cga = clampi(ga, 0, g.mx - 1), cgb = clampi(gb, 0, g.my - 1);
      if (cga != ga || cgb != gb) {
        const int src = (cga - ua0) * UB + (cgb - ub0);
        su[idx] = su[src];
        se[idx] = se[src];
        sie[idx] = sie[src];
      }
    }
    __syncthreads();
  }

  // ---- 3. dual-cell means and normals ----------------------------------
  // U_x, U_y on the tile's cells plus a one-cell halo (Yee-level bc)
  for (int idx = tid; idx < S::HN; idx += NTHREADS) {
    const int hr = idx / S::HP;
    const int hc = idx - hr * S::HP;
    int ci = i0 - 1 + hr, cj = j0 - 1 + hc;
    if (g.bc == EPS_BC_CLAMP) {
      ci = clampi(ci, 0, g.nx - 1);
      cj = clampi(cj, 0, g.ny - 1);
    }
    const int ra = 2 * ci - ua0, rb = 2 * cj - ub0;
    // Omega_x: a in {2i, 2i+1}, b in {2j-1, 2j};  Omega_y: a in {2i-1, 2i}, b in {2j, 2j+1}
    sUx[idx] = 0.25f * ((su[ra * UB + rb - 1] + su[ra * UB + rb]) +
                        (su[(ra + 1) * UB + rb - 1] + su[(ra + 1) * UB + rb]));
    sUy[idx] = 0.25f * ((su[(ra - 1) * UB + rb] + su[(ra - 1) * UB + rb + 1]) +
                        (su[ra * UB + rb] + su[ra * UB + rb + 1]));
  }

  const int cr = tid / TJ, cc = tid - (tid / TJ) * TJ;
  const int ci = i0 + cr, cj = j0 + cc;
  const bool valid = ci < g.nx && cj < g.ny;
  const int ra = 2 * cr + 3, rb = 2 * cc + 3;
  const float Ax = 0.25f * ((se[ra * UB + rb - 1] + se[ra * UB + rb]) +
                            (se[(ra + 1) * UB + rb - 1] + se[(ra + 1) * UB + rb]));
  const float Hx = 0.25f * ((sie[ra * UB + rb - 1] + sie[ra * UB + rb]) +
                            (sie[(ra + 1) * UB + rb - 1] + sie[(ra + 1) * UB + rb]));
  const float Ay = 0.25f * ((se[(ra - 1) * UB + rb] + se[(ra - 1) * UB + rb + 1]) +
                            (se[ra * UB + rb] + se[ra * UB + rb + 1]));
  const float Hy = 0.25f * ((sie[(ra - 1) * UB + rb] + sie[(ra - 1) * UB + rb + 1]) +
                            (sie[ra * UB + rb] + sie[ra * UB + rb + 1]));
  const float Az = 0.25f * ((se[(ra - 1) * UB + rb - 1] + se[(ra - 1) * UB + rb]) +
                            (se[ra * UB + rb - 1] + se[ra * UB + rb]));
  const float Hz = 0.25f * ((sie[(ra - 1) * UB + rb - 1] + sie[(ra - 1) * UB + rb]) +
                            (sie[ra * UB + rb - 1] + sie[ra * UB + rb]));
  __syncthreads();

  float gxx, gyx, gxy, gyy;
  {
    constexpr int P = S::HP;
    const int h = (cr + 1) * P + (cc + 1);
    gxx = (sUx[h + P - 1] - sUx[h - P - 1]) + 2.f * (sUx[h + P] - sUx[h - P]) +
          (sUx[h + P + 1] - sUx[h - P + 1]);
    gyx = (sUx[h - P + 1] - sUx[h - P - 1]) + 2.f * (sUx[h + 1] - sUx[h - 1]) +
          (sUx[h + P + 1] - sUx[h + P - 1]);
    gxy = (sUy[h + P - 1] - sUy[h - P - 1]) + 2.f * (sUy[h + P] - sUy[h - P]) +
          (sUy[h + P + 1] - sUy[h - P + 1]);
    gyy = (sUy[h - P + 1] - sUy[h - P - 1]) + 2.f * (sUy[h + 1] - sUy[h - 1]) +
          (sUy[h + P + 1] - sUy[h + P - 1]);
  }
  const float g2x = gxx * gxx + gyx * gyx;
  const float g2y = gxy * gxy + gyy * gyy;
  const bool okx = g2x > NORMAL_TAU2, oky = g2y > NORMAL_TAU2;
  const float mx_ = okx ? gxx * gxx / g2x : 0.f;
  const float my_ = oky ? gyy * gyy / g2y : 0.f;

  // ---- 4. Eq. 7 and the eps_hat store ----------------------------------
  const float ex = 1.0f / fmaf(mx_, Hx, (1.f - mx_) / Ax);
  const float ey = 1.0f / fmaf(my_, Hy, (1.f - my_) / Ay);
  const float ezi = Az;
  const float ezf = 1.0f / fmaf(0.5f, Hz, 0.5f / g.eps_clad);
  sE[0 * NTHREADS + tid] = ex;
  sE[1 * NTHREADS + tid] = ey;
  sE[2 * NTHREADS + tid] = ezi;
  sE[3 * NTHREADS + tid] = ezf;
  if (a.write_offdiag) {
    sE[4 * NTHREADS + tid] = okx ? gxx * gyx / g2x * (Hx - 1.f / Ax) : 0.f;
    sE[5 * NTHREADS + tid] = oky ? gxy * gyy / g2y * (Hy - 1.f / Ay) : 0.f;
  }
  __syncthreads();

  const int nvi = min(TI, g.nx - i0);
  const int nvj = min(TJ, g.ny - j0);
  if (a.write_eps || a.write_offdiag) {
    const int ncomp_eps = a.write_eps ? 3 : 0;
    const int ncomp = ncomp_eps + (a.write_offdiag ? 2 : 0);
    if ((g.nz & 3) == 0) {
      const int nz4 = g.nz >> 2;
      const FastDiv dz4(nz4);
      const int per_row = nvj * nz4;
      for (int t = 0; t < ncomp; ++t) {
        const bool od = t >= ncomp_eps;
        const int comp = od ? t - ncomp_eps : t;
        float *base = od ? a.offdiag : a.eps;
        for (int r = 0; r < nvi; ++r) {
          float4 *dst = reinterpret_cast<float4 *>(
              base + (((size_t)comp * g.nx + i0 + r) * g.ny + j0) * g.nz);
          for (int f = tid; f < per_row; f += NTHREADS) {
            const int c = dz4.div(f);
            const int k = 4 * (f - c * nz4);
            const int col = r * TJ + c;
            float4 v;
            if (od) {
              const float val = sE[(4 + comp) * NTHREADS + col];
              v.x = (k + 0 >= g.k0 + 1 && k + 0 <= g.k0 + g.nk) ? val : 0.f;
              v.y = (k + 1 >= g.k0 + 1 && k + 1 <= g.k0 + g.nk) ? val : 0.f;
              v.z = (k + 2 >= g.k0 + 1 && k + 2 <= g.k0 + g.nk) ? val : 0.f;
              v.w = (k + 3 >= g.k0 + 1 && k + 3 <= g.k0 + g.nk) ? val : 0.f;
            } else {
              const float exy = sE[comp * NTHREADS + col];
              const float vzi = sE[2 * NTHREADS + col], vzf = sE[3 * NTHREADS + col];
              v.x = plane_value(comp, k + 0, g.k0, g.nk, exy, vzi, vzf, g.eps_clad);
              v.y = plane_value(comp, k + 1, g.k0, g.nk, exy, vzi, vzf, g.eps_clad);
              v.z = plane_value(comp, k + 2, g.k0, g.nk, exy, vzi, vzf, g.eps_clad);
              v.w = plane_value(comp, k + 3, g.k0, g.nk, exy, vzi, vzf, g.eps_clad);
            }
            __stcs(dst + f, v);
          }
        }
      }
    } else {
      const FastDiv dz(g.nz);
      const int per_row = nvj * g.nz;
      for (int t = 0; t < ncomp; ++t) {
        const bool od = t >= ncomp_eps;
        const int comp = od ? t - ncomp_eps : t;
        float *base = od ? a.offdiag : a.eps;
        for (int r = 0; r < nvi; ++r) {
          float *dst = base + (((size_t)comp * g.nx + i0 + r) * g.ny + j0) * g.nz;
          for (int f = tid; f < per_row; f += NTHREADS) {
            const int c = dz.div(f);
            const int k = f - c * g.nz;
            const int col = r * TJ + c;
            float v;
            if (od) {
              v = (k >= g.k0 + 1 && k <= g.k0 + g.nk) ? sE[(4 + comp) * NTHREADS + col] : 0.f;
            } else {
              v = plane_value(comp, k, g.k0, g.nk, sE[comp * NTHREADS + col],
                              sE[2 * NTHREADS + col], sE[3 * NTHREADS + col], g.eps_clad);
            }
            __stcs(dst + f, v);
          }
        }
      }
    }
  }
  if (a.mode == MODE_FWD) return;

  // ---- 5. Eq. 1 contraction over the J-support planes ------------------
  {
    const int warp = tid >> 5, lane = tid & 31;
    const int grp = lane >> 3, gl = lane & 7;
    const int klo = g.k0, khi = g.k0 + g.nk;
    for (int pass = 0; pass < NTHREADS / 32; ++pass) {
      const int slot = pass * 32 + warp * 4 + grp;
      const int r = slot / TJ, c = slot - (slot / TJ) * TJ;
      const int pi = i0 + r, pj = j0 + c;
      float wx = 0.f, wy = 0.f, wzi = 0.f, wzf = 0.f;
      if (pi < g.nx && pj < g.ny) {
        if (a.mode == MODE_C64) {
          const int nz2 = g.nz >> 1;
          const size_t cs = (size_t)g.nx * g.ny * nz2;       // component stride, float4
          const size_t col = ((size_t)pi * g.ny + pj) * nz2;
          const int plo = klo >> 1, phi = khi >> 1;
          for (int l = 0; l < a.nlambda; ++l) {
            const float4 *ef = a.EF[l] + col;
            const float4 *ea = a.EA[l] + col;
            for (int pc = plo + gl; pc <= phi; pc += 8) {
              const float4 fx = ld_stream(ef + pc), ax = ld_stream(ea + pc);
              const float4 fy = ld_stream(ef + cs + pc), ay = ld_stream(ea + cs + pc);
              const float4 fz = ld_stream(ef + 2 * cs + pc), az = ld_stream(ea + 2 * cs + pc);
              const int k = 2 * pc;
              const bool s0 = k >= klo + 1 && k <= khi;
              const bool s1 = k + 1 >= klo + 1 && k + 1 <= khi;
              const bool i0z = k >= klo + 1 && k <= khi - 1;
              const bool i1z = k + 1 >= klo + 1 && k + 1 <= khi - 1;
              const bool f0z = k == klo || k == khi;
              const bool f1z = k + 1 == klo || k + 1 == khi;
              const float x0 = fx.x * ax.x - fx.y * ax.y, x1 = fx.z * ax.z - fx.w * ax.w;
              const float y0 = fy.x * ay.x - fy.y * ay.y, y1 = fy.z * ay.z - fy.w * ay.w;
              const float z0 = fz.x * az.x - fz.y * az.y, z1 = fz.z * az.z - fz.w * az.w;
              wx = fmaf(a.fs[l][0], (s0 ? x0 : 0.f) + (s1 ? x1 : 0.f), wx);
              wy = fmaf(a.fs[l][1], (s0 ? y0 : 0.f) + (s1 ? y1 : 0.f), wy);
              wzi = fmaf(a.fs[l][2], (i0z ? z0 : 0.f) + (i1z ? z1 : 0.f), wzi);
              wzf = fmaf(a.fs[l][2], (f0z ? z0 : 0.f) + (f1z ? z1 : 0.f), wzf);
            }
          }
        } else {   // MODE_REAL: G is the cotangent of eps_hat itself
          const size_t cs = (size_t)g.nx * g.ny * g.nz;
          const float *gc = a.G + ((size_t)pi * g.ny + pj) * g.nz;
          for (int k = klo + gl; k <= khi; k += 8) {
            const float gx_ = __ldg(gc + k), gy_ = __ldg(gc + cs + k), gz_ = __ldg(gc + 2 * cs + k);
            if (k >= klo + 1) {
              wx += gx_;
              wy += gy_;
            }
            if (k >= klo + 1 && k <= khi - 1) wzi += gz_;
            if (k == klo || k == khi) wzf += gz_;
          }
        }
      }
#pragma unroll
      for (int off = 4; off > 0; off >>= 1) {
        wx += __shfl_xor_sync(0xffffffffu, wx, off);
        wy += __shfl_xor_sync(0xffffffffu, wy, off);
        wzi += __shfl_xor_sync(0xffffffffu, wzi, off);
        wzf += __shfl_xor_sync(0xffffffffu, wzf, off);
      }
      if (gl == 0) {
        sW[0 * NTHREADS + slot] = wx;
        sW[1 * NTHREADS + slot] = wy;
        sW[2 * NTHREADS + slot] = wzi;
        sW[3 * NTHREADS + slot] = wzf;
      }
    }
  }
  __syncthreads();

  // ---- 6. adjoint seeds and the tile's u -------------------------------
  if (valid) {
    const float Wx = sW[0 * NTHREADS + tid], Wy = sW[1 * NTHREADS + tid];
    const float Wzi = sW[2 * NTHREADS + tid], Wzf = sW[3 * NTHREADS + tid];
    // eps = 1/(m H + (1-m)/A):  de/dH = -eps^2 m, de/dA = eps^2 (1-m)/A^2, de/dm = -eps^2 (H - 1/A)
    const float e2x = ex * ex * Wx, e2y = ey * ey * Wy;
    const float dAx = e2x * (1.f - mx_) / (Ax * Ax), dHx = -e2x * mx_;
    const float dmx = -e2x * (Hx - 1.f / Ax);
    const float dAy = e2y * (1.f - my_) / (Ay * Ay), dHy = -e2y * my_;
    const float dmy = -e2y * (Hy - 1.f / Ay);
    float dgxx = 0.f, dgyx = 0.f, dgxy = 0.f, dgyy = 0.f;
    if (okx) {   // m = gx^2/|g|^2: dm/dgx = 2 gx gy^2/|g|^4, dm/dgy = -2 gx^2 gy/|g|^4
      const float t = 2.f * dmx / (g2x * g2x);
      dgxx = t * gxx * gyx * gyx;
      dgyx = -t * gxx * gxx * gyx;
    }
    if (oky) {   // m = gy^2/|g|^2: dm/dgx = -2 gx gy^2/|g|^4, dm/dgy = 2 gx^2 gy/|g|^4
      const float t = 2.f * dmy / (g2y * g2y);
      dgxy = -t * gxy * gyy * gyy;
      dgyy = t * gxy * gxy * gyy;
    }
    const float dAz = Wzi;
    const float dHz = -0.5f * ezf * ezf * Wzf;
    const size_t plane = (size_t)g.nx * g.ny;
    float *sd = a.seeds + (size_t)ci * g.ny + cj;
    sd[S_DAX * plane] = dAx;
    sd[S_DHX * plane] = dHx;
    sd[S_GXX * plane] = dgxx;
    sd[S_GYX * plane] = dgyx;
    sd[S_DAY * plane] = dAy;
    sd[S_DHY * plane] = dHy;
    sd[S_GXY * plane] = dgxy;
    sd[S_GYY * plane] = dgyy;
    sd[S_DAZ * plane] = dAz;
    sd[S_DHZ * plane] = dHz;
  }
  {
    const int na = 2 * nvi, nb = 2 * nvj;
    for (int idx = tid; idx < 4 * TI * TJ; idx += NTHREADS) {
      const int r = idx / (2 * TJ);
      const int c = idx - r * (2 * TJ);
      if (r < na && c < nb)
        a.uws[(size_t)(2 * i0 + r) * g.my + 2 * j0 + c] = su[(r + 3) * UB + c + 3];
    }
  }
}

}  // namespace epsc
