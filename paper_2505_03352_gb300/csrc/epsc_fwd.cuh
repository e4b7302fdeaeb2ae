// Forward chain + adjoint seeds, one 8 x 32 tile of Yee columns per block.
//
// Stages (all in shared memory except the field reads and the outputs):
//   1. C tile with a halo of R + 3 subpixels (asynchronous copies), boundary
//      rule applied on load.
//   2. u = K * C (Eq. 2) on the (2 TI + 5) x (2 TJ + 5) subpixel region the
//      dual cells and the Sobel halo touch, then rho (Eq. 6), eps = mix(rho)
//      and 1/eps.
//   3. Dual-cell means (Eq. 8): A_c, H_c for the tile's cells, U_x, U_y for
//      the tile plus a one-cell halo; Sobel gradients and normal weights.
//   4. Eq. 7 per column; eps_hat rows written with warp-contiguous 16-byte
//      streaming stores.
//   5. (VJP) per-column seeds dJ/dA_c, dJ/dH_c, dJ/dg = W * factor, after
//      waiting for the contraction's column sums W, or (defer_seeds) the
//      W-independent factors alone, finished by the seeds kernel; stage 2
//      already wrote the per-subpixel adjoint factors P'(u) (eps_core -
//      eps_clad) / 4 and 1/eps^2 of the tile.
#pragma once

#include "epsc_common.cuh"

namespace epsc {

template <int RP1>
struct FwdSmem {
  static constexpr int R = RP1 - 1;
  static constexpr int CA = UA + 2 * R;
  static constexpr int CB = UB + 2 * R;
  // row pitch of the staged C tile: whole 16-byte runs with room for a row
  // that starts up to 3 floats after a 16-byte boundary
  static constexpr int CBP = (CB + 3 + 3) & ~3;
  static constexpr int HP = TJ + 2;              // pitch of the halo cell maps
  static constexpr int HN = (TI + 2) * HP;
  static constexpr int OFF_C = 0;
  static constexpr int OFF_U = OFF_C + CA * CBP;
  static constexpr int OFF_E = OFF_U + UA * UB;
  static constexpr int OFF_IE = OFF_E + UA * UB;
  static constexpr int OFF_UX = OFF_IE + UA * UB;
  static constexpr int OFF_UY = OFF_UX + HN;
  static constexpr int OFF_UZ = OFF_UY + HN;       // U_z with halo (3-D face normals)
  static constexpr int TOTAL = OFF_UZ + HN;
  static constexpr size_t BYTES = sizeof(float) * TOTAL;
  // dynamic shared memory of a launch: max(BYTES, the eps_hat staging area)
};

// Value of output component `comp` on plane k: comp 0/1 = eps_xx/yy and
// 3/4 = off-diagonal at the Ex/Ey points take `vmain` on the slab planes;
// comp 2 = eps_zz takes vzi inside the slab and vzf on the two face planes;
// comp 5/6 = eta_zx/zy at the Ez points take vmain on the lower face plane,
// -vmain on the upper one and 0 elsewhere.
__device__ __forceinline__ float plane_value(int comp, int k, int k0, int nk, float vmain,
                                             float vzi, float vzf, float clad) {
  const bool slab = k >= k0 + 1 && k <= k0 + nk;
  if (comp < 2) return slab ? vmain : clad;
  if (comp > 4) return k == k0 ? vmain : (k == k0 + nk ? -vmain : 0.f);
  if (comp > 2) return slab ? vmain : 0.f;
  if (k >= k0 + 1 && k <= k0 + nk - 1) return vzi;
  if (k == k0 || k == k0 + nk) return vzf;
  return clad;
}

// Planes 4 k4 .. 4 k4 + 3 of one eps_hat component of a column: `vin` on
// the value run [lo, hi], `vf` on the face planes kf0, kf1 (eps_zz), `out`
// elsewhere.  Groups of four planes wholly inside the run or wholly outside
// [flo, fhi] take one branch (uniform over a warp when k4 is); the rest
// select per plane.
__device__ __forceinline__ float4 eps_planes4(int k4, float vin, float vf, float out, int lo,
                                              int hi, int flo, int fhi, int kf0, int kf1) {
  const int k = 4 * k4;
  if (k >= lo && k + 3 <= hi) return make_float4(vin, vin, vin, vin);
  if (k + 3 < flo || k > fhi) return make_float4(out, out, out, out);
  float t[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int kk = k + q;
    const bool in = kk >= lo && kk <= hi;
    const bool face = kk == kf0 || kk == kf1;
    t[q] = in ? vin : (face ? vf : out);
  }
  return make_float4(t[0], t[1], t[2], t[3]);
}

template <int BC>
__device__ __forceinline__ int bc_map_t(int x, int n) {
  return BC == EPS_BC_CLAMP ? clampi(x, 0, n - 1) : wrapi(x, n);
}

// One tile (rows i0 .., columns j0 ..) of one region `rg`; `a` supplies the
// conic weights as compile-time-indexed kernel parameters.  `eps_map` (the
// single-region kernel's parameter, or null) is the tensor map of eps_hat
// for the swizzled staging form (rg.eps_tma).
template <int RP1, int BC, class Args>
__device__ __forceinline__ void fwd_tile(const Args &a, const FwdRegion &rg, const int i0,
                                         const int j0, const CUtensorMap *eps_map = nullptr) {
  using S = FwdSmem<RP1>;
  constexpr int R = S::R;
  constexpr int CB = S::CB;
  extern __shared__ __align__(16) float smem[];
  float *sC = smem + S::OFF_C;
  float *su = smem + S::OFF_U;
  float *se = smem + S::OFF_E;
  float *sie = smem + S::OFF_IE;
  float *sUx = smem + S::OFF_UX;
  float *sUy = smem + S::OFF_UY;
  float *sUz = smem + S::OFF_UZ;

  const Geometry &g = rg.g;
  const int tid = threadIdx.x;
  const int ua0 = 2 * i0 - 3;
  const int ub0 = 2 * j0 - 3;
  const int ca0 = ua0 - R;
  const int cb0 = ub0 - R;
  const int nvi = min(TI, g.nx - i0);
  const int nvj = min(TJ, g.ny - j0);

  // the scatter kernel queued behind this grid may start launching; it
  // waits for this grid's results before reading them
  griddep_launch_dependents();

  // ---- 1. control tile with halo (asynchronous copies) ----------------
  // A tile whose halo lies inside the region, in a control map whose rows
  // are whole 16-byte runs, copies 16 bytes at a time from the 16-byte
  // boundary at or below its first column (the staged view is shifted by
  // the remainder, csh); the others copy element by element with the
  // boundary rule applied.  Every copy stays inside the map.
  constexpr int CBP = S::CBP;
  const int xa = cb0 & ~3;                       // (floor to a multiple of 4)
  const int ncv = (cb0 + CB - xa + 3) >> 2;      // float4 per row
  const bool cvec = (g.my & 3) == 0 && ((uintptr_t)rg.C & 15) == 0 && ca0 >= 0 &&
                    ca0 + S::CA <= g.mx && xa >= 0 && xa + 4 * ncv <= g.my;
  const int csh = cvec ? cb0 - xa : 0;
  if (cvec) {
    for (int idx = tid; idx < S::CA * ncv; idx += NTHREADS) {
      const int r = idx / ncv, k = idx - r * ncv;
      const size_t o = (size_t)(ca0 + r) * g.my + xa + 4 * k;
      if (!EPSC_IN_BOUNDS(o, 4, (size_t)g.mx * g.my, a.err)) continue;
      cp_async16(sC + r * CBP + 4 * k, rg.C + o);
    }
  } else {
    for (int idx = tid; idx < S::CA * CB; idx += NTHREADS) {
      const int r = idx / CB;
      const int c = idx - r * CB;
      const int ga = bc_map_t<BC>(ca0 + r, g.mx);
      const int gb = bc_map_t<BC>(cb0 + c, g.my);
      const size_t o = (size_t)ga * g.my + gb;
      const bool ok = EPSC_IN_BOUNDS(o, 1, (size_t)g.mx * g.my, a.err);
      cp_async4(sC + r * CBP + c, rg.C + (ok ? o : 0), ok);
    }
  }
  cp_async_wait_all();
  __syncthreads();

  // ---- 2. filtered density, projection, mixing -------------------------
  // rho = (1 + tanh(x)) / 2, x = beta (u - eta), from t = exp(-2|x|) <= 1
  // (no overflow at any beta): rho = 1/(1+t) for x >= 0 and t/(1+t) below,
  // rho (1 - rho) = t/(1+t)^2.  The adjoint factor P'(u) (eps_core -
  // eps_clad) / 4 = beta/2 deps rho (1 - rho) and 1/eps^2 of the core
  // subpixels go to the workspace for the scatter kernel.
  constexpr int NSTRIP = UA / NA_F;
  const bool vjp = rg.mode != MODE_FWD;
  for (int item = tid; item < NSTRIP * UB; item += NTHREADS) {
    const int s = item / UB;
    const int col = item - s * UB;
    const int r0 = s * NA_F;
    float hi[NA_F];
    strip_stencil<RP1, NA_F>(sC + csh + r0 * CBP + col, CBP, a, hi);
#pragma unroll
    for (int k = 0; k < NA_F; ++k) {
      const int o = (r0 + k) * UB + col;
      const float x = g.beta * (hi[k] - g.eta);
      const float t = __expf(-2.f * fabsf(x));
      const float inv = __fdividef(1.f, 1.f + t);
      const float rho = x >= 0.f ? inv : t * inv;
      const float e = fmaf(rho, g.deps, g.eps_clad);
      const float ie = __frcp_rn(e);
      su[o] = hi[k];
      se[o] = e;
      sie[o] = ie;
      if (vjp) {
        const int ra = r0 + k - 3, rb = col - 3;   // core subpixel of the tile?
        if (ra >= 0 && ra < 2 * nvi && rb >= 0 && rb < 2 * nvj) {
          const size_t go = (size_t)(2 * i0 + ra) * g.my + 2 * j0 + rb;
          if (EPSC_IN_BOUNDS(go, 1, (size_t)g.mx * g.my, a.err)) {
            rg.pd4[go] = 0.5f * g.beta * g.deps * (t * inv * inv);
            rg.ie2[go] = ie * ie;
          }
        }
      }
    }
  }
  __syncthreads();

  // edge replicate: subpixels outside the region take the edge subpixel's values
  if (BC == EPS_BC_CLAMP && (ua0 < 0 || ub0 < 0 || ua0 + UA > g.mx || ub0 + UB > g.my)) {
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
    if (BC == EPS_BC_CLAMP) {
      ci = clampi(ci, 0, g.nx - 1);
      cj = clampi(cj, 0, g.ny - 1);
    }
    const int ra = 2 * ci - ua0, rb = 2 * cj - ub0;
    // Omega_x: a in {2i, 2i+1}, b in {2j-1, 2j};  Omega_y: a in {2i-1, 2i}, b in {2j, 2j+1}
    sUx[idx] = 0.25f * ((su[ra * UB + rb - 1] + su[ra * UB + rb]) +
                        (su[(ra + 1) * UB + rb - 1] + su[(ra + 1) * UB + rb]));
    sUy[idx] = 0.25f * ((su[(ra - 1) * UB + rb] + su[(ra - 1) * UB + rb + 1]) +
                        (su[ra * UB + rb] + su[ra * UB + rb + 1]));
    // Omega_z: a in {2i-1, 2i}, b in {2j-1, 2j}
    if (rg.normals3d)
      sUz[idx] = 0.25f * ((su[(ra - 1) * UB + rb - 1] + su[(ra - 1) * UB + rb]) +
                          (su[ra * UB + rb - 1] + su[ra * UB + rb]));
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
  // explicit fma: the result must not depend on how the compiler contracts
  const float g2x = fmaf(gxx, gxx, gyx * gyx);
  const float g2y = fmaf(gxy, gxy, gyy * gyy);
  const bool okx = g2x > NORMAL_TAU2, oky = g2y > NORMAL_TAU2;
  const float ig2x = okx ? __frcp_rn(g2x) : 0.f;
  const float ig2y = oky ? __frcp_rn(g2y) : 0.f;
  const float mx_ = gxx * gxx * ig2x;
  const float my_ = gyy * gyy * ig2y;

  // ---- 4. Eq. 7 and the eps_hat store ----------------------------------
  const float iAx = __frcp_rn(Ax), iAy = __frcp_rn(Ay);
  const float ex = __frcp_rn(fmaf(mx_, Hx, (1.f - mx_) * iAx));
  const float ey = __frcp_rn(fmaf(my_, Hy, (1.f - my_) * iAy));
  const float ezf = __frcp_rn(fmaf(0.5f, Hz, 0.5f / g.eps_clad));
  const float ezi = Az;   // n_z = 0 inside the slab: eps_zz = <eps>_z
  const float odx = gxx * gyx * ig2x * (Hx - iAx);
  const float ody = gxy * gyy * ig2y * (Hy - iAy);

  // 3-D normals at the slab faces (forward only).  The Ez cells of planes
  // k0 and k0 + nk are half slab, half cladding.  Sobel-consistent central
  // differences of the cell-averaged density: in plane half the Sobel of
  // U_z, along z +4 U_z at the lower face and -4 U_z at the upper face.
  // Row z of eps^-1 = n n^T <eps^-1> + (I - n n^T) / <eps> with
  // <eps> = (A_z + eps_clad)/2, <eps^-1> = (H_z + 1/eps_clad)/2; without a
  // defined normal the base rule n = z stays.  ezf3 is eps_zz on both face
  // planes; ezx3, ezy3 are eta_zx, eta_zy on the lower face (negated on the
  // upper one).
  float ezf3 = ezf, ezx3 = 0.f, ezy3 = 0.f;
  if (rg.normals3d) {
    constexpr int P = S::HP;
    const int h = (cr + 1) * P + (cc + 1);
    const float gx = 0.5f * ((sUz[h + P - 1] - sUz[h - P - 1]) + 2.f * (sUz[h + P] - sUz[h - P]) +
                             (sUz[h + P + 1] - sUz[h - P + 1]));
    const float gy = 0.5f * ((sUz[h - P + 1] - sUz[h - P - 1]) + 2.f * (sUz[h + 1] - sUz[h - 1]) +
                             (sUz[h + P + 1] - sUz[h + P - 1]));
    const float gz = 4.f * sUz[h];
    const float g2 = fmaf(gx, gx, fmaf(gy, gy, gz * gz));
    if (g2 > NORMAL_TAU2) {
      const float ig = __frcp_rn(g2);
      const float a_inv = fmaf(0.5f, Hz, 0.5f / g.eps_clad);
      const float b = __frcp_rn(fmaf(0.5f, Az, 0.5f * g.eps_clad));
      const float nz2 = gz * gz * ig;
      ezf3 = __frcp_rn(fmaf(nz2, a_inv, (1.f - nz2) * b));
      ezx3 = gz * gx * ig * (a_inv - b);
      ezy3 = gz * gy * ig * (a_inv - b);
    }
  }

  // ---- eps_hat store: whole-tile staging + bulk (TMA) stores ------------
  // Each thread writes its column's planes of `ncomp` components into shared
  // memory (rows of TJ * nz floats per component and tile row), then one
  // thread issues one bulk copy per contiguous row span.  The copies run
  // while the block goes on to the seeds; the block waits for them only
  // before it exits.  When the staging does not fit, components go in
  // rounds (waiting for the previous round's copies to read shared memory),
  // and plane counts that are not a multiple of 4 use direct stores.
  bool bulk_pending = false;
  if (rg.write_eps || rg.write_offdiag) {
    const int c_first = rg.write_eps ? 0 : 3;
    const int c_last = rg.write_offdiag ? (rg.normals3d ? 6 : 4) : 2;
    const size_t cplane = (size_t)g.nx * g.ny * g.nz;
    const int comp_floats = TI * TJ * g.nz;
    const int per_round = rg.stage_floats / comp_floats;
    if ((g.nz & 3) == 0 && rg.direct_eps) {
      // Warp-cooperative stores, no shared memory: warp cr (one tile row,
      // lane = column) writes its row's contiguous run of nvj * nz floats per
      // component, 16 coalesced bytes a lane per store; each lane takes the
      // owning column's values from that column's lane by shuffle.  The
      // values are those the staging below writes.
      const int nz4 = g.nz >> 2;
      if (cr < nvi) {   // uniform over the warp
        const size_t roff = ((size_t)(i0 + cr) * g.ny + j0) * g.nz;
        const int nf4 = nvj * nz4;
        for (int comp = c_first; comp <= c_last; ++comp) {
          const float vm = comp == 0 ? ex : comp == 1 ? ey : comp == 2 ? ezi : comp == 3 ? odx
                           : comp == 4 ? ody : comp == 5 ? ezx3 : ezy3;
          const float outv = comp < 3 ? g.eps_clad : 0.f;
          float *base = comp < 3 ? rg.eps + comp * cplane : rg.offdiag + (comp - 3) * cplane;
          if (!EPSC_IN_BOUNDS((comp < 3 ? comp : comp - 3) * cplane + roff, (size_t)nf4 * 4,
                              (comp < 3 ? 3 : (rg.normals3d ? 4 : 2)) * cplane, a.err))
            continue;
          float4 *dst = reinterpret_cast<float4 *>(base + roff);
          if ((32 % nz4) == 0) {
            // nz4 divides 32, so a lane keeps the same four planes k .. k+3
            // at every step: classify them once per component (the owning
            // column's value, its negation, the face value, or a constant)
            const int k = 4 * (cc % nz4);
            int kind[4];
            float cst[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
              const int kk = k + q;
              const bool slab = kk >= g.k0 + 1 && kk <= g.k0 + g.nk;
              cst[q] = 0.f;
              if (comp < 2) {
                kind[q] = slab ? 0 : 3;
                cst[q] = outv;
              } else if (comp == 2) {
                const bool inside = kk >= g.k0 + 1 && kk <= g.k0 + g.nk - 1;
                const bool face = kk == g.k0 || kk == g.k0 + g.nk;
                kind[q] = inside ? 0 : (face ? 2 : 3);
                cst[q] = outv;
              } else if (comp <= 4) {
                kind[q] = slab ? 0 : 3;
              } else {
                kind[q] = kk == g.k0 ? 0 : (kk == g.k0 + g.nk ? 1 : 3);
              }
            }
            const int jbase = cc / nz4;
            for (int f0 = 0; f0 < nf4; f0 += 32) {
              const int jj = min(f0 / nz4 + jbase, 31);
              const float v = __shfl_sync(0xffffffffu, vm, jj);
              const float vf = comp == 2 ? __shfl_sync(0xffffffffu, ezf3, jj) : 0.f;
              float t[4];
#pragma unroll
              for (int q = 0; q < 4; ++q)
                t[q] = kind[q] == 0 ? v : (kind[q] == 1 ? -v : (kind[q] == 2 ? vf : cst[q]));
              if (f0 + cc < nf4) __stcs(dst + f0 + cc, make_float4(t[0], t[1], t[2], t[3]));
            }
          } else {
            for (int f0 = 0; f0 < nf4; f0 += 32) {
              const int f = f0 + cc;
              const int jj = min(f / nz4, 31);
              const float v = __shfl_sync(0xffffffffu, vm, jj);
              const float vf = __shfl_sync(0xffffffffu, ezf3, jj);
              if (f < nf4) {
                const int k = 4 * (f - (f / nz4) * nz4);
                float t[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) t[q] = plane_value(comp, k + q, g.k0, g.nk, v, v, vf, outv);
                __stcs(dst + f, make_float4(t[0], t[1], t[2], t[3]));
              }
            }
          }
        }
      }
    } else if (eps_map && rg.eps_tma && g.nz == 32 && c_first == 0 && c_last == 2 &&
               per_round >= 1) {
      // Swizzled staging: each column's 32 planes are one 128-byte row of a
      // 1024-byte-aligned buffer, its 16-byte chunk k4 at chunk k4 ^ (row &
      // 7), the layout of the map's 128-byte swizzle.  The eight lanes of a
      // quarter-warp then store to eight different bank groups; in a plain
      // row-major buffer the 128-byte row pitch puts all 32 lanes' 16-byte
      // stores on the same four banks (eight times the shared-memory
      // wavefronts).  One tensor store per component writes the tile's
      // TI x TJ x nz box (clipped at the region edge).  Components rotate
      // through min(per_round, 3) buffers, one bulk group each.
      float *sbuf = smem;   // the stencil buffers are dead from here on; the
                            // launch leaves 1 KB of slack for the alignment
      sbuf += ((1024u - ((unsigned)__cvta_generic_to_shared(smem) & 1023u)) & 1023u) >> 2;
      const int nbuf = min(per_round, 3);
      const int sw = cc & 7;   // row = cr * TJ + cc, TJ a multiple of 8
      __syncthreads();
      for (int comp = 0; comp <= 2; ++comp) {
        float *buf = sbuf + (comp % nbuf) * comp_floats;
        if (comp >= nbuf) {   // the store that read this buffer must be done reading
          if (tid == 0) {
            if (nbuf == 1) bulk_wait_read_n<0>();
            else bulk_wait_read_n<1>();
          }
          __syncthreads();
        }
        if (cr < nvi && cc < nvj) {
          const float vin = comp == 0 ? ex : comp == 1 ? ey : ezi;
          const int zlen = comp == 2 ? g.nk - 1 : g.nk;   // planes k0+1 .. k0+zlen take vin
          const int lo = g.k0 + 1, hi = g.k0 + zlen;
          const int flo = comp == 2 ? g.k0 : lo, fhi = comp == 2 ? g.k0 + g.nk : hi;
          const int kf0 = comp == 2 ? g.k0 : -8, kf1 = comp == 2 ? g.k0 + g.nk : -8;
          float4 *row = reinterpret_cast<float4 *>(buf + (cr * TJ + cc) * 32);
#pragma unroll
          for (int k4 = 0; k4 < 8; ++k4)
            row[k4 ^ sw] = eps_planes4(k4, vin, ezf3, g.eps_clad, lo, hi, flo, fhi, kf0, kf1);
        }
        fence_proxy_async_smem();
        __syncthreads();
        if (tid == 0) {
          tma_store_4d(eps_map, buf, 0, j0, i0, comp);
          bulk_commit();
        }
      }
      bulk_pending = true;
    } else if ((g.nz & 3) == 0 && per_round >= 1) {
      float *sbuf = smem;   // the stencil buffers are dead from here on
      const int nz4 = g.nz >> 2;
      __syncthreads();
      for (int c0 = c_first; c0 <= c_last; c0 += per_round) {
        const int c1 = min(c_last, c0 + per_round - 1);
        if (c0 != c_first) {   // previous round's copies must have read the buffer
          if (tid == 0) bulk_wait_read();
          __syncthreads();
        }
        if (cr < nvi && cc < nvj) {
          for (int comp = c0; comp <= c1; ++comp) {
            if (comp > 4) {
              // eta_zx / eta_zy: the two face planes only
              const float v = comp == 5 ? ezx3 : ezy3;
              float4 *dz = reinterpret_cast<float4 *>(sbuf + (comp - c0) * comp_floats +
                                                      (cr * TJ + cc) * g.nz);
              const int f0 = g.k0, f1 = g.k0 + g.nk;
              for (int k4 = 0; k4 < nz4; ++k4) {
                const int k = 4 * k4;
                float t[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) t[q] = k + q == f0 ? v : (k + q == f1 ? -v : 0.f);
                dz[k4] = make_float4(t[0], t[1], t[2], t[3]);
              }
              continue;
            }
            const float vin = comp == 0 ? ex : comp == 1 ? ey : comp == 2 ? ezi : comp == 3 ? odx : ody;
            const float out = comp < 3 ? g.eps_clad : 0.f;
            const int zlen = comp == 2 ? g.nk - 1 : g.nk;   // planes k0+1 .. k0+zlen take vin
            const int kf0 = comp == 2 ? g.k0 : -8, kf1 = comp == 2 ? g.k0 + g.nk : -8;
            float4 *dst = reinterpret_cast<float4 *>(sbuf + (comp - c0) * comp_floats +
                                                     (cr * TJ + cc) * g.nz);
            // The plane pattern is the same for every column, so each group
            // of four planes is classified once (warp-uniform): all inside
            // the value run, all outside it, or mixed (per-plane selects).
            const int lo = g.k0 + 1, hi = g.k0 + zlen;       // value run [lo, hi]
            const int flo = comp == 2 ? g.k0 : lo, fhi = comp == 2 ? g.k0 + g.nk : hi;
            for (int k4 = 0; k4 < nz4; ++k4)
              dst[k4] = eps_planes4(k4, vin, ezf3, out, lo, hi, flo, fhi, kf0, kf1);
          }
        }
        fence_proxy_async_smem();
        __syncthreads();
        if (tid == 0) {
          for (int comp = c0; comp <= c1; ++comp) {
            float *base = comp < 3 ? rg.eps + comp * cplane : rg.offdiag + (comp - 3) * cplane;
            for (int r = 0; r < nvi; ++r) {
              const size_t off = ((size_t)(i0 + r) * g.ny + j0) * g.nz;
              if (EPSC_IN_BOUNDS((comp < 3 ? comp : comp - 3) * cplane + off, nvj * g.nz,
                                 (comp < 3 ? 3 : (rg.normals3d ? 4 : 2)) * cplane, a.err))
                bulk_store(base + off, sbuf + (comp - c0) * comp_floats + r * TJ * g.nz,
                           (unsigned)(nvj * g.nz * 4));
            }
          }
          bulk_commit();
        }
        bulk_pending = true;
      }
    } else if (valid) {
      // plane counts not a multiple of 4: thread per column
      for (int comp = c_first; comp <= c_last; ++comp) {
        float *base = comp < 3 ? rg.eps + comp * cplane : rg.offdiag + (comp - 3) * cplane;
        const float vm = comp == 0 ? ex : comp == 1 ? ey : comp == 3 ? odx : comp == 4 ? ody
                         : comp == 5 ? ezx3 : ezy3;
        const size_t off = ((size_t)ci * g.ny + cj) * g.nz;
        if (!EPSC_IN_BOUNDS((comp < 3 ? comp : comp - 3) * cplane + off, g.nz,
                            (comp < 3 ? 3 : (rg.normals3d ? 4 : 2)) * cplane, a.err))
          continue;
        float *dst = base + off;
        for (int k = 0; k < g.nz; ++k)
          dst[k] = plane_value(comp, k, g.k0, g.nk, vm, ezi, ezf3, g.eps_clad);
      }
    }
  }
  // Before the block may leave (or the next tile reuse shared memory) its
  // bulk stores must have read the staging area; their global writes
  // complete on their own and are visible once the grid has completed.
  if (rg.mode == MODE_FWD) {
    if (bulk_pending && tid == 0) bulk_wait_read();
    return;
  }

  // ---- 5. adjoint seeds ----------------------------------------------------
  // Every adjoint seed of a column is linear in that column's Eq. 1 sum of
  // its component: seed = W * factor (dJ/dA_z = W_zi itself).  In the
  // default form the tile waits here for the contraction grid and writes
  // the seeds; with defer_seeds it writes the W-independent factors and
  // leaves dJ/dA_z to the seeds kernel, so the stencil never waits (larger
  // problems: tiles do not hold their SM slot while the fields stream).
  float fAx = 0.f, fHx = 0.f, fgxx = 0.f, fgyx = 0.f;
  float fAy = 0.f, fHy = 0.f, fgxy = 0.f, fgyy = 0.f, fHz = 0.f;
  if (valid) {
    // eps = 1/(m H + (1-m)/A):  de/dH = -eps^2 m, de/dA = eps^2 (1-m)/A^2, de/dm = -eps^2 (H - 1/A)
    const float e2x = ex * ex, e2y = ey * ey;
    fAx = e2x * (1.f - mx_) * (iAx * iAx);
    fHx = -e2x * mx_;
    const float fmx = -e2x * (Hx - iAx);
    fAy = e2y * (1.f - my_) * (iAy * iAy);
    fHy = -e2y * my_;
    const float fmy = -e2y * (Hy - iAy);
    if (okx) {   // m = gx^2/|g|^2: dm/dgx = 2 gx gy^2/|g|^4, dm/dgy = -2 gx^2 gy/|g|^4
      const float t = 2.f * fmx * (ig2x * ig2x);
      fgxx = t * gxx * gyx * gyx;
      fgyx = -t * gxx * gxx * gyx;
    }
    if (oky) {   // m = gy^2/|g|^2: dm/dgx = -2 gx gy^2/|g|^4, dm/dgy = 2 gx^2 gy/|g|^4
      const float t = 2.f * fmy * (ig2y * ig2y);
      fgxy = -t * gxy * gyy * gyy;
      fgyy = t * gxy * gxy * gyy;
    }
    fHz = -0.5f * ezf * ezf;
  }
  float Wx = 1.f, Wy = 1.f, Wzi = 0.f, Wzf = 1.f;
  if (!rg.defer_seeds) griddep_wait();   // the contraction grid has completed
  double s_col = 0.0;                    // this column's eps . W (Eq. 1 surrogate)
  if (valid && EPSC_IN_BOUNDS((size_t)ci * g.ny + cj, 1, (size_t)g.nx * g.ny, a.err)) {
    const size_t plane = (size_t)g.nx * g.ny;
    if (!rg.defer_seeds) {
      const float *wc = rg.W + (size_t)ci * g.ny + cj;
      Wx = wc[0 * plane];
      Wy = wc[1 * plane];
      Wzi = wc[2 * plane];
      Wzf = wc[3 * plane];
      // eps_hat is constant along z on each support run: eps_xx, eps_yy on
      // planes k0+1 .. k0+nk, eps_zz = A_z inside, ezf on the two faces
      s_col = fmaf(ex, Wx, ey * Wy) + fmaf(ezi, Wzi, ezf * Wzf);
    } else if (rg.epsc) {
      float *ec = rg.epsc + (size_t)ci * g.ny + cj;
      ec[0 * plane] = ex;
      ec[1 * plane] = ey;
      ec[2 * plane] = ezi;
      ec[3 * plane] = ezf;
    }
    float *sd = rg.seeds + (size_t)ci * g.ny + cj;
    sd[S_DAX * plane] = fAx * Wx;
    sd[S_DHX * plane] = fHx * Wx;
    sd[S_GXX * plane] = fgxx * Wx;
    sd[S_GYX * plane] = fgyx * Wx;
    sd[S_DAY * plane] = fAy * Wy;
    sd[S_DHY * plane] = fHy * Wy;
    sd[S_GXY * plane] = fgxy * Wy;
    sd[S_GYY * plane] = fgyy * Wy;
    if (!rg.defer_seeds) sd[S_DAZ * plane] = Wzi;
    sd[S_DHZ * plane] = fHz * Wzf;
  }
  if (rg.S && !rg.defer_seeds) block_add_to(rg.S, s_col);   // uniform over the block
  if (bulk_pending && tid == 0) bulk_wait_read();
}

// Single-region stencil over a 1-D grid: block b takes tiles b,
// b + gridDim.x, ... of the row-major tile grid (one tile per block when the
// grid covers them all).
// (radius classes up to 8: at most 64 registers a thread, so four blocks fit
// on an SM when the eps_hat staging is one component per round; larger
// classes would spill at that bound and keep three)
template <int RP1, int BC>
__global__ void __launch_bounds__(NTHREADS, (RP1 <= 8 ? 4 : 3)) fwd_kernel(const __grid_constant__ FwdArgsR<RP1> a) {
  const Geometry &g = a.r.g;
  const int tiles_j = (g.ny + TJ - 1) / TJ;
  const int ntiles = tiles_j * ((g.nx + TI - 1) / TI);
  for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const int ti = t / tiles_j;
    fwd_tile<RP1, BC>(a, a.r, ti * TI, (t - ti * tiles_j) * TJ, &a.eps_map);
    __syncthreads();   // the next tile reuses shared memory (bulk stores have read it)
  }
}

template <int RP1, int BC>
__global__ void __launch_bounds__(NTHREADS, 3) fwd_batched_kernel(const __grid_constant__ FwdBatchArgs a) {
  int k, t;
  batch_tile(a, blockIdx.x, k, t);
  const int tj = a.tiles_j[k];
  const int ti = t / tj;
  fwd_tile<RP1, BC>(a, a.r[k], ti * TI, (t - ti * tj) * TJ);
}

}  // namespace epsc
