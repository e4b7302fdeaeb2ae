// Adjoint scatter: per-column seeds -> dJ/dC, one TA x TB tile of control
// subpixels per block.  Applies, in gather form, the transposes of the
// forward stages in reverse order:
//   Sobel^T (Yee level)  ->  dual-cell mean^T (Eq. 8)  ->  1/eps and mixing
//   ->  projection P'(u) (analytic, Eq. 6)  ->  K^T (Eq. 2).
// Edge replicate is a many-to-one index map; its transpose folds every
// contribution that landed outside the region back onto the edge element.
#pragma once

#include "epsc_common.cuh"

namespace epsc {

template <int RP1>
struct BwdSmem {
  static constexpr int R = RP1 - 1;
  static constexpr int GA_MAX = TA + 2 * R;                    // gather rows incl. fold halo
  static constexpr int GB_MAX = TB + 2 * R;
  static constexpr int NSTRIP_MAX = (GA_MAX + NA_B - 1) / NA_B;
  static constexpr int DA_ALLOC = NSTRIP_MAX * NA_B + 2 * R;   // du rows readable by strips
  static constexpr int DBP = TB + 4 * R;                       // du pitch
  static constexpr int NCI = (TA + 4 * R) / 2 + 3;             // cell rows covering du
  static constexpr int NCJ = (TB + 4 * R) / 2 + 3;
  static constexpr int OFF_DUX = 0;
  static constexpr int OFF_DUY = OFF_DUX + NCI * NCJ;
  static constexpr int OFF_DU = OFF_DUY + NCI * NCJ;
  static constexpr int OFF_DCE = OFF_DU + DA_ALLOC * DBP;
  static constexpr int TOTAL = OFF_DCE + GA_MAX * GB_MAX;
  static constexpr size_t BYTES = sizeof(float) * TOTAL;
};

// Transposed 3-tap Sobel factors along one axis: for target cell t, three
// source cells s with weights wd = sum_{d: bc(s+d)=t} D(d) and
// ws = sum_{d: bc(s+d)=t} S(d), D = (-1, 0, 1), S = (1, 2, 1).  Sources that
// do not exist (edge replicate at the region edge) get zero weights.
struct SobelT {
  int src[3];
  float wd[3], ws[3];
};

__device__ __forceinline__ SobelT sobel_t_axis(int t, int n, int bc) {
  SobelT r;
  if (bc == EPS_BC_PERIODIC) {
    // each (s, d) with wrap(s + d) = t is s = wrap(t - d): one term per d
#pragma unroll
    for (int d = -1; d <= 1; ++d) {
      r.src[d + 1] = wrapi(t - d, n);
      r.wd[d + 1] = (float)d;
      r.ws[d + 1] = d == 0 ? 2.f : 1.f;
    }
  } else {
#pragma unroll
    for (int e = 0; e < 3; ++e) {
      const int s = t - 1 + e;
      float wd = 0.f, ws = 0.f;
      if (s >= 0 && s < n) {
#pragma unroll
        for (int d = -1; d <= 1; ++d) {
          if (clampi(s + d, 0, n - 1) == t) {
            wd += (float)d;
            ws += d == 0 ? 2.f : 1.f;
          }
        }
      }
      r.src[e] = clampi(s, 0, n - 1);
      r.wd[e] = wd;
      r.ws[e] = ws;
    }
  }
  return r;
}

template <int RP1>
__global__ void __launch_bounds__(NTHREADS) bwd_kernel(const __grid_constant__ BwdArgs a) {
  using S = BwdSmem<RP1>;
  constexpr int R = S::R;
  constexpr int DBP = S::DBP;
  extern __shared__ float smem[];
  float *sdUx = smem + S::OFF_DUX;
  float *sdUy = smem + S::OFF_DUY;
  float *sdu = smem + S::OFF_DU;
  float *sdc = smem + S::OFF_DCE;

  const Geometry &g = a.g;
  const int tid = threadIdx.x;
  const bool clamp = g.bc == EPS_BC_CLAMP;
  const int a0 = blockIdx.y * TA, b0 = blockIdx.x * TB;
  const int aend = min(a0 + TA, g.mx), bend = min(b0 + TB, g.my);
  // gather region: the tile, plus R extended positions where edge replicate folds
  const int ga_lo = a0 - ((clamp && a0 == 0) ? R : 0);
  const int ga_hi = aend + ((clamp && aend == g.mx) ? R : 0);
  const int gb_lo = b0 - ((clamp && b0 == 0) ? R : 0);
  const int gb_hi = bend + ((clamp && bend == g.my) ? R : 0);
  const int GA = ga_hi - ga_lo, GB = gb_hi - gb_lo;
  // du region: gather region +- R (virtual subpixel coordinates)
  const int da_lo = ga_lo - R, db_lo = gb_lo - R;
  const int DA = GA + 2 * R, DB = GB + 2 * R;
  // cells touched by the du region: floor(a/2) .. floor((a+1)/2)
  const int ci_lo = da_lo >> 1, cj_lo = db_lo >> 1;
  const int NCI = ((da_lo + DA) >> 1) - ci_lo + 1;
  const int NCJ = ((db_lo + DB) >> 1) - cj_lo + 1;
  const size_t plane = (size_t)g.nx * g.ny;

  // ---- Sobel^T: dU_c at the touched cells -------------------------------
  for (int idx = tid; idx < NCI * NCJ; idx += NTHREADS) {
    const int r = idx / NCJ, c = idx - (idx / NCJ) * NCJ;
    int vi = ci_lo + r, vj = cj_lo + c;
    float ux = 0.f, uy = 0.f;
    bool real = true;
    if (clamp) {
      real = vi >= 0 && vi < g.nx && vj >= 0 && vj < g.ny;
    } else {
      vi = wrapi(vi, g.nx);
      vj = wrapi(vj, g.ny);
    }
    if (real) {
      const SobelT tx = sobel_t_axis(vi, g.nx, g.bc);
      const SobelT ty = sobel_t_axis(vj, g.ny, g.bc);
#pragma unroll
      for (int p = 0; p < 3; ++p) {
#pragma unroll
        for (int q = 0; q < 3; ++q) {
          const size_t o = (size_t)tx.src[p] * g.ny + ty.src[q];
          const float wdx_sy = tx.wd[p] * ty.ws[q];   // d g_x / d U
          const float wsx_dy = tx.ws[p] * ty.wd[q];   // d g_y / d U
          ux += wdx_sy * __ldg(a.seeds + S_GXX * plane + o) + wsx_dy * __ldg(a.seeds + S_GYX * plane + o);
          uy += wdx_sy * __ldg(a.seeds + S_GXY * plane + o) + wsx_dy * __ldg(a.seeds + S_GYY * plane + o);
        }
      }
    }
    sdUx[r * S::NCJ + c] = ux;
    sdUy[r * S::NCJ + c] = uy;
  }
  __syncthreads();

  // ---- du on the du region ---------------------------------------------
  const int NSTRIP = (GA + NA_B - 1) / NA_B;
  const int DA_USED = NSTRIP * NA_B + 2 * R;   // rows the strips read
  const float q4 = 0.25f;
  for (int idx = tid; idx < DA_USED * DB; idx += NTHREADS) {
    const int r = idx / DB, c = idx - (idx / DB) * DB;
    const int va = da_lo + r, vb = db_lo + c;
    float du = 0.f;
    const bool inside = va >= 0 && va < g.mx && vb >= 0 && vb < g.my;
    if (r < DA && (inside || !clamp)) {
      const int wa = clamp ? va : wrapi(va, g.mx);
      const int wb = clamp ? vb : wrapi(vb, g.my);
      const float u = __ldg(a.uws + (size_t)wa * g.my + wb);
      const float t = tanhf(g.beta * (u - g.eta));
      const float pprime = 0.5f * g.beta * (1.f - t * t);
      const float e = fmaf(fmaf(0.5f, t, 0.5f), g.deps, g.eps_clad);
      const float ie2 = 1.f / (e * e);
      // cells containing (va, vb): centred axis -> v >> 1, shifted axis -> (v+1) >> 1
      const int ia_c = va >> 1, jb_c = vb >> 1;
      const int ia_s = (va + 1) >> 1, jb_s = (vb + 1) >> 1;
      // multiplicities of the shifted axis (edge replicate maps subpixel -1 onto 0)
      float ma = 1.f, mb = 1.f;
      if (clamp) {
        ma = ia_s >= g.nx ? 0.f : (va == 0 ? 2.f : 1.f);
        mb = jb_s >= g.ny ? 0.f : (vb == 0 ? 2.f : 1.f);
      }
      float de = 0.f, dus = 0.f;
      // x: centred in a, shifted in b
      if (mb != 0.f) {
        const size_t o = (size_t)(clamp ? ia_c : wrapi(ia_c, g.nx)) * g.ny + (clamp ? jb_s : wrapi(jb_s, g.ny));
        de += mb * (__ldg(a.seeds + S_DAX * plane + o) - __ldg(a.seeds + S_DHX * plane + o) * ie2);
        dus += mb * sdUx[(ia_c - ci_lo) * S::NCJ + (jb_s - cj_lo)];
      }
      // y: shifted in a, centred in b
      if (ma != 0.f) {
        const size_t o = (size_t)(clamp ? ia_s : wrapi(ia_s, g.nx)) * g.ny + (clamp ? jb_c : wrapi(jb_c, g.ny));
        de += ma * (__ldg(a.seeds + S_DAY * plane + o) - __ldg(a.seeds + S_DHY * plane + o) * ie2);
        dus += ma * sdUy[(ia_s - ci_lo) * S::NCJ + (jb_c - cj_lo)];
      }
      // z: shifted in both
      if (ma != 0.f && mb != 0.f) {
        const size_t o = (size_t)(clamp ? ia_s : wrapi(ia_s, g.nx)) * g.ny + (clamp ? jb_s : wrapi(jb_s, g.ny));
        de += ma * mb * (__ldg(a.seeds + S_DAZ * plane + o) - __ldg(a.seeds + S_DHZ * plane + o) * ie2);
      }
      du = q4 * fmaf(pprime * g.deps, de, dus);
    }
    sdu[r * DBP + c] = du;
  }
  __syncthreads();

  // ---- K^T gather on the gather region ----------------------------------
  for (int item = tid; item < NSTRIP * GB; item += NTHREADS) {
    const int s = item / GB, col = item - (item / GB) * GB;
    const int r0 = s * NA_B;
    float hi[NA_B], lo[NA_B];
    strip_stencil<RP1, NA_B, false>(sdu + r0 * DBP + col, DBP, a, hi, lo);
#pragma unroll
    for (int k = 0; k < NA_B; ++k) {
      if (r0 + k < GA) sdc[(r0 + k) * S::GB_MAX + col] = hi[k];
    }
  }
  __syncthreads();

  // ---- fold extended positions onto the edge and write ------------------
  const int na = aend - a0, nb = bend - b0;
  for (int idx = tid; idx < na * nb; idx += NTHREADS) {
    const int r = idx / nb, c = idx - (idx / nb) * nb;
    const int ga = a0 + r, gb = b0 + c;
    int ra0 = ga - ga_lo, ra1 = ra0, rb0 = gb - gb_lo, rb1 = rb0;
    if (clamp) {
      if (ga == 0) ra0 = 0;
      if (ga == g.mx - 1) ra1 = GA - 1;
      if (gb == 0) rb0 = 0;
      if (gb == g.my - 1) rb1 = GB - 1;
    }
    float acc = 0.f;
    for (int x = ra0; x <= ra1; ++x)
      for (int y = rb0; y <= rb1; ++y) acc += sdc[x * S::GB_MAX + y];
    a.dJdC[(size_t)ga * g.my + gb] = acc;
  }
}

}  // namespace epsc
