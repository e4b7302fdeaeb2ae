// Subpixel-map kernels of the chain with morphological filtering (Eq. 2-5)
// and of its adjoint.  One templated kernel, four kinds:
//
//   MAP_FRONT    u = K * C (conic, Eq. 2);  rho_0 = (1 + tanh(beta (u - eta))) / 2
//                (Eq. 3) and its derivative P'(u) = 2 beta rho_0 (1 - rho_0)
//   MAP_LSE      one soft dilate (Eq. 4) or erode (Eq. 5) with the normalised
//                disk K_m:  s = rho (dilate) or 1 - rho (erode),
//                S = sum_d w_d exp(alpha (s[x+d] - 1)),  s_out = 1 + log(S) / alpha
//   MAP_LSE_T    adjoint of one MAP_LSE:  with T[x] = g_out[x] exp(alpha (1 - s_out[x])),
//                g_in[y] = exp(alpha (s_in[y] - 1)) sum_{(x,d): bc(x+d) = y} w_d T[x]
//                (the softmax weights of the disk, both factors bounded by e^alpha)
//   MAP_FRONT_T  dJ/dC[y] = sum_{(x,d): bc(x+d) = y} w_d (g_0[x] P'(u)[x])
//
// Each block computes one 32 x 32 tile of outputs.  The forward kinds stage
// the tile's input with a halo of R (boundary rule applied on load) and run
// the register-blocked strip stencil; the transposes under edge replicate
// gather over the tile extended by R past the domain edge (inputs outside
// the domain are zero) and fold the extension back onto the edge elements,
// under wrap they gather with wrapped indices.  All weights are symmetric
// under d -> -d, so the gather form uses the forward weight table.
#pragma once

#include "epsc_common.cuh"

namespace epsc {

constexpr int MT_A = 32, MT_B = 32;   // output tile (subpixels)
constexpr int NA_M = 4;               // outputs per strip

enum MapKind { MAP_FRONT = 0, MAP_LSE = 1, MAP_LSE_T = 2, MAP_FRONT_T = 3 };

// The weights come last: each kernel takes the struct with its own (2 RP1 -
// 1)^2 box, the host fills the full-size one (a common prefix).
template <int NW>
struct MapArgsN {
  int mx, my;
  float beta, eta;      // FRONT: first projection (Eq. 3)
  float alpha;          // LSE, LSE_T
  int erode;            // LSE, LSE_T: 0 dilate, 1 erode
  const float *in;      // FRONT: C; LSE: rho_k; LSE_T: g_{k+1}; FRONT_T: g_0
  const float *aux;     // LSE_T: rho_{k+1}; FRONT_T: P'(u)
  const float *aux2;    // LSE_T: rho_k
  float *out;           // FRONT: rho_0; LSE: rho_{k+1}; LSE_T: g_k; FRONT_T: dJ/dC
  float *out2;          // FRONT: P'(u)
  int *err;             // error flag (debug bounds checks)
  float w[NW];
};
using MapArgs = MapArgsN<MAX_BOX * MAX_BOX>;

template <int RP1>
struct MapSmem {
  static constexpr int R = RP1 - 1;
  static constexpr int GA_MAX = MT_A + 2 * R;                     // gather rows incl. fold extension
  static constexpr int GB_MAX = MT_B + 2 * R;
  static constexpr int NSTRIP_MAX = (GA_MAX + NA_M - 1) / NA_M;
  static constexpr int SA = NSTRIP_MAX * NA_M + 2 * R;            // staged rows the strips can read
  static constexpr int SP = GB_MAX + 2 * R;                       // staged pitch
  static constexpr int OFF_IN = 0;
  static constexpr int OFF_H = OFF_IN + SA * SP;                  // gather results (fold only)
  static constexpr int TOTAL = OFF_H + GA_MAX * GB_MAX;
  static constexpr size_t BYTES = sizeof(float) * TOTAL;
};

__device__ __forceinline__ float lse_s(float rho, int erode) { return erode ? 1.f - rho : rho; }

template <int RP1, int BC, int KIND>
__global__ void __launch_bounds__(NTHREADS) map_kernel(
    const __grid_constant__ MapArgsN<(2 * RP1 - 1) * (2 * RP1 - 1)> a) {
  using S = MapSmem<RP1>;
  constexpr int R = S::R;
  constexpr bool TRANS = KIND == MAP_LSE_T || KIND == MAP_FRONT_T;
  constexpr bool FOLD = TRANS && BC == EPS_BC_CLAMP;
  extern __shared__ __align__(16) float smem[];
  float *sIn = smem + S::OFF_IN;
  float *sH = smem + S::OFF_H;
  const int tid = threadIdx.x;

  const int a0 = blockIdx.y * MT_A, b0 = blockIdx.x * MT_B;
  const int aend = min(a0 + MT_A, a.mx), bend = min(b0 + MT_B, a.my);
  // gather region: the tile, extended past the domain edge under fold
  const int ga_lo = (FOLD && a0 == 0) ? -R : a0;
  const int ga_hi = (FOLD && aend == a.mx) ? a.mx + R : aend;
  const int gb_lo = (FOLD && b0 == 0) ? -R : b0;
  const int gb_hi = (FOLD && bend == a.my) ? a.my + R : bend;
  const int GA = ga_hi - ga_lo, GB = gb_hi - gb_lo;
  const int NSTRIP = (GA + NA_M - 1) / NA_M;
  const int SA_USED = NSTRIP * NA_M + 2 * R;
  const int SB_USED = GB + 2 * R;

  // Launched behind the previous kernel of the chain (programmatic dependent
  // launch): let the next one start launching, then wait for the previous
  // grid's results before the first global read or write.
  griddep_launch_dependents();
  griddep_wait();

  // ---- stage the (transformed) input with its halo ----------------------
#pragma unroll 4
  for (int idx = tid; idx < SA_USED * SB_USED; idx += NTHREADS) {
    const int r = idx / SB_USED, c = idx - r * SB_USED;
    int x = ga_lo - R + r, y = gb_lo - R + c;
    float v = 0.f;
    if (r < GA + 2 * R) {
      bool inside = true;
      if (TRANS && BC == EPS_BC_CLAMP) {
        inside = x >= 0 && x < a.mx && y >= 0 && y < a.my;
      } else {
        x = bc_map(x, a.mx, BC);
        y = bc_map(y, a.my, BC);
      }
      if (inside && EPSC_IN_BOUNDS((size_t)x * a.my + y, 1, (size_t)a.mx * a.my, a.err)) {
        const size_t o = (size_t)x * a.my + y;
        if (KIND == MAP_FRONT) {
          v = __ldg(a.in + o);
        } else if (KIND == MAP_LSE) {
          v = expf(a.alpha * (lse_s(__ldg(a.in + o), a.erode) - 1.f));
        } else if (KIND == MAP_LSE_T) {
          v = __ldg(a.in + o) * expf(a.alpha * (1.f - lse_s(__ldg(a.aux + o), a.erode)));
        } else {
          v = __ldg(a.in + o) * __ldg(a.aux + o);
        }
      }
    }
    sIn[r * S::SP + c] = v;
  }
  __syncthreads();

  // ---- strips: H = sum_d w_d in[x + d] on the gather region ---------------
  for (int item = tid; item < NSTRIP * GB; item += NTHREADS) {
    const int st = item / GB, col = item - st * GB;
    const int r0 = st * NA_M;
    float hi[NA_M];
    strip_stencil<RP1, NA_M>(sIn + r0 * S::SP + col, S::SP, a, hi);
#pragma unroll
    for (int k = 0; k < NA_M; ++k) {
      const int r = r0 + k;
      if (r >= GA) break;
      if (FOLD) {
        sH[r * S::GB_MAX + col] = hi[k];
        continue;
      }
      const size_t o = (size_t)(ga_lo + r) * a.my + (gb_lo + col);
      if (!EPSC_IN_BOUNDS(o, 1, (size_t)a.mx * a.my, a.err)) continue;
      if (KIND == MAP_FRONT) {
        // with x = beta (u - eta) and t = exp(-2|x|) <= 1 (no overflow at any
        // beta): rho_0 = 1/(1+t) for x >= 0, t/(1+t) below, and
        // P'(u) = (beta/2)(1 - tanh^2 x) = 2 beta t / (1+t)^2.  The accurate
        // exp keeps rho_0 to a few ulp: the final projection amplifies its error.
        const float x = a.beta * (hi[k] - a.eta);
        const float t = expf(-2.f * fabsf(x));
        const float inv = 1.f / (1.f + t);
        a.out[o] = x >= 0.f ? inv : t * inv;
        a.out2[o] = 2.f * a.beta * (t * inv * inv);
      } else if (KIND == MAP_LSE) {
        const float s_out = 1.f + logf(hi[k]) / a.alpha;
        a.out[o] = a.erode ? 1.f - s_out : s_out;
      } else if (KIND == MAP_LSE_T) {
        a.out[o] = expf(a.alpha * (lse_s(__ldg(a.aux2 + o), a.erode) - 1.f)) * hi[k];
      } else {
        a.out[o] = hi[k];
      }
    }
  }
  if (!FOLD) return;
  __syncthreads();

  // ---- fold the extension onto the edge elements and write ---------------
  for (int idx = tid; idx < (aend - a0) * (bend - b0); idx += NTHREADS) {
    const int r = idx / (bend - b0), c = idx - r * (bend - b0);
    const int x = a0 + r, y = b0 + c;
    int ra0 = x - ga_lo, ra1 = ra0, rb0 = y - gb_lo, rb1 = rb0;
    if (x == 0) ra0 = 0;
    if (x == a.mx - 1) ra1 = GA - 1;
    if (y == 0) rb0 = 0;
    if (y == a.my - 1) rb1 = GB - 1;
    float acc = 0.f;
    for (int i = ra0; i <= ra1; ++i)
      for (int j = rb0; j <= rb1; ++j) acc += sH[i * S::GB_MAX + j];
    const size_t o = (size_t)x * a.my + y;
    if (!EPSC_IN_BOUNDS(o, 1, (size_t)a.mx * a.my, a.err)) continue;
    if (KIND == MAP_LSE_T) acc *= expf(a.alpha * (lse_s(__ldg(a.aux2 + o), a.erode) - 1.f));
    a.out[o] = acc;
  }
}

}  // namespace epsc
