// One optimiser iteration on the device (Sec. 4): Adam (Eq. 10-11) over
// the controls, fused with the unbinarity count of the design, then the
// beta_max control (Eq. 15) and the beta schedule (Eq. 14).
//
// The count reads the per-subpixel adjoint factor the VJP's stencil pass
// left in its workspace, P = (beta/2)(eps_core - eps_clad) rho (1 - rho),
// so the design is not recomputed: a subpixel is gray when
// P * pscale > gray_tol (1 - gray_tol), pscale = 1 / ((beta/2) deps).
//
// Each block adds its gray count to the state and takes a ticket; the last
// block to finish (no block waits for another) reads the total, applies
// Eq. 15 and Eq. 14, advances the iteration index and clears the
// accumulators for the next iteration.
#pragma once

#include "epsc_common.cuh"

namespace epsc {

struct OptArgs {
  long n4;                   // controls / 4
  float lr, b1, b2, omb1, omb2, adam_eps;
  float gray_p;              // gray_tol (1 - gray_tol)
  float pscale;              // 1 / ((beta/2) deps)
  float ln_b1, ln_b2;        // log(b1), log(b2) for the bias corrections
  float gamma, inv_u0_m1, beta_min, inv_n_iter, inv_e_m1;   // inv_u0_m1 = 1/u0 - 1
  long n;                    // controls
  float4 *C;
  const float4 *G;
  float4 *M, *V;
  const float4 *P;           // the VJP's per-subpixel factor
  eps_opt_state_t *state;
};

__device__ __forceinline__ void adam_elem(float &c, float g, float &m, float &v, float bc1,
                                          float bc2, const OptArgs &a) {
  m = fmaf(a.b1, m, a.omb1 * g);
  v = fmaf(a.b2, v, a.omb2 * (g * g));
  const float mh = m * bc1, vh = v * bc2;
  c -= a.lr * mh / (sqrtf(vh) + a.adam_eps);
}

__global__ void __launch_bounds__(NTHREADS) opt_step_kernel(const __grid_constant__ OptArgs a) {
  __shared__ unsigned s_gray[NTHREADS / 32];
  __shared__ bool s_last;
  // iteration i = completed + 1; the state was last written by the previous
  // launch's final block, which completed before this grid started
  const int i = a.state->step + 1;
  // 1 / (1 - b^i) with 1 - b^i = -expm1(i log b): no cancellation at small i
  // (FP32 here: this GPU's FP64 rate is far below its FP32 rate)
  const float bc1 = -1.f / expm1f((float)i * a.ln_b1);
  const float bc2 = -1.f / expm1f((float)i * a.ln_b2);

  unsigned gray = 0;
  for (long k = (long)blockIdx.x * NTHREADS + threadIdx.x; k < a.n4; k += (long)gridDim.x * NTHREADS) {
    float4 c = a.C[k], m = a.M[k], v = a.V[k];
    const float4 g = __ldg(a.G + k), p = __ldg(a.P + k);
    adam_elem(c.x, g.x, m.x, v.x, bc1, bc2, a);
    adam_elem(c.y, g.y, m.y, v.y, bc1, bc2, a);
    adam_elem(c.z, g.z, m.z, v.z, bc1, bc2, a);
    adam_elem(c.w, g.w, m.w, v.w, bc1, bc2, a);
    a.C[k] = c;
    a.M[k] = m;
    a.V[k] = v;
    gray += (p.x * a.pscale > a.gray_p) + (p.y * a.pscale > a.gray_p) +
            (p.z * a.pscale > a.gray_p) + (p.w * a.pscale > a.gray_p);
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) gray += __shfl_xor_sync(0xffffffffu, gray, off);
  if ((threadIdx.x & 31) == 0) s_gray[threadIdx.x >> 5] = gray;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned tot = 0;
    for (int w = 0; w < NTHREADS / 32; ++w) tot += s_gray[w];
    atomicAdd(&a.state->gray_acc, tot);
    __threadfence();
    s_last = atomicAdd(&a.state->ticket, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!s_last || threadIdx.x != 0) return;

  // ---- final block: Eq. 15, then Eq. 14 for the next iteration ----------
  // FP32 in forms without cancellation: (1/u - 1)/beta = (n - g)/(g beta)
  // with the integer n - g exact, and exp(x^2) - 1 = expm1(x^2)
  __threadfence();
  volatile eps_opt_state_t *st = a.state;
  const unsigned total = atomicAdd(&a.state->gray_acc, 0u);
  const unsigned g = total > 0u ? total : 1u;   // floor: one subpixel
  const float beta = st->beta;
  const float sample = (float)(a.n - (long)g) / ((float)g * beta);
  float t = st->t;
  t = t <= 0.f ? sample : fmaf(a.gamma, t, (1.f - a.gamma) * sample);
  const float beta_max = fmaf(a.gamma, st->beta_max, (1.f - a.gamma) * a.inv_u0_m1 / t);
  const float x = (float)(i + 1) * a.inv_n_iter;
  const float beta_next = fmaf(beta_max - a.beta_min, expm1f(x * x) * a.inv_e_m1, a.beta_min);
  st->t = t;
  st->beta_max = beta_max;
  st->beta = beta_next;
  st->unbinarity = (float)((double)g / (double)a.n);
  st->gray = total;
  st->gray_acc = 0u;
  st->ticket = 0u;
  st->step = i;
  __threadfence();
}

// Initial state: no iteration done, beta of iteration 1 from Eq. 14.
__global__ void opt_init_kernel(eps_opt_state_t *state, float beta1, float beta_max0) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  state->step = 0;
  state->beta = beta1;
  state->beta_max = beta_max0;
  state->t = 0.f;
  state->unbinarity = 0.f;
  state->gray = 0u;
  state->gray_acc = 0u;
  state->ticket = 0u;
}

}  // namespace epsc
