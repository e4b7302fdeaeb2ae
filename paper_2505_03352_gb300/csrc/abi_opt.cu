// C ABI of the on-device optimiser iteration (Sec. 4, Eq. 10-15).
#include <algorithm>
#include <cmath>
#include <cstring>

#include "epschain.h"
#include "epsc_host.h"
#include "epsc_opt.cuh"

using namespace epsc;

namespace {

bool aligned(const void *p, size_t a) { return ((uintptr_t)p % a) == 0; }

eps_status_t check_opt(const eps_opt_t *o) {
  if (!o) return EPS_ERR_INVALID_ARG;
  const float f[] = {o->lr, o->b1, o->b2, o->adam_eps, o->gray_tol, o->gamma, o->u0, o->beta_min,
                     o->beta_max0};
  for (float v : f)
    if (!std::isfinite(v)) return EPS_ERR_INVALID_ARG;
  if (!(o->lr > 0.f) || o->b1 < 0.f || !(o->b1 < 1.f) || o->b2 < 0.f || !(o->b2 < 1.f) ||
      o->adam_eps < 0.f)
    return EPS_ERR_INVALID_ARG;
  if (!(o->gray_tol > 0.f) || !(o->gray_tol < 0.5f) || o->gamma < 0.f || !(o->gamma < 1.f) ||
      !(o->u0 > 0.f) || !(o->u0 < 1.f))
    return EPS_ERR_INVALID_ARG;
  if (!(o->beta_min > 0.f) || o->beta_max0 < o->beta_min || o->n_iter < 1) return EPS_ERR_INVALID_ARG;
  return EPS_OK;
}

// Eq. 14 at iteration i
double schedule(int i, const eps_opt_t *o, double beta_max) {
  const double x = (double)i / o->n_iter;
  return o->beta_min + (beta_max - o->beta_min) * (std::exp(x * x) - 1.0) / (std::exp(1.0) - 1.0);
}

}  // namespace

extern "C" {

eps_status_t eps_opt_init(const eps_opt_t *opt, eps_opt_state_t *state, eps_stream_t stream) {
  eps_status_t st = check_opt(opt);
  if (st != EPS_OK) return st;
  if (!state || !aligned(state, 4)) return EPS_ERR_INVALID_ARG;
  const float beta1 = (float)schedule(1, opt, opt->beta_max0);
  opt_init_kernel<<<1, 32, 0, (cudaStream_t)stream>>>(state, beta1, opt->beta_max0);
  if (cudaGetLastError() != cudaSuccess) return EPS_ERR_CUDA;
  epsc_host::note_launch();
  return EPS_OK;
}

eps_status_t eps_opt_step(const eps_problem_t *prob, const eps_morph_t *morph, const eps_opt_t *opt,
                          eps_opt_state_t *state, float *C, const float *G, float *M, float *V,
                          const void *ws, size_t ws_bytes, eps_stream_t stream) {
  eps_status_t st = check_opt(opt);
  if (st != EPS_OK) return st;
  if (!prob) return EPS_ERR_INVALID_ARG;
  // where the VJP's stencil pass left the per-subpixel factor
  size_t base = 0, need = 0, off = 0, base_need = 0;
  if (morph) {
    if ((st = epsc_host::morph_base_offset(prob, morph, &base, &need)) != EPS_OK) return st;
    eps_problem_t yee = *prob;   // the morphology path's base chain: identity filter, eta = 1/2
    yee.radius = 1.0f;
    yee.eta = 0.5f;
    if ((st = epsc_host::subpixel_factor_offset(&yee, &off, &base_need)) != EPS_OK) return st;
  } else {
    if ((st = epsc_host::subpixel_factor_offset(prob, &off, &need)) != EPS_OK) return st;
  }
  if (!(prob->beta > 0.f) || prob->eps_core == prob->eps_clad) return EPS_ERR_INVALID_ARG;
  const long n = (long)prob->mx * prob->my;
  if (n == 0) return EPS_OK;
  if (!state || !aligned(state, 4)) return EPS_ERR_INVALID_ARG;
  if (!C || !G || !M || !V) return EPS_ERR_INVALID_ARG;
  if (!aligned(C, 16) || !aligned(G, 16) || !aligned(M, 16) || !aligned(V, 16))
    return EPS_ERR_INVALID_ARG;
  if (!ws || !aligned(ws, 256) || ws_bytes < need) return EPS_ERR_WORKSPACE;
  int nsm = 0;
  if ((st = epsc_host::sm_count_current(&nsm)) != EPS_OK) return st;

  OptArgs a;
  std::memset(&a, 0, sizeof(a));
  a.n = n;
  a.n4 = n / 4;   // mx, my even: n is a multiple of 4
  a.lr = opt->lr;
  a.b1 = opt->b1;
  a.b2 = opt->b2;
  a.omb1 = (float)(1.0 - (double)opt->b1);
  a.omb2 = (float)(1.0 - (double)opt->b2);
  a.adam_eps = opt->adam_eps;
  a.gray_p = (float)((double)opt->gray_tol * (1.0 - (double)opt->gray_tol));
  a.pscale = (float)(1.0 / (0.5 * (double)prob->beta * ((double)prob->eps_core - prob->eps_clad)));
  a.ln_b1 = (float)std::log((double)opt->b1);
  a.ln_b2 = (float)std::log((double)opt->b2);
  a.gamma = opt->gamma;
  a.inv_u0_m1 = (float)(1.0 / (double)opt->u0 - 1.0);
  a.beta_min = opt->beta_min;
  a.inv_n_iter = (float)(1.0 / (double)opt->n_iter);
  a.inv_e_m1 = (float)(1.0 / (std::exp(1.0) - 1.0));
  a.C = reinterpret_cast<float4 *>(C);
  a.G = reinterpret_cast<const float4 *>(G);
  a.M = reinterpret_cast<float4 *>(M);
  a.V = reinterpret_cast<float4 *>(V);
  a.P = reinterpret_cast<const float4 *>((const char *)ws + base + off);
  a.state = state;
  const long blocks = std::max<long>(1, std::min<long>((a.n4 + NTHREADS - 1) / NTHREADS, (long)nsm * 4));
  return epsc_host::launch_kernel("eps_opt_step", (const void *)&opt_step_kernel,
                                  dim3((unsigned)blocks), 0, &a, (cudaStream_t)stream, false);
}

}  // extern "C"
