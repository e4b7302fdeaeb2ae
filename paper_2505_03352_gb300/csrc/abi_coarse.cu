// C ABI of the chain with coarse control variables (Eq. 2 on a node grid).
//
// Phi = basis expansion of the node values (one kernel), then the base chain
// on Phi with an identity filter (Eq. 3/6 onwards: projection at prob->eta,
// mixing, dual-cell means, Sobel normals from Phi, Eq. 7), and for the
// adjoint the transpose of the expansion on the base chain's d/dPhi.
#include <algorithm>
#include <cstring>

#include "epschain.h"
#include "epsc_coarse.cuh"
#include "epsc_host.h"

using namespace epsc;

namespace {

inline size_t align256(size_t b) { return (b + 255) & ~size_t(255); }
bool aligned(const void *p, size_t a) { return ((uintptr_t)p % a) == 0; }

struct CoarsePlan {
  eps_problem_t yee;
  size_t map_bytes, yee_off, yee_bytes, total;
  bool empty;
};

// Workspace: Phi [mx][my] | d/dPhi [mx][my] | base chain
eps_status_t plan(const eps_problem_t *prob, const eps_coarse_t *cg, CoarsePlan *P) {
  if (!prob || !cg || !P) return EPS_ERR_INVALID_ARG;
  std::memset(P, 0, sizeof(*P));
  P->yee = *prob;
  P->yee.radius = 1.0f;   // the basis replaces the conic filter
  size_t yb = 0;
  eps_status_t st = eps_workspace_size(&P->yee, 0, &yb);
  if (st != EPS_OK) return st;
  if (cg->ncx < 2 || cg->ncy < 2 || cg->ncx > (1 << 20) || cg->ncy > (1 << 20)) return EPS_ERR_SHAPE;
  P->empty = prob->mx == 0 || prob->my == 0;
  P->map_bytes = align256(sizeof(float) * (size_t)prob->mx * prob->my);
  P->yee_off = 2 * P->map_bytes;
  P->yee_bytes = yb;
  P->total = P->empty ? 0 : P->yee_off + yb;
  return EPS_OK;
}

CoarseArgs args_of(const eps_problem_t *prob, const eps_coarse_t *cg) {
  CoarseArgs a;
  std::memset(&a, 0, sizeof(a));
  a.mx = prob->mx;
  a.my = prob->my;
  a.ncx = cg->ncx;
  a.ncy = cg->ncy;
  return a;
}

eps_status_t run_expand(const eps_problem_t *prob, const eps_coarse_t *cg, const float *c, float *phi,
                        cudaStream_t s) {
  int nsm = 0;
  eps_status_t st = epsc_host::sm_count_current(&nsm);
  if (st != EPS_OK) return st;
  CoarseArgs a = args_of(prob, cg);
  a.c = c;
  a.phi = phi;
  if ((st = epsc_host::error_flag(&a.err)) != EPS_OK) return st;
  const long n = (long)prob->mx * prob->my;
  const long blocks = std::max<long>(1, std::min<long>((n + NTHREADS - 1) / NTHREADS, (long)nsm * 8));
  return epsc_host::launch_kernel("eps_coarse_expand", (const void *)&coarse_expand_kernel,
                                  dim3((unsigned)blocks), 0, &a, s, true);
}

eps_status_t run_transpose(const eps_problem_t *prob, const eps_coarse_t *cg, const float *g,
                           float *dc, cudaStream_t s) {
  CoarseArgs a = args_of(prob, cg);
  a.g = g;
  a.dc = dc;
  eps_status_t st = epsc_host::error_flag(&a.err);
  if (st != EPS_OK) return st;
  const long blocks = (long)cg->ncx * cg->ncy;   // one block per node
  if (blocks > 0x7fffffffL) return EPS_ERR_SHAPE;
  return epsc_host::launch_kernel("eps_coarse_transpose", (const void *)&coarse_transpose_kernel,
                                  dim3((unsigned)blocks), 0, &a, s, true);
}

}  // namespace

extern "C" {

eps_status_t eps_coarse_workspace_size(const eps_problem_t *prob, const eps_coarse_t *coarse,
                                       int32_t n_lambda, size_t *bytes) {
  if (!bytes) return EPS_ERR_INVALID_ARG;
  if (n_lambda < 0 || n_lambda > EPS_MAX_LAMBDA) return EPS_ERR_INVALID_ARG;
  CoarsePlan P;
  const eps_status_t st = plan(prob, coarse, &P);
  if (st != EPS_OK) return st;
  *bytes = P.total;
  return EPS_OK;
}

eps_status_t eps_forward_coarse(const eps_problem_t *prob, const eps_coarse_t *coarse,
                                const float *c, float *eps, float *offdiag, void *ws,
                                size_t ws_bytes, eps_stream_t stream) {
  CoarsePlan P;
  eps_status_t st = plan(prob, coarse, &P);
  if (st != EPS_OK) return st;
  if (P.empty) return EPS_OK;
  const bool od = (prob->flags & EPS_FLAG_OFFDIAG) != 0;
  if (!c || !eps || (od && !offdiag)) return EPS_ERR_INVALID_ARG;
  if (!aligned(c, 4) || !aligned(eps, 16) || (od && !aligned(offdiag, 16))) return EPS_ERR_INVALID_ARG;
  if (!ws || !aligned(ws, 256) || ws_bytes < P.total) return EPS_ERR_WORKSPACE;
  float *phi = (float *)ws;
  if ((st = run_expand(prob, coarse, c, phi, (cudaStream_t)stream)) != EPS_OK) return st;
  return eps_forward(&P.yee, phi, eps, offdiag, stream);
}

eps_status_t eps_vjp_coarse(const eps_problem_t *prob, const eps_coarse_t *coarse, const float *c,
                            int32_t n_lambda, int32_t field_type, const void *const *EF,
                            const void *const *EA, const float *field_scales, float scale,
                            float *dJdc, float *eps_out, void *ws, size_t ws_bytes,
                            eps_stream_t stream) {
  CoarsePlan P;
  eps_status_t st = plan(prob, coarse, &P);
  if (st != EPS_OK) return st;
  const void *yee_ws = ws ? (const char *)ws + P.yee_off : nullptr;
  const size_t yee_room = ws_bytes > P.yee_off ? ws_bytes - P.yee_off : 0;
  if ((st = epsc_host::check_vjp_args(prob, c, n_lambda, field_type, EF, EA, field_scales, scale,
                                      dJdc, eps_out, yee_ws, yee_room)) != EPS_OK)
    return st;
  if (P.empty) return EPS_OK;
  if (!ws || !aligned(ws, 256) || ws_bytes < P.total) return EPS_ERR_WORKSPACE;
  float *phi = (float *)ws;
  float *gphi = (float *)((char *)ws + P.map_bytes);
  cudaStream_t s = (cudaStream_t)stream;
  if ((st = run_expand(prob, coarse, c, phi, s)) != EPS_OK) return st;
  st = eps_vjp(&P.yee, phi, n_lambda, field_type, EF, EA, field_scales, scale, gphi, eps_out,
               (char *)ws + P.yee_off, P.yee_bytes, stream);
  if (st != EPS_OK) return st;
  return run_transpose(prob, coarse, gphi, dJdc, s);
}

eps_status_t eps_vjp_real_coarse(const eps_problem_t *prob, const eps_coarse_t *coarse,
                                 const float *c, const float *G, float *dJdc, void *ws,
                                 size_t ws_bytes, eps_stream_t stream) {
  CoarsePlan P;
  eps_status_t st = plan(prob, coarse, &P);
  if (st != EPS_OK) return st;
  if (prob->flags & EPS_FLAG_NORMALS_3D) return EPS_ERR_UNSUPPORTED;   // forward only
  if (P.empty) return EPS_OK;
  if (!c || !G || !dJdc) return EPS_ERR_INVALID_ARG;
  if (!aligned(c, 4) || !aligned(G, 4) || !aligned(dJdc, 4)) return EPS_ERR_INVALID_ARG;
  if (!ws || !aligned(ws, 256) || ws_bytes < P.total) return EPS_ERR_WORKSPACE;
  float *phi = (float *)ws;
  float *gphi = (float *)((char *)ws + P.map_bytes);
  cudaStream_t s = (cudaStream_t)stream;
  if ((st = run_expand(prob, coarse, c, phi, s)) != EPS_OK) return st;
  if ((st = eps_vjp_real(&P.yee, phi, G, gphi, (char *)ws + P.yee_off, P.yee_bytes, stream)) != EPS_OK)
    return st;
  return run_transpose(prob, coarse, gphi, dJdc, s);
}

}  // extern "C"
