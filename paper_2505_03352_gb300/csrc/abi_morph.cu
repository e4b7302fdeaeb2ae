// C ABI of the chain with morphological filtering (Sec. 3, Eq. 3-6).
//
// The front of the chain runs on subpixel maps kept in the workspace:
//   FRONT       C -> rho_0 (Eq. 2 + Eq. 3) and P'(u)
//   LSE x n     rho_k -> rho_{k+1} (Eq. 4 / Eq. 5)
// then the base chain runs on rho_n with an identity filter and eta = 1/2
// (Eq. 6 onwards: mixing, dual-cell means, normals from rho_n, Eq. 7).  The
// adjoint takes the base chain's d/d rho_n and runs LSE_T x n and FRONT_T
// back to dJ/dC.  Every argument is checked before the first launch.
#include <cmath>
#include <cstring>

#include "epschain.h"
#include "epsc_host.h"
#include "epsc_launch.h"
#include "epsc_morph.cuh"

using namespace epsc;

namespace {

inline size_t align256(size_t b) { return (b + 255) & ~size_t(255); }
bool aligned(const void *p, size_t a) { return ((uintptr_t)p % a) == 0; }

struct MorphPlan {
  eps_problem_t yee;                   // base chain on rho_n
  int rp1_cone, rp1_disk;
  float w_cone[MAX_BOX * MAX_BOX];
  float w_disk[MAX_BOX * MAX_BOX];
  size_t map_bytes;                    // one subpixel map, 256-byte aligned
  size_t yee_off, yee_bytes, total;    // base-chain workspace after the maps
  bool empty;
};

// Workspace: rho_0 .. rho_n | P'(u) | adjoint map a | adjoint map b | base chain
eps_status_t plan(const eps_problem_t *prob, const eps_morph_t *m, MorphPlan *P) {
  if (!prob || !m || !P) return EPS_ERR_INVALID_ARG;
  std::memset(P, 0, sizeof(*P));
  eps_status_t st = epsc_host::conic_filter(prob, P->w_cone, &P->rp1_cone);
  if (st != EPS_OK) return st;
  if (!std::isfinite(m->alpha) || !(m->alpha > 0.f) || m->alpha > EPS_MORPH_MAX_ALPHA)
    return EPS_ERR_INVALID_ARG;
  if (!std::isfinite(m->radius) || m->radius < 0.f) return EPS_ERR_INVALID_ARG;
  if (m->radius >= EPS_MAX_RADIUS) return EPS_ERR_UNSUPPORTED;
  if (m->n_ops < 0 || m->n_ops > EPS_MORPH_MAX_OPS) return EPS_ERR_INVALID_ARG;
  for (int k = 0; k < m->n_ops; ++k)
    if (m->ops[k] != EPS_MORPH_DILATE && m->ops[k] != EPS_MORPH_ERODE) return EPS_ERR_INVALID_ARG;

  // normalised disk: integer offsets with p^2 + q^2 <= radius^2, weight 1/count
  const double r = m->radius;
  const int h = (int)std::floor(r);
  P->rp1_disk = h + 1;
  const int bw = 2 * h + 1;
  int count = 0;
  for (int p = -h; p <= h; ++p)
    for (int q = -h; q <= h; ++q)
      if ((double)(p * p + q * q) <= r * r) ++count;
  for (int p = -h; p <= h; ++p)
    for (int q = -h; q <= h; ++q)
      if ((double)(p * p + q * q) <= r * r) P->w_disk[(p + h) * bw + q + h] = (float)(1.0 / count);

  P->yee = *prob;
  P->yee.radius = 1.0f;   // identity filter: the single tap at r = 0
  P->yee.eta = 0.5f;      // Eq. 6 projects rho_tilde at 1/2
  size_t yb = 0;
  if ((st = eps_workspace_size(&P->yee, 0, &yb)) != EPS_OK) return st;
  P->empty = prob->mx == 0 || prob->my == 0;
  P->map_bytes = align256(sizeof(float) * (size_t)prob->mx * prob->my);
  P->yee_off = (size_t)(m->n_ops + 4) * P->map_bytes;
  P->yee_bytes = yb;
  P->total = P->empty ? 0 : P->yee_off + yb;
  return EPS_OK;
}

struct Maps {
  float *rho[EPS_MORPH_MAX_OPS + 1];
  float *pp, *ga, *gb;
  void *yee_ws;
};

Maps maps_of(const MorphPlan &P, const eps_morph_t *m, void *ws) {
  Maps M;
  char *b = (char *)ws;
  for (int k = 0; k <= m->n_ops; ++k) M.rho[k] = (float *)(b + k * P.map_bytes);
  M.pp = (float *)(b + (m->n_ops + 1) * P.map_bytes);
  M.ga = (float *)(b + (m->n_ops + 2) * P.map_bytes);
  M.gb = (float *)(b + (m->n_ops + 3) * P.map_bytes);
  M.yee_ws = b + P.yee_off;
  return M;
}

eps_status_t check_ws(const MorphPlan &P, const void *ws, size_t ws_bytes) {
  if (!ws || !aligned(ws, 256) || ws_bytes < P.total) return EPS_ERR_WORKSPACE;
  return EPS_OK;
}

eps_status_t run_map(const char *name, int kind, int rp1, const float *w, const eps_problem_t *prob,
                     float alpha, int erode, const float *in, const float *aux, const float *aux2,
                     float *out, float *out2, cudaStream_t s) {
  MapArgs ma;
  std::memset(&ma, 0, sizeof(ma));
  ma.mx = prob->mx;
  ma.my = prob->my;
  ma.beta = prob->beta;
  ma.eta = prob->eta;
  ma.alpha = alpha;
  ma.erode = erode;
  ma.in = in;
  ma.aux = aux;
  ma.aux2 = aux2;
  ma.out = out;
  ma.out2 = out2;
  eps_status_t st = epsc_host::error_flag(&ma.err);
  if (st != EPS_OK) return st;
  std::memcpy(ma.w, w, sizeof(ma.w));
  const KernelEntry k = map_entry(rp1, prob->bc, kind);
  const dim3 grid((prob->my + MT_B - 1) / MT_B, (prob->mx + MT_A - 1) / MT_A);
  // programmatic dependent launch: the kernel waits for the previous grid
  // before touching global memory
  return epsc_host::launch_kernel(name, k.fn, grid, k.smem, &ma, s, true);
}

// C -> rho_0, P'(u) -> rho_1 .. rho_n
eps_status_t run_front(const MorphPlan &P, const eps_problem_t *prob, const eps_morph_t *m,
                       const float *C, const Maps &M, cudaStream_t s) {
  eps_status_t st = run_map("eps_morph_front", MAP_FRONT, P.rp1_cone, P.w_cone, prob, 0.f, 0, C,
                            nullptr, nullptr, M.rho[0], M.pp, s);
  for (int k = 0; k < m->n_ops && st == EPS_OK; ++k)
    st = run_map("eps_morph_lse", MAP_LSE, P.rp1_disk, P.w_disk, prob, m->alpha, m->ops[k],
                 M.rho[k], nullptr, nullptr, M.rho[k + 1], nullptr, s);
  return st;
}

// d/d rho_n (in M.ga) -> dJ/dC
eps_status_t run_back(const MorphPlan &P, const eps_problem_t *prob, const eps_morph_t *m,
                      const Maps &M, float *dJdC, cudaStream_t s) {
  float *g = M.ga, *other = M.gb;
  eps_status_t st = EPS_OK;
  for (int k = m->n_ops - 1; k >= 0 && st == EPS_OK; --k) {
    st = run_map("eps_morph_lse_T", MAP_LSE_T, P.rp1_disk, P.w_disk, prob, m->alpha, m->ops[k], g,
                 M.rho[k + 1], M.rho[k], other, nullptr, s);
    float *t = g;
    g = other;
    other = t;
  }
  if (st != EPS_OK) return st;
  return run_map("eps_morph_front_T", MAP_FRONT_T, P.rp1_cone, P.w_cone, prob, 0.f, 0, g, M.pp,
                 nullptr, dJdC, nullptr, s);
}

}  // namespace

extern "C" {

eps_status_t eps_morph_workspace_size(const eps_problem_t *prob, const eps_morph_t *morph,
                                      int32_t n_lambda, size_t *bytes) {
  if (!bytes) return EPS_ERR_INVALID_ARG;
  if (n_lambda < 0 || n_lambda > EPS_MAX_LAMBDA) return EPS_ERR_INVALID_ARG;
  MorphPlan P;
  const eps_status_t st = plan(prob, morph, &P);
  if (st != EPS_OK) return st;
  *bytes = P.total;
  return EPS_OK;
}

eps_status_t eps_forward_morph(const eps_problem_t *prob, const eps_morph_t *morph,
                               const float *C, float *eps, float *offdiag, void *ws,
                               size_t ws_bytes, eps_stream_t stream) {
  MorphPlan P;
  eps_status_t st = plan(prob, morph, &P);
  if (st != EPS_OK) return st;
  if (P.empty) return EPS_OK;
  const bool od = (prob->flags & EPS_FLAG_OFFDIAG) != 0;
  if (!C || !eps || (od && !offdiag)) return EPS_ERR_INVALID_ARG;
  if (!aligned(C, 4) || !aligned(eps, 16) || (od && !aligned(offdiag, 16)))
    return EPS_ERR_INVALID_ARG;
  if ((st = check_ws(P, ws, ws_bytes)) != EPS_OK) return st;
  const Maps M = maps_of(P, morph, ws);
  cudaStream_t s = (cudaStream_t)stream;
  if ((st = run_front(P, prob, morph, C, M, s)) != EPS_OK) return st;
  return eps_forward(&P.yee, M.rho[morph->n_ops], eps, offdiag, stream);
}

eps_status_t eps_vjp_morph(const eps_problem_t *prob, const eps_morph_t *morph, const float *C,
                           int32_t n_lambda, int32_t field_type, const void *const *EF,
                           const void *const *EA, const float *field_scales, float scale,
                           float *dJdC, float *eps_out, void *ws, size_t ws_bytes,
                           eps_stream_t stream) {
  MorphPlan P;
  eps_status_t st = plan(prob, morph, &P);
  if (st != EPS_OK) return st;
  // eps_vjp's own checks, with the base chain's part of the workspace
  const void *yee_ws = ws ? (const char *)ws + P.yee_off : nullptr;
  const size_t yee_room = ws_bytes > P.yee_off ? ws_bytes - P.yee_off : 0;
  if ((st = epsc_host::check_vjp_args(prob, C, n_lambda, field_type, EF, EA, field_scales, scale,
                                      dJdC, eps_out, yee_ws, yee_room)) != EPS_OK)
    return st;
  if (P.empty) return EPS_OK;
  if ((st = check_ws(P, ws, ws_bytes)) != EPS_OK) return st;
  const Maps M = maps_of(P, morph, ws);
  cudaStream_t s = (cudaStream_t)stream;
  if ((st = run_front(P, prob, morph, C, M, s)) != EPS_OK) return st;
  st = eps_vjp(&P.yee, M.rho[morph->n_ops], n_lambda, field_type, EF, EA, field_scales, scale,
               M.ga, eps_out, M.yee_ws, P.yee_bytes, stream);
  if (st != EPS_OK) return st;
  return run_back(P, prob, morph, M, dJdC, s);
}

eps_status_t eps_vjp_real_morph(const eps_problem_t *prob, const eps_morph_t *morph,
                                const float *C, const float *G, float *dJdC, void *ws,
                                size_t ws_bytes, eps_stream_t stream) {
  MorphPlan P;
  eps_status_t st = plan(prob, morph, &P);
  if (st != EPS_OK) return st;
  if (prob->flags & EPS_FLAG_NORMALS_3D) return EPS_ERR_UNSUPPORTED;   // forward only
  if (P.empty) return EPS_OK;
  if (!C || !G || !dJdC) return EPS_ERR_INVALID_ARG;
  if (!aligned(C, 4) || !aligned(G, 4) || !aligned(dJdC, 4)) return EPS_ERR_INVALID_ARG;
  if ((st = check_ws(P, ws, ws_bytes)) != EPS_OK) return st;
  const Maps M = maps_of(P, morph, ws);
  cudaStream_t s = (cudaStream_t)stream;
  if ((st = run_front(P, prob, morph, C, M, s)) != EPS_OK) return st;
  if ((st = eps_vjp_real(&P.yee, M.rho[morph->n_ops], G, M.ga, M.yee_ws, P.yee_bytes, stream)) !=
      EPS_OK)
    return st;
  return run_back(P, prob, morph, M, dJdC, s);
}

}  // extern "C"

namespace epsc_host {

eps_status_t morph_base_offset(const eps_problem_t *prob, const eps_morph_t *morph, size_t *offset,
                               size_t *ws_needed) {
  MorphPlan P;
  const eps_status_t st = plan(prob, morph, &P);
  if (st != EPS_OK) return st;
  *offset = P.yee_off;
  *ws_needed = P.total;
  return EPS_OK;
}

}  // namespace epsc_host
