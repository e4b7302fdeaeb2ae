// C ABI of the epschain library: argument validation, conic weights,
// workspace layout, kernel dispatch and per-kernel timing.  Every argument
// error returns before any launch.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <set>
#include <utility>
#include <vector>

#include "epschain.h"
#include "epsc_launch.h"

using namespace epsc;

// Device-side error flag (one per device that loads the library).
__device__ int g_eps_error_flag;

namespace {

struct Resolved {
  bool empty;
  Geometry g;
  int rp1;
  float w[MAX_BOX * MAX_BOX];
};

inline size_t align256(size_t b) { return (b + 255) & ~size_t(255); }

eps_status_t resolve(const eps_problem_t *p, Resolved *r) {
  if (!p || !r) return EPS_ERR_INVALID_ARG;
  std::memset(r, 0, sizeof(*r));
  if (p->sub != 2) return EPS_ERR_UNSUPPORTED;
  if (p->bc != EPS_BC_CLAMP && p->bc != EPS_BC_PERIODIC) return EPS_ERR_INVALID_ARG;
  if (p->flags & ~EPS_FLAG_OFFDIAG) return EPS_ERR_INVALID_ARG;
  if (!std::isfinite(p->radius) || !(p->radius > 0.f)) return EPS_ERR_INVALID_ARG;
  if (!std::isfinite(p->beta) || !std::isfinite(p->eta)) return EPS_ERR_INVALID_ARG;
  if (!std::isfinite(p->eps_core) || !std::isfinite(p->eps_clad) || !(p->eps_core > 0.f) ||
      !(p->eps_clad > 0.f))
    return EPS_ERR_INVALID_ARG;
  if (p->radius > EPS_MAX_RADIUS) return EPS_ERR_UNSUPPORTED;
  if (p->mx < 0 || p->my < 0 || (p->mx & 1) || (p->my & 1)) return EPS_ERR_SHAPE;
  if (p->mx > (1 << 20) || p->my > (1 << 20)) return EPS_ERR_SHAPE;
  if (p->nz < 1 || p->nz > 4096 || p->slab_nk < 1 || p->slab_k0 < -1) return EPS_ERR_SHAPE;
  const int k0 = p->slab_k0 >= 0 ? p->slab_k0 : (p->nz - p->slab_nk - 1) / 2;
  if (k0 < 0 || k0 + p->slab_nk > p->nz - 1) return EPS_ERR_SHAPE;

  r->empty = p->mx == 0 || p->my == 0;
  Geometry &g = r->g;
  g.mx = p->mx;
  g.my = p->my;
  g.nx = p->mx / 2;
  g.ny = p->my / 2;
  g.nz = p->nz;
  g.k0 = k0;
  g.nk = p->slab_nk;
  g.bc = p->bc;
  g.beta = p->beta;
  g.eta = p->eta;
  g.eps_core = p->eps_core;
  g.eps_clad = p->eps_clad;
  g.deps = p->eps_core - p->eps_clad;

  // Eq. 2 basis: normalised cone on integer offsets with r < R (float64 sums)
  const double R = p->radius;
  const int rp1 = std::max(1, (int)std::ceil(R));
  if (rp1 > MAX_RP1) return EPS_ERR_UNSUPPORTED;
  r->rp1 = rp1;
  const int h = rp1 - 1, bw = 2 * rp1 - 1;
  double total = 0.0;
  std::vector<double> wd(bw * bw, 0.0);
  for (int pp = -h; pp <= h; ++pp)
    for (int qq = -h; qq <= h; ++qq) {
      const double rr = std::hypot((double)pp, (double)qq);
      if (rr < R) {
        wd[(pp + h) * bw + qq + h] = 1.0 - rr / R;
        total += 1.0 - rr / R;
      }
    }
  for (int t = 0; t < bw * bw; ++t) r->w[t] = (float)(wd[t] / total);
  return EPS_OK;
}

size_t workspace_bytes(const Geometry &g) {
  return align256(sizeof(float) * NSEED * (size_t)g.nx * g.ny) +
         align256(sizeof(float) * (size_t)g.mx * g.my);
}

bool aligned(const void *p, size_t a) { return ((uintptr_t)p % a) == 0; }

// ---------------------------------------------------------------- profiling
struct ProfRec {
  const char *name;
  cudaEvent_t e0, e1;
};
std::mutex g_prof_mu;
bool g_prof_on = false;
std::vector<ProfRec> g_prof_recs;
std::vector<cudaEvent_t> g_event_pool;

cudaEvent_t pool_event() {
  if (!g_event_pool.empty()) {
    cudaEvent_t e = g_event_pool.back();
    g_event_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
  return e;
}

// --------------------------------------------------------------- launching
std::mutex g_attr_mu;
std::set<std::pair<int, const void *>> g_attr_done;

eps_status_t prepare(const KernelEntry &k) {
  if (!k.fn) return EPS_ERR_UNSUPPORTED;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return EPS_ERR_CUDA;
  std::lock_guard<std::mutex> lk(g_attr_mu);
  if (g_attr_done.count({dev, k.fn})) return EPS_OK;
  if (cudaFuncSetAttribute(k.fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)k.smem) !=
      cudaSuccess)
    return EPS_ERR_CUDA;
  g_attr_done.insert({dev, k.fn});
  return EPS_OK;
}

eps_status_t launch(const char *name, const KernelEntry &k, dim3 grid, void *args,
                    cudaStream_t s) {
  eps_status_t st = prepare(k);
  if (st != EPS_OK) return st;
  ProfRec rec{name, nullptr, nullptr};
  bool prof = false;
  {
    std::lock_guard<std::mutex> lk(g_prof_mu);
    if (g_prof_on) {
      rec.e0 = pool_event();
      rec.e1 = pool_event();
      prof = rec.e0 && rec.e1;
    }
  }
  if (prof && cudaEventRecord(rec.e0, s) != cudaSuccess) return EPS_ERR_CUDA;
  void *params[] = {args};
  if (cudaLaunchKernel(k.fn, grid, dim3(NTHREADS), params, k.smem, s) != cudaSuccess)
    return EPS_ERR_CUDA;
  if (prof) {
    if (cudaEventRecord(rec.e1, s) != cudaSuccess) return EPS_ERR_CUDA;
    std::lock_guard<std::mutex> lk(g_prof_mu);
    g_prof_recs.push_back(rec);
  }
  return EPS_OK;
}

eps_status_t error_flag_ptr(int **out) {
  if (cudaGetSymbolAddress((void **)out, g_eps_error_flag) != cudaSuccess) return EPS_ERR_CUDA;
  return EPS_OK;
}

dim3 fwd_grid(const Geometry &g) { return dim3((g.ny + TJ - 1) / TJ, (g.nx + TI - 1) / TI); }
dim3 bwd_grid(const Geometry &g) { return dim3((g.my + TB - 1) / TB, (g.mx + TA - 1) / TA); }

void fill_fwd_common(FwdArgs &fa, const Resolved &r, const float *C, int *err) {
  std::memset(&fa, 0, sizeof(fa));
  fa.g = r.g;
  fa.C = C;
  fa.err = err;
  std::memcpy(fa.w, r.w, sizeof(fa.w));
}

eps_status_t run_scatter(const Resolved &r, const float *seeds, const float *uws, float *dJdC,
                         int *err, cudaStream_t s) {
  BwdArgs ba;
  std::memset(&ba, 0, sizeof(ba));
  ba.g = r.g;
  ba.seeds = seeds;
  ba.uws = uws;
  ba.dJdC = dJdC;
  ba.err = err;
  std::memcpy(ba.w, r.w, sizeof(ba.w));
  return launch("eps_vjp_scatter", bwd_entry(r.rp1), bwd_grid(r.g), &ba, s);
}

}  // namespace

extern "C" {

const char *eps_status_string(eps_status_t status) {
  switch (status) {
    case EPS_OK: return "EPS_OK";
    case EPS_ERR_INVALID_ARG: return "EPS_ERR_INVALID_ARG";
    case EPS_ERR_SHAPE: return "EPS_ERR_SHAPE";
    case EPS_ERR_WORKSPACE: return "EPS_ERR_WORKSPACE";
    case EPS_ERR_UNSUPPORTED: return "EPS_ERR_UNSUPPORTED";
    case EPS_ERR_CUDA: return "EPS_ERR_CUDA";
    case EPS_ERR_DEVICE_TIMEOUT: return "EPS_ERR_DEVICE_TIMEOUT";
    case EPS_ERR_DEVICE_BOUNDS: return "EPS_ERR_DEVICE_BOUNDS";
  }
  return "EPS_ERR_UNKNOWN";
}

eps_status_t eps_workspace_size(const eps_problem_t *prob, int32_t n_lambda, size_t *bytes) {
  if (!bytes) return EPS_ERR_INVALID_ARG;
  if (n_lambda < 0 || n_lambda > EPS_MAX_LAMBDA) return EPS_ERR_INVALID_ARG;
  Resolved r;
  eps_status_t st = resolve(prob, &r);
  if (st != EPS_OK) return st;
  *bytes = r.empty ? 0 : workspace_bytes(r.g);
  return EPS_OK;
}

eps_status_t eps_forward(const eps_problem_t *prob, const float *C, float *eps, float *offdiag,
                         eps_stream_t stream) {
  Resolved r;
  eps_status_t st = resolve(prob, &r);
  if (st != EPS_OK) return st;
  if (r.empty) return EPS_OK;
  const bool od = (prob->flags & EPS_FLAG_OFFDIAG) != 0;
  if (!C || !eps || (od && !offdiag)) return EPS_ERR_INVALID_ARG;
  if (!aligned(C, 4) || !aligned(eps, 16) || (od && !aligned(offdiag, 16)))
    return EPS_ERR_INVALID_ARG;
  int *err = nullptr;
  if ((st = error_flag_ptr(&err)) != EPS_OK) return st;
  FwdArgs fa;
  fill_fwd_common(fa, r, C, err);
  fa.mode = MODE_FWD;
  fa.write_eps = 1;
  fa.write_offdiag = od ? 1 : 0;
  fa.eps = eps;
  fa.offdiag = od ? offdiag : nullptr;
  return launch("eps_forward", fwd_entry(r.rp1), fwd_grid(r.g), &fa, (cudaStream_t)stream);
}

eps_status_t eps_vjp(const eps_problem_t *prob, const float *C, int32_t n_lambda,
                     int32_t field_type, const void *const *EF, const void *const *EA,
                     const float *field_scales, float scale, float *dJdC, float *eps_out,
                     void *ws, size_t ws_bytes, eps_stream_t stream) {
  Resolved r;
  eps_status_t st = resolve(prob, &r);
  if (st != EPS_OK) return st;
  if (n_lambda < 0 || n_lambda > EPS_MAX_LAMBDA) return EPS_ERR_INVALID_ARG;
  if (field_type != EPS_FIELD_C64 && field_type != EPS_FIELD_BF16X2_SCALED &&
      field_type != EPS_FIELD_F16X2_SCALED)
    return EPS_ERR_INVALID_ARG;
  if (field_type != EPS_FIELD_C64) return EPS_ERR_UNSUPPORTED;
  if (!std::isfinite(scale)) return EPS_ERR_INVALID_ARG;
  if (r.empty) return EPS_OK;
  if (!C || !dJdC) return EPS_ERR_INVALID_ARG;
  if (n_lambda > 0 && (!EF || !EA)) return EPS_ERR_INVALID_ARG;
  for (int l = 0; l < n_lambda; ++l) {
    if (!EF[l] || !EA[l]) return EPS_ERR_INVALID_ARG;
    if (!aligned(EF[l], 16) || !aligned(EA[l], 16)) return EPS_ERR_INVALID_ARG;
  }
  if (field_scales)
    for (int t = 0; t < 6 * n_lambda; ++t)
      if (!std::isfinite(field_scales[t])) return EPS_ERR_INVALID_ARG;
  if (r.g.nz & 1) return EPS_ERR_SHAPE;   // complex64 planes are read in pairs
  if (!aligned(C, 4) || !aligned(dJdC, 4) || (eps_out && !aligned(eps_out, 16)))
    return EPS_ERR_INVALID_ARG;
  if (!ws || !aligned(ws, 256) || ws_bytes < workspace_bytes(r.g)) return EPS_ERR_WORKSPACE;
  int *err = nullptr;
  if ((st = error_flag_ptr(&err)) != EPS_OK) return st;

  float *seeds = (float *)ws;
  float *uws = (float *)((char *)ws + align256(sizeof(float) * NSEED * (size_t)r.g.nx * r.g.ny));
  FwdArgs fa;
  fill_fwd_common(fa, r, C, err);
  fa.mode = MODE_C64;
  fa.write_eps = eps_out ? 1 : 0;
  fa.eps = eps_out;
  fa.nlambda = n_lambda;
  fa.seeds = seeds;
  fa.uws = uws;
  for (int l = 0; l < n_lambda; ++l) {
    fa.EF[l] = (const float4 *)EF[l];
    fa.EA[l] = (const float4 *)EA[l];
    for (int c = 0; c < 3; ++c) {
      float s = scale;
      if (field_scales) s *= field_scales[(l * 2 + 0) * 3 + c] * field_scales[(l * 2 + 1) * 3 + c];
      fa.fs[l][c] = s;
    }
  }
  cudaStream_t s = (cudaStream_t)stream;
  st = launch(eps_out ? "eps_fwd_vjp_contract" : "eps_vjp_contract", fwd_entry(r.rp1),
              fwd_grid(r.g), &fa, s);
  if (st != EPS_OK) return st;
  return run_scatter(r, seeds, uws, dJdC, err, s);
}

eps_status_t eps_vjp_real(const eps_problem_t *prob, const float *C, const float *G, float *dJdC,
                          void *ws, size_t ws_bytes, eps_stream_t stream) {
  Resolved r;
  eps_status_t st = resolve(prob, &r);
  if (st != EPS_OK) return st;
  if (r.empty) return EPS_OK;
  if (!C || !G || !dJdC) return EPS_ERR_INVALID_ARG;
  if (!aligned(C, 4) || !aligned(G, 4) || !aligned(dJdC, 4)) return EPS_ERR_INVALID_ARG;
  if (!ws || !aligned(ws, 256) || ws_bytes < workspace_bytes(r.g)) return EPS_ERR_WORKSPACE;
  int *err = nullptr;
  if ((st = error_flag_ptr(&err)) != EPS_OK) return st;
  float *seeds = (float *)ws;
  float *uws = (float *)((char *)ws + align256(sizeof(float) * NSEED * (size_t)r.g.nx * r.g.ny));
  FwdArgs fa;
  fill_fwd_common(fa, r, C, err);
  fa.mode = MODE_REAL;
  fa.G = G;
  fa.seeds = seeds;
  fa.uws = uws;
  cudaStream_t s = (cudaStream_t)stream;
  st = launch("eps_vjp_real_contract", fwd_entry(r.rp1), fwd_grid(r.g), &fa, s);
  if (st != EPS_OK) return st;
  return run_scatter(r, seeds, uws, dJdC, err, s);
}

eps_status_t eps_sync_status(eps_stream_t stream) {
  if (cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess) return EPS_ERR_CUDA;
  int flag = 0;
  if (cudaMemcpyFromSymbol(&flag, g_eps_error_flag, sizeof(int)) != cudaSuccess)
    return EPS_ERR_CUDA;
  if (flag == 0) return EPS_OK;
  const int zero = 0;
  if (cudaMemcpyToSymbol(g_eps_error_flag, &zero, sizeof(int)) != cudaSuccess) return EPS_ERR_CUDA;
  return flag == EPS_ERR_DEVICE_TIMEOUT ? EPS_ERR_DEVICE_TIMEOUT : EPS_ERR_DEVICE_BOUNDS;
}

eps_status_t eps_profile_start(void) {
  std::lock_guard<std::mutex> lk(g_prof_mu);
  g_prof_on = true;
  return EPS_OK;
}

eps_status_t eps_profile_stop(eps_profile_entry_t *entries, int32_t max_entries,
                              int32_t *n_entries) {
  std::vector<ProfRec> recs;
  {
    std::lock_guard<std::mutex> lk(g_prof_mu);
    g_prof_on = false;
    recs.swap(g_prof_recs);
  }
  eps_status_t st = EPS_OK;
  std::vector<eps_profile_entry_t> agg;
  for (const ProfRec &rec : recs) {
    float ms = 0.f;
    if (cudaEventSynchronize(rec.e1) != cudaSuccess ||
        cudaEventElapsedTime(&ms, rec.e0, rec.e1) != cudaSuccess)
      st = EPS_ERR_CUDA;
    size_t t = 0;
    for (; t < agg.size(); ++t)
      if (std::strcmp(agg[t].name, rec.name) == 0) break;
    if (t == agg.size()) {
      eps_profile_entry_t e;
      std::memset(&e, 0, sizeof(e));
      std::snprintf(e.name, sizeof(e.name), "%s", rec.name);
      agg.push_back(e);
    }
    agg[t].launches += 1;
    agg[t].total_ms += ms;
  }
  {
    std::lock_guard<std::mutex> lk(g_prof_mu);
    for (const ProfRec &rec : recs) {
      g_event_pool.push_back(rec.e0);
      g_event_pool.push_back(rec.e1);
    }
  }
  int n = 0;
  for (size_t t = 0; t < agg.size() && entries && n < max_entries; ++t) entries[n++] = agg[t];
  if (n_entries) *n_entries = n;
  return st;
}

}  // extern "C"
