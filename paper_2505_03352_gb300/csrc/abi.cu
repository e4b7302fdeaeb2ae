// C ABI of the epschain library: argument validation, conic weights,
// workspace layout, kernel dispatch and per-kernel timing.  Every argument
// error returns before any launch.
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <algorithm>
#include <atomic>
#include <memory>
#include <mutex>
#include <set>
#include <utility>
#include <vector>

#include "epschain.h"
#include <cuda.h>

#include "epsc_contract.cuh"
#include "epsc_contract_tma.cuh"
#include "epsc_contract_tma_batch.cuh"
#include "epsc_contract_tma_real.cuh"
#include "epsc_pack.cuh"
#include "epsc_launch.h"
#include "epsc_multi.cuh"

using namespace epsc;

// Device-side error flag (one per device that loads the library).
__device__ int g_eps_error_flag;

namespace {

struct Resolved {
  bool empty;
  bool normals3d;   // EPS_FLAG_NORMALS_3D: forward only
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
  if (p->flags & ~(EPS_FLAG_OFFDIAG | EPS_FLAG_NORMALS_3D)) return EPS_ERR_INVALID_ARG;
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
  r->normals3d = (p->flags & EPS_FLAG_NORMALS_3D) != 0;
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

// Workspace: W [4][nx][ny] | seeds [NSEED][nx][ny] | pd4 [mx][my] | ie2 [mx][my]
// | epsc [4][nx][ny] (per-column eps values for the Eq. 1 surrogate, used by
// eps_vjp_surrogate only), each 256-byte aligned.
struct WsLayout {
  size_t w, seeds, pd4, ie2, epsc, total;
};

WsLayout ws_layout(const Geometry &g) {
  WsLayout L;
  const size_t cells = (size_t)g.nx * g.ny;
  const size_t subs = (size_t)g.mx * g.my;
  L.w = 0;
  L.seeds = L.w + align256(sizeof(float) * 4 * cells);
  L.pd4 = L.seeds + align256(sizeof(float) * NSEED * cells);
  L.ie2 = L.pd4 + align256(sizeof(float) * subs);
  L.epsc = L.ie2 + align256(sizeof(float) * subs);
  L.total = L.epsc + align256(sizeof(float) * 4 * cells);
  return L;
}

size_t workspace_bytes(const Geometry &g) { return ws_layout(g).total; }

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
int g_sm_count[64];

// Largest dynamic shared memory any launch of this library asks for.
constexpr size_t MAX_DYN_SMEM = 200 * 1024;

eps_status_t prepare(const void *fn, size_t smem) {
  if (!fn) return EPS_ERR_UNSUPPORTED;
  if (smem > MAX_DYN_SMEM) return EPS_ERR_UNSUPPORTED;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return EPS_ERR_CUDA;
  std::lock_guard<std::mutex> lk(g_attr_mu);
  if (g_attr_done.count({dev, fn})) return EPS_OK;
  if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)MAX_DYN_SMEM) !=
      cudaSuccess)
    return EPS_ERR_CUDA;
  g_attr_done.insert({dev, fn});
  return EPS_OK;
}

eps_status_t sm_count(int *n) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return EPS_ERR_CUDA;
  std::lock_guard<std::mutex> lk(g_attr_mu);
  if (g_sm_count[dev] == 0 &&
      cudaDeviceGetAttribute(&g_sm_count[dev], cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return EPS_ERR_CUDA;
  *n = g_sm_count[dev];
  return EPS_OK;
}

// Launch `fn` (one by-value argument struct) on stream s.  With `pdl` the
// kernel may begin while the previous kernel in the stream is still running
// (programmatic dependent launch); it must then wait on that grid
// (griddepcontrol.wait) before reading its results.  While profiling, each
// launch is bracketed by events and launched without overlap.
// Kernel launches made by the library in this process (eps_launch_count).
std::atomic<unsigned long long> g_launch_count{0};

eps_status_t launch(const char *name, const void *fn, dim3 grid, size_t smem, void *args,
                    cudaStream_t s, bool pdl = false, unsigned block = NTHREADS) {
  eps_status_t st = prepare(fn, smem);
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
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = grid;
  cfg.blockDim = dim3(block);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  if (pdl && !prof) {
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
  }
  void *params[] = {args};
  if (cudaLaunchKernelExC(&cfg, fn, params) != cudaSuccess) return EPS_ERR_CUDA;
  g_launch_count.fetch_add(1, std::memory_order_relaxed);
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
long fwd_ntiles(const Geometry &g) { return (long)fwd_grid(g).x * fwd_grid(g).y; }
// scatter tiles of TA x tbw subpixels (tbw: TB, or 64 for the batched calls' wide tiles)
dim3 bwd_grid(const Geometry &g, int tbw = TB) {
  return dim3((g.my + tbw - 1) / tbw, (g.mx + TA - 1) / TA);
}

// Dynamic shared memory of a forward launch: the stencil buffers, grown to
// stage all of the tile's eps_hat components (up to 3) for one round of bulk
// stores when that fits the budget.
// (ncomp = 0: eps_hat leaves by direct coalesced stores; only the stencil
// buffers are needed)
size_t fwd_smem(const KernelEntry &k, const Geometry &g, int ncomp, int *stage_floats) {
  const size_t comp_bytes = sizeof(float) * TI * TJ * (size_t)g.nz;
  size_t want = std::max(k.smem, std::min<size_t>(ncomp, 3) * comp_bytes);
  if (want > MAX_DYN_SMEM) want = std::max(k.smem, std::min(MAX_DYN_SMEM, comp_bytes));
  *stage_floats = (int)(want / sizeof(float));
  return want;
}

void fill_fwd_common(FwdArgs &fa, const Resolved &r, const float *C, int *err) {
  std::memset(&fa, 0, sizeof(fa));
  fa.r.g = r.g;
  fa.r.C = C;
  fa.err = err;
  std::memcpy(fa.w, r.w, sizeof(fa.w));
}

// Persistent contraction grid: a few blocks per SM, so that the stencil
// kernel launched behind it (programmatic dependent launch) finds room on
// every SM and its compute overlaps the field stream.
constexpr int CONTRACT_BLOCKS_PER_SM = 2;

eps_status_t run_contract(const ContractArgs &ca, int lanes, cudaStream_t s) {
  int nsm = 0;
  eps_status_t st = sm_count(&nsm);
  if (st != EPS_OK) return st;
  const long ncol = (long)ca.nx * ca.ny;
  const long per_block = (NTHREADS / lanes) * 2;   // columns per block per iteration
  long blocks = (ncol + per_block - 1) / per_block;
  blocks = std::min<long>(blocks, (long)nsm * CONTRACT_BLOCKS_PER_SM);
  return launch(ca.mode == MODE_C64 ? "eps_vjp_contract" : "eps_vjp_real_contract",
                contract_entry(lanes), dim3((unsigned)std::max<long>(blocks, 1)), 0,
                (void *)&ca, s);
}

// cuTensorMapEncodeTiled, resolved through the runtime (no link to libcuda)
typedef CUresult (*PFN_encodeTiled)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *,
                                    const cuuint64_t *, const cuuint64_t *, const cuuint32_t *,
                                    const cuuint32_t *, CUtensorMapInterleave, CUtensorMapSwizzle,
                                    CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

PFN_encodeTiled encode_tiled() {
  static PFN_encodeTiled fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (PFN_encodeTiled)p;
  });
  return fn;
}

// Tensor map of eps_hat [3][nx][ny][nz] for the stencil's swizzled staging
// form: a {nz, ny, nx, 3} float tensor with a {nz, TJ, TI, 1} box and the
// 128-byte swizzle.  nz = 32 only (a column's planes are exactly one
// swizzle row); false otherwise or when the map cannot be made (the plain
// staging then runs).
bool eps_store_map(const Geometry &g, float *eps, CUtensorMap *map) {
  PFN_encodeTiled enc = encode_tiled();
  if (!enc || !eps || g.nz != 32 || !aligned(eps, 16)) return false;
  const cuuint64_t col = (cuuint64_t)g.nz * 4;
  cuuint64_t dims[4] = {(cuuint64_t)g.nz, (cuuint64_t)g.ny, (cuuint64_t)g.nx, 3};
  cuuint64_t strides[3] = {col, col * g.ny, col * g.ny * g.nx};
  cuuint32_t box[4] = {(cuuint32_t)g.nz, (cuuint32_t)TJ, (cuuint32_t)TI, 1};
  cuuint32_t es[4] = {1, 1, 1, 1};
  return enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, (void *)eps, dims, strides, box, es,
             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
             CU_TENSOR_MAP_L2_PROMOTION_NONE, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// Dynamic shared memory of a single-region forward launch that stages
// `ncomp` (1 .. 3) eps_hat components through the swizzled form: the
// stencil buffers or the staging buffers, whichever is larger, plus 1 KB
// so that the staging can start on a 1024-byte boundary.
size_t fwd_smem_swizzled(const KernelEntry &k, const Geometry &g, int ncomp, int *stage_floats) {
  const int comp_floats = TI * TJ * g.nz;
  ncomp = std::max(1, std::min(ncomp, 3));
  *stage_floats = ncomp * comp_floats;
  return std::max(k.smem, sizeof(float) * ncomp * comp_floats + 1024);
}

// Sets up the eps_hat output of a single-region forward launch: the
// swizzled staging form (tensor map in `fa`) where eps_store_map allows,
// else plain staging of `ncomp` components per round (ncomp 0: direct
// stores, nz a multiple of 4); returns the launch's dynamic shared memory.
size_t fwd_eps_output(FwdArgs &fa, const KernelEntry &k, const Geometry &g, int ncomp,
                      int swz_comps) {
  if (swz_comps > 0 && !fa.r.write_offdiag && eps_store_map(g, fa.r.eps, &fa.eps_map)) {
    fa.r.eps_tma = 1;
    fa.r.direct_eps = 0;
    return fwd_smem_swizzled(k, g, swz_comps, &fa.r.stage_floats);
  }
  fa.r.eps_tma = 0;
  fa.r.direct_eps = (ncomp == 0 && (g.nz & 3) == 0) ? 1 : 0;
  return fwd_smem(k, g, fa.r.direct_eps ? 0 : std::max(ncomp, 1), &fa.r.stage_floats);
}

// J-support window of a column in floats: the 32-byte sectors holding
// planes k0 .. k0+nk (complex64, 8 bytes per plane).
void support_window(const Geometry &g, int *x0, int *bx) {
  const int lo = (2 * g.k0) & ~7;
  const int hi = (2 * (g.k0 + g.nk + 1) + 7) & ~7;
  *x0 = lo;
  *bx = hi - lo;
}

// Arguments of the contraction through bulk tensor copies (every column);
// EPS_ERR_UNSUPPORTED when the fields or the window do not fit its
// requirements (the caller falls back).
eps_status_t prepare_contract_tma(const Geometry &g, int n_lambda, const void *const *EF,
                                  const void *const *EA, const float (*fs)[3], float *Wm,
                                  int *err, ContractTmaArgs *ta) {
  PFN_encodeTiled enc = encode_tiled();
  if (!enc || n_lambda < 1) return EPS_ERR_UNSUPPORTED;
  int x0 = 0, bx = 0;
  support_window(g, &x0, &bx);
  if (bx > TMA_BX_MAX || (g.nz & 1)) return EPS_ERR_UNSUPPORTED;
  std::memset(ta, 0, sizeof(*ta));
  const long ncol = (long)g.nx * g.ny;
  const size_t comp_bytes = (size_t)ncol * g.nz * 8;
  for (int l = 0; l < n_lambda; ++l) {
    for (int f = 0; f < 2; ++f) {
      // (2 nz floats) x (columns) x (3 components)
      cuuint64_t dims[3] = {(cuuint64_t)(2 * g.nz), (cuuint64_t)ncol, 3};
      cuuint64_t strides[2] = {(cuuint64_t)g.nz * 8, (cuuint64_t)comp_bytes};
      cuuint32_t box[3] = {(cuuint32_t)bx, (cuuint32_t)TMA_BY, 3};
      cuuint32_t es[3] = {1, 1, 1};
      if (enc(&ta->maps[l * 2 + f], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3,
              (void *)(f == 0 ? EF[l] : EA[l]), dims, strides, box, es,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
              CU_TENSOR_MAP_L2_PROMOTION_NONE, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return EPS_ERR_UNSUPPORTED;
    }
    for (int c = 0; c < 3; ++c) ta->fs[l][c] = fs[l][c];
  }
  ta->W = Wm;
  ta->err = err;
  ta->nx = g.nx;
  ta->ny = g.ny;
  ta->k0 = g.k0;
  ta->nk = g.nk;
  ta->nlambda = n_lambda;
  ta->x0 = x0;
  ta->bx = bx;
  ta->col_lo = 0;
  ta->col_hi = ncol;
  return EPS_OK;
}

// One launch of the prepared contraction over the columns [col_lo, col_hi).
eps_status_t launch_contract_tma(ContractTmaArgs *ta, long col_lo, long col_hi,
                                 cudaStream_t s) {
  static_assert(sizeof(ContractTmaArgs) < 8192, "kernel parameter space");
  int nsm = 0;
  eps_status_t st = sm_count(&nsm);
  if (st != EPS_OK) return st;
  ta->col_lo = col_lo;
  ta->col_hi = col_hi;
  const long nchunks = (col_hi - col_lo + TMA_BY - 1) / TMA_BY;
  if (nchunks <= 0) return EPS_OK;
  const long blocks = std::max<long>(1, std::min<long>(nchunks, (long)nsm * CONTRACT_BLOCKS_PER_SM));
  const size_t smem = (size_t)TMA_NSTAGE * 6 * TMA_BY * ta->bx * 4 + 128;
  return launch("eps_vjp_contract", contract_tma_entry(ta->nlambda), dim3((unsigned)blocks), smem,
                ta, s);
}

// Contraction through bulk tensor copies over every column;
// EPS_ERR_UNSUPPORTED as prepare_contract_tma.
eps_status_t run_contract_tma(const Geometry &g, int n_lambda, const void *const *EF,
                              const void *const *EA, const float (*fs)[3], float *Wm, int *err,
                              cudaStream_t s) {
  ContractTmaArgs targs;
  const eps_status_t st = prepare_contract_tma(g, n_lambda, EF, EA, fs, Wm, err, &targs);
  if (st != EPS_OK) return st;
  return launch_contract_tma(&targs, 0, (long)g.nx * g.ny, s);
}

// Arguments of the batched TMA contraction over the regions of `ca`
// (geometries `gs`, same order); false when the batch or a region's fields
// or window do not suit it (the register-load contraction then runs).
bool prepare_contract_tma_batch(const std::vector<const Geometry *> &gs,
                                const ContractBatchArgs &ca, int n_lambda,
                                ContractTmaBatchArgs *ta, size_t *smem) {
  PFN_encodeTiled enc = encode_tiled();
  if (!enc || n_lambda < 1 || ca.n < 1 || ca.n * n_lambda * 2 > TMA_BATCH_MAX_MAPS) return false;
  std::memset(ta, 0, sizeof(*ta));
  long chunks = 0;
  int bx_max = 0;
  for (int k = 0; k < ca.n; ++k) {
    const Geometry &g = *gs[k];
    const ContractBatchRegion &cr = ca.r[k];
    int x0 = 0, bx = 0;
    support_window(g, &x0, &bx);
    if (bx > TMA_BX_MAX || (g.nz & 1)) return false;
    ContractTmaBatchRegion &tr = ta->r[k];
    tr.W = cr.W;
    tr.ncol = (long)g.nx * g.ny;
    tr.chunk_start = (int)chunks;
    tr.k0 = g.k0;
    tr.nk = g.nk;
    tr.x0 = x0;
    tr.bx = bx;
    tr.map0 = 2 * n_lambda * k;
    const size_t comp_bytes = (size_t)tr.ncol * g.nz * 8;
    for (int l = 0; l < n_lambda; ++l) {
      for (int c = 0; c < 3; ++c) tr.fs[l][c] = cr.fs[l][c];
      for (int f = 0; f < 2; ++f) {
        // (2 nz floats) x (columns) x (3 components)
        cuuint64_t dims[3] = {(cuuint64_t)(2 * g.nz), (cuuint64_t)tr.ncol, 3};
        cuuint64_t strides[2] = {(cuuint64_t)g.nz * 8, (cuuint64_t)comp_bytes};
        cuuint32_t box[3] = {(cuuint32_t)bx, (cuuint32_t)TMA_BY, 3};
        cuuint32_t es[3] = {1, 1, 1};
        if (enc(&ta->maps[tr.map0 + 2 * l + f], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3,
                (void *)(f == 0 ? cr.EF[l] : cr.EA[l]), dims, strides, box, es,
                CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                CU_TENSOR_MAP_L2_PROMOTION_NONE, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
          return false;
      }
    }
    chunks += (tr.ncol + TMA_BY - 1) / TMA_BY;
    bx_max = std::max(bx_max, bx);
  }
  if (chunks <= 0 || chunks > (1l << 30)) return false;
  ta->n = ca.n;
  ta->nlambda = n_lambda;
  ta->nchunks = (int)chunks;
  ta->stage_floats = 6 * TMA_BY * bx_max;
  *smem = (size_t)TMA_NSTAGE * ta->stage_floats * 4 + 128;
  return true;
}

// Column sums of a real cotangent G through bulk tensor copies;
// EPS_ERR_UNSUPPORTED when G's layout does not suit them (nz not a multiple
// of 4, G not 16-byte aligned, a support window wider than the box).
eps_status_t run_contract_tma_real(const Geometry &g, const float *G, float *Wm, int *err,
                                   cudaStream_t s) {
  PFN_encodeTiled enc = encode_tiled();
  if (!enc || (g.nz & 3) || !aligned(G, 16)) return EPS_ERR_UNSUPPORTED;
  const int lo = g.k0 & ~7;
  const int hi = (g.k0 + g.nk + 1 + 7) & ~7;
  if (hi - lo > TMA_REAL_BX_MAX) return EPS_ERR_UNSUPPORTED;
  ContractTmaRealArgs ta;
  std::memset(&ta, 0, sizeof(ta));
  const long ncol = (long)g.nx * g.ny;
  // (nz floats) x (columns) x (3 components)
  cuuint64_t dims[3] = {(cuuint64_t)g.nz, (cuuint64_t)ncol, 3};
  cuuint64_t strides[2] = {(cuuint64_t)g.nz * 4, (cuuint64_t)ncol * g.nz * 4};
  cuuint32_t box[3] = {(cuuint32_t)(hi - lo), (cuuint32_t)TMA_REAL_BY, 3};
  cuuint32_t es[3] = {1, 1, 1};
  if (enc(&ta.map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, (void *)G, dims, strides, box, es,
          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
          CU_TENSOR_MAP_L2_PROMOTION_NONE, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
    return EPS_ERR_UNSUPPORTED;
  ta.W = Wm;
  ta.err = err;
  ta.nx = g.nx;
  ta.ny = g.ny;
  ta.k0 = g.k0;
  ta.nk = g.nk;
  ta.x0 = lo;
  ta.bx = hi - lo;
  int nsm = 0;
  eps_status_t st = sm_count(&nsm);
  if (st != EPS_OK) return st;
  const long nchunks = (ncol + TMA_REAL_BY - 1) / TMA_REAL_BY;
  const long blocks = std::max<long>(1, std::min<long>(nchunks, (long)nsm * CONTRACT_BLOCKS_PER_SM));
  const size_t smem = (size_t)TMA_REAL_NSTAGE * 3 * TMA_REAL_BY * ta.bx * 4 + 128;
  return launch("eps_vjp_real_contract", contract_tma_real_entry(), dim3((unsigned)blocks), smem,
                &ta, s);
}

// Launch shape of the bulk-copy packed contraction (swept at the 3000 x
// 3000, eight-wavelength BF16 call: three blocks per SM of two stages of 96
// columns, 55 KB each, with the stencil beside them, 1.140 ms; two of 128
// columns 1.165-1.171 ms; 2 x 3 stages of 128 columns 1.35 ms; the
// register-load kernel, which fills every SM slot, 1.41 ms; more shapes at
// PK_BY).
constexpr int PACKED_BLOCKS_PER_SM = 3;
constexpr int PACKED_NSTAGE = 2;

// Packed planes per column (multiple of 4) and bytes of one packed field.
int packed_planes(const Geometry &g) { return (g.nk + 1 + 3) & ~3; }
size_t packed_bytes(const Geometry &g) {
  return 16 + (size_t)3 * g.nx * g.ny * packed_planes(g) * 4;
}

// Arguments of the packed contraction; *bulk is set when every field
// buffer suits the bulk-copy kernel (16-byte aligned), which alone takes a
// column range (launch_contract_packed).
eps_status_t prepare_contract_packed(const Geometry &g, int n_lambda, int type,
                                     const void *const *EF, const void *const *EA,
                                     const float (*fs)[3], float *Wm, int *err,
                                     ContractPackedArgs *pa, bool *bulk) {
  std::memset(pa, 0, sizeof(*pa));
  pa->nx = g.nx;
  pa->ny = g.ny;
  pa->k0 = g.k0;
  pa->nk = g.nk;
  pa->np = packed_planes(g);
  pa->nlambda = n_lambda;
  pa->type = type;
  for (int l = 0; l < n_lambda; ++l) {
    pa->EF[l] = (const unsigned char *)EF[l];
    pa->EA[l] = (const unsigned char *)EA[l];
    for (int c = 0; c < 3; ++c) pa->fs[l][c] = fs[l][c];
  }
  pa->W = Wm;
  pa->err = err;
  pa->col_lo = 0;
  pa->col_hi = (long)g.nx * g.ny;
  *bulk = n_lambda > 0;
  for (int l = 0; l < n_lambda; ++l) *bulk = *bulk && aligned(EF[l], 16) && aligned(EA[l], 16);
  return EPS_OK;
}

// The bulk-copy packed contraction over the columns [col_lo, col_hi): a ring
// of PACKED_NSTAGE stages of 6 x PK_BY x 4 np bytes (27.6 KB at nk = 11) in
// PACKED_BLOCKS_PER_SM blocks per SM, about 55 KB per block, so a stencil
// block (34 KB with one eps_hat component staged per round) still fits
// beside the three.
eps_status_t launch_contract_packed(ContractPackedArgs *pa, long col_lo, long col_hi,
                                    cudaStream_t s) {
  int nsm = 0;
  eps_status_t st = sm_count(&nsm);
  if (st != EPS_OK) return st;
  pa->nstage = PACKED_NSTAGE;
  pa->col_lo = col_lo;
  pa->col_hi = col_hi;
  const size_t smem = (size_t)PACKED_NSTAGE * 6 * PK_BY * pa->np * 4 + 128;
  const long nchunks = (col_hi - col_lo + PK_BY - 1) / PK_BY;
  if (nchunks <= 0) return EPS_OK;
  const long blocks = std::max<long>(1, std::min<long>(nchunks, (long)nsm * PACKED_BLOCKS_PER_SM));
  return launch("eps_vjp_contract_packed", contract_packed_bulk_entry(), dim3((unsigned)blocks),
                smem, pa, s, false, PK_THREADS);
}

eps_status_t run_contract_packed(const Geometry &g, int n_lambda, int type, const void *const *EF,
                                 const void *const *EA, const float (*fs)[3], float *Wm, int *err,
                                 cudaStream_t s) {
  ContractPackedArgs pa;
  bool bulk = false;
  eps_status_t st = prepare_contract_packed(g, n_lambda, type, EF, EA, fs, Wm, err, &pa, &bulk);
  if (st != EPS_OK) return st;
  const long ncol = (long)g.nx * g.ny;
  if (bulk) return launch_contract_packed(&pa, 0, ncol, s);
  int nsm = 0;
  if ((st = sm_count(&nsm)) != EPS_OK) return st;
  const long blocks = std::max<long>(1, std::min<long>((ncol + NTHREADS - 1) / NTHREADS, (long)nsm * 8));
  return launch("eps_vjp_contract_packed", contract_packed_entry(), dim3((unsigned)blocks), 0, &pa, s);
}

// seeds = factor * W over the given regions; launched in plain stream order,
// so it starts once the contraction and the stencil have both completed
eps_status_t run_seeds(const SeedsArgs &sa, cudaStream_t s) {
  int nsm = 0;
  eps_status_t st = sm_count(&nsm);
  if (st != EPS_OK) return st;
  if (sa.ncol == 0) return EPS_OK;
  // one thread per column, or per four columns for one region of whole float4
  // rows (a full-occupancy elementwise pass), capped for very large calls
  const long cols = sa.band_hi > 0 ? sa.band_hi - sa.band_lo : sa.ncol;
  if (cols <= 0) return EPS_OK;
  const bool vec = sa.n == 1 && (sa.r[0].ncol & 3) == 0 && (sa.band_lo & 3) == 0 &&
                   (sa.band_hi & 3) == 0;
  const long items = vec ? (cols + 3) / 4 : cols;
  const long blocks = std::max<long>(1, std::min<long>((items + NTHREADS - 1) / NTHREADS, (long)nsm * 64));
  return launch("eps_vjp_seeds", seeds_entry(), dim3((unsigned)blocks), 0, (void *)&sa, s, false);
}

// Launch form of a single-region VJP stencil (one block per tile): where
// the seeds are finished (0: each tile waits for the contraction; 1: the
// seeds kernel) and the eps_hat components staged per round.  Within one
// wave (at most 3 tiles per SM) waiting in the tile saves a launch; larger
// problems defer, so tiles never hold an SM slot while the fields stream.
// (Measured alternatives that lost: a persistent stencil of 2 or 3 blocks
// per SM finishing its seeds after its last tile, and 1-component staging.)
struct StencilForm {
  int defer, stage_comps;   // stage_comps 0: eps_hat by direct coalesced stores
};
constexpr int ONE_WAVE_TILES_PER_SM = 3;
constexpr StencilForm FORM_ONE_WAVE{0, 3};
// Multi-wave problems stage one eps_hat component per round: 32 KB of shared
// memory at nz = 32 instead of 98 KB, so four stencil blocks fit on an SM
// (or some beside the field contraction).  Measured: the 2000 x 2000,
// three-wavelength call 526 -> 519 us, the 3000 x 3000 eight-wavelength
// call 2.41 -> 2.39 ms (FP32) and 1.44 -> 1.23 ms (BF16).  Direct stores
// (stage_comps 0) measured no better in the fused calls (BF16 1.25 ms,
// 600 x 600 call 47.6 against 44.3 us), so the fused forms keep staging.
constexpr StencilForm FORM_MULTI_WAVE{1, 1};
// eps_forward's swizzled staging (nz = 32): eps_hat buffers per block
constexpr int FWD_SWZ_COMPS = 1;

eps_status_t stencil_form(const Geometry &g, StencilForm *f, long *blocks) {
  int nsm = 0;
  const eps_status_t st = sm_count(&nsm);
  if (st != EPS_OK) return st;
  const long tiles = fwd_ntiles(g);
  *f = tiles <= (long)ONE_WAVE_TILES_PER_SM * nsm ? FORM_ONE_WAVE : FORM_MULTI_WAVE;
  *blocks = tiles;
  return EPS_OK;
}

// (band_hi > 0: only the columns [band_lo, band_hi))
eps_status_t run_seeds_one(const Geometry &g, const float *W, float *seeds, int *err,
                           cudaStream_t s, const float *epsc = nullptr, double *S = nullptr,
                           long band_lo = 0, long band_hi = 0) {
  SeedsArgs sa;
  std::memset(&sa, 0, sizeof(sa));
  sa.n = 1;
  sa.ncol = (long)g.nx * g.ny;
  sa.band_lo = band_lo;
  sa.band_hi = band_hi;
  sa.r[0] = SeedsRegion{0, sa.ncol, W, seeds};
  sa.err = err;
  sa.epsc = epsc;
  sa.S = S;
  return run_seeds(sa, s);
}

// Box shapes of the scatter's bulk-copy staging for radius class rp1.
struct ScatterBoxes {
  int dbp, da, nci, ncj, ngj;
};
template <int RP1>
ScatterBoxes scatter_boxes_t(int tbw) {
  if (tbw == 64) {
    using S = BwdSmem<RP1, 64>;
    return ScatterBoxes{S::DBP, S::DA_BOX, S::NCI, S::NCJ, S::NGJ};
  }
  using S = BwdSmem<RP1>;
  return ScatterBoxes{S::DBP, S::DA_BOX, S::NCI, S::NCJ, S::NGJ};
}
ScatterBoxes scatter_boxes(int rp1, int tbw = TB) {
  switch (rp1) {
#define EPSC_BOX_CASE(R) \
  case R:                \
    return scatter_boxes_t<R>(tbw);
    EPSC_BOX_CASE(1) EPSC_BOX_CASE(2) EPSC_BOX_CASE(3) EPSC_BOX_CASE(4) EPSC_BOX_CASE(5)
    EPSC_BOX_CASE(6) EPSC_BOX_CASE(7) EPSC_BOX_CASE(8) EPSC_BOX_CASE(9) EPSC_BOX_CASE(10)
    EPSC_BOX_CASE(11) EPSC_BOX_CASE(12)
#undef EPSC_BOX_CASE
  }
  return ScatterBoxes{0, 0, 0, 0, 0};
}

// Tensor maps of the scatter's staged inputs: P' deps / 4 and 1/eps^2 as
// {my, mx, 1} with a {DBP, DA_BOX, 1} box, the seeds as {ny, nx, NSEED}
// with a box over the six mean seeds and one over the four Sobel seeds
// (one-cell halo).  False when the layout does not suit bulk copies (row
// pitches not multiples of 16 bytes, radius class below 3); the kernel then
// gathers element by element.
bool scatter_maps(const Resolved &r, const float *seeds, const float *pd4, const float *ie2,
                  CUtensorMap *maps, int tbw = TB) {
  PFN_encodeTiled enc = encode_tiled();
  const Geometry &g = r.g;
  if (!enc || r.rp1 < 3 || (g.my & 3) || (g.ny & 3)) return false;
  const ScatterBoxes b = scatter_boxes(r.rp1, tbw);
  cuuint32_t es[3] = {1, 1, 1};
  for (int m = 0; m < 2; ++m) {
    cuuint64_t dims[3] = {(cuuint64_t)g.my, (cuuint64_t)g.mx, 1};
    cuuint64_t strides[2] = {(cuuint64_t)g.my * 4, (cuuint64_t)g.mx * g.my * 4};
    cuuint32_t box[3] = {(cuuint32_t)b.dbp, (cuuint32_t)b.da, 1};
    if (enc(&maps[m], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, (void *)(m == 0 ? pd4 : ie2), dims,
            strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
            CU_TENSOR_MAP_L2_PROMOTION_NONE, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
      return false;
  }
  for (int m = 0; m < 2; ++m) {
    cuuint64_t dims[3] = {(cuuint64_t)g.ny, (cuuint64_t)g.nx, (cuuint64_t)NSEED};
    cuuint64_t strides[2] = {(cuuint64_t)g.ny * 4, (cuuint64_t)g.nx * g.ny * 4};
    cuuint32_t box[3] = {(cuuint32_t)(m == 0 ? b.ncj : b.ngj),
                         (cuuint32_t)(m == 0 ? b.nci : b.nci + 2), (cuuint32_t)(m == 0 ? 6 : 4)};
    if (enc(&maps[2 + m], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, (void *)seeds, dims, strides, box,
            es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
            CU_TENSOR_MAP_L2_PROMOTION_NONE, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
      return false;
  }
  return true;
}

// The scatter over the tile rows [t0, t1) (t1 < 0: to the last row), launched
// with programmatic dependent launch behind the kernel queued ahead of it
// when `pdl`.
eps_status_t run_scatter(const Resolved &r, const float *seeds, const float *pd4, const float *ie2,
                         float *dJdC, int *err, cudaStream_t s, int t0 = 0, int t1 = -1,
                         bool pdl = true) {
  // Bulk-copy staging pays from two waves of tiles up (of the whole grid).
  // Within one wave every block stages at once, and the element-wise copies
  // of all its threads deliver a block's inputs as soon (cfg3: 541 us
  // against 552 us for the call; cfg2 unchanged).
  int nsm = 0;
  eps_status_t st = sm_count(&nsm);
  if (st != EPS_OK) return st;
  const dim3 full = bwd_grid(r.g);
  if (t1 < 0 || t1 > (int)full.y) t1 = (int)full.y;
  if (t0 >= t1) return EPS_OK;
  const dim3 grid(full.x, (unsigned)(t1 - t0));
  if ((long)full.x * full.y > (long)ONE_WAVE_TILES_PER_SM * nsm) {
    const KernelEntry kt = bwd_tma_entry(r.rp1, r.g.bc);
    BwdTmaArgs ta;
    std::memset(&ta, 0, sizeof(ta));
    if (kt.fn && scatter_maps(r, seeds, pd4, ie2, ta.maps)) {
      ta.r.g = r.g;
      ta.r.seeds = seeds;
      ta.r.pd4 = pd4;
      ta.r.ie2 = ie2;
      ta.r.dJdC = dJdC;
      ta.err = err;
      ta.ty0 = t0;
      std::memcpy(ta.w, r.w, sizeof(ta.w));
      return launch("eps_vjp_scatter", kt.fn, grid, kt.smem, &ta, s, pdl);
    }
  }
  BwdArgs ba;
  std::memset(&ba, 0, sizeof(ba));
  ba.r.g = r.g;
  ba.r.seeds = seeds;
  ba.r.pd4 = pd4;
  ba.r.ie2 = ie2;
  ba.r.dJdC = dJdC;
  ba.err = err;
  ba.ty0 = t0;
  std::memcpy(ba.w, r.w, sizeof(ba.w));
  const KernelEntry k = bwd_entry(r.rp1, r.g.bc);
  return launch("eps_vjp_scatter", k.fn, grid, k.smem, &ba, s, pdl);
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
  fa.r.mode = MODE_FWD;
  fa.r.write_eps = 1;
  fa.r.write_offdiag = od ? 1 : 0;
  fa.r.normals3d = (prob->flags & EPS_FLAG_NORMALS_3D) ? 1 : 0;
  fa.r.eps = eps;
  fa.r.offdiag = od ? offdiag : nullptr;
  const KernelEntry k = fwd_entry(r.rp1, r.g.bc);
  // nz = 32: swizzled staging through one buffer (FWD_SWZ_COMPS).
  // Otherwise, more than one wave of tiles: eps_hat leaves by
  // warp-cooperative direct stores (no staging, only the stencil's 31 KB of
  // shared memory); within one wave, one component staged per round.
  // Measured on a GB300, the 2000 x 2000 forward (nz = 32): three
  // components staged plainly 197 us, one 154 us, direct stores 136 us,
  // swizzled staging through one buffer 101 us (two 106 us, three 134 us);
  // the 600 x 600 forward (nz = 24) 19.2 us staged, 21.2 us direct.
  int nsm = 0;
  if ((st = sm_count(&nsm)) != EPS_OK) return st;
  const bool multi = fwd_ntiles(r.g) > (long)ONE_WAVE_TILES_PER_SM * nsm;
  const size_t smem = fwd_eps_output(fa, k, r.g, multi ? 0 : (od ? 5 : 1), FWD_SWZ_COMPS);
  return launch("eps_forward", k.fn, dim3((unsigned)fwd_ntiles(r.g)), smem, &fa, (cudaStream_t)stream);
}

}  // extern "C"

namespace {

// Auxiliary streams of the concurrent grouped form: one set per device,
// created on first use and kept for the process.  A call forks them from the
// caller's stream with an event and joins them back before it returns, so
// ordering against other work on the caller's stream (and graph capture of
// that stream) is kept; the mutex makes the enqueue sequences of calls from
// different host threads, which share the set, follow one another.
// The set also holds the stream and events of the single-region band
// pipeline (vjp_pipelined).
constexpr int AUX_STREAMS = 8;
constexpr int MAX_PIPE_BANDS = 16;
struct AuxSet {
  bool ready = false;
  cudaStream_t st[AUX_STREAMS];
  cudaEvent_t fork, mid, join[AUX_STREAMS], join2[AUX_STREAMS];
  cudaStream_t pipe;
  cudaEvent_t pipe_fork, pipe_join, band[MAX_PIPE_BANDS];
};
std::mutex g_aux_mu;
AuxSet g_aux[64];

eps_status_t aux_set(AuxSet **out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return EPS_ERR_CUDA;
  AuxSet &a = g_aux[dev];
  if (!a.ready) {
    for (int i = 0; i < AUX_STREAMS; ++i) {
      if (cudaStreamCreateWithFlags(&a.st[i], cudaStreamNonBlocking) != cudaSuccess ||
          cudaEventCreateWithFlags(&a.join[i], cudaEventDisableTiming) != cudaSuccess ||
          cudaEventCreateWithFlags(&a.join2[i], cudaEventDisableTiming) != cudaSuccess)
        return EPS_ERR_CUDA;
    }
    if (cudaEventCreateWithFlags(&a.fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&a.mid, cudaEventDisableTiming) != cudaSuccess ||
        cudaStreamCreateWithFlags(&a.pipe, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&a.pipe_fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&a.pipe_join, cudaEventDisableTiming) != cudaSuccess)
      return EPS_ERR_CUDA;
    for (int i = 0; i < MAX_PIPE_BANDS; ++i)
      if (cudaEventCreateWithFlags(&a.band[i], cudaEventDisableTiming) != cudaSuccess)
        return EPS_ERR_CUDA;
    a.ready = true;
  }
  *out = &a;
  return EPS_OK;
}

// Every stream in `waiters` waits for the work enqueued so far on `s`.
eps_status_t fork_streams(cudaStream_t s, cudaEvent_t ev, const cudaStream_t *waiters, int n) {
  if (cudaEventRecord(ev, s) != cudaSuccess) return EPS_ERR_CUDA;
  for (int i = 0; i < n; ++i)
    if (cudaStreamWaitEvent(waiters[i], ev, 0) != cudaSuccess) return EPS_ERR_CUDA;
  return EPS_OK;
}

// `s` waits for the work enqueued so far on every stream in `workers`.
eps_status_t join_streams(cudaStream_t s, const cudaEvent_t *evs, const cudaStream_t *workers,
                          int n) {
  for (int i = 0; i < n; ++i) {
    if (cudaEventRecord(evs[i], workers[i]) != cudaSuccess) return EPS_ERR_CUDA;
    if (cudaStreamWaitEvent(s, evs[i], 0) != cudaSuccess) return EPS_ERR_CUDA;
  }
  return EPS_OK;
}

// Argument checks of eps_vjp (everything but the problem itself, which
// `r` already resolved); *skip is set for an empty problem.
eps_status_t vjp_args(const Resolved &r, const float *C, int32_t n_lambda, int32_t field_type,
                      const void *const *EF, const void *const *EA, const float *field_scales,
                      float scale, const float *dJdC, const float *eps_out, const void *ws,
                      size_t ws_bytes, bool *skip) {
  *skip = false;
  if (r.normals3d) return EPS_ERR_UNSUPPORTED;   // forward only
  if (n_lambda < 0 || n_lambda > EPS_MAX_LAMBDA) return EPS_ERR_INVALID_ARG;
  if (field_type != EPS_FIELD_C64 && field_type != EPS_FIELD_BF16X2_SCALED &&
      field_type != EPS_FIELD_F16X2_SCALED)
    return EPS_ERR_INVALID_ARG;
  if (!std::isfinite(scale)) return EPS_ERR_INVALID_ARG;
  if (r.empty) {
    *skip = true;
    return EPS_OK;
  }
  if (!C || !dJdC) return EPS_ERR_INVALID_ARG;
  if (n_lambda > 0 && (!EF || !EA)) return EPS_ERR_INVALID_ARG;
  for (int l = 0; l < n_lambda; ++l) {
    if (!EF[l] || !EA[l]) return EPS_ERR_INVALID_ARG;
    if (!aligned(EF[l], 16) || !aligned(EA[l], 16)) return EPS_ERR_INVALID_ARG;
  }
  if (field_scales)
    for (int t = 0; t < 6 * n_lambda; ++t)
      if (!std::isfinite(field_scales[t])) return EPS_ERR_INVALID_ARG;
  if (field_type == EPS_FIELD_C64 && (r.g.nz & 1)) return EPS_ERR_SHAPE;   // planes read in pairs
  if (!aligned(C, 4) || !aligned(dJdC, 4) || (eps_out && !aligned(eps_out, 16)))
    return EPS_ERR_INVALID_ARG;
  if (!ws || !aligned(ws, 256) || ws_bytes < workspace_bytes(r.g)) return EPS_ERR_WORKSPACE;
  return EPS_OK;
}

}  // namespace

namespace {

// Band pipeline of a multi-wave single-region call (edge-replicate rule,
// complex64 fields through the bulk-copy contraction).  The contraction
// runs band by band (consecutive column ranges) on the caller's stream; a
// pipeline stream runs the stencil alongside, then, as each band's column
// sums complete, that band's seeds and the scatter of every tile row whose
// seed maps are complete.  All but the last band's seeds and scatter then
// overlap the field stream instead of following it.
//
// Measured on a GB300 (L2 flushed, one box, medians; 0 bands = the
// single-stream order):
//   bands                     0      3      4      5      6      8
//   3000 x 3000, 8 lambda  2427   2373   2371   2364   2367   2345-2347 (another box: 0 -> 2415)
//   2000 x 2000, 3 lambda   516    501    514    524    533    561
// Each band boundary costs a contraction tail and ramp, and queued stencil
// or scatter blocks take the slots the next band's blocks would get; the
// shorter three-wavelength stream pays for that first.  Tried and not
// kept: the contraction bands on a stream of the highest priority (2494 us
// at 4 bands), the stencil as a persistent grid of two blocks per SM
// (2377 / 508 us at 4 bands).
// Packed (BF16 / FP16) fields keep the single-stream order: banding their
// contraction (chunks of 128 columns) measured 1.171 -> 1.257 ms at the
// 3000 x 3000, eight-wavelength call, whose shorter field stream leaves less
// to hide and more to lose at each boundary.
// Cumulative share of the contraction's rounds at each band's end.  Uneven
// splits moved the two workloads apart by about 1 % either way (one box:
// 0.5 / 0.85 / 1: 3000 x 3000 2372 us, 2000 x 2000 514 us; 0.6 / 1: 2393 /
// 501 us; 0.35 / 0.65 / 0.87 / 1: 2379 / 512 us; equal thirds 2394 / 505
// us), so the bands stay equal.
constexpr double PIPE_SPLIT[] = {1.0 / 3, 2.0 / 3, 1.0};
constexpr int PIPE_NSPLIT = (int)(sizeof(PIPE_SPLIT) / sizeof(double));
static_assert(PIPE_NSPLIT <= MAX_PIPE_BANDS, "band events");

// Highest Yee row of the seed maps that scatter tile row t reads, its
// bulk-copy boxes included (edge-replicate rule: no wrap).
int scatter_seed_row_hi(const Resolved &r, int t) {
  const int R = r.rp1 - 1;
  const int ga_lo = TA * t - (t == 0 ? R : 0);   // the fold halo of the first row
  const int da_lo = ga_lo - R;
  const int ci_lo = da_lo >= 0 ? da_lo / 2 : -((1 - da_lo) / 2);   // floor(da_lo / 2)
  return ci_lo + scatter_boxes(r.rp1).nci;
}

struct PipeCall {
  const Resolved *r;
  ContractTmaArgs *ta;          // prepared contraction (every column)
  FwdArgs *fa;                  // stencil arguments (seed factors: defer form)
  KernelEntry kf;
  size_t fsmem;
  long fblocks;
  const char *fname;
  float *W, *seeds, *pd4, *ie2, *dJdC, *epsc;
  double *S;
  int *err;
};

eps_status_t vjp_pipelined(const PipeCall &c, cudaStream_t s) {
  const Resolved &r = *c.r;
  const Geometry &g = r.g;
  int nsm = 0;
  eps_status_t st = sm_count(&nsm);
  if (st != EPS_OK) return st;
  std::lock_guard<std::mutex> lk(g_aux_mu);
  AuxSet *aux = nullptr;
  if ((st = aux_set(&aux)) != EPS_OK) return st;
  // Bands of whole rounds of the contraction grid (one chunk per block and
  // round), so every block of a band has the same number of chunks.
  const long ncol = (long)g.nx * g.ny;
  const long chunk_cols = TMA_BY;
  const long nchunks = (ncol + chunk_cols - 1) / chunk_cols;
  const long per_round = (long)nsm * CONTRACT_BLOCKS_PER_SM;
  const long rounds = (nchunks + per_round - 1) / per_round;
  const int nb = (int)std::max<long>(1, std::min<long>(PIPE_NSPLIT, rounds));
  auto band_end = [&](int b) {   // first round after band b
    if (b >= nb - 1) return rounds;
    if (nb < PIPE_NSPLIT) return rounds * (b + 1) / nb;
    return std::min(rounds, std::max<long>(b + 1, (long)(rounds * PIPE_SPLIT[b] + 0.5)));
  };
  const int T = (int)bwd_grid(g).y;

  if (cudaEventRecord(aux->pipe_fork, s) != cudaSuccess ||
      cudaStreamWaitEvent(aux->pipe, aux->pipe_fork, 0) != cudaSuccess)
    return EPS_ERR_CUDA;
  auto bands = [&]() -> eps_status_t {
    int t_done = 0;
    for (int b = 0; b < nb; ++b) {
      const long lo = b == 0 ? 0 : std::min(ncol, band_end(b - 1) * per_round * chunk_cols);
      const long hi = b == nb - 1 ? ncol : std::min(ncol, band_end(b) * per_round * chunk_cols);
      if ((st = launch_contract_tma(c.ta, lo, hi, s)) != EPS_OK) return st;
      if (cudaEventRecord(aux->band[b], s) != cudaSuccess) return EPS_ERR_CUDA;
      if (b == 0 && (st = launch(c.fname, c.kf.fn, dim3((unsigned)c.fblocks), c.fsmem, c.fa,
                                 aux->pipe, false)) != EPS_OK)
        return st;
      if (cudaStreamWaitEvent(aux->pipe, aux->band[b], 0) != cudaSuccess) return EPS_ERR_CUDA;
      if ((st = run_seeds_one(g, c.W, c.seeds, c.err, aux->pipe, c.S ? c.epsc : nullptr, c.S, lo,
                              hi)) != EPS_OK)
        return st;
      // tile rows whose seed rows (all below the first incomplete Yee row) are done
      int t_ready = T;
      if (b < nb - 1) {
        const long rows_done = hi / g.ny;
        t_ready = t_done;
        while (t_ready < T && scatter_seed_row_hi(r, t_ready) < rows_done) ++t_ready;
      }
      if (t_ready > t_done) {
        if ((st = run_scatter(r, c.seeds, c.pd4, c.ie2, c.dJdC, c.err, aux->pipe, t_done, t_ready,
                              false)) != EPS_OK)
          return st;
        t_done = t_ready;
      }
    }
    return EPS_OK;
  };
  st = bands();
  // joined back even after a failed enqueue, so that work queued on `s`
  // later never runs ahead of pipeline work already queued
  const bool joined = cudaEventRecord(aux->pipe_join, aux->pipe) == cudaSuccess &&
                      cudaStreamWaitEvent(s, aux->pipe_join, 0) == cudaSuccess;
  if (st != EPS_OK) return st;
  return joined ? EPS_OK : EPS_ERR_CUDA;
}

// The fused forward + Eq. 1 VJP of eps_vjp; with S non-null also the
// surrogate S = sum over the J-support voxels of eps_hat * w (zeroed here,
// accumulated by the stencil or the seeds kernel).
eps_status_t vjp_fused(const eps_problem_t *prob, const float *C, int32_t n_lambda,
                       int32_t field_type, const void *const *EF, const void *const *EA,
                       const float *field_scales, float scale, float *dJdC, float *eps_out,
                       double *S, void *ws, size_t ws_bytes, cudaStream_t s) {
  Resolved r;
  eps_status_t st = resolve(prob, &r);
  if (st != EPS_OK) return st;
  bool skip = false;
  st = vjp_args(r, C, n_lambda, field_type, EF, EA, field_scales, scale, dJdC, eps_out, ws,
                ws_bytes, &skip);
  if (st != EPS_OK) return st;
  if (S && cudaMemsetAsync(S, 0, sizeof(double), s) != cudaSuccess) return EPS_ERR_CUDA;
  if (skip) return EPS_OK;
  int *err = nullptr;
  if ((st = error_flag_ptr(&err)) != EPS_OK) return st;

  const WsLayout L = ws_layout(r.g);
  float *Wm = (float *)((char *)ws + L.w);
  float *seeds = (float *)((char *)ws + L.seeds);
  float *pd4 = (float *)((char *)ws + L.pd4);
  float *ie2 = (float *)((char *)ws + L.ie2);
  float *epsc = (float *)((char *)ws + L.epsc);

  // Eq. 1 column sums: per-wavelength scales of the components
  ContractArgs ca;
  std::memset(&ca, 0, sizeof(ca));
  ca.nx = r.g.nx;
  ca.ny = r.g.ny;
  ca.nz = r.g.nz;
  ca.k0 = r.g.k0;
  ca.nk = r.g.nk;
  ca.nlambda = n_lambda;
  ca.mode = MODE_C64;
  ca.err = err;
  ca.W = Wm;
  bool sector_ok = (r.g.nz & 3) == 0;
  for (int l = 0; l < n_lambda; ++l) {
    ca.EF[l] = (const float *)EF[l];
    ca.EA[l] = (const float *)EA[l];
    sector_ok = sector_ok && aligned(EF[l], 32) && aligned(EA[l], 32);
    for (int c = 0; c < 3; ++c) {
      float sc = scale;
      if (field_scales) sc *= field_scales[(l * 2 + 0) * 3 + c] * field_scales[(l * 2 + 1) * 3 + c];
      ca.fs[l][c] = sc;
    }
  }

  // forward chain + seeds (overlaps the contraction until it needs W)
  FwdArgs fa;
  fill_fwd_common(fa, r, C, err);
  fa.r.mode = MODE_C64;
  fa.r.write_eps = eps_out ? 1 : 0;
  fa.r.eps = eps_out;
  fa.r.W = Wm;
  fa.r.seeds = seeds;
  StencilForm form;
  long blocks = 0;
  if ((st = stencil_form(r.g, &form, &blocks)) != EPS_OK) return st;
  fa.r.defer_seeds = form.defer;
  fa.r.pd4 = pd4;
  fa.r.ie2 = ie2;
  if (S) {
    fa.r.S = form.defer ? nullptr : S;
    fa.r.epsc = form.defer ? epsc : nullptr;
  }
  const KernelEntry kf = fwd_entry(r.rp1, r.g.bc);
  const size_t smem = eps_out ? fwd_eps_output(fa, kf, r.g, std::min(3, form.stage_comps),
                                                form.stage_comps)
                              : fwd_smem(kf, r.g, 0, &fa.r.stage_floats);
  const char *fname = eps_out ? "eps_fwd_vjp_stencil" : "eps_vjp_stencil";

  // (profiling runs the kernels one after another, so each event pair
  // times one kernel alone)
  bool prof = false;
  {
    std::lock_guard<std::mutex> lk(g_prof_mu);
    prof = g_prof_on;
  }
  if (PIPE_NSPLIT > 1 && !prof && n_lambda > 0 && form.defer == 1 && r.g.bc == EPS_BC_CLAMP) {
    if (field_type == EPS_FIELD_C64) {
      std::unique_ptr<ContractTmaArgs> ta(new ContractTmaArgs);
      st = prepare_contract_tma(r.g, n_lambda, EF, EA, ca.fs, Wm, err, ta.get());
      if (st == EPS_OK) {
        PipeCall pc{&r, ta.get(), &fa, kf, smem, blocks, fname, Wm, seeds, pd4, ie2, dJdC, epsc,
                    S, err};
        return vjp_pipelined(pc, s);
      }
      if (st != EPS_ERR_UNSUPPORTED) return st;
    }
  }

  // 1. Eq. 1 column sums (streaming over the J-support planes)
  if (field_type == EPS_FIELD_C64) {
    st = (n_lambda > 0) ? run_contract_tma(r.g, n_lambda, EF, EA, ca.fs, Wm, err, s)
                        : EPS_ERR_UNSUPPORTED;
    if (st == EPS_ERR_UNSUPPORTED) st = run_contract(ca, sector_ok ? 4 : 8, s);
  } else {
    st = run_contract_packed(r.g, n_lambda, field_type, EF, EA, ca.fs, Wm, err, s);
  }
  if (st != EPS_OK) return st;
  // 2. the stencil, with programmatic dependent launch behind the contraction
  st = launch(fname, kf.fn, dim3((unsigned)blocks), smem, &fa, s, true);
  if (st != EPS_OK) return st;
  // 3. (seeds-kernel form) seeds = factor * W, once both grids are done
  if (form.defer == 1 &&
      (st = run_seeds_one(r.g, Wm, seeds, err, s, S ? epsc : nullptr, S)) != EPS_OK)
    return st;
  // 4. transposes down to dJ/dC
  return run_scatter(r, seeds, pd4, ie2, dJdC, err, s);
}

}  // namespace

extern "C" {

eps_status_t eps_vjp(const eps_problem_t *prob, const float *C, int32_t n_lambda,
                     int32_t field_type, const void *const *EF, const void *const *EA,
                     const float *field_scales, float scale, float *dJdC, float *eps_out,
                     void *ws, size_t ws_bytes, eps_stream_t stream) {
  return vjp_fused(prob, C, n_lambda, field_type, EF, EA, field_scales, scale, dJdC, eps_out,
                   nullptr, ws, ws_bytes, (cudaStream_t)stream);
}

eps_status_t eps_vjp_surrogate(const eps_problem_t *prob, const float *C, int32_t n_lambda,
                               int32_t field_type, const void *const *EF, const void *const *EA,
                               const float *field_scales, float scale, float *dJdC,
                               float *eps_out, double *S, void *ws, size_t ws_bytes,
                               eps_stream_t stream) {
  if (!S || !aligned(S, 8)) return EPS_ERR_INVALID_ARG;
  return vjp_fused(prob, C, n_lambda, field_type, EF, EA, field_scales, scale, dJdC, eps_out, S,
                   ws, ws_bytes, (cudaStream_t)stream);
}

eps_status_t eps_vjp_real(const eps_problem_t *prob, const float *C, const float *G, float *dJdC,
                          void *ws, size_t ws_bytes, eps_stream_t stream) {
  Resolved r;
  eps_status_t st = resolve(prob, &r);
  if (st != EPS_OK) return st;
  if (r.normals3d) return EPS_ERR_UNSUPPORTED;   // forward only
  if (r.empty) return EPS_OK;
  if (!C || !G || !dJdC) return EPS_ERR_INVALID_ARG;
  if (!aligned(C, 4) || !aligned(G, 4) || !aligned(dJdC, 4)) return EPS_ERR_INVALID_ARG;
  if (!ws || !aligned(ws, 256) || ws_bytes < workspace_bytes(r.g)) return EPS_ERR_WORKSPACE;
  int *err = nullptr;
  if ((st = error_flag_ptr(&err)) != EPS_OK) return st;
  const WsLayout L = ws_layout(r.g);
  float *Wm = (float *)((char *)ws + L.w);
  float *seeds = (float *)((char *)ws + L.seeds);
  float *pd4 = (float *)((char *)ws + L.pd4);
  float *ie2 = (float *)((char *)ws + L.ie2);
  cudaStream_t s = (cudaStream_t)stream;
  ContractArgs ca;
  std::memset(&ca, 0, sizeof(ca));
  ca.nx = r.g.nx;
  ca.ny = r.g.ny;
  ca.nz = r.g.nz;
  ca.k0 = r.g.k0;
  ca.nk = r.g.nk;
  ca.mode = MODE_REAL;
  ca.err = err;
  ca.G = G;
  ca.W = Wm;
  st = run_contract_tma_real(r.g, G, Wm, err, s);
  if (st == EPS_ERR_UNSUPPORTED) st = run_contract(ca, 8, s);
  if (st != EPS_OK) return st;
  FwdArgs fa;
  fill_fwd_common(fa, r, C, err);
  fa.r.mode = MODE_REAL;
  fa.r.W = Wm;
  fa.r.seeds = seeds;
  StencilForm form;
  long blocks = 0;
  if ((st = stencil_form(r.g, &form, &blocks)) != EPS_OK) return st;
  fa.r.defer_seeds = form.defer;
  fa.r.pd4 = pd4;
  fa.r.ie2 = ie2;
  const KernelEntry kf = fwd_entry(r.rp1, r.g.bc);
  const size_t smem = fwd_smem(kf, r.g, 0, &fa.r.stage_floats);
  st = launch("eps_vjp_real_stencil", kf.fn, dim3((unsigned)blocks), smem, &fa, s, true);
  if (st != EPS_OK) return st;
  if (form.defer == 1 && (st = run_seeds_one(r.g, Wm, seeds, err, s)) != EPS_OK) return st;
  return run_scatter(r, seeds, pd4, ie2, dJdC, err, s);
}

eps_status_t eps_packed_field_bytes(const eps_problem_t *prob, int32_t field_type,
                                    size_t *bytes) {
  if (!bytes) return EPS_ERR_INVALID_ARG;
  if (field_type != EPS_FIELD_BF16X2_SCALED && field_type != EPS_FIELD_F16X2_SCALED)
    return EPS_ERR_INVALID_ARG;
  Resolved r;
  eps_status_t st = resolve(prob, &r);
  if (st != EPS_OK) return st;
  *bytes = r.empty ? 0 : packed_bytes(r.g);
  return EPS_OK;
}

eps_status_t eps_field_pack(const eps_problem_t *prob, int32_t field_type, const void *src,
                            void *dst, size_t dst_bytes, eps_stream_t stream) {
  if (field_type != EPS_FIELD_BF16X2_SCALED && field_type != EPS_FIELD_F16X2_SCALED)
    return EPS_ERR_INVALID_ARG;
  Resolved r;
  eps_status_t st = resolve(prob, &r);
  if (st != EPS_OK) return st;
  if (r.empty) return EPS_OK;
  if (!src || !dst) return EPS_ERR_INVALID_ARG;
  if (!aligned(src, 8) || !aligned(dst, 16)) return EPS_ERR_INVALID_ARG;
  if (dst_bytes < packed_bytes(r.g)) return EPS_ERR_WORKSPACE;
  cudaStream_t s = (cudaStream_t)stream;
  PackArgs pa;
  std::memset(&pa, 0, sizeof(pa));
  pa.nx = r.g.nx;
  pa.ny = r.g.ny;
  pa.nz = r.g.nz;
  pa.k0 = r.g.k0;
  pa.nk = r.g.nk;
  pa.np = packed_planes(r.g);
  pa.type = field_type;
  pa.src = (const float2 *)src;
  pa.dst = (unsigned char *)dst;
  if ((st = error_flag_ptr(&pa.err)) != EPS_OK) return st;
  int nsm = 0;
  if ((st = sm_count(&nsm)) != EPS_OK) return st;
  if (cudaMemsetAsync(dst, 0, 16, s) != cudaSuccess) return EPS_ERR_CUDA;
  if ((st = launch("eps_field_pack_amax", pack_amax_entry(), dim3((unsigned)nsm * 2, 3), 0, &pa,
                   s)) != EPS_OK)
    return st;
  if ((st = launch("eps_field_pack", pack_entry(), dim3((unsigned)nsm * 8), 0, &pa, s)) != EPS_OK)
    return st;
  unsigned char *d = (unsigned char *)dst;
  void *args[] = {&d, &pa.type};
  if (cudaLaunchKernel(pack_finish_entry(), dim3(1), dim3(32), args, 0, s) != cudaSuccess)
    return EPS_ERR_CUDA;
  g_launch_count.fetch_add(1, std::memory_order_relaxed);
  return EPS_OK;
}

eps_status_t eps_sync_status(eps_stream_t stream) {
  if (cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess) return EPS_ERR_CUDA;
  int flag = 0;
  if (cudaMemcpyFromSymbol(&flag, g_eps_error_flag, sizeof(int)) != cudaSuccess)
    return EPS_ERR_CUDA;
  if (flag == 0) return EPS_OK;
  const int zero = 0;
  if (cudaMemcpyToSymbol(g_eps_error_flag, &zero, sizeof(int)) != cudaSuccess) return EPS_ERR_CUDA;
  return (flag & ERRFLAG_TIMEOUT) ? EPS_ERR_DEVICE_TIMEOUT : EPS_ERR_DEVICE_BOUNDS;
}

eps_status_t eps_selftest_timeout(int64_t cycles, eps_stream_t stream) {
  if (cycles < 1 || cycles > (1ll << 31)) return EPS_ERR_INVALID_ARG;
  SelftestArgs a;
  eps_status_t st = error_flag_ptr(&a.err);
  if (st != EPS_OK) return st;
  a.cycles = (long long)cycles;
  return launch("eps_selftest_timeout", selftest_timeout_entry(), dim3(1), 0, &a,
                (cudaStream_t)stream);
}

eps_status_t eps_selftest_bounds(eps_stream_t stream) {
#ifdef EPS_DEBUG_BOUNDS
  SelftestArgs a;
  eps_status_t st = error_flag_ptr(&a.err);
  if (st != EPS_OK) return st;
  a.cycles = 0;
  return launch("eps_selftest_bounds", selftest_bounds_entry(), dim3(1), 0, &a,
                (cudaStream_t)stream);
#else
  (void)stream;
  return EPS_ERR_UNSUPPORTED;
#endif
}

eps_status_t eps_set_l2_fetch_granularity(int32_t bytes, int32_t *previous) {
  if (bytes < 0 || bytes > 128) return EPS_ERR_INVALID_ARG;
  size_t old = 0;
  if (cudaDeviceGetLimit(&old, cudaLimitMaxL2FetchGranularity) != cudaSuccess) return EPS_ERR_CUDA;
  if (previous) *previous = (int32_t)old;
  if (cudaDeviceSetLimit(cudaLimitMaxL2FetchGranularity, (size_t)bytes) != cudaSuccess)
    return EPS_ERR_CUDA;
  return EPS_OK;
}

eps_status_t eps_launch_count(uint64_t *count) {
  if (!count) return EPS_ERR_INVALID_ARG;
  *count = g_launch_count.load(std::memory_order_relaxed);
  return EPS_OK;
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

// ------------------------------------------------------------- batched calls

namespace {

// Launch shapes of a batched call.  Two launch forms:
//  * multi:   one mixed-radius persistent stencil launch and one scatter
//             launch per boundary rule (`fwd_bps` / `bwd_bps` blocks per SM
//             walk the tile list, heaviest radius class first);
//  * grouped: one stencil and one scatter launch per (radius, boundary
//             rule) group, one block per tile.
// eps_autotune_batched times these choices on the caller's batch and caches
// the fastest per batch signature; other calls use the cache or the default.
struct BatchTuning {
  int multi;          // 1: multi form, 0: grouped form
  int fwd_bps;        // persistent stencil blocks per SM (multi form)
  int bwd_bps;        // persistent scatter blocks per SM (multi form)
  int contract_bps;   // batched contraction blocks per SM (TMA form; 4x for register loads)
  int stage_comps;    // eps_hat components staged per round of bulk stores (1 or 3)
  int defer_seeds;    // 1: stencil writes seed factors, the seeds kernel applies W
  int bwd_bulk;       // grouped form: 1 = the scatter stages interior tiles by bulk copies
  int bwd_cols;       // grouped form: scatter tile width in subpixels (32 or 64)
  int group_streams;  // grouped form: 1 = each radius group's launches on a stream of its own
};
// Default: the grouped form, measured faster on the 64-region batch (radius
// classes 2 .. 8): one kernel holding all twelve radius bodies runs them side
// by side on an SM and lost to per-class launches there.  Three TMA
// contraction blocks per SM streamed that batch's fields in 304 us against
// 368 us with two; one eps_hat component per staging round took the call
// from 0.916 to 0.897 ms.
constexpr BatchTuning DEFAULT_TUNING{0, 3, 3, 3, 1, 0, 1, TB, 0};
// The TMA contraction's ring (2 stages of up to 6 x 32 x 64 floats) leaves
// room for at most this many blocks per SM.
constexpr int TMA_BATCH_MAX_BPS = 4;

std::mutex g_tune_mu;
std::vector<std::pair<uint64_t, BatchTuning>> g_tune;   // small: one entry per tuned batch

uint64_t batch_signature(int32_t n, const eps_problem_t *probs, int32_t n_lambda) {
  uint64_t h = 1469598103934665603ull;   // FNV-1a over the problem structs
  auto mix = [&](const void *p, size_t bytes) {
    const unsigned char *c = (const unsigned char *)p;
    for (size_t i = 0; i < bytes; ++i) h = (h ^ c[i]) * 1099511628211ull;
  };
  mix(&n, sizeof(n));
  mix(&n_lambda, sizeof(n_lambda));
  for (int k = 0; k < n; ++k) mix(&probs[k], sizeof(eps_problem_t));
  return h;
}

BatchTuning lookup_tuning(uint64_t sig) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  for (const auto &e : g_tune)
    if (e.first == sig) return e.second;
  return DEFAULT_TUNING;
}

void store_tuning(uint64_t sig, const BatchTuning &t) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  for (auto &e : g_tune)
    if (e.first == sig) {
      e.second = t;
      return;
    }
  g_tune.push_back({sig, t});
}

// Regions that share one conic filter and boundary rule (grouped form).
struct Group {
  int rp1, bc;
  float radius;
  std::vector<int> regions;   // indices, largest tile count first
};

eps_status_t resolve_batch(int32_t n, const eps_problem_t *probs, std::vector<Resolved> &rs,
                           std::vector<size_t> &ws_off, size_t *ws_total) {
  if (n < 0 || n > EPS_MAX_BATCH || (n > 0 && !probs)) return EPS_ERR_INVALID_ARG;
  rs.resize(n);
  ws_off.resize(n);
  size_t off = 0;
  for (int k = 0; k < n; ++k) {
    eps_status_t st = resolve(&probs[k], &rs[k]);
    if (st != EPS_OK) return st;
    if (rs[k].normals3d) return EPS_ERR_UNSUPPORTED;   // single-region forward only
    ws_off[k] = off;
    off += rs[k].empty ? 0 : workspace_bytes(rs[k].g);
  }
  *ws_total = off;
  return EPS_OK;
}

long fwd_tiles(const Resolved &r) { return (long)fwd_grid(r.g).x * fwd_grid(r.g).y; }

std::vector<Group> make_groups(const std::vector<Resolved> &rs, const eps_problem_t *probs) {
  std::vector<Group> gs;
  for (int k = 0; k < (int)rs.size(); ++k) {
    if (rs[k].empty) continue;
    size_t gi = 0;
    for (; gi < gs.size(); ++gi)
      if (gs[gi].rp1 == rs[k].rp1 && gs[gi].bc == rs[k].g.bc && gs[gi].radius == probs[k].radius)
        break;
    if (gi == gs.size()) gs.push_back(Group{rs[k].rp1, rs[k].g.bc, probs[k].radius, {}});
    gs[gi].regions.push_back(k);
  }
  for (Group &g : gs)
    std::stable_sort(g.regions.begin(), g.regions.end(),
                     [&](int x, int y) { return fwd_tiles(rs[x]) > fwd_tiles(rs[y]); });
  return gs;
}

// Launch sets of the multi form: one boundary rule, at most one radius per
// radius class; regions ordered heaviest class first, then largest first.
struct LaunchSet {
  int bc;
  float radius_of[MAX_RP1 + 1];   // radius of each class present, 0 if absent
  std::vector<int> regions;
};

std::vector<LaunchSet> make_sets(const std::vector<Resolved> &rs, const eps_problem_t *probs) {
  std::vector<LaunchSet> sets;
  for (int k = 0; k < (int)rs.size(); ++k) {
    if (rs[k].empty) continue;
    const int c = rs[k].rp1;
    size_t si = 0;
    for (; si < sets.size(); ++si)
      if (sets[si].bc == rs[k].g.bc &&
          (sets[si].radius_of[c] == 0.f || sets[si].radius_of[c] == probs[k].radius))
        break;
    if (si == sets.size()) {
      LaunchSet ls;
      ls.bc = rs[k].g.bc;
      for (float &r : ls.radius_of) r = 0.f;
      sets.push_back(ls);
    }
    sets[si].radius_of[c] = probs[k].radius;
    sets[si].regions.push_back(k);
  }
  for (LaunchSet &ls : sets)
    std::stable_sort(ls.regions.begin(), ls.regions.end(), [&](int x, int y) {
      if (rs[x].rp1 != rs[y].rp1) return rs[x].rp1 > rs[y].rp1;
      return fwd_tiles(rs[x]) > fwd_tiles(rs[y]);
    });
  return sets;
}

// Grouped form: one batched stencil launch per group.
// gstreams (optional): the stream of each group's launch (concurrent form)
eps_status_t run_fwd_grouped(const std::vector<Group> &gs, const std::vector<Resolved> &rs,
                             const std::vector<FwdRegion> &regions, int ncomp, int *err,
                             cudaStream_t s, bool pdl,
                             const std::vector<cudaStream_t> *gstreams = nullptr) {
  FwdBatchArgs *ba = new FwdBatchArgs;
  eps_status_t st = EPS_OK;
  for (size_t gi = 0; gi < gs.size(); ++gi) {
    const Group &g = gs[gi];
    const cudaStream_t gst = gstreams ? (*gstreams)[gi] : s;
    std::memset(ba, 0, sizeof(*ba));
    ba->n = (int)g.regions.size();
    ba->err = err;
    std::memcpy(ba->w, rs[g.regions[0]].w, sizeof(ba->w));
    const KernelEntry k = fwd_entry(g.rp1, g.bc, true);
    size_t smem = 0;
    int tiles = 0;
    for (int q = 0; q < ba->n; ++q) {
      const int ri = g.regions[q];
      int sf = 0;
      smem = std::max(smem, fwd_smem(k, rs[ri].g, ncomp, &sf));
      const dim3 grid = fwd_grid(rs[ri].g);
      ba->tile_start[q] = tiles;
      ba->tiles_j[q] = (int)grid.x;
      tiles += (int)(grid.x * grid.y);
      ba->r[q] = regions[ri];
    }
    ba->tile_start[ba->n] = tiles;
    for (int q = 0; q < ba->n; ++q) ba->r[q].stage_floats = (int)(smem / sizeof(float));
    st = launch("eps_batched_stencil", k.fn, dim3((unsigned)tiles), smem, ba, gst,
                pdl && !gstreams);
    if (st != EPS_OK) break;
  }
  delete ba;
  return st;
}

// One scatter launch per group whose interior tiles stage through bulk
// tensor copies: at most BWD_TMA_BATCH regions a launch, each region's four
// maps in the parameters (regions whose layout does not suit bulk copies
// gather element by element inside the same launch).
static_assert(sizeof(BwdTmaBatchArgs) <= 32764, "kernel parameter space");
eps_status_t run_bwd_group_bulk(const Group &g, const std::vector<Resolved> &rs,
                                const std::vector<BwdRegion> &regions, const KernelEntry &k,
                                int tbw, int *err, cudaStream_t s, bool pdl) {
  std::unique_ptr<BwdTmaBatchArgs> ta(new BwdTmaBatchArgs);
  eps_status_t st = EPS_OK;
  for (size_t q0 = 0; q0 < g.regions.size() && st == EPS_OK; q0 += BWD_TMA_BATCH) {
    const int cnt = (int)std::min<size_t>(BWD_TMA_BATCH, g.regions.size() - q0);
    std::memset(ta.get(), 0, sizeof(*ta));
    ta->n = cnt;
    ta->err = err;
    std::memcpy(ta->w, rs[g.regions[q0]].w, sizeof(ta->w));
    int tiles = 0;
    for (int q = 0; q < cnt; ++q) {
      const int ri = g.regions[q0 + q];
      const BwdRegion &br = regions[ri];
      const dim3 grid = bwd_grid(rs[ri].g, tbw);
      ta->tile_start[q] = tiles;
      ta->tiles_j[q] = (int)grid.x;
      tiles += (int)(grid.x * grid.y);
      ta->r[q] = br;
      ta->has_maps[q] =
          scatter_maps(rs[ri], br.seeds, br.pd4, br.ie2, &ta->maps[4 * q], tbw) ? 1 : 0;
    }
    ta->tile_start[cnt] = tiles;
    st = launch("eps_batched_scatter", k.fn, dim3((unsigned)tiles), k.smem, ta.get(), s, pdl);
  }
  return st;
}

// tbw: scatter tile width in subpixels (TB, or 64: wide tiles, fewer
// halo subpixels per output at two blocks per SM instead of three)
eps_status_t run_bwd_grouped(const std::vector<Group> &gs, const std::vector<Resolved> &rs,
                             const std::vector<BwdRegion> &regions, int bulk, int tbw, int *err,
                             cudaStream_t s,
                             const std::vector<cudaStream_t> *gstreams = nullptr) {
  BwdBatchArgs *ba = new BwdBatchArgs;
  eps_status_t st = EPS_OK;
  const bool wide = tbw == 64;
  for (size_t gi = 0; gi < gs.size(); ++gi) {
    const Group &g = gs[gi];
    const cudaStream_t gst = gstreams ? (*gstreams)[gi] : s;
    if (bulk) {
      const KernelEntry kb =
          wide ? bwd_tma_batched_wide_entry(g.rp1, g.bc) : bwd_tma_batched_entry(g.rp1, g.bc);
      if (kb.fn) {
        st = run_bwd_group_bulk(g, rs, regions, kb, tbw, err, gst, !gstreams);
        if (st != EPS_OK) break;
        continue;
      }
    }
    std::memset(ba, 0, sizeof(*ba));
    ba->n = (int)g.regions.size();
    ba->err = err;
    std::memcpy(ba->w, rs[g.regions[0]].w, sizeof(ba->w));
    const KernelEntry k = wide ? bwd_batched_wide_entry(g.rp1, g.bc) : bwd_entry(g.rp1, g.bc, true);
    int tiles = 0;
    for (int q = 0; q < ba->n; ++q) {
      const int ri = g.regions[q];
      const dim3 grid = bwd_grid(rs[ri].g, tbw);
      ba->tile_start[q] = tiles;
      ba->tiles_j[q] = (int)grid.x;
      tiles += (int)(grid.x * grid.y);
      ba->r[q] = regions[ri];
    }
    ba->tile_start[ba->n] = tiles;
    st = launch("eps_batched_scatter", k.fn, dim3((unsigned)tiles), k.smem, ba, gst, !gstreams);
    if (st != EPS_OK) break;
  }
  delete ba;
  return st;
}

// Multi form: one persistent mixed-radius launch per set.
eps_status_t run_fwd_multi(const std::vector<LaunchSet> &sets, const std::vector<Resolved> &rs,
                           const std::vector<FwdRegion> &regions, int ncomp, int bps, int *err,
                           cudaStream_t s, bool pdl) {
  int nsm = 0;
  eps_status_t st = sm_count(&nsm);
  if (st != EPS_OK) return st;
  FwdMultiArgs *ma = new FwdMultiArgs;
  for (const LaunchSet &ls : sets) {
    std::memset(ma, 0, sizeof(*ma));
    ma->n = (int)ls.regions.size();
    ma->err = err;
    size_t smem = 0;
    int tiles = 0;
    for (int q = 0; q < ma->n; ++q) {
      const int ri = ls.regions[q];
      const int c = rs[ri].rp1;
      std::memcpy(ma->w + woff(c), rs[ri].w, sizeof(float) * (2 * c - 1) * (2 * c - 1));
      int sf = 0;
      smem = std::max(smem, fwd_smem(fwd_entry(c, ls.bc), rs[ri].g, ncomp, &sf));
      const dim3 grid = fwd_grid(rs[ri].g);
      ma->tile_start[q] = tiles;
      ma->tiles_j[q] = (int)grid.x;
      ma->rp1[q] = c;
      tiles += (int)(grid.x * grid.y);
      ma->r[q] = regions[ri];
    }
    ma->tile_start[ma->n] = tiles;
    for (int q = 0; q < ma->n; ++q) ma->r[q].stage_floats = (int)(smem / sizeof(float));
    const long blocks = std::max<long>(1, std::min<long>(tiles, (long)nsm * bps));
    st = launch("eps_batched_stencil", fwd_multi_entry(ls.bc), dim3((unsigned)blocks), smem, ma, s,
                pdl);
    if (st != EPS_OK) break;
  }
  delete ma;
  return st;
}

eps_status_t run_bwd_multi(const std::vector<LaunchSet> &sets, const std::vector<Resolved> &rs,
                           const std::vector<BwdRegion> &regions, int bps, int *err,
                           cudaStream_t s) {
  int nsm = 0;
  eps_status_t st = sm_count(&nsm);
  if (st != EPS_OK) return st;
  BwdMultiArgs *ma = new BwdMultiArgs;
  for (const LaunchSet &ls : sets) {
    std::memset(ma, 0, sizeof(*ma));
    ma->n = (int)ls.regions.size();
    ma->err = err;
    size_t smem = 0;
    int tiles = 0;
    for (int q = 0; q < ma->n; ++q) {
      const int ri = ls.regions[q];
      const int c = rs[ri].rp1;
      std::memcpy(ma->w + woff(c), rs[ri].w, sizeof(float) * (2 * c - 1) * (2 * c - 1));
      smem = std::max(smem, bwd_entry(c, ls.bc).smem);
      const dim3 grid = bwd_grid(rs[ri].g);
      ma->tile_start[q] = tiles;
      ma->tiles_j[q] = (int)grid.x;
      ma->rp1[q] = c;
      tiles += (int)(grid.x * grid.y);
      ma->r[q] = regions[ri];
    }
    ma->tile_start[ma->n] = tiles;
    const long blocks = std::max<long>(1, std::min<long>(tiles, (long)nsm * bps));
    st = launch("eps_batched_scatter", bwd_multi_entry(ls.bc), dim3((unsigned)blocks), smem, ma, s,
                true);
    if (st != EPS_OK) break;
  }
  delete ma;
  return st;
}

eps_status_t run_fwd_batch(const std::vector<Resolved> &rs, const eps_problem_t *probs,
                           const std::vector<FwdRegion> &regions, int ncomp,
                           const BatchTuning &t, int *err, cudaStream_t s, bool pdl) {
  const int nc = std::min(ncomp, t.stage_comps);
  if (t.multi) return run_fwd_multi(make_sets(rs, probs), rs, regions, nc, t.fwd_bps, err, s, pdl);
  return run_fwd_grouped(make_groups(rs, probs), rs, regions, nc, err, s, pdl);
}

eps_status_t run_bwd_batch(const std::vector<Resolved> &rs, const eps_problem_t *probs,
                           const std::vector<BwdRegion> &regions, const BatchTuning &t, int *err,
                           cudaStream_t s) {
  if (t.multi) return run_bwd_multi(make_sets(rs, probs), rs, regions, t.bwd_bps, err, s);
  return run_bwd_grouped(make_groups(rs, probs), rs, regions, t.bwd_bulk, t.bwd_cols, err, s);
}

eps_status_t vjp_batched_impl(int32_t n, const eps_problem_t *probs, const float *const *C,
                              int32_t n_lambda, int32_t field_type, const void *const *EF,
                              const void *const *EA, const float *field_scales, float scale,
                              float *const *dJdC, float *const *eps_out, void *ws, size_t ws_bytes,
                              cudaStream_t s, const BatchTuning *forced) {
  std::vector<Resolved> rs;
  std::vector<size_t> off;
  size_t total = 0;
  eps_status_t st = resolve_batch(n, probs, rs, off, &total);
  if (st != EPS_OK) return st;
  if (n_lambda < 0 || n_lambda > EPS_MAX_BATCH_LAMBDA) return EPS_ERR_INVALID_ARG;
  if (field_type != EPS_FIELD_C64) {
    if (field_type == EPS_FIELD_BF16X2_SCALED || field_type == EPS_FIELD_F16X2_SCALED)
      return EPS_ERR_UNSUPPORTED;
    return EPS_ERR_INVALID_ARG;
  }
  if (!std::isfinite(scale)) return EPS_ERR_INVALID_ARG;
  if (n == 0) return EPS_OK;
  if (!C || !dJdC || (n_lambda > 0 && (!EF || !EA))) return EPS_ERR_INVALID_ARG;
  if (!ws || !aligned(ws, 256) || ws_bytes < total) return EPS_ERR_WORKSPACE;
  int *err = nullptr;
  if ((st = error_flag_ptr(&err)) != EPS_OK) return st;
  const BatchTuning t = forced ? *forced : lookup_tuning(batch_signature(n, probs, n_lambda));

  std::unique_ptr<ContractBatchArgs> ca_owner(new ContractBatchArgs);
  std::unique_ptr<SeedsArgs> sa_owner(new SeedsArgs);
  ContractBatchArgs *ca = ca_owner.get();
  SeedsArgs *sa = sa_owner.get();
  std::memset(ca, 0, sizeof(*ca));
  std::memset(sa, 0, sizeof(*sa));
  std::vector<FwdRegion> fr(n);
  std::vector<BwdRegion> br(n);
  std::vector<const Geometry *> gs;
  long ncol = 0;
  for (int k = 0; k < n; ++k) {
    std::memset(&fr[k], 0, sizeof(FwdRegion));
    std::memset(&br[k], 0, sizeof(BwdRegion));
    if (rs[k].empty) continue;
    const Geometry &g = rs[k].g;
    float *out_eps = eps_out ? eps_out[k] : nullptr;
    if (!C[k] || !dJdC[k] || !aligned(C[k], 4) || !aligned(dJdC[k], 4) ||
        (out_eps && !aligned(out_eps, 16)) || (g.nz & 1)) {
      return (g.nz & 1) ? EPS_ERR_SHAPE : EPS_ERR_INVALID_ARG;
    }
    const WsLayout L = ws_layout(g);
    char *base = (char *)ws + off[k];
    float *Wm = (float *)(base + L.w);
    float *seeds = (float *)(base + L.seeds);
    float *pd4 = (float *)(base + L.pd4);
    float *ie2 = (float *)(base + L.ie2);
    gs.push_back(&rs[k].g);
    ContractBatchRegion &cr = ca->r[ca->n++];
    cr.col_start = ncol;
    cr.nz = g.nz;
    cr.k0 = g.k0;
    cr.nk = g.nk;
    cr.nlambda = n_lambda;
    cr.W = Wm;
    for (int l = 0; l < n_lambda; ++l) {
      const void *ef = EF[k * n_lambda + l], *ea = EA[k * n_lambda + l];
      if (!ef || !ea || !aligned(ef, 16) || !aligned(ea, 16)) {
        return EPS_ERR_INVALID_ARG;
      }
      cr.EF[l] = (const float *)ef;
      cr.EA[l] = (const float *)ea;
      for (int c = 0; c < 3; ++c) {
        float sc = scale;
        if (field_scales) {
          const float *fsr = field_scales + (size_t)(k * n_lambda + l) * 6;
          sc *= fsr[c] * fsr[3 + c];
          if (!std::isfinite(sc)) {
            return EPS_ERR_INVALID_ARG;
          }
        }
        cr.fs[l][c] = sc;
      }
    }
    sa->r[sa->n++] = SeedsRegion{ncol, (long)g.nx * g.ny, Wm, seeds};
    ncol += (long)g.nx * g.ny;
    fr[k].g = g;
    fr[k].mode = MODE_C64;
    fr[k].write_eps = out_eps ? 1 : 0;
    // the concurrent form's stencils never wait for the contraction
    fr[k].defer_seeds = (t.defer_seeds || (t.group_streams && !t.multi)) ? 1 : 0;
    fr[k].C = C[k];
    fr[k].eps = out_eps;
    fr[k].W = Wm;
    fr[k].seeds = seeds;
    fr[k].pd4 = pd4;
    fr[k].ie2 = ie2;
    br[k].g = g;
    br[k].seeds = seeds;
    br[k].pd4 = pd4;
    br[k].ie2 = ie2;
    br[k].dJdC = dJdC[k];
  }
  ca->ncol = ncol;
  ca->err = err;
  sa->ncol = ncol;
  sa->err = err;
  // Concurrent grouped form: each radius group's stencil and scatter launches
  // go to an auxiliary stream of their own, so the groups' partial waves run
  // side by side.  The stencils (seed factors only) start with the
  // contraction; the seeds kernel runs on `s` once the contraction and every
  // stencil are done; then the scatters run on the auxiliary streams again.
  const bool conc = t.group_streams && !t.multi;
  std::unique_lock<std::mutex> aux_lock(g_aux_mu, std::defer_lock);
  AuxSet *aux = nullptr;
  std::vector<Group> groups;
  std::vector<cudaStream_t> gstreams;
  int naux = 0;
  if (conc) {
    aux_lock.lock();
    if ((st = aux_set(&aux)) != EPS_OK) return st;
    groups = make_groups(rs, probs);
    naux = (int)std::min<size_t>(groups.size(), AUX_STREAMS);
    for (size_t gi = 0; gi < groups.size(); ++gi) gstreams.push_back(aux->st[gi % AUX_STREAMS]);
    if (naux > 0 && (st = fork_streams(s, aux->fork, aux->st, naux)) != EPS_OK) return st;
  }
  if (ncol > 0) {
    int nsm = 0;
    if ((st = sm_count(&nsm)) != EPS_OK) return st;
    std::unique_ptr<ContractTmaBatchArgs> ta(new ContractTmaBatchArgs);
    size_t tsmem = 0;
    if (prepare_contract_tma_batch(gs, *ca, n_lambda, ta.get(), &tsmem)) {
      ta->err = err;
      const int bps = std::max(1, std::min(t.contract_bps, TMA_BATCH_MAX_BPS));
      const long blocks = std::max<long>(1, std::min<long>(ta->nchunks, (long)nsm * bps));
      st = launch("eps_batched_contract", contract_tma_batch_entry(ta->n * ta->nlambda * 2),
                  dim3((unsigned)blocks), tsmem, ta.get(), s);
    } else {
      const long per_block = (NTHREADS / 32) * 4;
      const long blocks = std::max<long>(
          1, std::min<long>((ncol + per_block - 1) / per_block, (long)nsm * 4 * t.contract_bps));
      st = launch("eps_batched_contract", contract_batched_entry(), dim3((unsigned)blocks), 0, ca,
                  s);
    }
  }
  if (st != EPS_OK) return st;
  bool any_eps = false;
  for (int k = 0; k < n; ++k) any_eps = any_eps || (eps_out && eps_out[k]);
  if (conc) {
    const int nc = std::min(any_eps ? 3 : 0, t.stage_comps);
    if ((st = run_fwd_grouped(groups, rs, fr, nc, err, s, false, &gstreams)) != EPS_OK) return st;
    if ((st = join_streams(s, aux->join, aux->st, naux)) != EPS_OK) return st;
    if ((st = run_seeds(*sa, s)) != EPS_OK) return st;
    if (naux > 0 && (st = fork_streams(s, aux->mid, aux->st, naux)) != EPS_OK) return st;
    if ((st = run_bwd_grouped(groups, rs, br, t.bwd_bulk, t.bwd_cols, err, s, &gstreams)) !=
        EPS_OK)
      return st;
    return join_streams(s, aux->join2, aux->st, naux);
  }
  st = run_fwd_batch(rs, probs, fr, any_eps ? 3 : 0, t, err, s, true);
  if (st == EPS_OK && t.defer_seeds) st = run_seeds(*sa, s);
  if (st != EPS_OK) return st;
  return run_bwd_batch(rs, probs, br, t, err, s);
}

}  // namespace

extern "C" {

eps_status_t eps_batched_workspace_size(int32_t n, const eps_problem_t *probs, int32_t n_lambda,
                                        size_t *bytes) {
  if (!bytes) return EPS_ERR_INVALID_ARG;
  if (n_lambda < 0 || n_lambda > EPS_MAX_BATCH_LAMBDA) return EPS_ERR_INVALID_ARG;
  std::vector<Resolved> rs;
  std::vector<size_t> off;
  return resolve_batch(n, probs, rs, off, bytes);
}

eps_status_t eps_forward_batched(int32_t n, const eps_problem_t *probs, const float *const *C,
                                 float *const *eps, eps_stream_t stream) {
  std::vector<Resolved> rs;
  std::vector<size_t> off;
  size_t total = 0;
  eps_status_t st = resolve_batch(n, probs, rs, off, &total);
  if (st != EPS_OK) return st;
  if (n == 0) return EPS_OK;
  if (!C || !eps) return EPS_ERR_INVALID_ARG;
  std::vector<FwdRegion> regions(n);
  for (int k = 0; k < n; ++k) {
    if (rs[k].empty) continue;
    if (probs[k].flags & EPS_FLAG_OFFDIAG) return EPS_ERR_UNSUPPORTED;
    if (!C[k] || !eps[k] || !aligned(C[k], 4) || !aligned(eps[k], 16)) return EPS_ERR_INVALID_ARG;
    std::memset(&regions[k], 0, sizeof(FwdRegion));
    regions[k].g = rs[k].g;
    regions[k].mode = MODE_FWD;
    regions[k].write_eps = 1;
    regions[k].C = C[k];
    regions[k].eps = eps[k];
  }
  int *err = nullptr;
  if ((st = error_flag_ptr(&err)) != EPS_OK) return st;
  const BatchTuning t = lookup_tuning(batch_signature(n, probs, -1));
  return run_fwd_batch(rs, probs, regions, 3, t, err, (cudaStream_t)stream, false);
}

eps_status_t eps_vjp_batched(int32_t n, const eps_problem_t *probs, const float *const *C,
                             int32_t n_lambda, int32_t field_type, const void *const *EF,
                             const void *const *EA, const float *field_scales, float scale,
                             float *const *dJdC, float *const *eps_out, void *ws, size_t ws_bytes,
                             eps_stream_t stream) {
  return vjp_batched_impl(n, probs, C, n_lambda, field_type, EF, EA, field_scales, scale, dJdC,
                          eps_out, ws, ws_bytes, (cudaStream_t)stream, nullptr);
}

eps_status_t eps_batched_set_tuning(int32_t n, const eps_problem_t *probs, int32_t n_lambda,
                                   const eps_tuning_t *tuning) {
  if (!tuning || n < 0 || n > EPS_MAX_BATCH || (n > 0 && !probs)) return EPS_ERR_INVALID_ARG;
  if (n_lambda < -1 || n_lambda > EPS_MAX_BATCH_LAMBDA) return EPS_ERR_INVALID_ARG;
  const eps_tuning_t &u = *tuning;
  if ((u.multi != 0 && u.multi != 1) || u.stencil_blocks_per_sm < 1 || u.stencil_blocks_per_sm > 16 ||
      u.scatter_blocks_per_sm < 1 || u.scatter_blocks_per_sm > 16 || u.contract_blocks_per_sm < 1 ||
      u.contract_blocks_per_sm > 64 || (u.stage_components != 1 && u.stage_components != 3) ||
      (u.defer_seeds != 0 && u.defer_seeds != 1) ||
      (u.scatter_bulk_staging != 0 && u.scatter_bulk_staging != 1) ||
      (u.scatter_tile_cols != 0 && u.scatter_tile_cols != 32 && u.scatter_tile_cols != 64) ||
      (u.concurrent_groups != 0 && u.concurrent_groups != 1))
    return EPS_ERR_INVALID_ARG;
  const BatchTuning t{u.multi, u.stencil_blocks_per_sm, u.scatter_blocks_per_sm,
                      u.contract_blocks_per_sm, u.stage_components, u.defer_seeds,
                      u.scatter_bulk_staging, u.scatter_tile_cols ? u.scatter_tile_cols : TB,
                      u.concurrent_groups};
  store_tuning(batch_signature(n, probs, n_lambda), t);
  return EPS_OK;
}

eps_status_t eps_autotune_batched(int32_t n, const eps_problem_t *probs, const float *const *C,
                                  int32_t n_lambda, int32_t field_type, const void *const *EF,
                                  const void *const *EA, const float *field_scales, float scale,
                                  float *const *dJdC, float *const *eps_out, void *ws,
                                  size_t ws_bytes, int32_t reps, eps_tuning_t *result,
                                  eps_stream_t stream) {
  if (reps < 1 || reps > 1000) return EPS_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s, &cap) != cudaSuccess) return EPS_ERR_CUDA;
  if (cap != cudaStreamCaptureStatusNone) return EPS_ERR_UNSUPPORTED;   // it synchronises
  // a dry run with the default shapes checks every argument before timing
  BatchTuning best = DEFAULT_TUNING;
  eps_status_t st = vjp_batched_impl(n, probs, C, n_lambda, field_type, EF, EA, field_scales,
                                     scale, dJdC, eps_out, ws, ws_bytes, s, &best);
  if (st != EPS_OK) return st;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    if (e0) cudaEventDestroy(e0);
    return EPS_ERR_CUDA;
  }
  int evals = 0;
  // mean milliseconds of `reps` calls with shapes t, after one warm-up call
  auto timeit = [&](const BatchTuning &t, float *ms) -> eps_status_t {
    eps_status_t r = vjp_batched_impl(n, probs, C, n_lambda, field_type, EF, EA, field_scales,
                                      scale, dJdC, eps_out, ws, ws_bytes, s, &t);
    if (r != EPS_OK) return r;
    if (cudaEventRecord(e0, s) != cudaSuccess) return EPS_ERR_CUDA;
    for (int i = 0; i < reps && r == EPS_OK; ++i)
      r = vjp_batched_impl(n, probs, C, n_lambda, field_type, EF, EA, field_scales, scale, dJdC,
                           eps_out, ws, ws_bytes, s, &t);
    if (r != EPS_OK) return r;
    if (cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
        cudaEventElapsedTime(ms, e0, e1) != cudaSuccess)
      return EPS_ERR_CUDA;
    *ms /= reps;
    ++evals;
    return EPS_OK;
  };
  float best_ms = 0.f, default_ms = 0.f;
  st = timeit(best, &best_ms);
  default_ms = best_ms;
  // coordinate descent over the launch form and shapes, two sweeps
  for (int sweep = 0; sweep < 2 && st == EPS_OK; ++sweep) {
    for (int param = 0; param < 9 && st == EPS_OK; ++param) {
      static const int values[9][4] = {{0, 1, -1, -1}, {1, 3, -1, -1}, {1, 2, 3, 4},
                                       {1, 2, 3, 4},   {1, 2, 3, 4}, {0, 1, -1, -1},
                                       {0, 1, -1, -1}, {32, 64, -1, -1}, {0, 1, -1, -1}};
      for (int v = 0; v < 4 && st == EPS_OK; ++v) {
        const int val = values[param][v];
        if (val < 0) continue;
        BatchTuning t = best;
        int *field[9] = {&t.multi, &t.stage_comps, &t.fwd_bps, &t.bwd_bps, &t.contract_bps,
                         &t.defer_seeds, &t.bwd_bulk, &t.bwd_cols, &t.group_streams};
        if (*field[param] == val) continue;
        if ((param == 2 || param == 3) && !t.multi) continue;   // grouped form: one block per tile
        // multi form: element-wise gather on TA x TB tiles, one stream
        if ((param == 6 || param == 7 || param == 8) && t.multi) continue;
        *field[param] = val;
        float ms = 0.f;
        st = timeit(t, &ms);
        if (st == EPS_OK && ms < 0.99f * best_ms) {
          best = t;
          best_ms = ms;
        }
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st != EPS_OK) return st;
  store_tuning(batch_signature(n, probs, n_lambda), best);
  if (result) {
    result->multi = best.multi;
    result->stencil_blocks_per_sm = best.fwd_bps;
    result->scatter_blocks_per_sm = best.bwd_bps;
    result->contract_blocks_per_sm = best.contract_bps;
    result->stage_components = best.stage_comps;
    result->defer_seeds = best.defer_seeds;
    result->scatter_bulk_staging = best.bwd_bulk;
    result->scatter_tile_cols = best.bwd_cols;
    result->concurrent_groups = best.group_streams;
    result->evaluations = evals;
    result->default_ms = default_ms;
    result->tuned_ms = best_ms;
  }
  return EPS_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Internal host interface for the library's other translation units.
namespace epsc_host {

eps_status_t conic_filter(const eps_problem_t *prob, float *w, int *rp1) {
  Resolved r;
  const eps_status_t st = resolve(prob, &r);
  if (st != EPS_OK) return st;
  std::memcpy(w, r.w, sizeof(r.w));
  *rp1 = r.rp1;
  return EPS_OK;
}

eps_status_t check_vjp_args(const eps_problem_t *prob, const float *C, int32_t n_lambda,
                            int32_t field_type, const void *const *EF, const void *const *EA,
                            const float *field_scales, float scale, const float *dJdC,
                            const float *eps_out, const void *ws, size_t ws_bytes) {
  Resolved r;
  eps_status_t st = resolve(prob, &r);
  if (st != EPS_OK) return st;
  bool skip = false;
  return vjp_args(r, C, n_lambda, field_type, EF, EA, field_scales, scale, dJdC, eps_out, ws,
                  ws_bytes, &skip);
}

eps_status_t launch_kernel(const char *name, const void *fn, dim3 grid, size_t smem, void *args,
                           cudaStream_t s, bool pdl) {
  return launch(name, fn, grid, smem, args, s, pdl);
}

void note_launch() { g_launch_count.fetch_add(1, std::memory_order_relaxed); }

eps_status_t subpixel_factor_offset(const eps_problem_t *prob, size_t *offset, size_t *ws_needed) {
  Resolved r;
  const eps_status_t st = resolve(prob, &r);
  if (st != EPS_OK) return st;
  const WsLayout L = ws_layout(r.g);
  *offset = L.pd4;
  *ws_needed = r.empty ? 0 : L.total;
  return EPS_OK;
}

eps_status_t sm_count_current(int *n) { return sm_count(n); }

eps_status_t error_flag(int **flag) { return error_flag_ptr(flag); }

}  // namespace epsc_host
