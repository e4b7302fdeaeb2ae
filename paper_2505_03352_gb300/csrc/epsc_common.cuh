// Shared definitions of the epschain CUDA kernels (sm_103a).
//
// Tiling.  The forward pass works on tiles of TI x TJ Yee columns (x rows,
// y contiguous), one thread per column in the per-column stages.  The
// backward scatter works on tiles of TA x TB control subpixels.  Both use
// 256-thread blocks.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "epschain.h"

namespace epsc {

constexpr int NTHREADS = 256;

// forward tile (Yee cells) and its subpixel region
constexpr int TI = 8;
constexpr int TJ = 32;
constexpr int UA = 2 * TI + 5;   // subpixel rows a in [2 i0 - 3, 2 i0 + 2 TI + 1]
constexpr int UB = 2 * TJ + 5;   // subpixel cols b in [2 j0 - 3, 2 j0 + 2 TJ + 1]
constexpr int NA_F = 7;          // filter outputs per thread (rows of a strip)
static_assert(UA % NA_F == 0, "forward strips must tile the subpixel rows");

// backward tile (subpixels)
constexpr int TA = 32;
constexpr int TB = 32;
constexpr int NA_B = 4;

// filter radius limit: RP1 = ceil(R) taps per half-axis including the centre
constexpr int MAX_RP1 = 12;
constexpr int MAX_BOX = 2 * MAX_RP1 - 1;

// |g|^2 threshold below which the interface normal is undefined (m = 0)
constexpr float NORMAL_TAU2 = 1e-12f;

enum Mode : int { MODE_FWD = 0, MODE_C64 = 1, MODE_REAL = 2 };

// bits of the device-side error flag
constexpr int ERRFLAG_TIMEOUT = 1;   // a bounded wait gave up
constexpr int ERRFLAG_BOUNDS = 2;    // a bounds check fired

// Debug bounds checks.  Built with -DEPS_DEBUG_BOUNDS, EPSC_IN_BOUNDS(lo,
// cnt, n, err) tests that elements [lo, lo + cnt) lie inside a buffer of n
// elements (lo is taken as unsigned, so a negative index fails); a failure
// sets ERRFLAG_BOUNDS in *err and the caller skips the access (a load
// reads zero).  Release builds compile every check to `true`.
#ifdef EPS_DEBUG_BOUNDS
__device__ __forceinline__ bool dbg_in_bounds(size_t lo, size_t cnt, size_t n, int *err) {
  if (lo <= n && cnt <= n - lo) return true;
  if (err) atomicOr(err, ERRFLAG_BOUNDS);
  return false;
}
#define EPSC_IN_BOUNDS(lo, cnt, n, err) \
  ::epsc::dbg_in_bounds((size_t)(lo), (size_t)(cnt), (size_t)(n), (err))
#else
#define EPSC_IN_BOUNDS(lo, cnt, n, err) true
#endif

// seed planes, [NSEED][nx][ny]: the stencil writes W-independent factors,
// the seeds kernel multiplies them by the column's Eq. 1 sums
// (the six mean seeds first, then the four Sobel seeds: each group is one
// contiguous block of planes, which the scatter stages as one box)
enum Seed : int {
  S_DAX = 0, S_DHX, S_DAY, S_DHY, S_DAZ, S_DHZ,   // dJ/dA_c, dJ/dH_c for c = x, y, z
  S_GXX, S_GYX, S_GXY, S_GYY,                     // dJ/dg_x, dJ/dg_y of U_x, then of U_y
  NSEED
};

struct Geometry {
  int mx, my, nx, ny, nz, k0, nk, bc;
  float beta, eta, eps_core, eps_clad, deps;
};

// One design region as seen by the stencil kernel.
struct FwdRegion {
  Geometry g;
  int mode;
  int write_eps;
  int write_offdiag;
  int normals3d;                 // 3-D normals at the slab faces (forward only)
  int defer_seeds;               // VJP: 0 = wait for the contraction and write the seeds,
                                 //      1 = write seed factors (the seeds kernel applies W)
  int stage_floats;              // shared floats available for eps_hat staging
  int direct_eps;                // 1: eps_hat leaves by warp-cooperative coalesced stores
                                 //    (no staging; nz a multiple of 4)
  const float *C;
  float *eps;
  float *offdiag;
  const float *W;                // [4][nx][ny] Eq. 1 column sums (contraction kernel)
  float *seeds;                  // [NSEED][nx][ny]
  float *pd4;                    // [mx][my] P'(u) (eps_core - eps_clad) / 4
  float *ie2;                    // [mx][my] 1 / eps^2
  // Eq. 1 surrogate S = sum over the J-support voxels of eps_hat * w (null:
  // not requested).  A tile that waits for the contraction adds its
  // columns' eps . W to *S itself; with defer_seeds it writes the column
  // values (eps_xx, eps_yy, eps_zz inside, eps_zz on the faces) to epsc
  // [4][nx][ny] and the seeds kernel adds them up.
  double *S;
  float *epsc;
  int eps_tma;                   // 1: eps_hat components leave the 128-byte-swizzled
                                 //    staging by one 4-D tensor store each (nz = 32;
                                 //    single-region kernel, its args carry the map)
};

// Seeds kernel: regions laid end to end in one column space.
struct SeedsRegion {
  long col_start, ncol;          // first column in the launch's column space, columns
  const float *W;                // [4][nx][ny] Eq. 1 column sums
  float *seeds;                  // [NSEED][nx][ny]: factors in, seeds out
};

struct SeedsArgs {
  int n;
  long ncol;
  // single-region calls: only the columns [band_lo, band_hi) (one band of a
  // pipelined call); band_hi == 0: every column
  long band_lo, band_hi;
  int *err;                      // error flag (debug bounds checks)
  // Eq. 1 surrogate (single-region calls; null: not requested): *S +=
  // sum over columns of epsc . W, epsc [4][nx][ny] from the stencil
  const float *epsc;
  double *S;
  SeedsRegion r[EPS_MAX_BATCH];
};

// Sum of v over the block (NTHREADS threads), added to *S by thread 0.  Every
// thread of the block must call it.  FP64 from the per-thread values on, so
// that the order of the block's and the grid's additions hardly matters.
__device__ __forceinline__ void block_add_to(double *S, double v) {
  __shared__ double part[NTHREADS / 32];
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  __syncthreads();   // part[] may still be read by an earlier call
  if (lane == 0) part[warp] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
#pragma unroll
    for (int w = 0; w < NTHREADS / 32; ++w) t += part[w];
    atomicAdd(S, t);
  }
}

// Kernel arguments end with the conic weights, a dense (2 RP1 - 1)^2 box,
// row-major.  Each kernel takes the struct with exactly its box (NW = (2 RP1
// - 1)^2); the host fills the full-size struct (NW = MAX_BOX^2) and passes
// it, and the launch copies only the kernel's parameter bytes, a common
// prefix.  Smaller parameter blocks launch faster.
template <int NW>
struct FwdArgsN {
  FwdRegion r;
  int *err;
  // eps_hat as a {nz, ny, nx, 3} float tensor, box {nz, TJ, TI, 1}, 128-byte
  // swizzle (used when r.eps_tma is set)
  CUtensorMap eps_map;
  float w[NW];
};
using FwdArgs = FwdArgsN<MAX_BOX * MAX_BOX>;
template <int RP1>
using FwdArgsR = FwdArgsN<(2 * RP1 - 1) * (2 * RP1 - 1)>;

// Batched stencil launch: regions sharing one conic filter; block b works on
// tile b - tile_start[k] of region k, tile_start[k] <= b < tile_start[k+1].
struct FwdBatchArgs {
  int n;
  int tile_start[EPS_MAX_BATCH + 1];
  int tiles_j[EPS_MAX_BATCH];
  FwdRegion r[EPS_MAX_BATCH];
  int *err;
  float w[MAX_BOX * MAX_BOX];
};

// One design region as seen by the adjoint scatter kernel.
struct BwdRegion {
  Geometry g;
  const float *seeds;
  const float *pd4;
  const float *ie2;
  float *dJdC;
};

template <int NW>
struct BwdArgsN {
  BwdRegion r;
  int *err;
  int ty0;                       // first tile row of the launch (grid row 0)
  float w[NW];
};

// Arguments of the scatter that stages through bulk tensor copies (larger
// problems; the tensor maps make its parameter block 0.5 KB larger, which
// would cost the one-wave launch about 1 us).
template <int NW>
struct __align__(128) BwdTmaArgsN {
  BwdRegion r;
  int *err;
  int ty0;                       // first tile row of the launch (grid row 0)
  // P' deps / 4 and 1 / eps^2 ({my, mx, 1}); the six mean seeds and the four
  // Sobel seeds ({ny, nx, NSEED}, one box each)
  CUtensorMap maps[4];
  float w[NW];
};
using BwdArgs = BwdArgsN<MAX_BOX * MAX_BOX>;
template <int RP1>
using BwdArgsR = BwdArgsN<(2 * RP1 - 1) * (2 * RP1 - 1)>;
using BwdTmaArgs = BwdTmaArgsN<MAX_BOX * MAX_BOX>;
template <int RP1>
using BwdTmaArgsR = BwdTmaArgsN<(2 * RP1 - 1) * (2 * RP1 - 1)>;

struct BwdBatchArgs {
  int n;
  int tile_start[EPS_MAX_BATCH + 1];
  int tiles_j[EPS_MAX_BATCH];
  BwdRegion r[EPS_MAX_BATCH];
  int *err;
  float w[MAX_BOX * MAX_BOX];
};

// Batched scatter that stages interior tiles through bulk tensor copies: up
// to BWD_TMA_BATCH regions of one radius group per launch, each with its own
// four tensor maps in the parameter block (has_maps[k] = 0: that region's
// layout does not suit bulk copies and its tiles gather element by element).
constexpr int BWD_TMA_BATCH = 32;
struct __align__(128) BwdTmaBatchArgs {
  int n;
  int tile_start[BWD_TMA_BATCH + 1];
  int tiles_j[BWD_TMA_BATCH];
  int has_maps[BWD_TMA_BATCH];
  BwdRegion r[BWD_TMA_BATCH];
  int *err;
  float w[MAX_BOX * MAX_BOX];
  CUtensorMap maps[4 * BWD_TMA_BATCH];   // region k: maps[4 k .. 4 k + 3]
};

// Region and tile of block b in a batched launch (regions scanned in order).
template <class BA>
__device__ __forceinline__ void batch_tile(const BA &a, int b, int &k, int &t) {
  k = 0;
  while (k + 1 < a.n && b >= a.tile_start[k + 1]) ++k;
  t = b - a.tile_start[k];
}

__device__ __forceinline__ int clampi(int x, int lo, int hi) { return min(max(x, lo), hi); }

__device__ __forceinline__ int wrapi(int x, int n) {
  int r = x % n;
  return r < 0 ? r + n : r;
}

__device__ __forceinline__ int bc_map(int x, int n, int bc) {
  return bc == EPS_BC_CLAMP ? clampi(x, 0, n - 1) : wrapi(x, n);
}

// Asynchronous 4-byte global -> shared copy (cp.async); zero-fills the
// destination when `valid` is false (no bytes are read from `src` then).
__device__ __forceinline__ void cp_async4(float *dst, const float *src, bool valid) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(dst);
  const int n = valid ? 4 : 0;
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(s), "l"(src), "r"(n)
               : "memory");
}

// 16-byte asynchronous copy; both addresses 16-byte aligned.
__device__ __forceinline__ void cp_async16(float *dst, const float *src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(src) : "memory");
}

__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.wait_all;\n" ::: "memory");
}

// Bulk (TMA) copy of `bytes` contiguous bytes from shared to global memory,
// tracked by the calling thread's bulk async-group.  Both addresses 16-byte
// aligned, bytes a multiple of 16.
__device__ __forceinline__ void bulk_store(void *gdst, const void *ssrc, unsigned bytes) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(ssrc);
  asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;\n" ::"l"(gdst), "r"(s),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;\n" ::: "memory"); }
// shared memory read by earlier bulk stores of this thread may be reused
__device__ __forceinline__ void bulk_wait_read() {
  asm volatile("cp.async.bulk.wait_group.read 0;\n" ::: "memory");
}
// ... all but the most recent N groups of them
template <int N>
__device__ __forceinline__ void bulk_wait_read_n() {
  asm volatile("cp.async.bulk.wait_group.read %0;\n" ::"n"(N) : "memory");
}
// 4-D tensor store of a shared-memory box at coordinates {x, y, z, w},
// tracked by the calling thread's bulk async-group; elements outside the
// tensor are not written.  The box's shared-memory layout is the map's
// (dense, swizzled as the map says); x * element size a multiple of 16.
__device__ __forceinline__ void tma_store_4d(const CUtensorMap *map, const void *ssrc, int x, int y,
                                             int z, int w) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(ssrc);
  asm volatile(
      "cp.async.bulk.tensor.4d.global.shared::cta.bulk_group [%0, {%2, %3, %4, %5}], [%1];\n" ::"l"(
          map),
      "r"(s), "r"(x), "r"(y), "r"(z), "r"(w)
      : "memory");
}
// earlier bulk stores of this thread have completed
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;\n" ::: "memory"); }
// make this thread's generic-proxy shared-memory writes visible to bulk copies
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
}

// Programmatic dependent launch: wait until the grids this grid depends on
// have completed and their writes are visible (no-op without a dependency).
__device__ __forceinline__ void griddep_wait() {
  asm volatile("griddepcontrol.wait;\n" ::: "memory");
}
// Let the dependent grid in the stream start launching its blocks.
__device__ __forceinline__ void griddep_launch_dependents() {
  asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory");
}

// Register-blocked conic stencil over a strip of NA outputs stacked along the
// row direction.  `src` points at the input element that lies R rows above and
// R columns left of output 0; output k is
//     sum_{p,q} w[(p+R)(2R+1) + q+R] * src[(k + p + R) * pitch + q + R].
// Every input row is read once from shared memory and reused by all NA
// outputs.  The cone is symmetric in q (w depends on p^2 + q^2 only, and the
// host table is exactly symmetric), so each row first pairs the inputs at
// +q and -q, and each output takes R + 1 taps per row instead of 2R + 1.
// Each output adds the per-row partial sums of its taps: fewer rounding
// steps in sequence than one long fma chain, which matters where a
// projection amplifies u's error by up to beta/2 (twice on the morphology
// path).
template <int RP1, int NA, class Args>
__device__ __forceinline__ void strip_stencil(const float *__restrict__ src, int pitch,
                                              const Args &a, float (&out)[NA]) {
  constexpr int R = RP1 - 1;
  constexpr int BW = 2 * R + 1;
#pragma unroll
  for (int k = 0; k < NA; ++k) out[k] = 0.f;
#pragma unroll
  for (int rr = 0; rr < NA + 2 * R; ++rr) {
    float sp[R + 1];   // sp[0] = centre, sp[j] = src(+j) + src(-j)
    sp[0] = src[rr * pitch + R];
#pragma unroll
    for (int j = 1; j <= R; ++j) sp[j] = src[rr * pitch + R + j] + src[rr * pitch + R - j];
#pragma unroll
    for (int k = 0; k < NA; ++k) {
      const int p = rr - k - R;
      if (p >= -R && p <= R) {
        float part = 0.f;
#pragma unroll
        for (int j = 0; j <= R; ++j) {
          if (p * p + j * j < RP1 * RP1) part = fmaf(a.w[(p + R) * BW + j + R], sp[j], part);
        }
        out[k] += part;
      }
    }
  }
}

// Fast unsigned division by a runtime divisor d for small numerators:
// q = umulhi(n, m) with m = ceil(2^32 / d) is exact whenever n * d^2 < 2^32
// (the rounding excess of m is below d, so n * excess / 2^32 < 1 / d).
struct FastDiv {
  unsigned d, m;
  __device__ __forceinline__ explicit FastDiv(unsigned d_)
      : d(d_), m(d_ > 1u ? 0xFFFFFFFFu / d_ + 1u : 0u) {}
  __device__ __forceinline__ unsigned div(unsigned n) const { return d == 1u ? n : __umulhi(n, m); }
};

}  // namespace epsc
