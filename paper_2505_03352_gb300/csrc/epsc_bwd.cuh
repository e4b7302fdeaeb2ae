// Adjoint scatter: per-column seeds -> dJ/dC, one TA x TB tile of control
// subpixels per block.  Applies, in gather form, the transposes of the
// forward stages in reverse order:
//   Sobel^T (Yee level)  ->  dual-cell mean^T (Eq. 8)  ->  1/eps and mixing
//   ->  projection P'(u) (analytic, Eq. 6)  ->  K^T (Eq. 2).
// Edge replicate is a many-to-one index map; its transpose folds every
// contribution that landed outside the region back onto the edge element.
//
// Everything the tile needs (P'(u) and 1/eps^2 of its subpixels, the seed
// maps of the touched cells and the Sobel seeds with a one-cell halo) is
// staged into shared memory first, so the global reads are all in flight at
// once: by per-element asynchronous copies (bwd_kernel, the batched
// kernels, and tiles next to the region edge), or, in bwd_tma_kernel (larger
// problems), by four bulk tensor copies per tile clear of the edge.
#pragma once

#include "epsc_common.cuh"
#include "epsc_contract_tma.cuh"   // mbarrier and bulk tensor copy helpers

namespace epsc {

// Shared-memory layout of a scatter tile of TA x TBW subpixels (TBW = TB,
// 32, or the wide batched tiles' 64).
template <int RP1, int TBW = TB>
struct BwdSmem {
  static constexpr int R = RP1 - 1;
  static constexpr int GA_MAX = TA + 2 * R;                    // gather rows incl. fold halo
  static constexpr int GB_MAX = TBW + 2 * R;
  static constexpr int NSTRIP_MAX = (GA_MAX + NA_B - 1) / NA_B;
  static constexpr int DA_ALLOC = NSTRIP_MAX * NA_B + 2 * R;   // du rows readable by strips
  static constexpr int DBP = TBW + 4 * R;                      // du pitch
  static constexpr int NCI = (TA + 4 * R) / 2 + 3;             // cell rows covering du
  static constexpr int NCJ0 = (TBW + 4 * R) / 2 + 3;           // cell columns covering du
  // Row pitches of the cell maps leave room for a row that starts up to 3
  // floats after a 16-byte boundary (bulk tensor copies start on one).
  static constexpr int NCJ = (NCJ0 + 3 + 3) & ~3;
  static constexpr int NC = NCI * NCJ;
  static constexpr int NGJ = (NCJ0 + 2 + 3 + 3) & ~3;          // Sobel seeds: one-cell halo
  static constexpr int NG = (NCI + 2) * NGJ;
  // sections start on 128-byte boundaries
  static constexpr int OFF_U = 0;                              // P' deps / 4, then du in place
  static constexpr int OFF_IE2 = OFF_U + ((DA_ALLOC * DBP + 31) & ~31);     // 1 / eps^2
  static constexpr int OFF_SEED = OFF_IE2 + ((DA_ALLOC * DBP + 31) & ~31);  // 6 maps: dA, dH of x, y, z
  static constexpr int OFF_G = OFF_SEED + ((6 * NC + 31) & ~31);            // 4 maps: dg of U_x, U_y
  static constexpr int OFF_DU = OFF_G + ((4 * NG + 31) & ~31);              // 2 maps: dU_x, dU_y
  // K^T results: written after the last read of 1 / eps^2, in its place
  static constexpr int OFF_DCE = OFF_IE2;
  static_assert(GA_MAX * GB_MAX <= DA_ALLOC * DBP, "K^T results fit in the 1/eps^2 section");
  static constexpr int TOTAL = OFF_DU + 2 * NC;
  // rows of the P' / 1/eps^2 box of a tile clear of the region edge
  static constexpr int DA_BOX = TA + 2 * R;
  // bytes the four bulk copies of such a tile deliver
  static constexpr unsigned TMA_BYTES = 4u * (2 * DBP * DA_BOX + 6 * NC + 4 * NG);
  static constexpr unsigned TMA_BYTES_G = 4u * (4 * NG);   // the Sobel seeds' box alone
  static constexpr size_t BYTES = sizeof(float) * TOTAL;
};

// Transposed 3-tap Sobel weights along one axis for target cell t and the
// sources s = t - 1 + e (e = 0, 1, 2):  wd = sum_{d: bc(s+d)=t} D(d),
// ws = sum_{d: bc(s+d)=t} S(d), D = (-1, 0, 1), S = (1, 2, 1).  Under edge
// replicate, sources outside [0, n) do not exist and get zero weights.
__device__ __forceinline__ void sobel_t_weights(int t, int n, int bc, float (&wd)[3],
                                                float (&ws)[3]) {
#pragma unroll
  for (int e = 0; e < 3; ++e) {
    if (bc == EPS_BC_PERIODIC) {
      const int d = 1 - e;   // the single offset with s + d = t
      wd[e] = (float)d;
      ws[e] = d == 0 ? 2.f : 1.f;
    } else {
      const int s = t - 1 + e;
      float a = 0.f, b = 0.f;
      if (s >= 0 && s < n) {
#pragma unroll
        for (int d = -1; d <= 1; ++d) {
          if (clampi(s + d, 0, n - 1) == t) {
            a += (float)d;
            b += d == 0 ? 2.f : 1.f;
          }
        }
      }
      wd[e] = a;
      ws[e] = b;
    }
  }
}

// One tile (subpixel rows a0 .., columns b0 ..) of one region `rg`.  With
// TMA, `maps` points at the region's four tensor maps of the staged inputs
// in the kernel parameters (bwd_tma_kernel: single region; the batched
// bwd_tma_batched_kernel: the tile's region), or is null for a region whose
// layout does not suit bulk copies; radius class 3 and up.
template <int RP1, int BC, bool TMA = false, int TBW = TB, class Args>
__device__ __forceinline__ void bwd_tile(const Args &a, const BwdRegion &rg, const int a0,
                                         const int b0, const CUtensorMap *maps = nullptr) {
  using S = BwdSmem<RP1, TBW>;
  constexpr int R = S::R;
  constexpr int DBP = S::DBP;
  constexpr bool clamp = BC == EPS_BC_CLAMP;
  extern __shared__ __align__(128) float bwd_smem[];
  float *sU = bwd_smem + S::OFF_U;
  float *sIE2 = bwd_smem + S::OFF_IE2;
  float *sSeed = bwd_smem + S::OFF_SEED;
  float *sG = bwd_smem + S::OFF_G;
  float *sdU = bwd_smem + S::OFF_DU;
  float *sdc = bwd_smem + S::OFF_DCE;

  const Geometry &g = rg.g;
  const int tid = threadIdx.x;
  const int ty = tid >> 5, tx = tid & 31;       // 8 x 32 thread grid for 2-D loops
  const int aend = min(a0 + TA, g.mx), bend = min(b0 + TBW, g.my);
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
  const int NSTRIP = (GA + NA_B - 1) / NA_B;
  const int DA_USED = NSTRIP * NA_B + 2 * R;   // rows the strips read

  // everything staged below is written by the stencil kernel queued ahead
  griddep_wait();

  // ---- stage P' deps / 4, 1/eps^2, the dA/dH seeds and the Sobel seeds ---
  // A tile whose staged windows lie inside the region (no edge fold, no wrap)
  // takes four bulk tensor copies in the single-region kernel.  Each box
  // starts at the 16-byte boundary at or below its window's first column;
  // the views of the staged maps are shifted by the remainder (sh, shj,
  // shg).  The staged values are those of the element-wise gather below,
  // which every other tile (and the batched launches) takes.
  bool staged = false;
  bool rest_pending = false;   // bulk copies of everything but the Sobel seeds in flight
  int sh = 0, shj = 0, shg = 0;
  __shared__ uint64_t s_bar[2];
  __shared__ int s_fail;
  if constexpr (TMA) {
    // (the sections sit on 128-byte boundaries of the dynamic shared memory,
    // declared 128-byte aligned; a base that were not falls back to the
    // element-wise gather)
    if (maps && R >= 2 && (smem_addr(bwd_smem) & 127u) == 0u && da_lo >= 0 && da_lo + DA <= g.mx &&
        db_lo >= 0 && db_lo + DB <= g.my && ci_lo >= 1 && ci_lo + NCI + 1 <= g.nx && cj_lo >= 1 &&
        cj_lo + NCJ + 1 <= g.ny) {
      const int xa = db_lo & ~3, xs = cj_lo & ~3, xg = (cj_lo - 1) & ~3;
      sh = db_lo - xa;
      shj = cj_lo - xs;
      shg = cj_lo - 1 - xg;
      // two barriers: the Sobel seeds' box (Sobel^T starts on it) and the
      // other three (waited for after Sobel^T, below)
      if (tid == 0) {
        mbar_init(&s_bar[0], 1);
        mbar_init(&s_bar[1], 1);
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
        mbar_arrive_expect_tx(&s_bar[0], S::TMA_BYTES_G);
        mbar_arrive_expect_tx(&s_bar[1], S::TMA_BYTES - S::TMA_BYTES_G);
        tma_load_3d(sG, &maps[3], xg, ci_lo - 1, S_GXX, &s_bar[0]);
        tma_load_3d(sU, &maps[0], xa, da_lo, 0, &s_bar[1]);
        tma_load_3d(sIE2, &maps[1], xa, da_lo, 0, &s_bar[1]);
        tma_load_3d(sSeed, &maps[2], xs, ci_lo, S_DAX, &s_bar[1]);
        s_fail = 0;
        if (!mbar_wait_bounded(&s_bar[0], 0u)) {
          // record the timeout; let every copy land before the block leaves
          atomicOr(a.err, ERRFLAG_TIMEOUT);
          mbar_wait_bounded(&s_bar[0], 0u);
          mbar_wait_bounded(&s_bar[1], 0u);
          s_fail = 1;
        }
      }
      __syncthreads();
      if (s_fail) return;
      staged = true;
      rest_pending = true;
    }
  }
  // Otherwise a tile whose windows lie inside the region, in maps whose rows
  // are whole float4 runs, copies 16 bytes at a time from the 16-byte
  // boundary at or below each window (the same shifted views); the rest
  // gather element by element.  Every copy stays inside its map.
  const int xa = db_lo & ~3, xs = cj_lo & ~3, xg = (cj_lo - 1) & ~3;
  const int nca = (db_lo + DB - xa + 3) >> 2;        // float4 per P' / 1/eps^2 row
  const int ncs = (cj_lo + NCJ - xs + 3) >> 2;       // per seed row
  const int ncg = (cj_lo + NCJ + 1 - xg + 3) >> 2;   // per Sobel-seed row
  const bool vec = !staged && (g.my & 3) == 0 && (g.ny & 3) == 0 && da_lo >= 0 &&
                   da_lo + DA <= g.mx && DA_USED == DA && db_lo >= 0 && xa + 4 * nca <= g.my &&
                   ci_lo >= 1 && ci_lo + NCI + 1 <= g.nx && cj_lo >= 1 && xs + 4 * ncs <= g.ny &&
                   xg + 4 * ncg <= g.ny && 4 * nca <= DBP && 4 * ncs <= S::NCJ && 4 * ncg <= S::NGJ;
  if (vec) {
    sh = db_lo - xa;
    shj = cj_lo - xs;
    shg = cj_lo - 1 - xg;
    for (int idx = tid; idx < DA * nca; idx += NTHREADS) {
      const int r = idx / nca, k = idx - r * nca;
      const size_t o = (size_t)(da_lo + r) * g.my + xa + 4 * k;
      if (!EPSC_IN_BOUNDS(o, 4, (size_t)g.mx * g.my, a.err)) continue;
      cp_async16(sU + r * DBP + 4 * k, rg.pd4 + o);
      cp_async16(sIE2 + r * DBP + 4 * k, rg.ie2 + o);
    }
    for (int idx = tid; idx < NCI * ncs; idx += NTHREADS) {
      const int r = idx / ncs, k = idx - r * ncs;
      const size_t o = (size_t)(ci_lo + r) * g.ny + xs + 4 * k;
      if (!EPSC_IN_BOUNDS(o, 4, plane, a.err)) continue;
      float *d = sSeed + r * S::NCJ + 4 * k;
      cp_async16(d + 0 * S::NC, rg.seeds + S_DAX * plane + o);
      cp_async16(d + 1 * S::NC, rg.seeds + S_DHX * plane + o);
      cp_async16(d + 2 * S::NC, rg.seeds + S_DAY * plane + o);
      cp_async16(d + 3 * S::NC, rg.seeds + S_DHY * plane + o);
      cp_async16(d + 4 * S::NC, rg.seeds + S_DAZ * plane + o);
      cp_async16(d + 5 * S::NC, rg.seeds + S_DHZ * plane + o);
    }
    for (int idx = tid; idx < (NCI + 2) * ncg; idx += NTHREADS) {
      const int r = idx / ncg, k = idx - r * ncg;
      const size_t o = (size_t)(ci_lo - 1 + r) * g.ny + xg + 4 * k;
      if (!EPSC_IN_BOUNDS(o, 4, plane, a.err)) continue;
      float *d = sG + r * S::NGJ + 4 * k;
      cp_async16(d + 0 * S::NG, rg.seeds + S_GXX * plane + o);
      cp_async16(d + 1 * S::NG, rg.seeds + S_GYX * plane + o);
      cp_async16(d + 2 * S::NG, rg.seeds + S_GXY * plane + o);
      cp_async16(d + 3 * S::NG, rg.seeds + S_GYY * plane + o);
    }
    cp_async_wait_all();
    __syncthreads();
  } else if (!staged) {
    for (int r = ty; r < DA_USED; r += 8) {
      const int va = da_lo + r;
      const bool row_ok = r < DA && (!clamp || (va >= 0 && va < g.mx));
      const size_t rowo = row_ok ? (size_t)(clamp ? va : wrapi(va, g.mx)) * g.my : 0;
      for (int c = tx; c < DB; c += 32) {
        const int vb = db_lo + c;
        bool ok = row_ok && (!clamp || (vb >= 0 && vb < g.my));
        size_t o = ok ? rowo + (clamp ? vb : wrapi(vb, g.my)) : 0;
        if (!EPSC_IN_BOUNDS(o, 1, (size_t)g.mx * g.my, a.err)) ok = false, o = 0;
        cp_async4(sU + r * DBP + c, rg.pd4 + o, ok);
        cp_async4(sIE2 + r * DBP + c, rg.ie2 + o, ok);
      }
    }
    for (int r = ty; r < NCI; r += 8) {
      const int vi = ci_lo + r;
      const bool row_ok = !clamp || (vi >= 0 && vi < g.nx);
      const size_t rowo = row_ok ? (size_t)(clamp ? vi : wrapi(vi, g.nx)) * g.ny : 0;
      for (int c = tx; c < NCJ; c += 32) {
        const int vj = cj_lo + c;
        bool ok = row_ok && (!clamp || (vj >= 0 && vj < g.ny));
        size_t o = ok ? rowo + (clamp ? vj : wrapi(vj, g.ny)) : 0;
        if (!EPSC_IN_BOUNDS(o, 1, plane, a.err)) ok = false, o = 0;
        float *d = sSeed + r * S::NCJ + c;
        cp_async4(d + 0 * S::NC, rg.seeds + S_DAX * plane + o, ok);
        cp_async4(d + 1 * S::NC, rg.seeds + S_DHX * plane + o, ok);
        cp_async4(d + 2 * S::NC, rg.seeds + S_DAY * plane + o, ok);
        cp_async4(d + 3 * S::NC, rg.seeds + S_DHY * plane + o, ok);
        cp_async4(d + 4 * S::NC, rg.seeds + S_DAZ * plane + o, ok);
        cp_async4(d + 5 * S::NC, rg.seeds + S_DHZ * plane + o, ok);
      }
    }
    for (int r = ty; r < NCI + 2; r += 8) {
      const int vi = ci_lo - 1 + r;
      const bool row_ok = !clamp || (vi >= 0 && vi < g.nx);
      const size_t rowo = row_ok ? (size_t)(clamp ? vi : wrapi(vi, g.nx)) * g.ny : 0;
      for (int c = tx; c < NCJ + 2; c += 32) {
        const int vj = cj_lo - 1 + c;
        bool ok = row_ok && (!clamp || (vj >= 0 && vj < g.ny));
        size_t o = ok ? rowo + (clamp ? vj : wrapi(vj, g.ny)) : 0;
        if (!EPSC_IN_BOUNDS(o, 1, plane, a.err)) ok = false, o = 0;
        float *d = sG + r * S::NGJ + c;
        cp_async4(d + 0 * S::NG, rg.seeds + S_GXX * plane + o, ok);
        cp_async4(d + 1 * S::NG, rg.seeds + S_GYX * plane + o, ok);
        cp_async4(d + 2 * S::NG, rg.seeds + S_GXY * plane + o, ok);
        cp_async4(d + 3 * S::NG, rg.seeds + S_GYY * plane + o, ok);
      }
    }
    cp_async_wait_all();
    __syncthreads();
  }
  // views of the staged maps (shifts are zero on the element-wise path)
  sU += sh;
  sIE2 += sh;
  sSeed += shj;
  sG += shg;

  // ---- Sobel^T: dU_c at the touched cells ----------------------------------
  // Cells whose three source rows and columns all exist and fold nothing
  // (every cell under the wrap rule; 1 <= cell <= n - 2 under edge
  // replicate) take the plain transposed stencil with its constant weights,
  //   d/dU of g_x: D(e) S(f),  of g_y: S(e) D(f),  D = (1, 0, -1), S = (1, 2, 1)
  // over source offsets e (rows) and f (columns); cells next to an edge
  // replicate use the folded weights.
  for (int c = tx; c < NCJ; c += 32) {
    const int vj = cj_lo + c;
    const bool col_real = vj >= 0 && vj < g.ny;
    const bool col_plain = !clamp || (vj >= 1 && vj <= g.ny - 2);
    float wdy[3], wsy[3];
    sobel_t_weights(clamp ? vj : wrapi(vj, g.ny), g.ny, BC, wdy, wsy);
    for (int r = ty; r < NCI; r += 8) {
      const int vi = ci_lo + r;
      float ux = 0.f, uy = 0.f;
      if (col_plain && (!clamp || (vi >= 1 && vi <= g.nx - 2))) {
        const float *a0 = sG + r * S::NGJ + c;   // source cell (vi - 1, vj - 1)
        const float *a2 = a0 + 2 * S::NGJ;        // source row vi + 1
        const float *b0 = a0 + S::NG;             // the g_y seeds of U_x
        const float *b1 = b0 + S::NGJ;
        const float *b2 = b0 + 2 * S::NGJ;
        ux = ((a0[0] + 2.f * a0[1] + a0[2]) - (a2[0] + 2.f * a2[1] + a2[2])) +
             ((b0[0] + 2.f * b1[0] + b2[0]) - (b0[2] + 2.f * b1[2] + b2[2]));
        const float *c0 = a0 + 2 * S::NG;         // the g_x, g_y seeds of U_y
        const float *c2 = c0 + 2 * S::NGJ;
        const float *d0 = a0 + 3 * S::NG;
        const float *d1 = d0 + S::NGJ;
        const float *d2 = d0 + 2 * S::NGJ;
        uy = ((c0[0] + 2.f * c0[1] + c0[2]) - (c2[0] + 2.f * c2[1] + c2[2])) +
             ((d0[0] + 2.f * d1[0] + d2[0]) - (d0[2] + 2.f * d1[2] + d2[2]));
      } else if (!clamp || (col_real && vi >= 0 && vi < g.nx)) {
        float wdx[3], wsx[3];
        sobel_t_weights(clamp ? vi : wrapi(vi, g.nx), g.nx, BC, wdx, wsx);
#pragma unroll
        for (int e = 0; e < 3; ++e) {
#pragma unroll
          for (int f = 0; f < 3; ++f) {
            const int o = (r + e) * S::NGJ + (c + f);   // source cell (vi - 1 + e, vj - 1 + f)
            const float gx_w = wdx[e] * wsy[f];          // d g_x / d U
            const float gy_w = wsx[e] * wdy[f];          // d g_y / d U
            ux += gx_w * sG[0 * S::NG + o] + gy_w * sG[1 * S::NG + o];
            uy += gx_w * sG[2 * S::NG + o] + gy_w * sG[3 * S::NG + o];
          }
        }
      }
      sdU[0 * S::NC + r * S::NCJ + c] = ux;
      sdU[1 * S::NC + r * S::NCJ + c] = uy;
    }
  }
  if (rest_pending && tid == 0 && !mbar_wait_bounded(&s_bar[1], 0u)) {
    atomicOr(a.err, ERRFLAG_TIMEOUT);
    mbar_wait_bounded(&s_bar[1], 0u);
    s_fail = 1;
  }
  __syncthreads();
  if (rest_pending && s_fail) return;

  // ---- du on the du region (in place over P' deps / 4) -----------------------
  const float q4 = 0.25f;
  // A du region clear of the edge-replicate fold (every subpixel inside the
  // region, none on row or column 0 or the last shifted cell; always under
  // the wrap rule) has unit multiplicities: the same values without the
  // edge logic.
  const bool du_plain = !clamp || (da_lo >= 1 && da_lo + DA <= g.mx - 1 && db_lo >= 1 &&
                                   db_lo + DB <= g.my - 1);
  if (du_plain) {
    const FastDiv ddb((unsigned)DB);
    for (int idx = tid; idx < DA * DB; idx += NTHREADS) {
      const int r = (int)ddb.div((unsigned)idx), c = idx - r * DB;
      const int va = da_lo + r, vb = db_lo + c;
      const float pd4 = sU[r * DBP + c];
      const float ie2 = sIE2[r * DBP + c];
      const int ic = (va >> 1) - ci_lo, is = ((va + 1) >> 1) - ci_lo;
      const int jc = (vb >> 1) - cj_lo, js = ((vb + 1) >> 1) - cj_lo;
      const int ox = ic * S::NCJ + js;
      const int oy = is * S::NCJ + jc;
      const int oz = is * S::NCJ + js;
      const float de = (sSeed[0 * S::NC + ox] - sSeed[1 * S::NC + ox] * ie2) +
                       (sSeed[2 * S::NC + oy] - sSeed[3 * S::NC + oy] * ie2) +
                       (sSeed[4 * S::NC + oz] - sSeed[5 * S::NC + oz] * ie2);
      const float dus = sdU[0 * S::NC + ox] + sdU[1 * S::NC + oy];
      sU[r * DBP + c] = fmaf(pd4, de, q4 * dus);
    }
  } else {
    const FastDiv ddb((unsigned)DB);
    for (int idx = tid; idx < DA * DB; idx += NTHREADS) {
      const int r = (int)ddb.div((unsigned)idx), c = idx - r * DB;
      const int va = da_lo + r, vb = db_lo + c;
      if (clamp && (va < 0 || va >= g.mx || vb < 0 || vb >= g.my)) continue;   // stays zero
      const float pd4 = sU[r * DBP + c];       // P'(u) (eps_core - eps_clad) / 4
      const float ie2 = sIE2[r * DBP + c];     // 1 / eps^2
      // cells containing (va, vb): centred axis -> v >> 1, shifted axis -> (v+1) >> 1
      const int ic = (va >> 1) - ci_lo, is = ((va + 1) >> 1) - ci_lo;
      const int jc = (vb >> 1) - cj_lo, js = ((vb + 1) >> 1) - cj_lo;
      // multiplicities of the shifted axis (edge replicate maps subpixel -1 onto 0)
      float ma = 1.f, mb = 1.f;
      if (clamp) {
        ma = ((va + 1) >> 1) >= g.nx ? 0.f : (va == 0 ? 2.f : 1.f);
        mb = ((vb + 1) >> 1) >= g.ny ? 0.f : (vb == 0 ? 2.f : 1.f);
      }
      const int ox = ic * S::NCJ + js;   // x: centred in a, shifted in b
      const int oy = is * S::NCJ + jc;   // y: shifted in a, centred in b
      const int oz = is * S::NCJ + js;   // z: shifted in both
      const float de = mb * (sSeed[0 * S::NC + ox] - sSeed[1 * S::NC + ox] * ie2) +
                       ma * (sSeed[2 * S::NC + oy] - sSeed[3 * S::NC + oy] * ie2) +
                       ma * mb * (sSeed[4 * S::NC + oz] - sSeed[5 * S::NC + oz] * ie2);
      const float dus = mb * sdU[0 * S::NC + ox] + ma * sdU[1 * S::NC + oy];
      sU[r * DBP + c] = fmaf(pd4, de, q4 * dus);
    }
  }
  __syncthreads();

  // ---- K^T gather on the gather region ----------------------------------
  {
    const FastDiv dgb((unsigned)GB);
    for (int item = tid; item < NSTRIP * GB; item += NTHREADS) {
      const int st = (int)dgb.div((unsigned)item), col = item - st * GB;
      const int r0 = st * NA_B;
      float hi[NA_B];
      strip_stencil<RP1, NA_B>(sU + r0 * DBP + col, DBP, a, hi);
#pragma unroll
      for (int k = 0; k < NA_B; ++k) {
        if (r0 + k < GA) sdc[(r0 + k) * S::GB_MAX + col] = hi[k];
      }
    }
  }
  __syncthreads();

  // ---- fold extended positions onto the edge and write ------------------
  if (ga_lo == a0 && gb_lo == b0 && ga_hi == aend && gb_hi == bend) {
    // no extended positions: each output is its own K^T result
    for (int r = ty; r < aend - a0; r += 8) {
      for (int c = tx; c < bend - b0; c += 32) {
        const size_t go = (size_t)(a0 + r) * g.my + b0 + c;
        if (EPSC_IN_BOUNDS(go, 1, (size_t)g.mx * g.my, a.err)) rg.dJdC[go] = sdc[r * S::GB_MAX + c];
      }
    }
    return;
  }
  for (int r = ty; r < aend - a0; r += 8) {
    const int ga = a0 + r;
    int ra0 = ga - ga_lo, ra1 = ra0;
    if (clamp) {
      if (ga == 0) ra0 = 0;
      if (ga == g.mx - 1) ra1 = GA - 1;
    }
    for (int c = tx; c < bend - b0; c += 32) {
      const int gb = b0 + c;
      int rb0 = gb - gb_lo, rb1 = rb0;
      if (clamp) {
        if (gb == 0) rb0 = 0;
        if (gb == g.my - 1) rb1 = GB - 1;
      }
      float acc = 0.f;
      for (int x = ra0; x <= ra1; ++x)
        for (int y = rb0; y <= rb1; ++y) acc += sdc[x * S::GB_MAX + y];
      const size_t go = (size_t)ga * g.my + gb;
      if (EPSC_IN_BOUNDS(go, 1, (size_t)g.mx * g.my, a.err)) rg.dJdC[go] = acc;
    }
  }
}

template <int RP1, int BC>
__global__ void __launch_bounds__(NTHREADS) bwd_kernel(const __grid_constant__ BwdArgsR<RP1> a) {
  bwd_tile<RP1, BC>(a, a.r, (blockIdx.y + a.ty0) * TA, blockIdx.x * TB);
}

// The same scatter with bulk-copy staging of the interior tiles.
template <int RP1, int BC>
__global__ void __launch_bounds__(NTHREADS) bwd_tma_kernel(const __grid_constant__ BwdTmaArgsR<RP1> a) {
  bwd_tile<RP1, BC, true>(a, a.r, (blockIdx.y + a.ty0) * TA, blockIdx.x * TB, &a.maps[0]);
}

// Batched scatter of one radius group with bulk-copy staging: block b takes
// tile b - tile_start[k] of region k (tiles of TA x TBW subpixels), staged
// through region k's maps.
template <int RP1, int BC, int TBW = TB>
__global__ void __launch_bounds__(NTHREADS) bwd_tma_batched_kernel(const __grid_constant__ BwdTmaBatchArgs a) {
  int k, t;
  batch_tile(a, blockIdx.x, k, t);
  const int tj = a.tiles_j[k];
  const int ti = t / tj;
  bwd_tile<RP1, BC, true, TBW>(a, a.r[k], ti * TA, (t - ti * tj) * TBW,
                               a.has_maps[k] ? &a.maps[4 * k] : nullptr);
}

template <int RP1, int BC, int TBW = TB>
__global__ void __launch_bounds__(NTHREADS) bwd_batched_kernel(const __grid_constant__ BwdBatchArgs a) {
  int k, t;
  batch_tile(a, blockIdx.x, k, t);
  const int tj = a.tiles_j[k];
  const int ti = t / tj;
  bwd_tile<RP1, BC, false, TBW>(a, a.r[k], ti * TA, (t - ti * tj) * TBW);
}

}  // namespace epsc
