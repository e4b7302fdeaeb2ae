/*
 * epschain — GB300 (sm_103a) library for the differentiable map from
 * topology-optimisation control variables C to the subpixel-smoothed
 * anisotropic permittivity eps_hat on an FDTD Yee grid, and its adjoint.
 *
 * Method: Sofronov, Yakovleva, Yakubovich, "Accelerated inverse design of
 * passive Si photonics" (arXiv 2505.03352).
 *   - density mixing and 2-D mask extruded in z ............. Sec. 3, par. 1
 *   - filter (conic basis, Eq. 2) and tanh projection ........ Eq. 2, 3, 6
 *   - per-component dual-cell means, half-cell shift ......... Eq. 8, Sec. 3
 *   - Sobel normals and anisotropic smoothing ................ Eq. 7, Sec. 3
 *   - vector-Jacobian product without forming J .............. Sec. 3 (end)
 *   - adjoint gradient dJ/dC = -2 Re(deps/dC . (E_F E_A)) .... Eq. 1 + footnote
 *
 * Conventions shared by every entry point:
 *   * Layouts are C order.  C and dJ/dC are float32 [mx][my] (controls at
 *     pitch d, `sub` = 2 subpixels per Yee cell per in-plane axis, so the Yee
 *     grid is nx = mx/2 by ny = my/2 by nz).  eps_hat and real cotangents G
 *     are float32 [3][nx][ny][nz] (component xx, yy, zz; z fastest).  Fields
 *     are complex64 [3][nx][ny][nz] with interleaved (re, im), one array per
 *     wavelength; only the planes where eps_hat depends on C are read.
 *   * Every pointer marked "device" is device memory owned by the caller.
 *     The library never allocates device memory inside a call; scratch space
 *     is the caller's workspace, sized by eps_workspace_size().
 *   * Calls are asynchronous on `stream` (a cudaStream_t; NULL is the legacy
 *     default stream).  Argument errors return before any launch, with
 *     nothing written.  Launch failures return EPS_ERR_CUDA.  Device-side
 *     error flags are reported by eps_sync_status().
 *   * Calls on different streams are independent and may run concurrently
 *     when each has its own workspace (the pipelined part of multi-wave
 *     eps_vjp calls runs on one library stream per device: see eps_vjp).
 */
#ifndef EPSCHAIN_H
#define EPSCHAIN_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Same type as cudaStream_t. */
typedef struct CUstream_st *eps_stream_t;

typedef enum {
  EPS_OK = 0,
  EPS_ERR_INVALID_ARG = 1,   /* null pointer, bad enum, non-finite parameter */
  EPS_ERR_SHAPE = 2,         /* sizes inconsistent or out of range */
  EPS_ERR_WORKSPACE = 3,     /* workspace null, misaligned or too small */
  EPS_ERR_UNSUPPORTED = 4,   /* valid request outside what is built (sub != 2, radius > max) */
  EPS_ERR_CUDA = 5,          /* a CUDA runtime call failed */
  EPS_ERR_DEVICE_TIMEOUT = 6,/* a bounded device-side wait gave up */
  EPS_ERR_DEVICE_BOUNDS = 7  /* a device-side bounds check fired (debug-bounds builds) */
} eps_status_t;

typedef enum { EPS_BC_CLAMP = 0, EPS_BC_PERIODIC = 1 } eps_bc_t;

typedef enum {
  EPS_FIELD_C64 = 0,          /* complex64 [3][nx][ny][nz] */
  EPS_FIELD_BF16X2_SCALED = 1,/* bf16 (re, im) pairs, slab planes only; see eps_field_pack */
  EPS_FIELD_F16X2_SCALED = 2  /* fp16 (re, im) pairs, slab planes only; see eps_field_pack */
} eps_field_t;

/* flags */
#define EPS_FLAG_OFFDIAG 1  /* eps_forward also writes the xy inverse-permittivity term */
#define EPS_FLAG_NORMALS_3D 2 /* 3-D normals at the slab faces (forward only; see eps_forward) */

#define EPS_MAX_LAMBDA 16    /* wavelengths per eps_vjp call */
#define EPS_MAX_BATCH 64     /* regions per batched call */
#define EPS_MAX_BATCH_LAMBDA 4 /* wavelengths per region in a batched call */
#define EPS_MAX_RADIUS 12.0f /* largest conic filter radius (subpixels) */

/*
 * One design region.  Eq. 2 / 3 / 6 / 7 parameters plus the slab geometry.
 *   mx, my     control grid, both even, 2 <= mx, my
 *   sub        subpixels per Yee cell per in-plane axis; must be 2
 *   nz         Yee cells along z
 *   slab_k0    lower Ez face plane of the slab; -1 picks (nz - nk - 1) / 2.
 *              Faces sit at z = (k0 + 1/2) D and (k0 + nk + 1/2) D, so
 *              Ex/Ey planes k0+1 .. k0+nk and Ez planes k0+1 .. k0+nk-1 lie
 *              in the slab and Ez planes k0, k0+nk straddle its faces.
 *              Requires 0 <= k0 and k0 + nk <= nz - 1.
 *   slab_nk    slab thickness in Yee cells, >= 1
 *   radius     conic filter radius R in subpixels, 0 < R <= EPS_MAX_RADIUS;
 *              taps at integer offsets with r < R, weight (1 - r/R)/sum
 *   beta, eta  projection rho = (1 + tanh(beta (u - eta))) / 2
 *   eps_core, eps_clad  permittivities mixed by rho (Sec. 3)
 *   bc         eps_bc_t: edge rule for the filter, the dual cells and Sobel
 *   flags      EPS_FLAG_*
 */
typedef struct {
  int32_t mx, my, sub, nz, slab_k0, slab_nk;
  float radius, beta, eta, eps_core, eps_clad;
  int32_t bc, flags;
} eps_problem_t;

/* Human-readable name of a status code (static string, never NULL). */
const char *eps_status_string(eps_status_t status);

/*
 * Workspace bytes eps_vjp / eps_vjp_real need for `prob` (n_lambda is
 * accepted for forward compatibility; the size does not depend on it).
 * Workspace pointers must be 256-byte aligned.
 */
eps_status_t eps_workspace_size(const eps_problem_t *prob, int32_t n_lambda, size_t *bytes);

/*
 * Forward chain (Eq. 2 -> 6 -> mixing -> Eq. 8 -> Sobel normals -> Eq. 7):
 *   C        device, float32 [mx][my]
 *   eps      device, float32 [3][nx][ny][nz], written in full (cladding
 *            planes get eps_clad)
 *   offdiag  device, float32 [2][nx][ny][nz] or NULL; written only when
 *            flags has EPS_FLAG_OFFDIAG: n_x n_y (<1/eps> - 1/<eps>) at the
 *            Ex points (index 0) and Ey points (index 1) on the slab planes,
 *            0 elsewhere.  Forward only: Eq. 1 uses zero off-diagonals.
 * EPS_FLAG_NORMALS_3D (forward only; eps_vjp* and the batched calls return
 * EPS_ERR_UNSUPPORTED with it): the Ez cells of the two face planes k0 and
 * k0 + nk, half slab and half cladding, take Eq. 7 in tensor form with a
 * 3-D normal, eps^-1 = n n^T <eps^-1> + (I - n n^T) / <eps>, where
 * <eps> = (A_z + eps_clad)/2, <eps^-1> = (H_z + 1/eps_clad)/2 and n is the
 * normalised Sobel-consistent gradient of the cell-averaged 3-D density
 * (g_x, g_y = half the Sobel of U_z, g_z = +4 U_z at k0 and -4 U_z at
 * k0 + nk; n = z where |g|^2 <= 1e-12).  eps_zz on the face planes becomes
 * 1 / (eps^-1)_zz; with EPS_FLAG_OFFDIAG as well, offdiag is [4][nx][ny][nz]
 * and indices 2 and 3 hold (eps^-1)_zx and (eps^-1)_zy at the Ez points
 * (non-zero on the face planes only).  The xz and yz terms at the Ex and Ey
 * points vanish in this geometry (their dual cells do not cross a face).
 */
eps_status_t eps_forward(const eps_problem_t *prob, const float *C, float *eps,
                         float *offdiag, eps_stream_t stream);

/*
 * Adjoint gradient, Eq. 1:  dJdC = (d eps_hat / dC)^T W,
 *   W = scale * Re( sum_l  s_l * E_F,l (.) E_A,l ),  elementwise and
 *   unconjugated (Eq. 1 footnote), scale = -2 for d|alpha|^2/dC.
 *   n_lambda      1 .. EPS_MAX_LAMBDA wavelengths (host count)
 *   field_type    eps_field_t of EF / EA
 *   EF, EA        host arrays of n_lambda device pointers, each 16-byte
 *                 aligned.  C64: complex64 [3][nx][ny][nz] (nz even).
 *                 Packed types: buffers written by eps_field_pack.
 *   field_scales  host float [n_lambda][2][3] (wavelength, field F/A,
 *                 component) multiplying each stored component, or NULL
 *                 for all ones
 *   dJdC          device, float32 [mx][my], overwritten
 *   eps_out       device float32 [3][nx][ny][nz] or NULL; when given the
 *                 forward eps_hat is written by the same pass (fused
 *                 forward + VJP)
 *   ws, ws_bytes  device workspace of at least eps_workspace_size() bytes
 * The filtered density and projection are recomputed from C; nothing from
 * an earlier eps_forward is reused.
 * Streams: all work is ordered on `stream` as one operation.  Problems of
 * more than one wave of stencil tiles with the edge-replicate rule and
 * complex64 fields run as a band pipeline: the field contraction streams
 * the columns band by band on `stream`, and a library-owned stream of the
 * current device (created with its events on first use, kept for the
 * process, no device memory) runs the stencil, each band's seeds and the
 * finished rows' scatter alongside; it is forked from `stream` by an event
 * at the start of the call and joined back before the call's last
 * operation, so work queued on `stream` after the call (and graph capture
 * of `stream`) sees a completed call.  Calls from several host threads
 * share that stream, so their pipelined parts run one after another.
 */
eps_status_t eps_vjp(const eps_problem_t *prob, const float *C, int32_t n_lambda,
                     int32_t field_type, const void *const *EF, const void *const *EA,
                     const float *field_scales, float scale, float *dJdC, float *eps_out,
                     void *ws, size_t ws_bytes, eps_stream_t stream);

/*
 * eps_vjp plus the value of the Eq. 1 surrogate whose gradient dJdC is:
 *   S = sum over the J-support voxels of eps_hat * W,
 * W as for eps_vjp (scale * Re(sum_l s_l E_F,l (.) E_A,l)).  The J-support
 * voxels are those whose eps_hat depends on C: Ex and Ey planes k0+1 ..
 * k0+nk and Ez planes k0 .. k0+nk (Sec. 3 extrusion with the z rules of
 * eps_forward); the other voxels hold eps_clad and would add a constant
 * independent of C.  This is the adjoint method's linearisation of the
 * objective around the current design (Eq. 1: dS/dC = dJ/dC) and gives
 * automatic-differentiation frameworks a scalar to hang the gradient on.
 *   S   device double, 8-byte aligned, overwritten (set to 0 on the stream
 *       first, then accumulated by the kernels in FP64; the order of the
 *       additions is not fixed, so S can differ between calls in its last
 *       bits)
 * Other arguments, results and errors as eps_vjp; a NULL or misaligned S
 * returns EPS_ERR_INVALID_ARG.  An empty problem or n_lambda = 0 gives S = 0.
 */
eps_status_t eps_vjp_surrogate(const eps_problem_t *prob, const float *C, int32_t n_lambda,
                               int32_t field_type, const void *const *EF, const void *const *EA,
                               const float *field_scales, float scale, float *dJdC,
                               float *eps_out, double *S, void *ws, size_t ws_bytes,
                               eps_stream_t stream);

/*
 * Vector-Jacobian product for an arbitrary real cotangent (Sec. 3, end):
 *   dJdC = (d eps_hat / dC)^T G,   G device float32 [3][nx][ny][nz].
 * Used by autograd backward passes; recomputes the forward from C.
 */
eps_status_t eps_vjp_real(const eps_problem_t *prob, const float *C, const float *G,
                          float *dJdC, void *ws, size_t ws_bytes, eps_stream_t stream);

/*
 * Batched calls: n <= EPS_MAX_BATCH independent design regions, each with
 * its own eps_problem_t (sizes, radius, beta, slab, boundary rule), in one
 * call.  Host arrays of n device pointers (C, eps / dJdC / eps_out); EF and
 * EA are host arrays of n * n_lambda device pointers, region-major
 * (EF[k * n_lambda + l]); field_scales, if not NULL, is host float
 * [n][n_lambda][2][3].  n_lambda <= EPS_MAX_BATCH_LAMBDA; complex64 fields
 * only; eps_out may be NULL or hold NULL entries.  The workspace is the
 * regions' eps_workspace_size() laid end to end (eps_batched_workspace_size).
 * One contraction launch covers every region; the stencil and scatter
 * launches follow the batch's launch shapes (below: by default one launch
 * each per radius group).  Results equal the per-region calls'.
 */
eps_status_t eps_batched_workspace_size(int32_t n, const eps_problem_t *probs, int32_t n_lambda,
                                        size_t *bytes);
eps_status_t eps_forward_batched(int32_t n, const eps_problem_t *probs, const float *const *C,
                                 float *const *eps, eps_stream_t stream);
eps_status_t eps_vjp_batched(int32_t n, const eps_problem_t *probs, const float *const *C,
                             int32_t n_lambda, int32_t field_type, const void *const *EF,
                             const void *const *EA, const float *field_scales, float scale,
                             float *const *dJdC, float *const *eps_out, void *ws, size_t ws_bytes,
                             eps_stream_t stream);

/*
 * Launch shapes of the batched calls, and their autotuner.
 *
 * eps_vjp_batched runs in one of two launch forms: one persistent
 * mixed-radius stencil launch and one scatter launch per boundary rule
 * (`multi` = 1; a batch that holds two different radii of the same radius
 * class ceil(R) needs one more launch per extra radius), or one stencil
 * and one scatter launch per (radius, boundary rule) group with one block
 * per tile (`multi` = 0, the default).  The shapes are: that form, the persistent
 * stencil and scatter blocks per SM, the contraction's blocks per SM, and
 * how many eps_hat components are staged per round of bulk stores (1 or
 * 3; fewer means less shared memory per block), and where the adjoint
 * seeds (linear in the Eq. 1 column sums W) are finished: in the stencil,
 * which then waits for the contraction, or by a separate seeds kernel
 * (`defer_seeds` = 1) so that stencil tiles never wait.  Results do not depend on
 * the shapes (every output element is computed the same way).
 *
 * eps_autotune_batched takes the arguments of eps_vjp_batched plus `reps`
 * (1 .. 1000): it runs the batched call with candidate shapes (coordinate
 * descent, two sweeps, each candidate timed with CUDA events over `reps`
 * calls after one warm-up call), keeps the fastest, and caches it for this
 * batch (keyed by n, n_lambda and every eps_problem_t) in the process, where
 * later eps_vjp_batched calls on the same batch pick it up.  It writes the
 * same outputs as eps_vjp_batched, synchronises `stream`, and returns
 * EPS_ERR_UNSUPPORTED while `stream` is capturing (tune first, then
 * capture).  `result` (host, may be NULL) receives the choice and the mean
 * milliseconds per call with the default and the chosen shapes.
 */
typedef struct {
  int32_t multi, stencil_blocks_per_sm, scatter_blocks_per_sm, contract_blocks_per_sm;
  int32_t stage_components, defer_seeds, evaluations;
  float default_ms, tuned_ms;
  int32_t scatter_bulk_staging, scatter_tile_cols, concurrent_groups;
} eps_tuning_t;

/*
 * eps_batched_set_tuning stores launch shapes for a batch directly (the same
 * cache eps_autotune_batched fills; evaluations, default_ms and tuned_ms are
 * ignored).  n_lambda is the wavelength count of the eps_vjp_batched calls
 * it applies to, or -1 for eps_forward_batched.  Fields: multi 0 or 1,
 * blocks per SM 1 .. 16 (stencil, scatter) and 1 .. 64 (contraction),
 * stage_components 1 or 3, defer_seeds 0 or 1, scatter_bulk_staging 0 or 1,
 * scatter_tile_cols 0 (= 32), 32 or 64, concurrent_groups 0 or 1; else
 * EPS_ERR_INVALID_ARG.
 * scatter_bulk_staging (grouped form, radius classes 3 and up): 1 stages the
 * scatter's interior tiles through bulk tensor copies (each launch carries
 * up to 32 regions' tensor maps in its parameters), 0 gathers element by
 * element.  scatter_tile_cols (grouped form): the scatter's tile shape,
 * 32 x 32 or 32 x 64 control subpixels (the wide tile recomputes fewer halo
 * subpixels per output but fits two blocks on an SM instead of three).
 * concurrent_groups (grouped form): 1 puts each radius group's stencil and
 * scatter launches on an auxiliary stream of their own (one set of up to 8
 * per device, created on first use and kept for the process; forked from and
 * joined back to `stream` with events, so stream order and graph capture of
 * `stream` hold), the stencils writing seed factors beside the contraction
 * and a seeds launch on `stream` applying the column sums; calls from
 * several host threads share the set and enqueue one after another.
 * The contraction streams the fields of every region through bulk tensor
 * copies (up to 4 blocks per SM, so larger values act as 4) when the batch
 * needs at most 192 tensor maps (n * n_lambda * 2); larger batches use
 * register loads with 4 * contract_blocks_per_sm blocks per SM.  Default
 * shapes: grouped form, 3 contraction blocks per SM, 1 component staged,
 * seeds finished in the stencil, bulk-copy scatter staging, 32 x 32 scatter
 * tiles.
 */
eps_status_t eps_batched_set_tuning(int32_t n, const eps_problem_t *probs, int32_t n_lambda,
                                   const eps_tuning_t *tuning);
eps_status_t eps_autotune_batched(int32_t n, const eps_problem_t *probs, const float *const *C,
                                  int32_t n_lambda, int32_t field_type, const void *const *EF,
                                  const void *const *EA, const float *field_scales, float scale,
                                  float *const *dJdC, float *const *eps_out, void *ws,
                                  size_t ws_bytes, int32_t reps, eps_tuning_t *result,
                                  eps_stream_t stream);

/*
 * Reduced-precision field storage (BF16 / FP16 complex pairs with one
 * scale per component) for eps_vjp's contraction.  A packed field buffer
 * holds only the planes eps_hat depends on:
 *   bytes [0, 16)    float scale[3], float pad
 *   bytes [16, ...)  [3][nx][ny][NP] (re, im) pairs of bf16 or fp16, the
 *                    planes k0 .. k0+NP-1 of each component divided by its
 *                    scale, NP = slab_nk + 1 rounded up to a multiple of 4
 * and decodes as value = scale[c] * stored.  scale = max(|re|, |im|) over
 * the component's support planes / target (1 for bf16, 2^14 for fp16).
 * Accumulation in the contraction is FP32.  The reduced precision of the
 * stored fields is the only source of extra error (stated, not bounded).
 *
 * eps_packed_field_bytes: size of one packed field buffer for `prob`.
 * eps_field_pack: pack one complex64 field [3][nx][ny][nz] (device, 8-byte
 *   aligned) into `dst` (device, 16-byte aligned, dst_bytes at least
 *   eps_packed_field_bytes); asynchronous on `stream`.
 * eps_vjp with field_type EPS_FIELD_BF16X2_SCALED / EPS_FIELD_F16X2_SCALED
 * takes packed buffers in EF / EA; field_scales (host, optional) multiply
 * on top of the buffers' own scales.
 */
eps_status_t eps_packed_field_bytes(const eps_problem_t *prob, int32_t field_type, size_t *bytes);
eps_status_t eps_field_pack(const eps_problem_t *prob, int32_t field_type, const void *src,
                            void *dst, size_t dst_bytes, eps_stream_t stream);

/*
 * Morphological filtering (Sec. 3, Eq. 3-6).  The chain becomes
 *   u = K * C (Eq. 2),  rho_0 = (1 + tanh(beta (u - eta))) / 2 (Eq. 3),
 *   rho_{k+1} = op_k(rho_k) for the listed operations, with the normalised
 *     disk K_m (integer subpixel offsets with p^2 + q^2 <= radius^2, each
 *     weight 1/count) and the prob's boundary rule:
 *       dilate (Eq. 4):  (1/alpha) log sum_d K_m(d) exp(alpha rho[x+d])
 *       erode  (Eq. 5):  1 - (1/alpha) log sum_d K_m(d) exp(alpha (1 - rho[x+d]))
 *   then the final projection at 1/2 (Eq. 6) and the rest of the chain, with
 *   the Sobel normals taken from rho_tilde = rho_n (the density whose 1/2
 *   level set the final projection draws).  That is: the base chain of
 *   eps_forward applied to rho_n with an identity filter and eta = 1/2.
 *   alpha   (0, EPS_MORPH_MAX_ALPHA]; App. B uses 20
 *   radius  disk radius d/2 in subpixels, 0 <= radius < EPS_MAX_RADIUS
 *   n_ops   0 .. EPS_MORPH_MAX_OPS operations ops[0 .. n_ops-1], each an
 *           eps_morph_op_t, applied in order (a closing then an opening is
 *           DILATE, ERODE, ERODE, DILATE)
 * The calls take a workspace of eps_morph_workspace_size() bytes (256-byte
 * aligned); it holds the density maps rho_0 .. rho_n, P'(u), two adjoint
 * maps and, after them, the base chain's workspace.  eps_vjp_morph and
 * eps_vjp_real_morph have the arguments and results of eps_vjp /
 * eps_vjp_real with dJ/dC taken through the whole chain.  Errors return
 * before any launch.
 */
#define EPS_MORPH_MAX_OPS 8
#define EPS_MORPH_MAX_ALPHA 60.0f
typedef enum { EPS_MORPH_DILATE = 0, EPS_MORPH_ERODE = 1 } eps_morph_op_t;
typedef struct {
  float alpha;
  float radius;
  int32_t n_ops;
  int32_t ops[EPS_MORPH_MAX_OPS];
} eps_morph_t;

eps_status_t eps_morph_workspace_size(const eps_problem_t *prob, const eps_morph_t *morph,
                                      int32_t n_lambda, size_t *bytes);
eps_status_t eps_forward_morph(const eps_problem_t *prob, const eps_morph_t *morph,
                               const float *C, float *eps, float *offdiag, void *ws,
                               size_t ws_bytes, eps_stream_t stream);
eps_status_t eps_vjp_morph(const eps_problem_t *prob, const eps_morph_t *morph, const float *C,
                           int32_t n_lambda, int32_t field_type, const void *const *EF,
                           const void *const *EA, const float *field_scales, float scale,
                           float *dJdC, float *eps_out, void *ws, size_t ws_bytes,
                           eps_stream_t stream);
eps_status_t eps_vjp_real_morph(const eps_problem_t *prob, const eps_morph_t *morph,
                                const float *C, const float *G, float *dJdC, void *ws,
                                size_t ws_bytes, eps_stream_t stream);

/*
 * Coarse control variables (Eq. 2 with the basis functions shifted to the
 * nodes of a rectangular grid that spans the design region, as in the
 * paper's 36 x 36 controls over 210 x 210 cells).  The node values c are
 * float32 [ncx][ncy] (device); node i sits at X_i = i h_x, h_x =
 * mx / (ncx - 1) subpixels (edge to edge), subpixel a's centre at a + 1/2,
 * and the basis is the tensor-product hat B(t) = max(0, 1 - |t|) (a reading:
 * compact, a partition of unity, exact on linear functions):
 *   Phi[a][b] = sum_{i,j} c[i][j] B((a + 1/2 - X_i)/h_x) B((b + 1/2 - Y_j)/h_y).
 * Phi replaces the conic filter's output: the base chain runs on Phi with
 * an identity filter (prob->radius is validated but not used) and
 * projection threshold prob->eta.  eps_vjp_coarse / eps_vjp_real_coarse
 * have the arguments of eps_vjp / eps_vjp_real with dJdc float32
 * [ncx][ncy] (device).  ncx, ncy >= 2.  Workspace: Phi, d/dPhi and the
 * base chain's workspace, eps_coarse_workspace_size() bytes, 256-byte
 * aligned.
 */
typedef struct {
  int32_t ncx, ncy;
} eps_coarse_t;

eps_status_t eps_coarse_workspace_size(const eps_problem_t *prob, const eps_coarse_t *coarse,
                                       int32_t n_lambda, size_t *bytes);
eps_status_t eps_forward_coarse(const eps_problem_t *prob, const eps_coarse_t *coarse,
                                const float *c, float *eps, float *offdiag, void *ws,
                                size_t ws_bytes, eps_stream_t stream);
eps_status_t eps_vjp_coarse(const eps_problem_t *prob, const eps_coarse_t *coarse, const float *c,
                            int32_t n_lambda, int32_t field_type, const void *const *EF,
                            const void *const *EA, const float *field_scales, float scale,
                            float *dJdc, float *eps_out, void *ws, size_t ws_bytes,
                            eps_stream_t stream);
eps_status_t eps_vjp_real_coarse(const eps_problem_t *prob, const eps_coarse_t *coarse,
                                 const float *c, const float *G, float *dJdc, void *ws,
                                 size_t ws_bytes, eps_stream_t stream);

/*
 * One optimiser iteration on the device (Sec. 4): Adam (Eq. 10-11) over the
 * controls, fused with the count of gray subpixels of the design, then the
 * beta_max control (Eq. 15) and the beta schedule (Eq. 14).
 *
 * Readings (the paper is silent): a subpixel is gray when its projected
 * density rho satisfies gray_tol < rho < 1 - gray_tol; the unbinarity is
 * u = max(gray count, 1) / (mx my); t starts at its first sample
 * (1/u - 1)/beta, then t <- gamma t + (1 - gamma)(1/u - 1)/beta and
 * beta_max <- gamma beta_max + (1 - gamma)(1/u0 - 1)/t; iteration i is
 * 1-based, the same i as Adam's bias correction, and the beta of iteration
 * i is beta_min + (beta_max - beta_min)(exp((i/n_iter)^2) - 1)/(e - 1).
 *
 * eps_opt_t (host):  lr (the paper's eta), b1, b2, adam_eps, gray_tol in
 *   (0, 1/2), gamma in [0, 1), u0 in (0, 1), beta_min > 0,
 *   beta_max0 >= beta_min (initial beta_max), n_iter >= 1 (N_i).
 *   App. B: b1 = 0.9, b2 = 0.999, lr = 0.001, gamma = 0.95, u0 = 0.01,
 *   beta_min = 10.
 * eps_opt_state_t (DEVICE memory, 32 bytes, 4-byte aligned, caller-owned):
 *   step        completed iterations (the next is step + 1)
 *   beta        beta of the next iteration: pass it as prob->beta of the
 *               next eps_vjp call (read it back, or keep the loop on the
 *               device with the same value)
 *   beta_max, t the Eq. 15 state;  unbinarity, gray: u and the gray count
 *               of the last iteration;  gray_acc, ticket: scratch, zero
 *               between calls.
 * eps_opt_init writes the initial state (step 0, beta of iteration 1,
 *   beta_max0) with a kernel on `stream`.
 * eps_opt_step performs iteration step + 1:
 *   prob, morph   the problem (and the morphology, or NULL) of the eps_vjp /
 *                 eps_vjp_real / eps_vjp_morph / eps_vjp_real_morph call
 *                 whose workspace `ws` (ws_bytes) holds the design of C at
 *                 beta = prob->beta; prob->beta must equal state->beta, be
 *                 > 0, and eps_core must differ from eps_clad.  The gray
 *                 count reads the per-subpixel factor that call left there.
 *   C, M, V       device float32 [mx][my], 16-byte aligned, updated in place
 *                 (M and V start at zero)
 *   G             device float32 [mx][my], 16-byte aligned: the gradient of
 *                 the objective being minimised at C
 * Successive steps on one state must be ordered on one stream.
 */
typedef struct {
  float lr, b1, b2, adam_eps, gray_tol, gamma, u0, beta_min, beta_max0;
  int32_t n_iter;
} eps_opt_t;

typedef struct {
  int32_t step;
  float beta, beta_max, t, unbinarity;
  uint32_t gray, gray_acc, ticket;
} eps_opt_state_t;

eps_status_t eps_opt_init(const eps_opt_t *opt, eps_opt_state_t *state, eps_stream_t stream);
eps_status_t eps_opt_step(const eps_problem_t *prob, const eps_morph_t *morph, const eps_opt_t *opt,
                          eps_opt_state_t *state, float *C, const float *G, float *M, float *V,
                          const void *ws, size_t ws_bytes, eps_stream_t stream);

/*
 * Synchronise `stream`, then return (and clear) any device-side error flag
 * raised by earlier calls on this device: EPS_ERR_DEVICE_TIMEOUT or
 * EPS_ERR_DEVICE_BOUNDS, else EPS_OK; EPS_ERR_CUDA if the sync failed.
 */
eps_status_t eps_sync_status(eps_stream_t stream);

/*
 * Self-test of the device-side timeout path.  Launches one block that
 * waits, with the same bounded mbarrier wait the contraction kernels use,
 * on a barrier nothing arrives at, giving up after `cycles` SM clock cycles
 * (1 .. 2^31; the kernels' own limit is 2^31, about one second).  The block
 * then records EPS_ERR_DEVICE_TIMEOUT in the device error flag and returns:
 * no fault, trap or hang, and the context stays usable.  The next
 * eps_sync_status(stream) reports the timeout and clears it.  Out-of-range
 * `cycles`: EPS_ERR_INVALID_ARG before any launch.
 */
eps_status_t eps_selftest_timeout(int64_t cycles, eps_stream_t stream);

/*
 * Debug bounds checks.  A library built with -DEPS_DEBUG_BOUNDS
 * (libepschain_debug.so, `build_lib --debug-bounds`) tests the index of
 * every global load and store of its kernels that is not bounded by its
 * own loop (staging gathers, stores, the register-load field reads; TMA
 * copies are bounded by their tensor maps) against the extent of its
 * buffer; an index outside records EPS_ERR_DEVICE_BOUNDS in the device
 * error flag and the access is skipped (a load reads zero).  Nothing traps.
 * eps_selftest_bounds launches one thread whose check fails without
 * touching memory, so eps_sync_status then reports EPS_ERR_DEVICE_BOUNDS;
 * in a release build it returns EPS_ERR_UNSUPPORTED.
 */
eps_status_t eps_selftest_bounds(eps_stream_t stream);

/*
 * eps_vjp without a caller workspace.  The paper has no counterpart: this
 * is for host programs that cannot allocate device memory where they need
 * the gradient (a framework pool that already holds the whole device, or a
 * loop that must not call cudaMalloc after start-up because it can
 * synchronise the device).  It allocates nothing: its scratch is one static
 * device array of EPS_STATIC_WS_BYTES per GPU, created when the library's
 * device code is loaded on that GPU and held until the process exits.
 *   - Arguments are those of eps_vjp minus ws / ws_bytes; results are the
 *     same as eps_vjp's.
 *   - Problems whose eps_workspace_size() exceeds EPS_STATIC_WS_BYTES are
 *     rejected with EPS_ERR_WORKSPACE before any launch (104 bytes per Yee
 *     column: about 161 000 columns, e.g. 400 x 400).
 *   - The first call on a device looks up the array's device address (set-up,
 *     once per device, with that device current); make that first call
 *     before any stream capture.  The address is kept for the rest of the
 *     process and belongs to the device's primary context: calls made with
 *     another context current on that device, or after cudaDeviceReset()
 *     on it, are not supported.
 *   - All calls on a device share the one array: calls that can overlap on
 *     the GPU (different streams, or host threads without ordering) race and
 *     must be serialised by the caller.  Nothing in the array needs to start
 *     at zero; it keeps whatever the last call left there.
 *   - Streams as in eps_vjp: a problem of more than one wave of stencil
 *     tiles runs as its band pipeline, whose first call on a device creates
 *     the library's pipeline stream and events (no device memory); make
 *     such a call once before any stream capture as well.
 */
#define EPS_STATIC_WS_BYTES (16 * 1024 * 1024)
eps_status_t eps_vjp_static(const eps_problem_t *prob, const float *C, int32_t n_lambda,
                            int32_t field_type, const void *const *EF, const void *const *EA,
                            const float *field_scales, float scale, float *dJdC, float *eps_out,
                            eps_stream_t stream);

/*
 * Set the L2 fetch granularity hint (cudaLimitMaxL2FetchGranularity, 0 ..
 * 128 bytes) of the calling thread's current CUDA context and return the
 * previous value in *previous (may be NULL).  The field reads of eps_vjp
 * touch 32-byte sectors scattered at the column pitch, so a 32-byte
 * granularity avoids DRAM fetches of the cladding planes between them.  The
 * setting belongs to the context: it lasts until changed or until the
 * process ends, and applies to every kernel in that context.
 */
eps_status_t eps_set_l2_fetch_granularity(int32_t bytes, int32_t *previous);

/*
 * Per-kernel timing.  While enabled, each launch made by this library is
 * bracketed by CUDA events on its stream, and the kernels of a call run one
 * after another on the caller's stream (no programmatic dependent launch,
 * no band pipeline), so each record is the kernel's own duration; calls are
 * slower than unprofiled ones.  eps_profile_stop() waits for the
 * recorded events and fills up to max_entries records (kernel name, number
 * of launches, summed milliseconds); *n_entries gets the number written.
 * Host-side state is process-global: do not profile from several host
 * threads at once.
 */
typedef struct {
  char name[48];
  int32_t launches;
  double total_ms;
} eps_profile_entry_t;

eps_status_t eps_profile_start(void);
eps_status_t eps_profile_stop(eps_profile_entry_t *entries, int32_t max_entries,
                              int32_t *n_entries);

/*
 * Number of kernel launches this library has made in the process, on every
 * device and stream (a host-side counter, incremented when a launch is
 * accepted; no synchronisation).  The difference of two readings counts the
 * launches of the calls made in between, whatever form they took (a band
 * pipeline launches more kernels than the single-stream order).
 * EPS_ERR_INVALID_ARG for a null pointer.  Instrumentation; the paper has no
 * counterpart.
 */
eps_status_t eps_launch_count(uint64_t *count);

#ifdef __cplusplus
}
#endif

#endif /* EPSCHAIN_H */
