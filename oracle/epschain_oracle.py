"""FP64 CPU oracle for the control-variables -> Yee-grid permittivity chain
and its adjoint, after Sofronov, Yakovleva and Yakubovich, "Accelerated
inverse design of passive Si photonics" (arXiv 2505.03352), Sec. 3 and Eq. 1.

TEST INFRASTRUCTURE, NOT PRODUCT CODE.  Only the test-suite, the smoke check
and the CPU-baseline leg of the benchmark may import this module.  It shares
no code with the CUDA library: every step below is the plain definition,
written with whole-array numpy operations in float64 (or complex128 for the
complex-step derivative checks), with no blocking, fusion or reordering.

The chain, per paper section:

  1. Density filter (Eq. 2, read as a normalised conic filter at control
     pitch):  u = K * C,  K_pq proportional to (1 - r/R) on integer offsets
     with r = sqrt(p^2 + q^2) < R, normalised to sum 1.
  2. Projection (Eq. 3 / Eq. 6):  rho = (1 + tanh(beta (u - eta))) / 2.
  3. Density mixing (Sec. 3, first paragraph):
     eps = eps_clad + rho (eps_core - eps_clad).
  4. Per-component dual-cell averages (Eq. 8, finite-sum form of the
     half-cell shift + downsample): A_c = <eps>_c, H_c = <1/eps>_c and the
     averaged filtered density U_c = <u>_c over the Yee-cell-sized box
     Omega_c centred on the E_c sample point.
  5. Normals (Sec. 3, Sobel edge detection), taken from the gradient of the
     filtered density on the Yee grid:  m_x = g_x^2/|g|^2 from U_x and
     m_y = g_y^2/|g|^2 from U_y; n_z = 0 inside the slab.
  6. Anisotropic smoothing (Eq. 7):
     eps_cc = 1 / (m_c H_c + (1 - m_c) / A_c), extruded through the slab
     (Sec. 3: the 2-D mask is extruded along z), with the Ez slab-face
     planes half filled and smoothed with n = z.
  7. Adjoint (Eq. 1):  dJ/dC = J^T (scale * Re(sum_lambda E_F * E_A)),
     J = d eps_hat / dC, elementwise unconjugated field product, scale = -2.

Readings where the paper is silent or garbled (each also listed in the
design notes of the repository):
  * boundary rule `bc` (CLAMP = edge replicate, PERIODIC = wrap) applied
    separately at each stage: to C in the filter, to subpixel indices in the
    dual-cell means, and to Yee indices in the Sobel stencil;
  * normal threshold: |g|^2 <= NORMAL_TAU2 gives m = 0 (normal undefined);
  * geometry: subpixel (a, b) covers [a d, (a+1) d] x [b d, (b+1) d], the
    Yee cell is D = s d, Ex sits at ((i+1/2)D, jD), Ey at (iD, (j+1/2)D),
    Ez at (iD, jD, (k+1/2)D); slab faces at z = (k0 + 1/2) D and
    (k0 + nk + 1/2) D;
  * Ex/Ey planes k0+1 .. k0+nk and Ez planes k0+1 .. k0+nk-1 take Eq. 7; Ez
    planes k0 and k0+nk take 1/(H_z/2 + 1/(2 eps_clad)); other planes are
    cladding;
  * off-diagonal (optional, forward only): eta_xy = n_x n_y (H - 1/A), the
    xy element of the inverse-permittivity tensor of Eq. 7 in tensor form.
"""

from __future__ import annotations

from dataclasses import dataclass

import numpy as np

CLAMP = 0
PERIODIC = 1

# Gradient magnitude threshold (on |g|^2) below which the interface normal is
# undefined and the cell is treated as having no in-plane interface (m = 0).
NORMAL_TAU2 = 1e-12


@dataclass(frozen=True)
class Problem:
    """Shape and material parameters of one design region.

    mx, my   control grid (subpixels), pitch d; C has shape (mx, my)
    sub      subpixels per Yee cell along x and y (s); the Yee grid is
             (mx/s, my/s, nz)
    nz       Yee cells along z
    slab_nk  slab thickness in Yee cells
    slab_k0  lower Ez face plane; -1 centres the slab
    radius   conic filter radius R in subpixels
    beta, eta  projection strength and threshold (Eq. 3 / Eq. 6)
    eps_core, eps_clad  permittivities mixed by rho (Sec. 3)
    bc       CLAMP or PERIODIC
    """

    mx: int
    my: int
    nz: int
    radius: float
    beta: float
    eta: float = 0.5
    eps_core: float = 12.11
    eps_clad: float = 2.085
    sub: int = 2
    slab_nk: int = 11
    slab_k0: int = -1
    bc: int = CLAMP

    @property
    def nx(self) -> int:
        return self.mx // self.sub

    @property
    def ny(self) -> int:
        return self.my // self.sub

    @property
    def k0(self) -> int:
        if self.slab_k0 >= 0:
            return self.slab_k0
        return (self.nz - self.slab_nk - 1) // 2


# --------------------------------------------------------------------------
# index helpers
# --------------------------------------------------------------------------

def bc_index(idx, n: int, bc: int):
    """Map (possibly out-of-range) integer indices onto [0, n) by the
    boundary rule: CLAMP replicates the edge, PERIODIC wraps."""
    idx = np.asarray(idx)
    if bc == CLAMP:
        return np.clip(idx, 0, n - 1)
    if bc == PERIODIC:
        return np.mod(idx, n)
    raise ValueError(f"unknown boundary rule {bc}")


def _grid(nx: int, ny: int):
    i = np.arange(nx)[:, None]
    j = np.arange(ny)[None, :]
    return i, j


def _full(idx_a, idx_b):
    a, b = np.broadcast_arrays(idx_a, idx_b)
    return a, b


# --------------------------------------------------------------------------
# 1. density filter (Eq. 2)
# --------------------------------------------------------------------------

def conic_taps(radius: float):
    """Offsets (p, q) with p^2 + q^2 < R^2 and their normalised conic
    weights (1 - r/R) / sum, in float64.  Eq. 2 with a compact cone basis."""
    if not radius > 0:
        raise ValueError("radius must be positive")
    n = int(np.ceil(radius))
    taps = []
    for p in range(-n, n + 1):
        for q in range(-n, n + 1):
            r = np.hypot(p, q)
            if r < radius:
                taps.append((p, q, 1.0 - r / radius))
    total = sum(t[2] for t in taps)
    return [(p, q, w / total) for p, q, w in taps]


def filter_density(C, radius: float, bc: int):
    """u[a, b] = sum_pq w_pq C[bc(a+p), bc(b+q)]  (Eq. 2)."""
    mx, my = C.shape
    a, b = _grid(mx, my)
    u = np.zeros(C.shape, dtype=np.result_type(C.dtype, np.float64))
    for p, q, w in conic_taps(radius):
        u = u + w * C[bc_index(a + p, mx, bc), bc_index(b + q, my, bc)]
    return u


def filter_density_T(du, radius: float, bc: int):
    """Transpose of filter_density: scatter-add w_pq du[a, b] onto
    C[bc(a+p), bc(b+q)]."""
    mx, my = du.shape
    a, b = _grid(mx, my)
    dC = np.zeros(du.shape, dtype=np.result_type(du.dtype, np.float64))
    for p, q, w in conic_taps(radius):
        ia, ib = _full(bc_index(a + p, mx, bc), bc_index(b + q, my, bc))
        np.add.at(dC, (ia, ib), w * du)
    return dC


# --------------------------------------------------------------------------
# 2. projection (Eq. 3 / Eq. 6) and 3. mixing (Sec. 3)
# --------------------------------------------------------------------------

def project(u, beta: float, eta: float):
    """rho = (1 + tanh(beta (u - eta))) / 2   (Eq. 6 with threshold eta)."""
    return 0.5 * (1.0 + np.tanh(beta * (u - eta)))


def project_grad(u, beta: float, eta: float):
    """d rho / d u = (beta / 2) (1 - tanh^2(beta (u - eta))), the analytic
    derivative the paper uses in place of autodiff (Sec. 3)."""
    t = np.tanh(beta * (u - eta))
    return 0.5 * beta * (1.0 - t * t)


def mix(rho, eps_core: float, eps_clad: float):
    """eps = rho eps_core + (1 - rho) eps_clad   (Sec. 3)."""
    return eps_clad + rho * (eps_core - eps_clad)


# --------------------------------------------------------------------------
# 4. dual-cell averages (Eq. 8)
# --------------------------------------------------------------------------

def dual_cell_offsets(component: int, s: int):
    """Subpixel offsets, relative to s*i (x) and s*j (y), of the subpixels
    inside Omega_c.  Along an axis where the E_c sample sits at a cell centre
    ((i + 1/2) D) the box spans subpixels s*i .. s*i + s - 1; where it sits
    on a grid node (i D) the box spans s*i - s/2 .. s*i + s/2 - 1."""
    centred = np.arange(s)
    noded = np.arange(s) - s // 2
    if component == 0:
        return centred, noded
    if component == 1:
        return noded, centred
    if component == 2:
        return noded, noded
    raise ValueError(component)


def dual_cell_mean(f, component: int, prob: Problem):
    """<f>_c on the Yee grid: mean of f over the s x s subpixels of
    Omega_c, out-of-range subpixel indices mapped by bc (Eq. 8)."""
    s, bc = prob.sub, prob.bc
    mx, my = f.shape
    i, j = _grid(prob.nx, prob.ny)
    offa, offb = dual_cell_offsets(component, s)
    acc = np.zeros((prob.nx, prob.ny), dtype=np.result_type(f.dtype, np.float64))
    for da in offa:
        for db in offb:
            acc = acc + f[bc_index(s * i + da, mx, bc), bc_index(s * j + db, my, bc)]
    return acc / (s * s)


def dual_cell_mean_T(g, component: int, prob: Problem):
    """Transpose of dual_cell_mean: scatter g/s^2 onto the subpixels."""
    s, bc = prob.sub, prob.bc
    i, j = _grid(prob.nx, prob.ny)
    offa, offb = dual_cell_offsets(component, s)
    out = np.zeros((prob.mx, prob.my), dtype=np.result_type(g.dtype, np.float64))
    for da in offa:
        for db in offb:
            ia, ib = _full(bc_index(s * i + da, prob.mx, bc),
                           bc_index(s * j + db, prob.my, bc))
            np.add.at(out, (ia, ib), g / (s * s))
    return out


# --------------------------------------------------------------------------
# 5. Sobel normals (Sec. 3)
# --------------------------------------------------------------------------

SOBEL_DIFF = {-1: -1.0, 0: 0.0, 1: 1.0}
SOBEL_SMOOTH = {-1: 1.0, 0: 2.0, 1: 1.0}


def sobel(U, bc: int):
    """3x3 Sobel gradient of a Yee-grid map, indices mapped by bc:
    g_x = sum diff(di) smooth(dj) U[i+di, j+dj],
    g_y = sum smooth(di) diff(dj) U[i+di, j+dj]."""
    nx, ny = U.shape
    i, j = _grid(nx, ny)
    gx = np.zeros(U.shape, dtype=np.result_type(U.dtype, np.float64))
    gy = np.zeros_like(gx)
    for di in (-1, 0, 1):
        for dj in (-1, 0, 1):
            v = U[bc_index(i + di, nx, bc), bc_index(j + dj, ny, bc)]
            gx = gx + SOBEL_DIFF[di] * SOBEL_SMOOTH[dj] * v
            gy = gy + SOBEL_SMOOTH[di] * SOBEL_DIFF[dj] * v
    return gx, gy


def sobel_T(dgx, dgy, bc: int):
    """Transpose of sobel: scatter the gradient cotangents back onto U."""
    nx, ny = dgx.shape
    i, j = _grid(nx, ny)
    dU = np.zeros(dgx.shape, dtype=np.result_type(dgx.dtype, np.float64))
    for di in (-1, 0, 1):
        for dj in (-1, 0, 1):
            ia, ib = _full(bc_index(i + di, nx, bc), bc_index(j + dj, ny, bc))
            w = SOBEL_DIFF[di] * SOBEL_SMOOTH[dj] * dgx + SOBEL_SMOOTH[di] * SOBEL_DIFF[dj] * dgy
            np.add.at(dU, (ia, ib), w)
    return dU


def normal_fraction(gx, gy, axis: int):
    """m = n_axis^2 = g_axis^2 / |g|^2, and 0 where |g|^2 <= NORMAL_TAU2."""
    g2 = gx * gx + gy * gy
    ok = np.real(g2) > NORMAL_TAU2
    num = gx * gx if axis == 0 else gy * gy
    return np.where(ok, num / np.where(ok, g2, 1.0), 0.0)


def normal_fraction_grad(gx, gy, axis: int):
    """(dm/dg_x, dm/dg_y) of normal_fraction; zero on the threshold branch."""
    g2 = gx * gx + gy * gy
    ok = np.real(g2) > NORMAL_TAU2
    inv4 = np.where(ok, 1.0 / np.where(ok, g2 * g2, 1.0), 0.0)
    if axis == 0:   # m = gx^2 / g2
        return 2.0 * gx * gy * gy * inv4, -2.0 * gx * gx * gy * inv4
    return -2.0 * gx * gy * gy * inv4, 2.0 * gx * gx * gy * inv4


def normal_cross(gx, gy):
    """n_x n_y = g_x g_y / |g|^2 (0 on the threshold branch)."""
    g2 = gx * gx + gy * gy
    ok = np.real(g2) > NORMAL_TAU2
    return np.where(ok, gx * gy / np.where(ok, g2, 1.0), 0.0)


# --------------------------------------------------------------------------
# 6. Eq. 7 and the z rules
# --------------------------------------------------------------------------

def support_planes(prob: Problem):
    """z-plane index ranges, as (start, stop) pairs, where eps_hat depends on
    C:  Ex/Ey (k0+1 .. k0+nk), Ez interior (k0+1 .. k0+nk-1) and the two Ez
    face planes k0 and k0+nk."""
    k0, nk = prob.k0, prob.slab_nk
    return {
        "xy": (k0 + 1, k0 + nk + 1),
        "z_int": (k0 + 1, k0 + nk),
        "z_face": (k0, k0 + nk),
    }


def check_problem(prob: Problem):
    if prob.sub < 2 or prob.sub % 2:
        raise ValueError("sub must be a positive even number")
    if prob.mx % prob.sub or prob.my % prob.sub:
        raise ValueError("mx, my must be multiples of sub")
    if prob.slab_nk < 1 or prob.k0 < 0 or prob.k0 + prob.slab_nk > prob.nz - 1:
        raise ValueError("slab does not fit in nz")


def forward(prob: Problem, C, offdiag: bool = False):
    """Full forward chain.  Returns a dict with eps_hat [3, nx, ny, nz] and
    every intermediate the adjoint needs."""
    check_problem(prob)
    C = np.asarray(C)
    if C.dtype.kind != "c":
        C = C.astype(np.float64)
    u = filter_density(C, prob.radius, prob.bc)                    # Eq. 2
    rho = project(u, prob.beta, prob.eta)                         # Eq. 6
    e = mix(rho, prob.eps_core, prob.eps_clad)                    # Sec. 3
    ie = 1.0 / e
    A = [dual_cell_mean(e, c, prob) for c in range(3)]            # Eq. 8
    H = [dual_cell_mean(ie, c, prob) for c in range(3)]
    U = [dual_cell_mean(u, c, prob) for c in range(2)]
    g = [sobel(U[c], prob.bc) for c in range(2)]                  # normals
    m = [normal_fraction(g[c][0], g[c][1], c) for c in range(2)]
    eps_c = [1.0 / (m[c] * H[c] + (1.0 - m[c]) / A[c]) for c in range(2)]   # Eq. 7
    eps_zi = A[2]                                                 # n_z = 0
    eps_zf = 1.0 / (0.5 * H[2] + 0.5 / prob.eps_clad)             # n = z, half filled

    sp = support_planes(prob)
    dtype = np.result_type(e.dtype, np.float64)
    eps_hat = np.full((3, prob.nx, prob.ny, prob.nz), prob.eps_clad, dtype=dtype)
    lo, hi = sp["xy"]
    eps_hat[0, :, :, lo:hi] = eps_c[0][:, :, None]
    eps_hat[1, :, :, lo:hi] = eps_c[1][:, :, None]
    lo, hi = sp["z_int"]
    eps_hat[2, :, :, lo:hi] = eps_zi[:, :, None]
    for k in sp["z_face"]:
        eps_hat[2, :, :, k] = eps_zf

    out = dict(u=u, rho=rho, e=e, A=A, H=H, U=U, g=g, m=m,
               eps_c=eps_c, eps_zi=eps_zi, eps_zf=eps_zf, eps_hat=eps_hat)
    if offdiag:
        od = np.zeros((2, prob.nx, prob.ny, prob.nz), dtype=dtype)
        lo, hi = sp["xy"]
        for c in range(2):
            nxny = normal_cross(g[c][0], g[c][1])
            od[c, :, :, lo:hi] = (nxny * (H[c] - 1.0 / A[c]))[:, :, None]
        out["offdiag"] = od
    return out


def eps_hat(prob: Problem, C):
    return forward(prob, C)["eps_hat"]


# --------------------------------------------------------------------------
# 7. adjoint (Eq. 1)
# --------------------------------------------------------------------------

def vjp_real(prob: Problem, C, G):
    """(d eps_hat / dC)^T G for a real cotangent G of eps_hat's shape: the
    vector-Jacobian product of Sec. 3, without forming the Jacobian.  The
    filtered density and projection are recomputed from C."""
    fw = forward(prob, C)
    G = np.asarray(G, dtype=np.float64)
    sp = support_planes(prob)
    lo, hi = sp["xy"]
    W = [G[0, :, :, lo:hi].sum(-1), G[1, :, :, lo:hi].sum(-1)]
    lo, hi = sp["z_int"]
    W_zi = G[2, :, :, lo:hi].sum(-1)
    W_zf = sum(G[2, :, :, k] for k in sp["z_face"])

    e = fw["e"]
    de = np.zeros_like(e)
    du = np.zeros_like(e)
    for c in range(2):
        eps, m, H, A = fw["eps_c"][c], fw["m"][c], fw["H"][c], fw["A"][c]
        eps2w = eps * eps * W[c]
        dH = -eps2w * m                          # d eps / d H
        dA = eps2w * (1.0 - m) / (A * A)         # d eps / d A
        dm = -eps2w * (H - 1.0 / A)              # d eps / d m
        gx, gy = fw["g"][c]
        mgx, mgy = normal_fraction_grad(gx, gy, c)
        dU = sobel_T(dm * mgx, dm * mgy, prob.bc)
        de = de + dual_cell_mean_T(dA, c, prob) - dual_cell_mean_T(dH, c, prob) / (e * e)
        du = du + dual_cell_mean_T(dU, c, prob)
    dA_z = W_zi
    dH_z = -0.5 * fw["eps_zf"] ** 2 * W_zf
    de = de + dual_cell_mean_T(dA_z, 2, prob) - dual_cell_mean_T(dH_z, 2, prob) / (e * e)
    du = du + de * (prob.eps_core - prob.eps_clad) * project_grad(fw["u"], prob.beta, prob.eta)
    return filter_density_T(du, prob.radius, prob.bc)


def field_cotangent(prob: Problem, EF, EA, scale: float = -2.0, field_scales=None):
    """scale * Re(sum_lambda E_F * E_A): the unconjugated elementwise field
    product of Eq. 1 (footnote: same array shape as eps_hat), accumulated in
    float64 one wavelength at a time.  field_scales[l][f][c], if given,
    multiplies component c of field f (0 = forward, 1 = adjoint) at
    wavelength l."""
    G = np.zeros((3, prob.nx, prob.ny, prob.nz), dtype=np.float64)
    for l, (ef, ea) in enumerate(zip(EF, EA)):
        ef = np.asarray(ef).astype(np.complex128)
        ea = np.asarray(ea).astype(np.complex128)
        prod = ef * ea
        if field_scales is not None:
            for c in range(3):
                prod[c] *= field_scales[l][0][c] * field_scales[l][1][c]
        G += prod.real
    return scale * G


def vjp_fields(prob: Problem, C, EF, EA, scale: float = -2.0, field_scales=None):
    """Eq. 1:  dJ/dC = J^T (scale * Re(sum_lambda E_F * E_A)), scale = -2."""
    return vjp_real(prob, C, field_cotangent(prob, EF, EA, scale, field_scales))
