"""FP64 CPU oracle for 3-D interface normals at the slab faces and the full
off-diagonal inverse-permittivity tensor (Eq. 7 in tensor form), for a
solver that accepts off-diagonal terms.

TEST INFRASTRUCTURE, NOT PRODUCT CODE.  Only the test-suite, the smoke check
and the CPU-baseline leg of the benchmark may import this module.  It shares
no code with the CUDA library; it builds on the base oracle.

Eq. 7 in tensor form:  eps^-1 = P <eps^-1> + (I - P) <eps>^-1,  P = n n^T.

Where the dual cells sit (the base chain's geometry): every Ex and Ey dual
cell lies entirely inside or entirely outside the slab in z, so their
normals are in-plane (n_z = 0) and their rows have only the xy term.  The
Ez cells of planes k0 and k0 + nk straddle the slab faces: they are half
slab, half cladding, and near a sidewall (the slab's edges and corners)
their interface normal is three-dimensional.  For those cells:

  <eps>    = (A_z + eps_clad) / 2,   <eps^-1> = (H_z + 1/eps_clad) / 2
  g        = (S_x rho3, S_y rho3, D_z rho3), Sobel-consistent central
             differences of the cell-averaged 3-D density rho3 at the cell:
             in plane the face cell holds half the slab's filtered density,
             rho3 = U_z / 2, so g_x, g_y = (Sobel of U_z) / 2; along z the
             density steps from 0 (cladding) to U_z across the cell, and a
             central difference over two cells scaled like the Sobel (8x the
             derivative) gives g_z = +4 U_z at the lower face (k0) and
             -4 U_z at the upper face (k0 + nk)
  n        = g / |g|; where |g|^2 <= NORMAL_TAU2 the cell has no defined
             normal and keeps the base rule n = z (flat cladding then gives
             the same eps_zz with and without this option)
  eps_zz   = 1 / (n_z^2 <eps^-1> + (1 - n_z^2) / <eps>)
  eta_zx   = n_z n_x (<eps^-1> - 1/<eps>),  eta_zy = n_z n_y (...)

The off-diagonal output is [4][nx][ny][nz]: eta_xy at the Ex points, eta_yx
at the Ey points (the base chain's two maps), then eta_zx and eta_zy at the
Ez points (non-zero on the two face planes only).  eta_xz at Ex and eta_yz
at Ey vanish identically in this geometry (n_z = 0 there).  Readings: the
half-filled cell's in-plane density, the Sobel-consistent z difference and
the fallback are this module's reading of the interface normal (Sec. 3)
for cells the paper's 2-D Sobel does not cover.
"""

from __future__ import annotations

import numpy as np

from .epschain_oracle import NORMAL_TAU2, Problem, dual_cell_mean, forward, sobel


def face_rows(prob: Problem, fw):
    """For the lower (k0) and upper (k0 + nk) face planes: (eps_zz,
    eta_zx, eta_zy), each [nx, ny], from the base chain's forward dict."""
    Uz = dual_cell_mean(fw["u"], 2, prob)
    sx, sy = sobel(Uz, prob.bc)
    a = 0.5 * (fw["H"][2] + 1.0 / prob.eps_clad)      # <eps^-1>
    am = 0.5 * (fw["A"][2] + prob.eps_clad)           # <eps>
    b = 1.0 / am
    rows = []
    for sign in (+1.0, -1.0):
        gx, gy, gz = 0.5 * sx, 0.5 * sy, sign * 4.0 * Uz
        g2 = gx * gx + gy * gy + gz * gz
        ok = np.real(g2) > NORMAL_TAU2
        inv = np.where(ok, 1.0 / np.where(ok, g2, 1.0), 0.0)
        nz2 = np.where(ok, gz * gz * inv, 1.0)
        nzx = np.where(ok, gz * gx * inv, 0.0)
        nzy = np.where(ok, gz * gy * inv, 0.0)
        eps_zz = 1.0 / (nz2 * a + (1.0 - nz2) * b)
        rows.append((eps_zz, nzx * (a - b), nzy * (a - b)))
    return rows


def forward_3d(prob: Problem, C):
    """eps_hat with the 3-D face rule and the 4-map off-diagonal output."""
    fw = forward(prob, C, offdiag=True)
    eps = fw["eps_hat"].copy()
    od2 = fw["offdiag"]
    od = np.zeros((4,) + od2.shape[1:], dtype=od2.dtype)
    od[:2] = od2
    k0, nk = prob.k0, prob.slab_nk
    for k, (ezz, ezx, ezy) in zip((k0, k0 + nk), face_rows(prob, fw)):
        eps[2, :, :, k] = ezz
        od[2, :, :, k] = ezx
        od[3, :, :, k] = ezy
    return eps, od
