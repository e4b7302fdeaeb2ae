"""FP64 CPU oracle for the chain with coarse control variables (Eq. 2 with
the basis functions shifted to the nodes of a coarse rectangular grid, as in
the paper's 36 x 36 controls over a 210 x 210-cell design region), and its
adjoint.

TEST INFRASTRUCTURE, NOT PRODUCT CODE.  Only the test-suite, the smoke check
and the CPU-baseline leg of the benchmark may import this module.  It shares
no code with the CUDA library; the Yee-grid stage is the base oracle.

  Eq. 2   Phi[a, b] = sum_{i, j} c[i, j] B((x_a - X_i) / h_x) B((y_b - Y_j) / h_y)
          then the base chain on Phi with an identity filter:
  Eq. 3/6 rho = (1 + tanh(beta (Phi - eta))) / 2, mixing, dual-cell means,
          Sobel normals from Phi, Eq. 7.
  adjoint dJ/dc = Bx^T (dJ/dPhi) By.

Readings where the paper is silent (each also listed in the design notes of
the repository):
  * the basis is the tensor-product hat B(t) = max(0, 1 - |t|): compact
    support, a partition of unity (uniform c gives uniform Phi) and exact on
    linear functions; Eq. 2's sum is used as written, without normalisation;
  * the node grid spans the region edge to edge: node i sits at
    X_i = i h_x, h_x = mx / (ncx - 1) in subpixel units (the paper's case,
    420 subpixels and 36 nodes, gives an integer stride of 12), and
    subpixel a's centre is at x_a = a + 1/2;
  * the coarse basis replaces the conic density filter: Phi plays the role
    of the filtered density u (projection threshold eta, Sobel normals).
"""

from __future__ import annotations

from dataclasses import replace

import numpy as np

from .epschain_oracle import Problem, field_cotangent, forward, vjp_real


def hat(t):
    return np.maximum(0.0, 1.0 - np.abs(t))


def basis_matrix(m: int, nc: int):
    """B[a, i] = hat((a + 1/2 - i h) / h), h = m / (nc - 1): float64 [m, nc]."""
    if nc < 2:
        raise ValueError("at least two nodes per axis")
    h = m / (nc - 1)
    a = np.arange(m)[:, None] + 0.5
    i = np.arange(nc)[None, :]
    return hat((a - i * h) / h)


def expand(c, mx: int, my: int):
    """Eq. 2 on the subpixel grid: Phi = Bx c By^T (same as the double sum)."""
    ncx, ncy = c.shape
    return basis_matrix(mx, ncx) @ c @ basis_matrix(my, ncy).T


def expand_T(g, ncx: int, ncy: int):
    mx, my = g.shape
    return basis_matrix(mx, ncx).T @ g @ basis_matrix(my, ncy)


def yee_problem(prob: Problem) -> Problem:
    """Base-chain problem on Phi: identity filter (the single tap at r = 0)."""
    return replace(prob, radius=1.0)


def forward_coarse(prob: Problem, c, offdiag: bool = False):
    c = np.asarray(c)
    if c.dtype.kind != "c":
        c = c.astype(np.float64)
    phi = expand(c, prob.mx, prob.my)
    out = forward(yee_problem(prob), phi, offdiag=offdiag)
    out["phi"] = phi
    return out


def eps_hat_coarse(prob: Problem, c):
    return forward_coarse(prob, c)["eps_hat"]


def vjp_real_coarse(prob: Problem, c, G):
    c = np.asarray(c, dtype=np.float64)
    phi = expand(c, prob.mx, prob.my)
    return expand_T(vjp_real(yee_problem(prob), phi, G), *c.shape)


def vjp_fields_coarse(prob: Problem, c, EF, EA, scale: float = -2.0, field_scales=None):
    return vjp_real_coarse(prob, c, field_cotangent(prob, EF, EA, scale, field_scales))
