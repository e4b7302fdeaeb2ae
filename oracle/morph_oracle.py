"""FP64 CPU oracle for the chain with morphological filtering (Sec. 3,
Eq. 3-6): controls -> filtered density -> first projection -> a sequence of
soft dilate / erode operations -> final projection -> the Yee-grid
permittivity of the base chain, and the adjoint of all of it.

TEST INFRASTRUCTURE, NOT PRODUCT CODE.  Only the test-suite, the smoke check
and the CPU-baseline leg of the benchmark may import this module.  It shares
no code with the CUDA library; it builds on the base oracle
(`epschain_oracle`) for the Yee-grid stage.

The chain, per paper equation:

  Eq. 2   u = K * C                      (conic density filter, as in the base chain)
  Eq. 3   rho_0 = (1 + tanh(beta (u - eta))) / 2
  Eq. 4   dilate:  D(rho)[x] = (1/alpha) log sum_y K_m(x - y) exp(alpha rho[y])
  Eq. 5   erode:   E(rho)[x] = 1 - (1/alpha) log sum_y K_m(x - y) exp(alpha (1 - rho[y]))
          rho_tilde = op_n( ... op_1(rho_0))
  Eq. 6   rho = (1 + tanh(beta (rho_tilde - 1/2))) / 2, then the base chain
          (mixing, dual-cell means, Sobel normals, Eq. 7, extrusion).

Readings where the paper is silent (each also listed in the design notes of
the repository):
  * K_m is the disk of the stated diameter d, on integer subpixel offsets
    (p, q) with p^2 + q^2 <= (d/2)^2 (closed disk), NORMALISED to sum 1 so
    that a uniform density is a fixed point of both operations (the integral
    of Eq. 4 with an unnormalised disk would shift a uniform density by
    log(area)/alpha);
  * the default sequence is a closing followed by an opening: dilate, erode,
    erode, dilate (the paper names both orders in which the two operations
    can be combined);
  * Phi of Eq. 3 is the filtered density minus the threshold, u - eta, as in
    the base chain;
  * the morphology uses the same boundary rule as the filter (edge replicate
    or wrap), applied to the subpixel indices;
  * with morphology on, the Sobel normals of the Yee stage are taken from
    rho_tilde: it is the smooth density whose 1/2 level set the final
    projection draws, i.e. it plays the role the filtered density has in the
    base chain.  The Yee stage is therefore exactly the base chain applied to
    rho_tilde with an identity filter (radius 1) and threshold 1/2.
"""

from __future__ import annotations

from dataclasses import dataclass, replace

import numpy as np

from .epschain_oracle import (
    Problem,
    _full,
    _grid,
    bc_index,
    field_cotangent,
    filter_density,
    filter_density_T,
    forward,
    project,
    project_grad,
    vjp_real,
)

DILATE = 0
ERODE = 1
CLOSE_THEN_OPEN = (DILATE, ERODE, ERODE, DILATE)


@dataclass(frozen=True)
class Morph:
    """alpha: sharpness of the soft max/min (App. B: 20); radius: disk
    radius d/2 in subpixels; ops: the sequence of DILATE / ERODE."""

    alpha: float = 20.0
    radius: float = 2.0
    ops: tuple = CLOSE_THEN_OPEN


def disk_taps(radius: float):
    """Offsets (p, q) with p^2 + q^2 <= radius^2, each with weight 1/N (the
    normalised disk K_m of Eq. 4/5)."""
    if radius < 0:
        raise ValueError("radius must be non-negative")
    n = int(np.floor(radius))
    offs = [(p, q) for p in range(-n, n + 1) for q in range(-n, n + 1)
            if p * p + q * q <= radius * radius]
    w = 1.0 / len(offs)
    return [(p, q, w) for p, q in offs]


def disk_sum(f, radius: float, bc: int):
    """S[x] = sum_d K_m(d) f[bc(x + d)]."""
    mx, my = f.shape
    a, b = _grid(mx, my)
    s = np.zeros(f.shape, dtype=np.result_type(f.dtype, np.float64))
    for p, q, w in disk_taps(radius):
        s = s + w * f[bc_index(a + p, mx, bc), bc_index(b + q, my, bc)]
    return s


def dilate(rho, morph: Morph, bc: int):
    """Eq. 4: (1/alpha) log sum K_m exp(alpha rho)."""
    return np.log(disk_sum(np.exp(morph.alpha * rho), morph.radius, bc)) / morph.alpha


def erode(rho, morph: Morph, bc: int):
    """Eq. 5: 1 - (1/alpha) log sum K_m exp(alpha (1 - rho))."""
    return 1.0 - np.log(disk_sum(np.exp(morph.alpha * (1.0 - rho)), morph.radius, bc)) / morph.alpha


def morph_forward(rho0, morph: Morph, bc: int):
    """[rho_0, rho_1, ..., rho_n]: rho_{k+1} = op_k(rho_k)."""
    maps = [rho0]
    for op in morph.ops:
        f = dilate if op == DILATE else erode
        maps.append(f(maps[-1], morph, bc))
    return maps


def morph_op_T(rho_in, g_out, op: int, morph: Morph, bc: int):
    """Adjoint of one operation.  For dilate, d rho_out[x] / d rho_in[y] at
    y = bc(x + d) is K_m(d) exp(alpha rho_in[y]) / S[x] with
    S[x] = sum_d K_m(d) exp(alpha rho_in[bc(x + d)]); for erode the same with
    exp(alpha (1 - rho_in)).  Both are positive: the softmax weights of the
    disk.  The transpose scatter-adds those weights times g_out[x] onto y."""
    mx, my = rho_in.shape
    a, b = _grid(mx, my)
    z = np.exp(morph.alpha * (rho_in if op == DILATE else 1.0 - rho_in))
    S = disk_sum(z, morph.radius, bc)
    g_in = np.zeros(rho_in.shape, dtype=np.result_type(rho_in.dtype, g_out.dtype, np.float64))
    for p, q, w in disk_taps(morph.radius):
        ia, ib = _full(bc_index(a + p, mx, bc), bc_index(b + q, my, bc))
        np.add.at(g_in, (ia, ib), w * z[ia, ib] / S * g_out)
    return g_in


def morph_T(maps, g_n, morph: Morph, bc: int):
    """Adjoint of the whole sequence: from d/d rho_n back to d/d rho_0."""
    g = g_n
    for k in range(len(morph.ops) - 1, -1, -1):
        g = morph_op_T(maps[k], g, morph.ops[k], morph, bc)
    return g


def yee_problem(prob: Problem) -> Problem:
    """The base-chain problem the Yee stage runs on rho_tilde: identity
    filter (radius 1 keeps only the centre tap) and threshold 1/2 (Eq. 6)."""
    return replace(prob, radius=1.0, eta=0.5)


def forward_morph(prob: Problem, morph: Morph, C, offdiag: bool = False):
    """Forward chain with morphology; returns the base chain's dict for the
    Yee stage plus u, rho0 and the morphology maps."""
    C = np.asarray(C)
    if C.dtype.kind != "c":
        C = C.astype(np.float64)
    u = filter_density(C, prob.radius, prob.bc)                  # Eq. 2
    rho0 = project(u, prob.beta, prob.eta)                      # Eq. 3
    maps = morph_forward(rho0, morph, prob.bc)                  # Eq. 4/5
    out = forward(yee_problem(prob), maps[-1], offdiag=offdiag)  # Eq. 6 + base chain
    out.update(u_filtered=u, rho0=rho0, morph_maps=maps)
    return out


def eps_hat_morph(prob: Problem, morph: Morph, C):
    return forward_morph(prob, morph, C)["eps_hat"]


def vjp_real_morph(prob: Problem, morph: Morph, C, G):
    """(d eps_hat / dC)^T G through the whole chain with morphology."""
    C = np.asarray(C, dtype=np.float64)
    u = filter_density(C, prob.radius, prob.bc)
    rho0 = project(u, prob.beta, prob.eta)
    maps = morph_forward(rho0, morph, prob.bc)
    g_tilde = vjp_real(yee_problem(prob), maps[-1], G)          # d/d rho_tilde
    g0 = morph_T(maps, g_tilde, morph, prob.bc)                 # d/d rho_0
    du = g0 * project_grad(u, prob.beta, prob.eta)              # Eq. 3
    return filter_density_T(du, prob.radius, prob.bc)           # Eq. 2


def vjp_fields_morph(prob: Problem, morph: Morph, C, EF, EA, scale: float = -2.0,
                     field_scales=None):
    """Eq. 1 through the chain with morphology."""
    return vjp_real_morph(prob, morph, C, field_cotangent(prob, EF, EA, scale, field_scales))
