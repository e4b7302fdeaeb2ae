"""FP64 CPU oracle for one optimiser step with dynamic control of binarity
(Sec. 4): Adam (Eq. 10-11), the unbinarity u of the design, the beta_max
control (Eq. 15) and the beta schedule (Eq. 14).

TEST INFRASTRUCTURE, NOT PRODUCT CODE.  Only the test-suite, the smoke check
and the CPU-baseline leg of the benchmark may import this module.  It shares
no code with the CUDA library.

One step, in the order the paper describes it (iteration i = 1 .. N, the
design and the gradient G of iteration i both taken at beta_i):
  1. u_i = (number of gray subpixels of rho(C_{i-1}, beta_i)) / (mx my)
  2. t <- gamma t + (1 - gamma) (1/u_i - 1) / beta_i                 (Eq. 15)
     beta_max <- gamma beta_max + (1 - gamma) (1/u_0 - 1) / t        (Eq. 15)
  3. M_i = b1 M + (1 - b1) G,  V_i = b2 V + (1 - b2) G^2,
     M^ = M_i / (1 - b1^i),  V^ = V_i / (1 - b2^i)                     (Eq. 10)
     C_i = C_{i-1} - lr M^ / (sqrt(V^) + adam_eps)                    (Eq. 11)
  4. beta_{i+1} = beta_min + (beta_max - beta_min)
                  (exp(((i+1)/N)^2) - 1) / (e - 1)                      (Eq. 14)

Readings where the paper is silent (each also listed in the design notes of
the repository):
  * a subpixel counts as gray when its projected density is strictly between
    gray_tol and 1 - gray_tol (default 0.05), i.e. rho (1 - rho) >
    gray_tol (1 - gray_tol);
  * u is floored at one subpixel (1 / (mx my)), so 1/u stays finite;
  * t has no stated initial value: it starts at its first sample
    (1/u_1 - 1) / beta_1, after which the moving average applies;
    beta_max starts at a given beta_max0;
  * adam_eps (the small constant the paper adds to the denominator)
    defaults to 1e-8, and the Adam learning rate is `lr` (the paper's eta,
    renamed to keep eta for the projection threshold); App. B: b1 = 0.9, b2 = 0.999, lr = 0.001,
    gamma = 0.95, u_0 = 0.01, beta_min = 10;
  * the schedule's i is the 1-based iteration index of Adam's bias
    correction, so beta_N = beta_max at the last iteration.
"""

from __future__ import annotations

from dataclasses import dataclass

import numpy as np


@dataclass(frozen=True)
class OptParams:
    lr: float = 0.001
    b1: float = 0.9
    b2: float = 0.999
    adam_eps: float = 1e-8
    gray_tol: float = 0.05
    gamma: float = 0.95
    u0: float = 0.01
    beta_min: float = 10.0
    beta_max0: float = 100.0
    n_iter: int = 100


@dataclass
class OptState:
    step: int            # completed iterations; the next one is step + 1
    beta: float          # beta of the next iteration
    beta_max: float
    t: float             # <= 0 until the first sample
    unbinarity: float    # u of the last completed iteration
    gray: int


def beta_schedule(i: int, n_iter: int, beta_min: float, beta_max: float) -> float:
    """Eq. 14."""
    x = (i / n_iter) ** 2
    return beta_min + (beta_max - beta_min) * (np.exp(x) - 1.0) / (np.e - 1.0)


def init_state(p: OptParams) -> OptState:
    return OptState(step=0, beta=beta_schedule(1, p.n_iter, p.beta_min, p.beta_max0),
                    beta_max=p.beta_max0, t=0.0, unbinarity=0.0, gray=0)


def gray_count(rho, gray_tol: float) -> int:
    """Number of subpixels with gray_tol < rho < 1 - gray_tol."""
    rho = np.asarray(rho, dtype=np.float64)
    return int(np.count_nonzero((rho > gray_tol) & (rho < 1.0 - gray_tol)))


def beta_max_control(t: float, beta_max: float, u: float, beta: float, gamma: float, u0: float):
    """Eq. 15, with t starting at its first sample."""
    sample = (1.0 / u - 1.0) / beta
    t = sample if t <= 0.0 else gamma * t + (1.0 - gamma) * sample
    beta_max = gamma * beta_max + (1.0 - gamma) * (1.0 / u0 - 1.0) / t
    return t, beta_max


def adam_update(C, G, M, V, i: int, p: OptParams):
    """Eq. 10-11 for iteration i (1-based); returns new (C, M, V)."""
    C = np.asarray(C, dtype=np.float64)
    G = np.asarray(G, dtype=np.float64)
    M = p.b1 * np.asarray(M, dtype=np.float64) + (1.0 - p.b1) * G
    V = p.b2 * np.asarray(V, dtype=np.float64) + (1.0 - p.b2) * G * G
    Mh = M / (1.0 - p.b1 ** i)
    Vh = V / (1.0 - p.b2 ** i)
    return C - p.lr * Mh / (np.sqrt(Vh) + p.adam_eps), M, V


def opt_step(p: OptParams, s: OptState, C, G, M, V, rho):
    """One iteration: rho is the projected subpixel density of C at s.beta.
    Returns (C, M, V, new state)."""
    i = s.step + 1
    n = np.asarray(rho).size
    gray = gray_count(rho, p.gray_tol)
    u = max(gray, 1) / n
    t, beta_max = beta_max_control(s.t, s.beta_max, u, s.beta, p.gamma, p.u0)
    C, M, V = adam_update(C, G, M, V, i, p)
    beta_next = beta_schedule(i + 1, p.n_iter, p.beta_min, beta_max)
    return C, M, V, OptState(step=i, beta=beta_next, beta_max=beta_max, t=t, unbinarity=u,
                             gray=gray)
