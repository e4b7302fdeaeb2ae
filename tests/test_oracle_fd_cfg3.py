"""FP64 central differences of the oracle at the differentiation form's
settings (R = 6, beta = 16, nz = 32, three wavelengths), on 32 randomly
chosen control pixels, by windowed recompute.

The Eq. 1 gradient dJ/dC is the derivative of the linear functional
J(C) = -2 sum eps_hat(C) * Re(sum_l E_F E_A).  A control pixel p moves
eps_hat only in cells within about R + 4 subpixels of it, and a cell's
eps_hat depends only on C within R + 4 subpixels.  So for each p the sum
over an interior box of half-width R + 6 around p, computed on a window
grown by another R + 6 (cut at the region edge, where the same clamp rule
applies), changes exactly as J does.  Its central difference must equal
the oracle's dJ/dC at p from the whole problem."""

import numpy as np

from oracle import epschain_oracle as orc
from paper_2505_03352_gb300 import synth

R, BETA, NZ, NL = 6.0, 16.0, 32, 3
MX, MY = 160, 144


def _inputs():
    C = synth.soi_layout(MX, MY, 3003)
    shape = (3, MX // 2, MY // 2, NZ)
    EF = [synth.complex_field(shape, 2030 + l) for l in range(NL)]
    EA = [synth.complex_field(shape, 3030 + l) for l in range(NL)]
    return C, EF, EA


def _window_sum(C, w_field, a0, a1, b0, b1, ia, ib):
    """-2 sum eps_hat * w over the interior cells [ia) x [ib) (Yee indices
    of the whole problem) of the eps_hat computed on the window
    [a0, a1) x [b0, b1) of C."""
    o = orc.Problem(mx=a1 - a0, my=b1 - b0, nz=NZ, radius=R, beta=BETA)
    e = orc.eps_hat(o, C[a0:a1, b0:b1])
    i0, i1 = ia[0] - a0 // 2, ia[1] - a0 // 2
    j0, j1 = ib[0] - b0 // 2, ib[1] - b0 // 2
    return -2.0 * float(np.sum(e[:, i0:i1, j0:j1, :] * w_field[:, ia[0]:ia[1], ib[0]:ib[1], :]))


def test_central_differences_on_32_random_pixels_cfg3_settings():
    C, EF, EA = _inputs()
    o = orc.Problem(mx=MX, my=MY, nz=NZ, radius=R, beta=BETA)
    g = orc.vjp_fields(o, C, EF, EA)
    w_field = sum((ef * ea).real for ef, ea in zip(EF, EA))
    rng = np.random.default_rng(33)
    pix = [(int(rng.integers(0, MX)), int(rng.integers(0, MY))) for _ in range(32)]
    pix[:2] = [(0, 5), (MX - 1, MY - 2)]              # two at the region edges
    reach = int(R) + 6
    h = 1e-6
    worst = 0.0
    for (pa, pb) in pix:
        # interior: Yee cells whose subpixels lie within `reach` of p
        ia = (max(0, (pa - reach) // 2), min(MX // 2, (pa + reach) // 2 + 1))
        ib = (max(0, (pb - reach) // 2), min(MY // 2, (pb + reach) // 2 + 1))
        # window: the interior grown by `reach` more subpixels, even-aligned
        a0, a1 = max(0, 2 * ia[0] - reach - 1) // 2 * 2, min(MX, 2 * ia[1] + reach + 1)
        b0, b1 = max(0, 2 * ib[0] - reach - 1) // 2 * 2, min(MY, 2 * ib[1] + reach + 1)
        a1 += a1 % 2
        b1 += b1 % 2
        Cp, Cm = C.astype(np.float64), C.astype(np.float64)
        Cp = Cp.copy()
        Cm = Cm.copy()
        Cp[pa, pb] += h
        Cm[pa, pb] -= h
        fd = (_window_sum(Cp, w_field, a0, a1, b0, b1, ia, ib)
              - _window_sum(Cm, w_field, a0, a1, b0, b1, ia, ib)) / (2 * h)
        worst = max(worst, abs(fd - g[pa, pb]))
    assert worst <= 1e-6 * np.max(np.abs(g)), (worst, np.max(np.abs(g)))
