"""The locality that the full-size GPU checks rest on, pinned on the CPU.

tests/test_gpu_large.py checks the cfg3 / cfg5 / cfg4 results on windows
(window_check, and window_check_device for fields held as tensors):
the oracle runs on a window grown by a margin of 2 ceil(R) + 8 subpixels
(cut at the region edge, where the same clamp rule applies) and is compared
with the full-size result in the window's interior.  Here the full-size
result is the oracle's own, so that comparison must agree to rounding for
eps_hat and for dJ/dC, at corners, edges and the centre, for the radii the
workloads use.  A window grown by too small a margin must not agree, so the
comparison is not vacuous."""

import numpy as np
import pytest

from oracle import epschain_oracle as orc
from paper_2505_03352_gb300 import synth
from tests.test_gpu_large import window_check, window_check_device


def _problem(radius, seed):
    w = synth.Workload("locality", 200, 176, 16, radius, 16.0, 1)
    C = synth.soi_layout(w.mx, w.my, seed)
    shape = (3, w.nx, w.ny, w.nz)
    EF = [synth.complex_field(shape, seed + 1)]
    EA = [synth.complex_field(shape, seed + 2)]
    o = orc.Problem(mx=w.mx, my=w.my, nz=w.nz, radius=w.radius, beta=w.beta)
    return w, C, EF, EA, o


@pytest.mark.parametrize("radius", [3.0, 6.0, 8.0])
def test_window_recompute_is_exact_in_the_interior(radius):
    w, C, EF, EA, o = _problem(radius, 4100 + int(radius))
    e = orc.eps_hat(o, C)
    g = orc.vjp_fields(o, C, EF, EA)
    windows = [(0, 0), (w.mx // 2, w.my // 2), (w.mx, w.my), (0, w.my), (77, 131)]
    worst_e, worst_g = window_check(w, C, EF, EA, e, g, windows, half=24)
    assert worst_e <= 1e-13, worst_e
    assert worst_g <= 1e-12, worst_g
    # the form the cfg5 check uses, slicing field tensors in place
    import torch
    worst_e, worst_g = window_check_device(w, C, [torch.from_numpy(x) for x in EF],
                                           [torch.from_numpy(x) for x in EA], e, g, windows, half=24)
    assert worst_e <= 1e-13, worst_e
    assert worst_g <= 1e-12, worst_g


def test_a_too_small_margin_is_visible():
    # the same interior, recomputed on a window grown by only 2 subpixels
    w, C, EF, EA, o = _problem(6.0, 4200)
    g = orc.vjp_fields(o, C, EF, EA)
    a0, a1, b0, b1, m = 80, 128, 64, 112, 2
    ow = orc.Problem(mx=a1 - a0 + 2 * m, my=b1 - b0 + 2 * m, nz=w.nz, radius=w.radius, beta=w.beta)
    sl = (slice(None), slice((a0 - m) // 2, (a1 + m) // 2), slice((b0 - m) // 2, (b1 + m) // 2),
          slice(None))
    gw = orc.vjp_fields(ow, C[a0 - m:a1 + m, b0 - m:b1 + m], [EF[0][sl]], [EA[0][sl]])
    ref = g[a0:a1, b0:b1]
    err = np.max(np.abs(gw[m:-m, m:-m] - ref)) / np.max(np.abs(ref))
    assert err > 1e-3, err
