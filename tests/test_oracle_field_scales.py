"""Pin of the oracle's per-component field scales (Eq. 1 with scaled fields).

The reduced-precision field formats store every component of E_F and E_A
divided by a scale, and the Eq. 1 contraction multiplies the product back
by the two scales.  The oracle's `field_scales[l][f][c]` branch must
therefore give exactly what the plain definition gives on fields that were
multiplied by those scales beforehand: component c of the forward field of
wavelength l by field_scales[l][0][c], the adjoint field's by
field_scales[l][1][c].  The pre-scaled reference takes the scales through
the arrays, not through the branch, so a slip in the branch (one factor
dropped, the forward scale used twice, the field and component indices
swapped) fails here.  Checked for the base chain, the morphology chain and
the coarse-control chain, each of which forwards the scales to the same
cotangent.
"""

import numpy as np
import pytest

from oracle import coarse_oracle as co
from oracle import epschain_oracle as orc
from oracle import morph_oracle as mo


def _inputs(p, n_lambda, seed):
    rng = np.random.default_rng(seed)
    shape = (3, p.nx, p.ny, p.nz)
    EF = [rng.standard_normal(shape) + 1j * rng.standard_normal(shape) for _ in range(n_lambda)]
    EA = [rng.standard_normal(shape) + 1j * rng.standard_normal(shape) for _ in range(n_lambda)]
    # distinct, asymmetric scales: [l][f][c] with no two equal, so swapping
    # f and c or using one field's scale for both changes the result
    fs = rng.uniform(0.3, 3.0, size=(n_lambda, 2, 3))
    return EF, EA, fs


def _prescaled(EF, EA, fs):
    EFs = [np.stack([ef[c] * fs[l, 0, c] for c in range(3)]) for l, ef in enumerate(EF)]
    EAs = [np.stack([ea[c] * fs[l, 1, c] for c in range(3)]) for l, ea in enumerate(EA)]
    return EFs, EAs


def _close(a, b):
    scale = np.max(np.abs(b))
    assert scale > 0
    assert np.max(np.abs(a - b)) <= 1e-12 * scale


@pytest.mark.parametrize("bc", [orc.CLAMP, orc.PERIODIC])
def test_base_chain_scales_equal_prescaled_fields(bc):
    p = orc.Problem(mx=20, my=16, nz=16, radius=3.0, beta=8.0, bc=bc)
    C = np.random.default_rng(5).random((p.mx, p.my))
    EF, EA, fs = _inputs(p, 3, 11)
    EFs, EAs = _prescaled(EF, EA, fs)
    _close(orc.field_cotangent(p, EF, EA, -2.0, fs), orc.field_cotangent(p, EFs, EAs, -2.0))
    _close(orc.vjp_fields(p, C, EF, EA, field_scales=fs), orc.vjp_fields(p, C, EFs, EAs))


def test_morphology_chain_scales_equal_prescaled_fields():
    p = orc.Problem(mx=20, my=20, nz=16, radius=3.0, beta=8.0)
    m = mo.Morph(alpha=20.0, radius=1.5)
    C = np.random.default_rng(6).random((p.mx, p.my))
    EF, EA, fs = _inputs(p, 2, 12)
    EFs, EAs = _prescaled(EF, EA, fs)
    _close(mo.vjp_fields_morph(p, m, C, EF, EA, field_scales=fs),
           mo.vjp_fields_morph(p, m, C, EFs, EAs))


def test_coarse_chain_scales_equal_prescaled_fields():
    p = orc.Problem(mx=24, my=20, nz=16, radius=1.0, beta=8.0)
    c = 0.5 + 0.3 * np.random.default_rng(7).standard_normal((5, 4))
    EF, EA, fs = _inputs(p, 2, 13)
    EFs, EAs = _prescaled(EF, EA, fs)
    _close(co.vjp_fields_coarse(p, c, EF, EA, field_scales=fs),
           co.vjp_fields_coarse(p, c, EFs, EAs))


def test_a_swapped_scale_index_would_be_caught():
    # the same comparison fails when the scales are read as [l][c][f]-like
    # misreadings: here the adjoint field's scales replaced by the forward
    # field's (the slip the pin must catch)
    p = orc.Problem(mx=16, my=16, nz=16, radius=3.0, beta=8.0)
    C = np.random.default_rng(8).random((p.mx, p.my))
    EF, EA, fs = _inputs(p, 2, 14)
    wrong = fs.copy()
    wrong[:, 1, :] = fs[:, 0, :]
    EFs, EAs = _prescaled(EF, EA, fs)
    ref = orc.vjp_fields(p, C, EFs, EAs)
    bad = orc.vjp_fields(p, C, EF, EA, field_scales=wrong)
    assert np.max(np.abs(bad - ref)) > 1e-3 * np.max(np.abs(ref))
