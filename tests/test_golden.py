"""Values the paper prints (tests/golden/paper_values.json, each with its
citation) against the defaults and readings of the oracles and the
binding."""

import json
import os

import numpy as np

from oracle import coarse_oracle as co
from oracle import epschain_oracle as orc
from oracle import morph_oracle as mo
from oracle import optimizer_oracle as oo

GOLDEN = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))


def test_optimiser_defaults_are_app_b():
    b = GOLDEN["app_b_defaults"]
    from paper_2505_03352_gb300.epschain import OptParams
    for p in (oo.OptParams(), OptParams()):
        assert (p.b1, p.b2, p.lr, p.gamma, p.u0, p.beta_min) == (
            b["b1"], b["b2"], b["eta"], b["gamma"], b["u0"], b["beta_min"])


def test_morphology_alpha_is_app_b():
    b = GOLDEN["app_b_defaults"]
    from paper_2505_03352_gb300.epschain import Morph
    assert mo.Morph().alpha == b["alpha"] == Morph().alpha


def test_app_b_permittivities_read_as_refractive_indices():
    # 3.4^2 and 1.44^2 are within 5 % of the Si / SiO2 permittivities the
    # chain uses; read literally, 3.4 / 1.44 would be a quite different contrast
    b, e = GOLDEN["app_b_defaults"], GOLDEN["permittivities_used"]
    assert abs(b["eps_core"] ** 2 - e["eps_si"]) / e["eps_si"] < 0.05
    assert abs(b["eps_clad"] ** 2 - e["eps_sio2"]) / e["eps_sio2"] < 0.01
    p = orc.Problem(mx=4, my=4, nz=14, radius=1.0, beta=1.0)
    assert (p.eps_core, p.eps_clad) == (e["eps_si"], e["eps_sio2"])


def test_coarse_layout_of_the_paper():
    g = GOLDEN["coarse_layout"]
    m = 2 * g["cells"]                      # two subpixels per Yee cell
    B = co.basis_matrix(m, g["controls"])
    assert m % (g["controls"] - 1) == 0     # an integer stride
    np.testing.assert_allclose(B.sum(axis=1), 1.0, atol=1e-14)


def test_morphology_diameters_at_10_nm_pitch():
    d = GOLDEN["morphology_diameters_nm"]
    r_min, r_max = d["d_min"] / 2 / 10, d["d_max"] / 2 / 10   # disk radii in subpixels
    assert len(mo.disk_taps(r_min)) == 5                        # the smallest non-trivial disk
    assert len(mo.disk_taps(r_max)) == sum(1 for p in range(-7, 8) for q in range(-7, 8)
                                           if p * p + q * q <= r_max * r_max)
