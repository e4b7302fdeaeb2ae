"""Chain with coarse control variables (Eq. 2 on a node grid): the CUDA path
(through the C ABI) against the FP64 coarse-control oracle, element by
element.  eps_hat: max relative error <= 1e-5; dJ/dc: max |delta| / max |ref|
<= 1e-4."""

import numpy as np
import pytest

from oracle import coarse_oracle as co
from oracle import epschain_oracle as orc
from paper_2505_03352_gb300 import synth

pytestmark = pytest.mark.gpu


def _ec():
    import paper_2505_03352_gb300 as ec
    return ec


def to_dev(x):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def eps_err(got, ref):
    return float(np.max(np.abs(got - ref) / np.abs(ref)))


def grad_err(got, ref):
    return float(np.max(np.abs(got - ref)) / np.max(np.abs(ref)))


@pytest.mark.parametrize("mx,my,nz,ncx,ncy,beta,bc", [
    (420, 420, 24, 36, 36, 16.0, 0),      # the paper's layout: 210 x 210 cells, 36 x 36 controls
    (420, 420, 24, 36, 36, 32.0, 1),      # periodic, beta = 32
    (70, 46, 16, 5, 9, 8.0, 0),           # ragged, non-integer spacing
    (64, 64, 16, 2, 2, 8.0, 0),           # one cell of the node grid
    (40, 36, 14, 33, 30, 8.0, 1),         # spacing below two subpixels
])
def test_coarse_chain_matches_oracle(mx, my, nz, ncx, ncy, beta, bc):
    ec = _ec()
    p = ec.Problem(mx=mx, my=my, nz=nz, radius=3.0, beta=beta, bc=bc)
    o = orc.Problem(mx=mx, my=my, nz=nz, radius=3.0, beta=beta, bc=bc)
    g = ec.Coarse(ncx, ncy)
    rng = np.random.default_rng(6100 + mx + ncx)
    c = (0.5 + 0.35 * rng.standard_normal((ncx, ncy))).astype(np.float32)
    shape = (3, p.nx, p.ny, p.nz)
    EF = [synth.complex_field(shape, 6101)]
    EA = [synth.complex_field(shape, 6102)]
    ref = co.eps_hat_coarse(o, c)
    e = ec.eps_forward_coarse(p, g, to_dev(c)).cpu().numpy()
    ec.eps_sync_status()
    assert eps_err(e, ref) <= 1e-5, eps_err(e, ref)
    ref_g = co.vjp_fields_coarse(o, c, EF, EA)
    d, e2 = ec.eps_vjp_coarse(p, g, to_dev(c), [to_dev(x) for x in EF], [to_dev(x) for x in EA],
                              eps_out=True)
    ec.eps_sync_status()
    assert grad_err(d.cpu().numpy(), ref_g) <= 1e-4, grad_err(d.cpu().numpy(), ref_g)
    assert eps_err(e2.cpu().numpy(), ref) <= 1e-5
    G = rng.standard_normal(shape).astype(np.float32)
    ref_r = co.vjp_real_coarse(o, c, G.astype(np.float64))
    dr = ec.eps_vjp_real_coarse(p, g, to_dev(c), to_dev(G)).cpu().numpy()
    ec.eps_sync_status()
    assert grad_err(dr, ref_r) <= 1e-4


def test_coarse_repeated_calls_are_bitwise_identical():
    ec = _ec()
    p = ec.Problem(mx=420, my=420, nz=24, radius=3.0, beta=16.0)
    g = ec.Coarse(36, 36)
    c = to_dev((0.5 + 0.3 * np.random.default_rng(1).standard_normal((36, 36))).astype(np.float32))
    shape = (3, p.nx, p.ny, p.nz)
    EF = [to_dev(synth.complex_field(shape, 1))]
    EA = [to_dev(synth.complex_field(shape, 2))]
    a = ec.eps_vjp_coarse(p, g, c, EF, EA).cpu().numpy()
    b = ec.eps_vjp_coarse(p, g, c, EF, EA).cpu().numpy()
    assert np.array_equal(a, b)
