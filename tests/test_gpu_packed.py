"""Reduced-precision (BF16 / FP16) field storage.

The packed bytes are read back and decoded on the host with numpy (bf16 is
the upper half of an IEEE float32, fp16 is numpy's float16), independently
of the CUDA code.  Feeding the decoded fields to the FP64 oracle must give
the GPU's packed-path gradient within the FP32 tolerance: that pins the
packed contraction.  The extra error of the reduced precision itself is
stated (measured against the oracle on the original complex64 fields), not
gated.
"""

import numpy as np
import pytest

from oracle import epschain_oracle as orc
from paper_2505_03352_gb300 import synth

pytestmark = pytest.mark.gpu


def decode(buf, p, field_type):
    raw = buf.cpu().numpy()
    scale = raw[:16].view(np.float32)[:3].astype(np.float64)
    npl = (p.slab_nk + 1 + 3) // 4 * 4
    data = raw[16:16 + 3 * p.nx * p.ny * npl * 4].view(np.uint16).reshape(3, p.nx, p.ny, npl, 2)
    if field_type == 1:   # bf16: the high 16 bits of a float32
        vals = (data.astype(np.uint32) << 16).view(np.float32).astype(np.float64)
    else:
        vals = data.view(np.float16).astype(np.float64)
    E = np.zeros((3, p.nx, p.ny, p.nz), np.complex128)
    k0, nk = p.k0, p.slab_nk
    n = min(nk + 1, p.nz - k0)
    for c in range(3):
        E[c, :, :, k0:k0 + n] = scale[c] * (vals[c, :, :, :n, 0] + 1j * vals[c, :, :, :n, 1])
    return E, scale


@pytest.mark.parametrize("field_type", [1, 2])
def test_pack_roundtrip_error_bound(field_type):
    import torch

    import paper_2505_03352_gb300 as ec
    p = ec.Problem(mx=96, my=160, nz=24, radius=3.0, beta=8.0)
    E = synth.complex_field((3, p.nx, p.ny, p.nz), 41)
    buf = ec.eps_field_pack(p, field_type, torch.from_numpy(E).cuda())
    ec.eps_sync_status()
    D, scale = decode(buf, p, field_type)
    k0, nk = p.k0, p.slab_nk
    orig = E[:, :, :, k0:k0 + nk + 1].astype(np.complex128)
    dec = D[:, :, :, k0:k0 + nk + 1]
    rel = 2.0 ** (-8 if field_type == 1 else -11)
    for part in (np.real, np.imag):
        err = np.abs(part(dec) - part(orig))
        assert np.all(err <= rel * np.abs(part(orig)) + 1e-30 + (0 if field_type == 1 else scale.max() * 2.0 ** -24))
    # scales: max |re|, |im| over the support planes / target
    target = 1.0 if field_type == 1 else 16384.0
    for c in range(3):
        amax = max(np.abs(orig[c].real).max(), np.abs(orig[c].imag).max())
        assert abs(scale[c] - np.float32(amax) / target) <= 1e-7 * scale[c]


@pytest.mark.parametrize("field_type", [1, 2])
@pytest.mark.parametrize("bc", [0, 1])
def test_packed_vjp_equals_oracle_on_decoded_fields(field_type, bc):
    import torch

    import paper_2505_03352_gb300 as ec
    mx, my, nz = 130, 98, 24
    p = ec.Problem(mx=mx, my=my, nz=nz, radius=6.0, beta=16.0, bc=bc)
    o = orc.Problem(mx=mx, my=my, nz=nz, radius=6.0, beta=16.0, bc=bc)
    C = synth.soi_layout(mx, my, 9)
    EF = [synth.complex_field((3, p.nx, p.ny, nz), 50 + l) for l in range(2)]
    EA = [synth.complex_field((3, p.nx, p.ny, nz), 60 + l) for l in range(2)]
    PF = [ec.eps_field_pack(p, field_type, torch.from_numpy(e).cuda()) for e in EF]
    PA = [ec.eps_field_pack(p, field_type, torch.from_numpy(e).cuda()) for e in EA]
    g, eps = ec.eps_vjp(p, torch.from_numpy(C).cuda(), PF, PA, eps_out=True, field_type=field_type)
    ec.eps_sync_status()
    g = g.cpu().numpy()
    DF = [decode(b, p, field_type)[0] for b in PF]
    DA = [decode(b, p, field_type)[0] for b in PA]
    ref = orc.vjp_fields(o, C, DF, DA)
    assert np.max(np.abs(g - ref)) / np.max(np.abs(ref)) <= 1e-4
    # the stated (not gated) error against the full-precision fields
    exact = orc.vjp_fields(o, C, EF, EA)
    err = float(np.max(np.abs(g - exact)) / np.max(np.abs(exact)))
    assert err < (5e-2 if field_type == 1 else 5e-3)
    np.testing.assert_allclose(eps.cpu().numpy(), orc.eps_hat(o, C), rtol=1e-5)
