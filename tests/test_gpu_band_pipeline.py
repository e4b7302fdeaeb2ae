"""The band pipeline of a multi-wave single-region call (edge-replicate
rule, complex64 fields): the contraction runs in column bands on the
caller's stream while a second stream runs the stencil, each band's seeds
and the scatter of the tile rows whose seed maps are complete.

- Against the FP64 oracle on a shape whose band boundaries fall inside Yee
  rows and whose last tile row and column are partial: dJ/dC within 1e-4 of
  its largest value, eps_hat within 1e-5 relative, and the Eq. 1 surrogate
  S within 1e-5 of the sum of its terms' magnitudes.
- Calls queued back to back on a side stream, into the same outputs and
  workspace, with C changed between them: the last call's result equals a
  lone call's bit for bit (no band of a later call overtakes an earlier
  call's scatter).
- Captured in a CUDA graph and replayed: the direct call's result bit for
  bit.
- Packed BF16 / FP16 fields on the same multi-wave shape (the packed
  contraction takes a column range too): against the oracle fed the
  decoded bytes, within the same tolerances.
- The library's launch counter over one call of each form (what the bench
  line's `gpu_launches` reports).
"""

import numpy as np
import pytest

from oracle import epschain_oracle as orc
from paper_2505_03352_gb300 import synth

pytestmark = pytest.mark.gpu


def _dev(x):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def _support_sum(o, e, w):
    k0, nk = o.k0, o.slab_nk
    return (float(np.sum(e[0:2, :, :, k0 + 1:k0 + nk + 1] * w[0:2, :, :, k0 + 1:k0 + nk + 1]))
            + float(np.sum(e[2, :, :, k0:k0 + nk + 1] * w[2, :, :, k0:k0 + nk + 1])))


def test_pipelined_call_matches_the_oracle():
    import paper_2505_03352_gb300 as ec
    mx, my, nz = 1202, 1042, 32      # 601 x 521 columns: 9786 chunks, 76 x 17 stencil tiles
    p = ec.Problem(mx=mx, my=my, nz=nz, radius=6.0, beta=16.0)
    o = orc.Problem(mx=mx, my=my, nz=nz, radius=6.0, beta=16.0)
    C = synth.soi_layout(mx, my, 9100)
    shape = (3, p.nx, p.ny, nz)
    EF = [synth.complex_field(shape, 9101 + l) for l in range(2)]
    EA = [synth.complex_field(shape, 9111 + l) for l in range(2)]
    g, e, S = ec.eps_vjp_surrogate(p, _dev(C), [_dev(x) for x in EF], [_dev(x) for x in EA],
                                   eps_out=True)
    ec.eps_sync_status()
    ref_g = orc.vjp_fields(o, C, EF, EA)
    ref_e = orc.eps_hat(o, C)
    g, e = g.cpu().numpy(), e.cpu().numpy()
    assert float(np.max(np.abs(g - ref_g)) / np.max(np.abs(ref_g))) <= 1e-4
    assert float(np.max(np.abs(e - ref_e) / ref_e)) <= 1e-5
    w = -2.0 * sum((ef.astype(np.complex128) * ea).real for ef, ea in zip(EF, EA))
    ref_S = _support_sum(o, ref_e, w)
    mag = _support_sum(o, ref_e, np.abs(w))
    assert abs(S.item() - ref_S) <= 1e-5 * mag, (S.item(), ref_S, mag)


def _case(mx=1600, my=1200, nz=32, nl=3, seed=9200):
    import paper_2505_03352_gb300 as ec
    p = ec.Problem(mx=mx, my=my, nz=nz, radius=6.0, beta=16.0)
    shape = (3, p.nx, p.ny, nz)
    EF = [_dev(synth.complex_field(shape, seed + l)) for l in range(nl)]
    EA = [_dev(synth.complex_field(shape, seed + 10 + l)) for l in range(nl)]
    C1 = _dev(synth.soi_layout(mx, my, seed + 20))
    C2 = _dev(synth.soi_layout(mx, my, seed + 21))
    return p, EF, EA, C1, C2


def _workspace(ec, p, nl):
    import torch
    return torch.empty(ec.eps_workspace_size(p, nl), dtype=torch.uint8, device="cuda")


def test_back_to_back_calls_on_a_side_stream():
    import torch

    import paper_2505_03352_gb300 as ec
    p, EF, EA, C1, C2 = _case()
    ref_g, ref_e = ec.eps_vjp(p, C2, EF, EA, eps_out=True)
    torch.cuda.synchronize()
    g = torch.empty_like(ref_g)
    e = torch.empty_like(ref_e)
    ws = _workspace(ec, p, len(EF))
    C = C1.clone()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        for _ in range(3):
            ec.eps_vjp(p, C, EF, EA, dJdC=g, eps_out=e, ws=ws, stream=s)
            C.copy_(C2)   # on s: after the call has joined its pipeline stream
            ec.eps_vjp(p, C, EF, EA, dJdC=g, eps_out=e, ws=ws, stream=s)
            C.copy_(C1)
        C.copy_(C2)
        ec.eps_vjp(p, C, EF, EA, dJdC=g, eps_out=e, ws=ws, stream=s)
    s.synchronize()
    ec.eps_sync_status()
    torch.testing.assert_close(g, ref_g, rtol=0, atol=0)
    torch.testing.assert_close(e, ref_e, rtol=0, atol=0)


def test_pipelined_call_in_a_cuda_graph():
    import torch

    import paper_2505_03352_gb300 as ec
    p, EF, EA, C1, _ = _case(nl=2, seed=9300)
    ref_g, ref_e = ec.eps_vjp(p, C1, EF, EA, eps_out=True)
    torch.cuda.synchronize()
    g = torch.zeros_like(ref_g)
    e = torch.zeros_like(ref_e)
    ws = _workspace(ec, p, len(EF))
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        ec.eps_vjp(p, C1, EF, EA, dJdC=g, eps_out=e, ws=ws, stream=s)   # warm-up
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        ec.eps_vjp(p, C1, EF, EA, dJdC=g, eps_out=e, ws=ws)
    g.zero_()
    e.zero_()
    graph.replay()
    torch.cuda.synchronize()
    ec.eps_sync_status()
    torch.testing.assert_close(g, ref_g, rtol=0, atol=0)
    torch.testing.assert_close(e, ref_e, rtol=0, atol=0)


def _decode(buf, p, field_type):
    """The packed planes of eps_field_pack back to complex128 fields (zero off
    the support planes): per-component scale times the stored pairs."""
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
    return E


@pytest.mark.parametrize("field_type", [1, 2])
def test_pipelined_packed_call_matches_the_oracle_on_decoded_fields(field_type):
    # BF16 / FP16 fields through the bulk-copy packed contraction (chunks of
    # 128 columns): against the oracle fed the decoded bytes, within the
    # FP32 path's tolerances
    import torch

    import paper_2505_03352_gb300 as ec
    mx, my, nz = 1202, 1042, 32
    p = ec.Problem(mx=mx, my=my, nz=nz, radius=6.0, beta=16.0)
    o = orc.Problem(mx=mx, my=my, nz=nz, radius=6.0, beta=16.0)
    C = synth.soi_layout(mx, my, 9400)
    shape = (3, p.nx, p.ny, nz)
    EF = [synth.complex_field(shape, 9401 + l) for l in range(2)]
    EA = [synth.complex_field(shape, 9411 + l) for l in range(2)]
    PF = [ec.eps_field_pack(p, field_type, torch.from_numpy(e).cuda()) for e in EF]
    PA = [ec.eps_field_pack(p, field_type, torch.from_numpy(e).cuda()) for e in EA]
    g, e = ec.eps_vjp(p, _dev(C), PF, PA, eps_out=True, field_type=field_type)
    ec.eps_sync_status()
    ref = orc.vjp_fields(o, C, [_decode(b, p, field_type) for b in PF],
                         [_decode(b, p, field_type) for b in PA])
    g = g.cpu().numpy()
    assert float(np.max(np.abs(g - ref)) / np.max(np.abs(ref))) <= 1e-4
    ref_e = orc.eps_hat(o, C)
    assert float(np.max(np.abs(e.cpu().numpy() - ref_e) / ref_e)) <= 1e-5


def test_launch_counter_counts_each_form():
    # eps_launch_count over one call: the one-wave form launches the
    # contraction, the stencil and the scatter; a pipelined multi-wave call
    # three contraction bands, the stencil, three seeds launches and up to
    # three scatter launches; under per-kernel profiling the same call keeps
    # the single-stream order (contraction, stencil, seeds, scatter)
    import torch

    import paper_2505_03352_gb300 as ec
    small = ec.Problem(mx=64, my=48, nz=16, radius=3.0, beta=8.0)
    shape = (3, small.nx, small.ny, small.nz)
    EF = [_dev(synth.complex_field(shape, 9501))]
    EA = [_dev(synth.complex_field(shape, 9502))]
    C = _dev(synth.soi_layout(64, 48, 9503))
    ec.eps_vjp(small, C, EF, EA)
    torch.cuda.synchronize()
    n0 = ec.eps_launch_count()
    ec.eps_vjp(small, C, EF, EA)
    assert ec.eps_launch_count() - n0 == 3
    p, EF, EA, C1, _ = _case(nl=1, seed=9510)
    ec.eps_vjp(p, C1, EF, EA)
    torch.cuda.synchronize()
    n0 = ec.eps_launch_count()
    ec.eps_vjp(p, C1, EF, EA)
    assert 8 <= ec.eps_launch_count() - n0 <= 10
    ec.eps_profile_start()
    n0 = ec.eps_launch_count()
    ec.eps_vjp(p, C1, EF, EA)
    assert ec.eps_launch_count() - n0 == 4
    ec.eps_profile_stop(64)
    ec.eps_sync_status()


@pytest.mark.parametrize("nz,nl", [(30, 2), (16, 16)],
                         ids=["planes_not_a_multiple_of_4", "sixteen_wavelengths"])
def test_pipelined_call_other_plane_counts_and_wavelengths(nz, nl):
    # nz = 30: the stencil writes eps_hat column by column (no staging form
    # takes it); 16 wavelengths: the contraction's largest map count
    import paper_2505_03352_gb300 as ec
    mx, my = 802, 722                 # 401 x 361 columns: ragged chunks and tiles
    p = ec.Problem(mx=mx, my=my, nz=nz, radius=4.0, beta=16.0)
    o = orc.Problem(mx=mx, my=my, nz=nz, radius=4.0, beta=16.0)
    C = synth.soi_layout(mx, my, 9600 + nz)
    shape = (3, p.nx, p.ny, nz)
    EF = [synth.complex_field(shape, 9610 + l) for l in range(nl)]
    EA = [synth.complex_field(shape, 9630 + l) for l in range(nl)]
    g, e = ec.eps_vjp(p, _dev(C), [_dev(x) for x in EF], [_dev(x) for x in EA], eps_out=True)
    ec.eps_sync_status()
    ref_g = orc.vjp_fields(o, C, EF, EA)
    ref_e = orc.eps_hat(o, C)
    g, e = g.cpu().numpy(), e.cpu().numpy()
    assert float(np.max(np.abs(g - ref_g)) / np.max(np.abs(ref_g))) <= 1e-4
    assert float(np.max(np.abs(e - ref_e) / ref_e)) <= 1e-5
