"""Batched calls: many regions of uneven size, radius, beta and boundary
rule in one call, against the per-region calls and the FP64 oracle; and the
batched call captured in a CUDA graph."""

import numpy as np
import pytest

from oracle import epschain_oracle as orc
from paper_2505_03352_gb300 import synth

pytestmark = pytest.mark.gpu


def region_set(n=14, seed=21):
    rng = np.random.default_rng(seed)
    regs = []
    for r in range(n):
        side_a = int(rng.integers(8, 90)) * 2
        side_b = int(rng.integers(8, 90)) * 2
        regs.append(dict(mx=side_a, my=side_b, nz=int(rng.choice([16, 24])),
                         radius=float(rng.integers(2, 9)), beta=float(rng.choice([4, 8, 16, 32])),
                         bc=int(rng.integers(0, 2)), seed=1000 + r))
    return regs


def inputs(regs):
    import torch

    import paper_2505_03352_gb300 as ec
    probs, Cs, EF, EA, raw = [], [], [], [], []
    for d in regs:
        p = ec.Problem(mx=d["mx"], my=d["my"], nz=d["nz"], radius=d["radius"], beta=d["beta"],
                       bc=d["bc"])
        C = synth.soi_layout(d["mx"], d["my"], d["seed"])
        ef = synth.complex_field((3, p.nx, p.ny, p.nz), d["seed"] + 1)
        ea = synth.complex_field((3, p.nx, p.ny, p.nz), d["seed"] + 2)
        probs.append(p)
        Cs.append(torch.from_numpy(C).cuda())
        EF.append([torch.from_numpy(ef).cuda()])
        EA.append([torch.from_numpy(ea).cuda()])
        raw.append((C, ef, ea))
    return probs, Cs, EF, EA, raw


def test_batched_equals_per_region_and_oracle():
    import paper_2505_03352_gb300 as ec
    regs = region_set()
    probs, Cs, EF, EA, raw = inputs(regs)
    bv = ec.BatchedVjp(probs, Cs, EF, EA)
    G, E = bv()
    ec.eps_sync_status()
    for k, p in enumerate(probs):
        g1, e1 = ec.eps_vjp(p, Cs[k], EF[k], EA[k], eps_out=True)
        ec.eps_sync_status()
        g1, e1 = g1.cpu().numpy(), e1.cpu().numpy()
        gb, eb = G[k].cpu().numpy(), E[k].cpu().numpy()
        np.testing.assert_array_equal(eb, e1)   # same stencil code per tile
        assert np.max(np.abs(gb - g1)) <= 1e-5 * np.max(np.abs(g1))
        C, ef, ea = raw[k]
        o = orc.Problem(mx=p.mx, my=p.my, nz=p.nz, radius=p.radius, beta=p.beta, bc=p.bc)
        ref = orc.vjp_fields(o, C, [ef], [ea])
        assert np.max(np.abs(gb - ref)) / np.max(np.abs(ref)) <= 1e-4
        assert np.max(np.abs(eb - orc.eps_hat(o, C)) / orc.eps_hat(o, C)) <= 1e-5


def test_forward_batched_equals_per_region():
    import paper_2505_03352_gb300 as ec
    regs = region_set(9, seed=5)
    probs, Cs, _, _, _ = inputs(regs)
    E = ec.eps_forward_batched(probs, Cs)
    ec.eps_sync_status()
    for k, p in enumerate(probs):
        e1 = ec.eps_forward(p, Cs[k])
        ec.eps_sync_status()
        np.testing.assert_array_equal(E[k].cpu().numpy(), e1.cpu().numpy())


def test_batched_call_in_a_cuda_graph():
    import torch

    import paper_2505_03352_gb300 as ec
    regs = region_set(10, seed=8)
    probs, Cs, EF, EA, _ = inputs(regs)
    bv = ec.BatchedVjp(probs, Cs, EF, EA)
    G0, E0 = bv()
    torch.cuda.synchronize()
    ref = [g.clone() for g in G0]
    refe = [e.clone() for e in E0]
    for g in G0:
        g.zero_()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        bv(stream=s)          # warm-up on the capture stream
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        bv()
    for g in G0:
        g.zero_()
    graph.replay()
    torch.cuda.synchronize()
    ec.eps_sync_status()
    for k in range(len(probs)):
        torch.testing.assert_close(G0[k], ref[k], rtol=0, atol=0)
        torch.testing.assert_close(E0[k], refe[k], rtol=0, atol=0)


def test_concurrent_groups_in_a_cuda_graph():
    # the concurrent form forks its auxiliary streams from the captured stream
    # and joins them back: the capture is valid and each replay equals the
    # direct call (the auxiliary set is created by the first, uncaptured call)
    import torch

    import paper_2505_03352_gb300 as ec
    probs, Cs, EF, EA, _ = inputs(region_set(n=10, seed=51))
    bv = ec.BatchedVjp(probs, Cs, EF, EA)
    bv.set_tuning(concurrent_groups=1)
    G0, E0 = bv()
    ec.eps_sync_status()
    ref_g = [g.clone() for g in G0]
    ref_e = [e.clone() for e in E0]
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=s):
        bv()
    for k in range(len(probs)):
        bv.dJdC[k].fill_(float("nan"))
        bv.eps[k].fill_(float("nan"))
    for _ in range(2):
        graph.replay()
        torch.cuda.synchronize()
        ec.eps_sync_status()
        for k in range(len(probs)):
            torch.testing.assert_close(bv.dJdC[k], ref_g[k], rtol=0, atol=0)
            torch.testing.assert_close(bv.eps[k], ref_e[k], rtol=0, atol=0)


def test_mixed_radius_classes_need_their_own_launch_set():
    # radii 5.5 and 6 share the radius class ceil(R) = 6: the batch takes an
    # extra launch set, and both match their per-region calls
    import paper_2505_03352_gb300 as ec
    regs = [dict(mx=64, my=48, nz=16, radius=5.5, beta=8.0, bc=0, seed=3001),
            dict(mx=40, my=72, nz=16, radius=6.0, beta=16.0, bc=0, seed=3002),
            dict(mx=36, my=36, nz=16, radius=1.0, beta=8.0, bc=0, seed=3003),
            dict(mx=50, my=42, nz=16, radius=11.5, beta=32.0, bc=1, seed=3004)]
    probs, Cs, EF, EA, raw = inputs(regs)
    G, E = ec.BatchedVjp(probs, Cs, EF, EA)()
    ec.eps_sync_status()
    for k, p in enumerate(probs):
        g1, e1 = ec.eps_vjp(p, Cs[k], EF[k], EA[k], eps_out=True)
        ec.eps_sync_status()
        np.testing.assert_array_equal(E[k].cpu().numpy(), e1.cpu().numpy())
        assert np.max(np.abs(G[k].cpu().numpy() - g1.cpu().numpy())) <= 1e-5 * g1.abs().max().item()


# the last capture is meant to stay empty: tuning refuses to launch while the
# stream is capturing, and torch warns when such a capture ends
@pytest.mark.filterwarnings("ignore:The CUDA Graph is empty")
def test_autotuned_shapes_give_identical_results():
    import torch

    import paper_2505_03352_gb300 as ec
    regs = region_set(n=10, seed=33)
    probs, Cs, EF, EA, _ = inputs(regs)
    bv = ec.BatchedVjp(probs, Cs, EF, EA)
    G0, E0 = bv()
    G0 = [g.clone() for g in G0]
    E0 = [e.clone() for e in E0]
    res = bv.autotune(reps=2)
    assert res["evaluations"] >= 5 and res["tuned_ms"] <= res["default_ms"] * 1.0001
    assert res["multi"] in (0, 1) and res["stage_components"] in (1, 3)
    G1, E1 = bv()          # picks up the cached shapes
    ec.eps_sync_status()
    for k in range(len(probs)):
        assert torch.equal(E0[k], E1[k])
        assert torch.equal(G0[k], G1[k])
    # tuning refuses to run while the stream is capturing
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        with pytest.raises(ec.EpsError):
            with torch.cuda.graph(graph, stream=s):
                bv.autotune(reps=1)


@pytest.mark.parametrize("shapes", [
    dict(multi=1),                                        # persistent mixed-radius launches
    dict(multi=1, stencil_blocks_per_sm=1, scatter_blocks_per_sm=2, stage_components=1),
    dict(multi=0, defer_seeds=1),                         # seeds finished by the seeds kernel
    dict(multi=1, defer_seeds=1, contract_blocks_per_sm=2),
    dict(multi=0, scatter_bulk_staging=0),                # scatter gathers element by element
    dict(multi=0, scatter_bulk_staging=1, stage_components=3),   # bulk-copy scatter staging
    dict(multi=0, scatter_tile_cols=64, scatter_bulk_staging=0),  # wide scatter tiles
    dict(multi=0, scatter_tile_cols=64, scatter_bulk_staging=1),
    dict(multi=0, concurrent_groups=1),                   # radius groups on streams of their own
    dict(multi=0, concurrent_groups=1, scatter_bulk_staging=0, scatter_tile_cols=64),
])
def test_every_launch_form_equals_per_region_calls(shapes):
    import paper_2505_03352_gb300 as ec
    regs = region_set(n=12, seed=41)
    regs[3]["radius"], regs[4]["radius"] = 5.5, 6.0      # one radius class twice
    probs, Cs, EF, EA, raw = inputs(regs)
    bv = ec.BatchedVjp(probs, Cs, EF, EA)
    bv.set_tuning(**shapes)
    G, E = bv()
    ec.eps_sync_status()
    for k, p in enumerate(probs):
        g1, e1 = ec.eps_vjp(p, Cs[k], EF[k], EA[k], eps_out=True)
        ec.eps_sync_status()
        np.testing.assert_array_equal(E[k].cpu().numpy(), e1.cpu().numpy())
        assert np.max(np.abs(G[k].cpu().numpy() - g1.cpu().numpy())) <= 1e-5 * g1.abs().max().item()
    # and one region against the oracle directly
    C, ef, ea = raw[5]
    p = probs[5]
    o = orc.Problem(mx=p.mx, my=p.my, nz=p.nz, radius=p.radius, beta=p.beta, bc=p.bc)
    ref = orc.vjp_fields(o, C, [ef], [ea])
    assert np.max(np.abs(G[5].cpu().numpy() - ref)) <= 1e-4 * np.max(np.abs(ref))


def test_bad_tuning_is_rejected():
    import paper_2505_03352_gb300 as ec
    probs, Cs, EF, EA, _ = inputs(region_set(n=2, seed=43))
    bv = ec.BatchedVjp(probs, Cs, EF, EA)
    for bad in (dict(multi=2), dict(stage_components=2), dict(stencil_blocks_per_sm=0),
                dict(defer_seeds=5), dict(contract_blocks_per_sm=65)):
        with pytest.raises(ec.EpsError):
            bv.set_tuning(**bad)


def test_batched_tma_contraction_is_bitwise_the_per_region_calls():
    # the batched contraction streams every region through bulk tensor copies
    # with the single-region kernel's lane order, and the stencil and scatter
    # run the same tile code: dJ/dC and eps_hat equal the per-region calls bit
    # for bit (regions of uneven size, slab position, nz and wavelengths)
    import paper_2505_03352_gb300 as ec
    import torch
    regs = region_set(n=16, seed=51)
    regs[2]["nz"], regs[7]["nz"] = 32, 20
    for nl in (1, 3):
        probs, Cs, EF, EA, _ = inputs(regs)
        if nl > 1:
            EF = [[e[0]] + [torch.randn_like(e[0]) for _ in range(nl - 1)] for e in EF]
            EA = [[e[0]] + [torch.randn_like(e[0]) for _ in range(nl - 1)] for e in EA]
        bv = ec.BatchedVjp(probs, Cs, EF, EA)
        G, E = bv()
        ec.eps_sync_status()
        for k, p in enumerate(probs):
            g1, e1 = ec.eps_vjp(p, Cs[k], EF[k], EA[k], eps_out=True)
            ec.eps_sync_status()
            np.testing.assert_array_equal(E[k].cpu().numpy(), e1.cpu().numpy())
            np.testing.assert_array_equal(G[k].cpu().numpy(), g1.cpu().numpy())


def test_register_load_contraction_for_batches_beyond_the_tensor_map_capacity():
    # 40 regions x 3 wavelengths need 240 tensor maps, more than one launch
    # carries: the register-load contraction runs, within rounding of the
    # per-region calls and within the oracle tolerance
    import paper_2505_03352_gb300 as ec
    import torch
    regs = region_set(n=40, seed=53)
    probs, Cs, EF, EA, raw = inputs(regs)
    EF = [[e[0]] + [torch.randn_like(e[0]) for _ in range(2)] for e in EF]
    EA = [[e[0]] + [torch.randn_like(e[0]) for _ in range(2)] for e in EA]
    G, E = ec.BatchedVjp(probs, Cs, EF, EA)()
    ec.eps_sync_status()
    for k in (0, 13, 39):
        p = probs[k]
        g1, e1 = ec.eps_vjp(p, Cs[k], EF[k], EA[k], eps_out=True)
        ec.eps_sync_status()
        np.testing.assert_array_equal(E[k].cpu().numpy(), e1.cpu().numpy())
        assert np.max(np.abs(G[k].cpu().numpy() - g1.cpu().numpy())) <= 1e-5 * g1.abs().max().item()
        C = raw[k][0]
        o = orc.Problem(mx=p.mx, my=p.my, nz=p.nz, radius=p.radius, beta=p.beta, bc=p.bc)
        ref = orc.vjp_fields(o, C, [e.cpu().numpy() for e in EF[k]], [e.cpu().numpy() for e in EA[k]])
        assert np.max(np.abs(G[k].cpu().numpy() - ref)) <= 1e-4 * np.max(np.abs(ref))


@pytest.mark.parametrize("mx,my,radius,bc", [
    (1000, 904, 6.0, 0),    # more than one wave of scatter tiles: bulk-copy staging
    (968, 1000, 3.0, 1),    # periodic: tiles clear of the wrap take the bulk copies
    (1024, 1000, 11.5, 0),  # the widest halo (radius class 12)
    (900, 1048, 2.5, 0),    # radius class 3, the smallest with bulk copies
])
def test_bulk_copy_staging_equals_elementwise_staging(mx, my, radius, bc):
    # a single call larger than one wave stages the scatter's inputs of its
    # interior tiles through bulk tensor copies; a one-region batch stages
    # every tile element by element: the results agree bit for bit
    import torch

    import paper_2505_03352_gb300 as ec
    p = ec.Problem(mx=mx, my=my, nz=16, radius=radius, beta=16.0, bc=bc)
    C = torch.from_numpy(synth.soi_layout(mx, my, mx + my + 7)).cuda()
    ef = [torch.from_numpy(synth.complex_field((3, p.nx, p.ny, p.nz), 61))]
    ea = [torch.from_numpy(synth.complex_field((3, p.nx, p.ny, p.nz), 62))]
    ef, ea = [x.cuda() for x in ef], [x.cuda() for x in ea]
    g1, e1 = ec.eps_vjp(p, C, ef, ea, eps_out=True)
    G, E = ec.BatchedVjp([p], [C], [ef], [ea])()
    ec.eps_sync_status()
    assert torch.equal(G[0], g1)
    assert torch.equal(E[0], e1)
