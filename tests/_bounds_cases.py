"""Calls that run every kernel family of the library once on shapes that
reach its edge cases (ragged tiles, both boundary rules, radius classes 1
to 12, the multi-wave forms, the register-load contraction, packed fields,
batches in both launch forms and beyond the tensor-map capacity, the
morphology chain, coarse controls, 3-D normals, the optimiser step).  Used
by the debug-bounds test, which runs them through the release build and
the debug-bounds build and compares the outputs.  Inputs come from seeded
numpy generators only, so both runs see the same values."""

import numpy as np


def _dev(torch, x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def _fields(torch, shape, nl, seed):
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(2 * nl):
        z = (rng.standard_normal(shape) + 1j * rng.standard_normal(shape)).astype(np.complex64)
        out.append(_dev(torch, z))
    return out[:nl], out[nl:]


def _controls(mx, my, seed):
    return np.random.default_rng(seed).random((mx, my), dtype=np.float32)


SINGLE = [
    # mx, my, nz, radius, beta, bc, slab_nk
    (66, 50, 16, 3.0, 8.0, 0, 11),
    (70, 94, 20, 5.5, 16.0, 1, 11),
    (130, 62, 24, 8.0, 32.0, 0, 11),
    (34, 34, 16, 1.0, 8.0, 0, 11),
    (90, 76, 16, 11.5, 16.0, 1, 11),
    (800, 720, 16, 4.0, 16.0, 0, 11),   # more than one wave of tiles: seeds kernel
    (60, 58, 48, 3.0, 8.0, 0, 40),      # window wider than a TMA box: register loads, 4 lanes
    (62, 54, 46, 2.0, 8.0, 1, 40),      # the same with nz % 4 != 0: 8 lanes
]


def run_cases(ec, torch):
    out = {}
    sync = ec.eps_sync_status
    for n, (mx, my, nz, radius, beta, bc, nk) in enumerate(SINGLE):
        p = ec.Problem(mx=mx, my=my, nz=nz, radius=radius, beta=beta, bc=bc, slab_nk=nk)
        C = _dev(torch, _controls(mx, my, 100 + n))
        EF, EA = _fields(torch, (3, p.nx, p.ny, p.nz), 2, 200 + n)
        g, e = ec.eps_vjp(p, C, EF, EA, eps_out=True)
        sync()
        out[f"vjp{n}"], out[f"eps{n}"] = g.cpu().numpy(), e.cpu().numpy()
        G = _dev(torch, np.random.default_rng(300 + n).standard_normal((3, p.nx, p.ny, p.nz)).astype(np.float32))
        out[f"real{n}"] = ec.eps_vjp_real(p, C, G).cpu().numpy()
        sync()
    # off-diagonal terms and 3-D face normals
    for n, flags in enumerate((ec.EPS_FLAG_OFFDIAG, ec.EPS_FLAG_OFFDIAG | ec.EPS_FLAG_NORMALS_3D)):
        p = ec.Problem(mx=78, my=66, nz=16, radius=4.0, beta=16.0, flags=flags)
        e, od = ec.eps_forward(p, _dev(torch, _controls(78, 66, 400 + n)))
        sync()
        out[f"fwd_eps{n}"], out[f"fwd_od{n}"] = e.cpu().numpy(), od.cpu().numpy()
    # packed fields
    for n, ft in enumerate((ec.EPS_FIELD_BF16X2_SCALED, ec.EPS_FIELD_F16X2_SCALED)):
        p = ec.Problem(mx=82, my=70, nz=20, radius=3.0, beta=8.0)
        C = _dev(torch, _controls(82, 70, 500 + n))
        EF, EA = _fields(torch, (3, p.nx, p.ny, p.nz), 3, 510 + n)
        PF = [ec.eps_field_pack(p, ft, x) for x in EF]
        PA = [ec.eps_field_pack(p, ft, x) for x in EA]
        out[f"packed{n}"] = ec.eps_vjp(p, C, PF, PA, field_type=ft).cpu().numpy()
        sync()
    # batches: grouped and multi forms (TMA contraction), and 25 regions x 4
    # wavelengths (200 tensor maps: register-load contraction)
    rng = np.random.default_rng(600)
    for n, (nreg, nl, shapes) in enumerate(((9, 1, {}), (9, 1, {"multi": 1, "defer_seeds": 1}),
                                           (25, 4, {}))):
        probs, Cs, EFs, EAs = [], [], [], []
        for k in range(nreg):
            mx, my = (int(v) * 2 for v in rng.integers(8, 60, size=2))
            p = ec.Problem(mx=mx, my=my, nz=int(rng.choice([16, 24])), radius=float(rng.integers(1, 10)),
                           beta=8.0, bc=int(rng.integers(0, 2)))
            probs.append(p)
            Cs.append(_dev(torch, _controls(mx, my, 700 + 100 * n + k)))
            ef, ea = _fields(torch, (3, p.nx, p.ny, p.nz), nl, 800 + 100 * n + k)
            EFs.append(ef)
            EAs.append(ea)
        bv = ec.BatchedVjp(probs, Cs, EFs, EAs)
        if shapes:
            bv.set_tuning(**shapes)
        G, E = bv()
        sync()
        for k in range(nreg):
            out[f"batch{n}_g{k}"], out[f"batch{n}_e{k}"] = G[k].cpu().numpy(), E[k].cpu().numpy()
    # morphology chain
    for n, (bc, rad) in enumerate(((0, 2.0), (1, 7.5))):
        p = ec.Problem(mx=72, my=60, nz=16, radius=3.0, beta=16.0, bc=bc)
        m = ec.Morph(alpha=20.0, radius=rad)
        C = _dev(torch, _controls(72, 60, 900 + n))
        EF, EA = _fields(torch, (3, p.nx, p.ny, p.nz), 1, 910 + n)
        g, e = ec.eps_vjp_morph(p, m, C, EF, EA, eps_out=True)
        sync()
        out[f"morph_g{n}"], out[f"morph_e{n}"] = g.cpu().numpy(), e.cpu().numpy()
    # coarse control nodes
    p = ec.Problem(mx=84, my=84, nz=16, radius=3.0, beta=16.0)
    cg = ec.Coarse(ncx=13, ncy=9)
    c = _dev(torch, np.random.default_rng(1000).random((13, 9), dtype=np.float32))
    EF, EA = _fields(torch, (3, p.nx, p.ny, p.nz), 1, 1001)
    dc, e = ec.eps_vjp_coarse(p, cg, c, EF, EA, eps_out=True)
    sync()
    out["coarse_g"], out["coarse_e"] = dc.cpu().numpy(), e.cpu().numpy()
    # one optimiser step after a VJP
    p = ec.Problem(mx=64, my=60, nz=16, radius=3.0, beta=8.0)
    opt = ec.OptParams(lr=0.01, n_iter=10)
    state = ec.eps_opt_init(opt)
    C = _dev(torch, _controls(64, 60, 1100))
    EF, EA = _fields(torch, (3, p.nx, p.ny, p.nz), 1, 1101)
    ws = torch.empty(ec.eps_workspace_size(p), dtype=torch.uint8, device="cuda")
    G = ec.eps_vjp(p, C, EF, EA, ws=ws)
    M, V = torch.zeros_like(C), torch.zeros_like(C)
    ec.eps_opt_step(p, opt, state, C, G, M, V, ws)
    sync()
    out["opt_C"], out["opt_M"], out["opt_V"] = C.cpu().numpy(), M.cpu().numpy(), V.cpu().numpy()
    return out
