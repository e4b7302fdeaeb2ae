"""Host-side argument checks of the batched, tuning, packed-field and L2
entry points of the C ABI, without a GPU: each case returns its status
before any CUDA call (pointers here are placeholders that the checks never
dereference)."""

import ctypes
import os

import pytest

from paper_2505_03352_gb300 import epschain as ec

OK, INVALID, SHAPE, WORKSPACE, UNSUPPORTED = 0, 1, 2, 3, 4


@pytest.fixture(scope="module")
def L():
    if not os.path.exists(ec.LIB_PATH):
        from paper_2505_03352_gb300 import build_lib
        build_lib.build()
    return ec.lib()


def prob(**kw):
    base = dict(mx=64, my=48, nz=16, radius=3.0, beta=8.0)
    base.update(kw)
    return ec.Problem(**base)


def probs_array(ps):
    return ec._probs(ps)


def ptrs(n, value=None):
    return (ctypes.c_void_p * max(n, 1))(*([value] * n))


def batched_ws(L, ps, n_lambda=1):
    n = ctypes.c_size_t(0)
    st = L.eps_batched_workspace_size(len(ps), probs_array(ps), n_lambda, ctypes.byref(n))
    return st, n.value


def test_batched_workspace_is_the_regions_laid_end_to_end(L):
    ps = [prob(), prob(mx=100, my=36, radius=6.0), prob(mx=0), prob(mx=32, my=32, nz=24)]
    st, total = batched_ws(L, ps)
    assert st == OK
    assert total == sum(ec.eps_workspace_size(p) for p in ps)
    assert ec.eps_workspace_size(prob(mx=0)) == 0


@pytest.mark.parametrize("ps,n_lambda,status", [
    ([prob()] * 65, 1, INVALID),                                  # more than 64 regions
    ([prob()], 5, INVALID),                                       # more than 4 wavelengths
    ([prob()], -1, INVALID),
    ([prob(), prob(mx=63)], 1, SHAPE),                            # a bad region
    ([prob(flags=ec.EPS_FLAG_NORMALS_3D)], 1, UNSUPPORTED),       # single-region forward only
])
def test_batched_workspace_rejects(L, ps, n_lambda, status):
    assert batched_ws(L, ps, n_lambda)[0] == status


def vjp_batched(L, ps, n_lambda=1, field_type=0, scale=-2.0, C=True, G=True, EF=True, ws=None,
                ws_bytes=0):
    n = len(ps)
    return L.eps_vjp_batched(n, probs_array(ps) if n else None, ptrs(n) if C else None, n_lambda,
                             field_type, ptrs(n * n_lambda) if EF else None,
                             ptrs(n * n_lambda) if EF else None, None, scale,
                             ptrs(n) if G else None, None, ws, ws_bytes, None)


def test_batched_vjp_checks_before_any_launch(L):
    ps = [prob(), prob(mx=96, my=40, radius=5.0)]
    total = batched_ws(L, ps)[1]
    assert vjp_batched(L, []) == OK                               # an empty batch is a no-op
    assert vjp_batched(L, [prob()] * 65) == INVALID
    assert vjp_batched(L, ps, n_lambda=5) == INVALID
    assert vjp_batched(L, ps, field_type=ec.EPS_FIELD_BF16X2_SCALED) == UNSUPPORTED
    assert vjp_batched(L, ps, field_type=ec.EPS_FIELD_F16X2_SCALED) == UNSUPPORTED
    assert vjp_batched(L, ps, field_type=9) == INVALID
    assert vjp_batched(L, ps, scale=float("nan")) == INVALID
    assert vjp_batched(L, ps, C=False) == INVALID
    assert vjp_batched(L, ps, G=False) == INVALID
    assert vjp_batched(L, ps, EF=False) == INVALID
    assert vjp_batched(L, ps, ws=None, ws_bytes=total) == WORKSPACE
    assert vjp_batched(L, ps, ws=8, ws_bytes=total) == WORKSPACE            # not 256-byte aligned
    assert vjp_batched(L, ps, ws=4096, ws_bytes=total - 1) == WORKSPACE     # too small
    assert vjp_batched(L, [prob(flags=ec.EPS_FLAG_NORMALS_3D)]) == UNSUPPORTED


def test_batched_forward_checks_before_any_launch(L):
    assert L.eps_forward_batched(0, None, None, None, None) == OK
    assert L.eps_forward_batched(65, probs_array([prob()] * 65), ptrs(65), ptrs(65), None) == INVALID
    assert L.eps_forward_batched(1, None, ptrs(1), ptrs(1), None) == INVALID
    assert L.eps_forward_batched(1, probs_array([prob()]), None, None, None) == INVALID
    assert L.eps_forward_batched(1, probs_array([prob(flags=ec.EPS_FLAG_NORMALS_3D)]), ptrs(1),
                                 ptrs(1), None) == UNSUPPORTED


def tuning(**kw):
    t = ec.eps_tuning_t()
    base = dict(multi=0, stencil_blocks_per_sm=3, scatter_blocks_per_sm=3, contract_blocks_per_sm=3,
                stage_components=3, defer_seeds=0)
    base.update(kw)
    for k, v in base.items():
        setattr(t, k, v)
    return t


@pytest.mark.parametrize("kw,status", [
    ({}, OK), (dict(multi=1, defer_seeds=1, stage_components=1), OK),
    (dict(stencil_blocks_per_sm=16, scatter_blocks_per_sm=1, contract_blocks_per_sm=64), OK),
    (dict(multi=2), INVALID), (dict(stencil_blocks_per_sm=0), INVALID),
    (dict(stencil_blocks_per_sm=17), INVALID), (dict(scatter_blocks_per_sm=0), INVALID),
    (dict(scatter_blocks_per_sm=17), INVALID), (dict(contract_blocks_per_sm=0), INVALID),
    (dict(contract_blocks_per_sm=65), INVALID), (dict(stage_components=2), INVALID),
    (dict(defer_seeds=2), INVALID), (dict(scatter_bulk_staging=1), OK),
    (dict(scatter_bulk_staging=2), INVALID), (dict(scatter_bulk_staging=-1), INVALID),
    (dict(scatter_tile_cols=64), OK), (dict(scatter_tile_cols=32), OK),
    (dict(scatter_tile_cols=0), OK), (dict(scatter_tile_cols=48), INVALID),
    (dict(concurrent_groups=1), OK), (dict(concurrent_groups=2), INVALID),
])
def test_set_tuning_ranges(L, kw, status):
    ps = [prob(), prob(mx=80)]
    assert L.eps_batched_set_tuning(len(ps), probs_array(ps), 1, ctypes.byref(tuning(**kw))) == status


def test_set_tuning_rejects_bad_batches(L):
    t = ctypes.byref(tuning())
    assert L.eps_batched_set_tuning(1, probs_array([prob()]), -1, t) == OK     # forward calls
    assert L.eps_batched_set_tuning(1, probs_array([prob()]), -2, t) == INVALID
    assert L.eps_batched_set_tuning(1, probs_array([prob()]), 5, t) == INVALID
    assert L.eps_batched_set_tuning(65, probs_array([prob()] * 65), 1, t) == INVALID
    assert L.eps_batched_set_tuning(1, None, 1, t) == INVALID
    assert L.eps_batched_set_tuning(1, probs_array([prob()]), 1, None) == INVALID


@pytest.mark.parametrize("reps", [0, -3, 1001])
def test_autotune_rejects_reps_out_of_range(L, reps):
    ps = [prob()]
    st = L.eps_autotune_batched(1, probs_array(ps), ptrs(1), 1, 0, ptrs(1), ptrs(1), None, -2.0,
                                ptrs(1), None, None, 0, reps, None, None)
    assert st == INVALID


@pytest.mark.parametrize("nbytes", [-1, 129, 1 << 20])
def test_l2_fetch_granularity_range(L, nbytes):
    prev = ctypes.c_int32(0)
    assert L.eps_set_l2_fetch_granularity(nbytes, ctypes.byref(prev)) == INVALID


@pytest.mark.parametrize("nk", [1, 3, 4, 7, 11])
def test_packed_field_bytes_follow_the_documented_layout(L, nk):
    # 16 bytes of scales, then [3][nx][ny][NP] pairs of 16-bit values, with
    # NP = nk + 1 rounded up to a multiple of 4
    p = prob(nz=16, slab_nk=nk)
    npl = (nk + 1 + 3) // 4 * 4
    for ft in (ec.EPS_FIELD_BF16X2_SCALED, ec.EPS_FIELD_F16X2_SCALED):
        assert ec.eps_packed_field_bytes(p, ft) == 16 + 3 * p.nx * p.ny * npl * 4
    assert ec.eps_packed_field_bytes(prob(mx=0), ec.EPS_FIELD_BF16X2_SCALED) == 0
    n = ctypes.c_size_t(0)
    assert L.eps_packed_field_bytes(ctypes.byref(p.c_struct()), ec.EPS_FIELD_C64, ctypes.byref(n)) == INVALID
    assert L.eps_packed_field_bytes(ctypes.byref(p.c_struct()), ec.EPS_FIELD_BF16X2_SCALED, None) == INVALID


def test_field_pack_checks_before_any_launch(L):
    P = ctypes.byref(prob().c_struct())
    assert L.eps_field_pack(P, ec.EPS_FIELD_C64, 4096, 4096, 1 << 20, None) == INVALID
    assert L.eps_field_pack(P, ec.EPS_FIELD_BF16X2_SCALED, None, 4096, 1 << 20, None) == INVALID
    assert L.eps_field_pack(P, ec.EPS_FIELD_BF16X2_SCALED, 4100, 4096, 1 << 20, None) == INVALID
    assert L.eps_field_pack(P, ec.EPS_FIELD_BF16X2_SCALED, 4096, 4104, 1 << 20, None) == INVALID
    E = ctypes.byref(prob(mx=0).c_struct())
    assert L.eps_field_pack(E, ec.EPS_FIELD_BF16X2_SCALED, None, None, 0, None) == OK   # empty region
