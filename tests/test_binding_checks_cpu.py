"""Argument checks of the Python binding, without a GPU.

The library is replaced by a recorder and CPU tensors stand in for CUDA
ones (the binding's accepted device type is switched to "cpu" for these
tests only).  Valid calls, in the forms the GPU tests and the benchmark
use, must reach the library with the caller's pointers.  Each malformed
argument must raise before any compute entry point is called: a wrong
shape, dtype, layout or device, a short or mismatched list, a workspace
that is not a byte buffer, or a stream of another device.  Without the
switch, host tensors are refused outright."""

import ctypes

import pytest
import torch

from paper_2505_03352_gb300 import epschain as eb

QUERIES = {"eps_workspace_size", "eps_morph_workspace_size", "eps_coarse_workspace_size",
           "eps_batched_workspace_size", "eps_packed_field_bytes"}


class _Stream:
    def __init__(self, device):
        self.device = device
        self.cuda_stream = 0


@pytest.fixture
def rec(monkeypatch):
    calls = []

    class Recorder:
        def __getattr__(self, name):
            def entry(*args):
                calls.append((name, args))
                return eb.EPS_OK
            return entry

    monkeypatch.setattr(eb, "_lib", Recorder())
    monkeypatch.setattr(eb, "_DEVICE_TYPE", "cpu")
    monkeypatch.setattr(torch.cuda, "current_stream", lambda *a, **k: _Stream(torch.device("cpu")))
    return calls


def launches(calls):
    return [name for name, _ in calls if name not in QUERIES]


P = eb.Problem(mx=16, my=12, nz=10, radius=2.0, beta=8.0, slab_nk=4)
SHAPE = (3, P.nx, P.ny, P.nz)


def _C():
    return torch.rand((P.mx, P.my))


def _fields(n=1):
    return ([torch.zeros(SHAPE, dtype=torch.complex64) for _ in range(n)],
            [torch.zeros(SHAPE, dtype=torch.complex64) for _ in range(n)])


def _val(a):
    return a.value if isinstance(a, ctypes.c_void_p) else a


def test_host_tensors_are_refused_by_the_product_checks():
    assert eb._DEVICE_TYPE == "cuda"
    with pytest.raises(ValueError, match="CUDA tensor"):
        eb.eps_forward(P, _C())


def test_valid_calls_reach_the_library_with_the_callers_pointers(rec):
    C = _C()
    EF, EA = _fields(2)
    eps = eb.eps_forward(P, C)
    assert eps.shape == SHAPE
    ws = torch.empty(64, dtype=torch.uint8)
    g, e = eb.eps_vjp(P, C, EF, EA, eps_out=True, ws=ws, field_scales=[[1.0] * 3, [1.0] * 3] * 2)
    name, args = rec[-1]
    assert name == "eps_vjp"
    assert _val(args[1]) == C.data_ptr() and args[2] == 2
    assert [args[4][i] for i in range(2)] == [t.data_ptr() for t in EF]
    assert _val(args[8]) == g.data_ptr() and _val(args[9]) == e.data_ptr()
    assert _val(args[10]) == ws.data_ptr() and args[11] == 64
    eb.eps_vjp(P, C, [], [])                                   # zero wavelengths
    eb.eps_vjp_real(P, C, torch.zeros(SHAPE))
    od_prob = eb.Problem(mx=16, my=12, nz=10, radius=2.0, beta=8.0, slab_nk=4,
                         flags=eb.EPS_FLAG_OFFDIAG | eb.EPS_FLAG_NORMALS_3D)
    e, od = eb.eps_forward(od_prob, C)
    assert od.shape == (4,) + SHAPE[1:]
    packed = eb.eps_field_pack(P, eb.EPS_FIELD_BF16X2_SCALED, EF[0])
    eb.eps_vjp(P, C, [packed], [packed.clone()], field_type=eb.EPS_FIELD_BF16X2_SCALED)
    probs = [P, eb.Problem(mx=8, my=10, nz=10, radius=1.0, beta=4.0, slab_nk=4)]
    Cs = [_C(), torch.rand((8, 10))]
    eb.eps_forward_batched(probs, Cs)
    assert eb.eps_forward_batched([], []) == []              # empty batch: a no-op call
    assert rec[-1][0] == "eps_forward_batched" and rec[-1][1][0] == 0
    EFb = [EF, [torch.zeros((3, 4, 5, 10), dtype=torch.complex64)] * 2]
    bv = eb.BatchedVjp(probs, Cs, EFb, EFb)
    bv()
    bv(stream=_Stream(torch.device("cpu")))
    pv = eb.PreparedVjp(P, C, EF, EA, torch.empty((P.mx, P.my)), eps_out=torch.empty(SHAPE))
    pv()
    m = eb.Morph()
    eb.eps_forward_morph(P, m, C)
    eb.eps_vjp_morph(P, m, C, EF, EA, eps_out=True)
    eb.eps_vjp_real_morph(P, m, C, torch.zeros(SHAPE))
    eb.PreparedVjpMorph(P, m, C, EF, EA, torch.empty((P.mx, P.my)))()
    state = eb.eps_opt_init(eb.OptParams(), device="cpu")
    M, V = torch.zeros_like(C), torch.zeros_like(C)
    eb.eps_opt_step(P, eb.OptParams(), state, C, torch.zeros_like(C), M, V, ws)
    cg, c = eb.Coarse(5, 4), torch.rand((5, 4))
    eb.eps_forward_coarse(P, cg, c)
    eb.eps_vjp_coarse(P, cg, c, EF, EA, eps_out=True)
    eb.eps_vjp_real_coarse(P, cg, c, torch.zeros(SHAPE))
    assert launches(rec) == [
        "eps_forward", "eps_vjp", "eps_vjp", "eps_vjp_real", "eps_forward", "eps_field_pack",
        "eps_vjp", "eps_forward_batched", "eps_forward_batched", "eps_vjp_batched",
        "eps_vjp_batched", "eps_vjp",
        "eps_forward_morph", "eps_vjp_morph", "eps_vjp_real_morph", "eps_vjp_morph",
        "eps_opt_init", "eps_opt_step", "eps_forward_coarse", "eps_vjp_coarse",
        "eps_vjp_real_coarse"]


def _bad_cases():
    C = _C()
    EF, EA = _fields(1)
    G = torch.zeros(SHAPE)
    probs = [P, P]
    return {
        "C float64": lambda: eb.eps_forward(P, C.double()),
        "C not contiguous": lambda: eb.eps_forward(P, torch.rand((P.my, P.mx)).t()),
        "C wrong shape": lambda: eb.eps_forward(P, torch.rand((P.mx, P.my + 2))),
        "C not a tensor": lambda: eb.eps_forward(P, C.numpy()),
        "C on another device type": lambda: eb.eps_forward(P, torch.empty((P.mx, P.my), device="meta")),
        "eps wrong shape": lambda: eb.eps_forward(P, C, eps=torch.empty((3, P.nx, P.ny, P.nz + 1))),
        "offdiag two maps for 3-D normals": lambda: eb.eps_forward(
            eb.Problem(mx=16, my=12, nz=10, radius=2.0, beta=8.0, slab_nk=4,
                       flags=eb.EPS_FLAG_OFFDIAG | eb.EPS_FLAG_NORMALS_3D),
            C, offdiag=torch.empty((2,) + SHAPE[1:])),
        "EF and EA lengths differ": lambda: eb.eps_vjp(P, C, EF, []),
        "field float32": lambda: eb.eps_vjp(P, C, [G], [G]),
        "17 wavelengths": lambda: eb.eps_vjp(P, C, EF * 17, EA * 17),
        "field_scales short": lambda: eb.eps_vjp(P, C, EF, EA, field_scales=[1.0] * 5),
        "eps_out wrong shape": lambda: eb.eps_vjp(P, C, EF, EA, eps_out=torch.empty(SHAPE[:3])),
        "dJdC wrong dtype": lambda: eb.eps_vjp(P, C, EF, EA, dJdC=torch.empty((P.mx, P.my),
                                                                             dtype=torch.float64)),
        "ws float32": lambda: eb.eps_vjp(P, C, EF, EA, ws=torch.empty(64)),
        "ws not contiguous": lambda: eb.eps_vjp_real(P, C, G, ws=torch.empty(128, dtype=torch.uint8)[::2]),
        "G complex": lambda: eb.eps_vjp_real(P, C, EF[0]),
        "packed field not contiguous": lambda: eb.eps_vjp(
            P, C, [torch.empty(64, dtype=torch.uint8)[::2]], [torch.empty(32, dtype=torch.uint8)],
            field_type=eb.EPS_FIELD_BF16X2_SCALED),
        "pack out float32": lambda: eb.eps_field_pack(P, eb.EPS_FIELD_BF16X2_SCALED, EF[0],
                                                      out=torch.empty(64)),
        "empty prepared batch": lambda: eb.BatchedVjp([], [], [], []),
        "batch controls without regions": lambda: eb.eps_forward_batched([], [C]),
        "batch controls short": lambda: eb.eps_forward_batched(probs, [C]),
        "batch eps short": lambda: eb.eps_forward_batched(probs, [C, C], eps=[torch.empty(SHAPE)]),
        "batch fields short": lambda: eb.BatchedVjp(probs, [C, C], [EF], [EA]),
        "batch region lacks a wavelength": lambda: eb.BatchedVjp(probs, [C, C], [EF * 2, EF],
                                                                 [EA * 2, EA]),
        "batch controls differ in dtype": lambda: eb.BatchedVjp(probs, [C, C.double()], [EF, EF],
                                                                [EA, EA]),
        "prepared field wrong shape": lambda: eb.PreparedVjp(
            P, C, [torch.zeros(SHAPE[:3] + (P.nz + 1,), dtype=torch.complex64)], EA,
            torch.empty((P.mx, P.my))),
        "prepared field_scales long": lambda: eb.PreparedVjp(P, C, EF, EA, torch.empty((P.mx, P.my)),
                                                             field_scales=[1.0] * 12),
        "prepared morph dJdC missing": lambda: eb.PreparedVjpMorph(P, eb.Morph(), C, EF, EA, None),
        "opt state short": lambda: eb.eps_opt_step(P, eb.OptParams(), torch.zeros(16, dtype=torch.uint8),
                                                   C, C, C.clone(), C.clone(),
                                                   torch.empty(8, dtype=torch.uint8)),
        "opt ws float32": lambda: eb.eps_opt_step(P, eb.OptParams(), torch.zeros(32, dtype=torch.uint8),
                                                  C, C, C.clone(), C.clone(), torch.empty(8)),
        "coarse nodes wrong shape": lambda: eb.eps_forward_coarse(P, eb.Coarse(5, 4), torch.rand((4, 5))),
        "stream of another device": lambda: eb.eps_forward(P, C, stream=_Stream(torch.device("cuda", 1))),
    }


@pytest.mark.parametrize("case", sorted(_bad_cases()))
def test_malformed_arguments_raise_before_any_launch(rec, case):
    with pytest.raises((ValueError, TypeError)):
        _bad_cases()[case]()
    assert launches(rec) == []


def test_prepared_call_refuses_a_stream_of_another_device(rec):
    C = _C()
    EF, EA = _fields(1)
    pv = eb.PreparedVjp(P, C, EF, EA, torch.empty((P.mx, P.my)))
    with pytest.raises(ValueError, match="stream"):
        pv(stream=_Stream(torch.device("cuda", 1)))
    assert launches(rec) == []


def test_tensors_on_another_device_than_the_calls_are_refused(monkeypatch):
    # the device-index comparison itself (a CPU tensor against cuda:1)
    monkeypatch.setattr(eb, "_DEVICE_TYPE", "cpu")
    with pytest.raises(ValueError, match="call's tensors are on cuda:1"):
        eb._need(torch.empty(3), (3,), torch.float32, "x", torch.device("cuda", 1))


def test_packed_field_buffers_must_hold_the_packed_size(rec, monkeypatch):
    monkeypatch.setattr(eb, "eps_packed_field_bytes", lambda prob, ft: 100)
    C = _C()
    ok = torch.empty(100, dtype=torch.uint8)
    eb.eps_vjp(P, C, [ok], [ok.clone()], field_type=eb.EPS_FIELD_F16X2_SCALED)
    with pytest.raises(ValueError, match="100 are needed"):
        eb.eps_vjp(P, C, [ok], [ok[:99]], field_type=eb.EPS_FIELD_F16X2_SCALED)
    assert launches(rec) == ["eps_vjp"]


def test_surrogate_call_reaches_the_library_and_checks_its_value_buffer(rec):
    # eps_vjp_surrogate: the S buffer is a float64 0-d tensor on the call's
    # device (allocated if not given); a wrong dtype or shape raises first
    C = _C()
    EF, EA = _fields(2)
    g, e, S = eb.eps_vjp_surrogate(P, C, EF, EA, eps_out=True)
    name, args = rec[-1]
    assert name == "eps_vjp_surrogate"
    assert S.dtype == torch.float64 and S.shape == ()
    assert _val(args[1]) == C.data_ptr() and _val(args[10]) == S.data_ptr()
    assert _val(args[8]) == g.data_ptr() and _val(args[9]) == e.data_ptr()
    g, S2 = eb.eps_vjp_surrogate(P, C, EF, EA)
    assert _val(rec[-1][1][9]) is None
    n = len(launches(rec))
    for bad in (torch.zeros((), dtype=torch.float32), torch.zeros(1, dtype=torch.float64)):
        with pytest.raises(ValueError):
            eb.eps_vjp_surrogate(P, C, EF, EA, S=bad)
    with pytest.raises(ValueError):
        eb.eps_vjp_surrogate(P, C, EF, EA[:1])
    assert len(launches(rec)) == n


def test_prepared_surrogate_marshals_the_fields_once(rec):
    # autograd.AdjointSurrogate: the field pointer arrays and the workspace
    # are built at construction; each call passes C's pointer and fresh
    # outputs, and a C of the wrong shape raises before any launch
    from paper_2505_03352_gb300 import autograd as ag
    EF, EA = _fields(3)
    surr = ag.AdjointSurrogate(P, EF, EA, with_eps=True)
    C = _C()
    dJdC, eps, S = surr.call(C)
    name, args = rec[-1]
    assert name == "eps_vjp_surrogate" and args[2] == 3
    assert [args[4][l] for l in range(3)] == [t.data_ptr() for t in EF]
    assert [args[5][l] for l in range(3)] == [t.data_ptr() for t in EA]
    assert _val(args[1]) == C.data_ptr() and _val(args[9]) == eps.data_ptr()
    ws_ptr = _val(args[11])
    surr.call(C)
    assert _val(rec[-1][1][11]) == ws_ptr          # the same workspace every call
    n = len(launches(rec))
    with pytest.raises(ValueError):
        surr.call(torch.rand((P.mx + 2, P.my)))
    assert len(launches(rec)) == n
