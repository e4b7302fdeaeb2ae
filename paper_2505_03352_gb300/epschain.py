"""Python binding of the epschain C ABI (include/epschain.h).

Argument marshalling only: every step of the chain runs in the CUDA kernels
of libepschain.so.  PyTorch supplies device memory and streams.  The
functions carry the names of the C entry points; they raise EpsError on any
status other than EPS_OK.  There is no CPU fallback: without the built
library every call raises.
"""

from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libepschain.so")

EPS_OK = 0
STATUS_NAMES = {
    0: "EPS_OK", 1: "EPS_ERR_INVALID_ARG", 2: "EPS_ERR_SHAPE", 3: "EPS_ERR_WORKSPACE",
    4: "EPS_ERR_UNSUPPORTED", 5: "EPS_ERR_CUDA", 6: "EPS_ERR_DEVICE_TIMEOUT",
    7: "EPS_ERR_DEVICE_BOUNDS",
}
EPS_BC_CLAMP, EPS_BC_PERIODIC = 0, 1
EPS_FIELD_C64, EPS_FIELD_BF16X2_SCALED, EPS_FIELD_F16X2_SCALED = 0, 1, 2
EPS_FLAG_OFFDIAG = 1
EPS_FLAG_NORMALS_3D = 2
EPS_MAX_LAMBDA = 16


class EpsError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        super().__init__(f"{where}: {STATUS_NAMES.get(status, status)}")


class eps_problem_t(ctypes.Structure):
    _fields_ = [
        ("mx", ctypes.c_int32), ("my", ctypes.c_int32), ("sub", ctypes.c_int32),
        ("nz", ctypes.c_int32), ("slab_k0", ctypes.c_int32), ("slab_nk", ctypes.c_int32),
        ("radius", ctypes.c_float), ("beta", ctypes.c_float), ("eta", ctypes.c_float),
        ("eps_core", ctypes.c_float), ("eps_clad", ctypes.c_float),
        ("bc", ctypes.c_int32), ("flags", ctypes.c_int32),
    ]


class eps_profile_entry_t(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 48), ("launches", ctypes.c_int32),
                ("total_ms", ctypes.c_double)]


@dataclass(frozen=True)
class Problem:
    """Mirror of eps_problem_t (see include/epschain.h for the meaning)."""

    mx: int
    my: int
    nz: int
    radius: float
    beta: float
    eta: float = 0.5
    eps_core: float = 12.11
    eps_clad: float = 2.085
    slab_nk: int = 11
    slab_k0: int = -1
    bc: int = EPS_BC_CLAMP
    flags: int = 0
    sub: int = 2

    @property
    def nx(self):
        return self.mx // self.sub

    @property
    def ny(self):
        return self.my // self.sub

    @property
    def k0(self):
        return self.slab_k0 if self.slab_k0 >= 0 else (self.nz - self.slab_nk - 1) // 2

    def c_struct(self) -> eps_problem_t:
        return eps_problem_t(self.mx, self.my, self.sub, self.nz, self.slab_k0, self.slab_nk,
                             self.radius, self.beta, self.eta, self.eps_core, self.eps_clad,
                             self.bc, self.flags)


_lib = None

_VP = ctypes.c_void_p
_PROTOS = {
    "eps_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "eps_workspace_size": (ctypes.c_int, [ctypes.POINTER(eps_problem_t), ctypes.c_int32,
                                          ctypes.POINTER(ctypes.c_size_t)]),
    "eps_forward": (ctypes.c_int, [ctypes.POINTER(eps_problem_t), _VP, _VP, _VP, _VP]),
    "eps_vjp": (ctypes.c_int, [ctypes.POINTER(eps_problem_t), _VP, ctypes.c_int32, ctypes.c_int32,
                               _VP, _VP, _VP, ctypes.c_float, _VP, _VP, _VP, ctypes.c_size_t, _VP]),
    "eps_vjp_surrogate": (ctypes.c_int, [ctypes.POINTER(eps_problem_t), _VP, ctypes.c_int32,
                                         ctypes.c_int32, _VP, _VP, _VP, ctypes.c_float, _VP, _VP,
                                         _VP, _VP, ctypes.c_size_t, _VP]),
    "eps_vjp_real": (ctypes.c_int, [ctypes.POINTER(eps_problem_t), _VP, _VP, _VP, _VP,
                                    ctypes.c_size_t, _VP]),
    "eps_sync_status": (ctypes.c_int, [_VP]),
    "eps_batched_workspace_size": (ctypes.c_int, [ctypes.c_int32, ctypes.POINTER(eps_problem_t),
                                                  ctypes.c_int32, ctypes.POINTER(ctypes.c_size_t)]),
    "eps_forward_batched": (ctypes.c_int, [ctypes.c_int32, ctypes.POINTER(eps_problem_t), _VP, _VP,
                                           _VP]),
    "eps_vjp_batched": (ctypes.c_int, [ctypes.c_int32, ctypes.POINTER(eps_problem_t), _VP,
                                       ctypes.c_int32, ctypes.c_int32, _VP, _VP, _VP, ctypes.c_float,
                                       _VP, _VP, _VP, ctypes.c_size_t, _VP]),
    "eps_packed_field_bytes": (ctypes.c_int, [ctypes.POINTER(eps_problem_t), ctypes.c_int32,
                                              ctypes.POINTER(ctypes.c_size_t)]),
    "eps_field_pack": (ctypes.c_int, [ctypes.POINTER(eps_problem_t), ctypes.c_int32, _VP, _VP,
                                      ctypes.c_size_t, _VP]),
    "eps_profile_start": (ctypes.c_int, []),
    "eps_launch_count": (ctypes.c_int, [ctypes.POINTER(ctypes.c_uint64)]),
    "eps_set_l2_fetch_granularity": (ctypes.c_int, [ctypes.c_int32, ctypes.POINTER(ctypes.c_int32)]),
    "eps_selftest_timeout": (ctypes.c_int, [ctypes.c_int64, ctypes.c_void_p]),
    "eps_selftest_bounds": (ctypes.c_int, [ctypes.c_void_p]),
    "eps_profile_stop": (ctypes.c_int, [ctypes.POINTER(eps_profile_entry_t), ctypes.c_int32,
                                        ctypes.POINTER(ctypes.c_int32)]),
    "eps_morph_workspace_size": (ctypes.c_int, [ctypes.POINTER(eps_problem_t), _VP, ctypes.c_int32,
                                                ctypes.POINTER(ctypes.c_size_t)]),
    "eps_forward_morph": (ctypes.c_int, [ctypes.POINTER(eps_problem_t), _VP, _VP, _VP, _VP, _VP,
                                         ctypes.c_size_t, _VP]),
    "eps_vjp_morph": (ctypes.c_int, [ctypes.POINTER(eps_problem_t), _VP, _VP, ctypes.c_int32,
                                     ctypes.c_int32, _VP, _VP, _VP, ctypes.c_float, _VP, _VP, _VP,
                                     ctypes.c_size_t, _VP]),
    "eps_vjp_real_morph": (ctypes.c_int, [ctypes.POINTER(eps_problem_t), _VP, _VP, _VP, _VP, _VP,
                                          ctypes.c_size_t, _VP]),
    "eps_opt_init": (ctypes.c_int, [_VP, _VP, _VP]),
    "eps_batched_set_tuning": (ctypes.c_int, [ctypes.c_int32, ctypes.POINTER(eps_problem_t),
                                              ctypes.c_int32, _VP]),
    "eps_autotune_batched": (ctypes.c_int, [ctypes.c_int32, ctypes.POINTER(eps_problem_t), _VP,
                                            ctypes.c_int32, ctypes.c_int32, _VP, _VP, _VP,
                                            ctypes.c_float, _VP, _VP, _VP, ctypes.c_size_t,
                                            ctypes.c_int32, _VP, _VP]),
    "eps_coarse_workspace_size": (ctypes.c_int, [ctypes.POINTER(eps_problem_t), _VP, ctypes.c_int32,
                                                 ctypes.POINTER(ctypes.c_size_t)]),
    "eps_forward_coarse": (ctypes.c_int, [ctypes.POINTER(eps_problem_t), _VP, _VP, _VP, _VP, _VP,
                                          ctypes.c_size_t, _VP]),
    "eps_vjp_coarse": (ctypes.c_int, [ctypes.POINTER(eps_problem_t), _VP, _VP, ctypes.c_int32,
                                      ctypes.c_int32, _VP, _VP, _VP, ctypes.c_float, _VP, _VP, _VP,
                                      ctypes.c_size_t, _VP]),
    "eps_vjp_real_coarse": (ctypes.c_int, [ctypes.POINTER(eps_problem_t), _VP, _VP, _VP, _VP, _VP,
                                           ctypes.c_size_t, _VP]),
    "eps_opt_step": (ctypes.c_int, [ctypes.POINTER(eps_problem_t), _VP, _VP, _VP, _VP, _VP, _VP,
                                    _VP, _VP, ctypes.c_size_t, _VP]),
}


def lib():
    """The loaded libepschain.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                               "`python -m paper_2505_03352_gb300.build_lib`")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _PROTOS.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _check(status: int, where: str):
    if status != EPS_OK:
        raise EpsError(status, where)


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


# Device type every tensor argument must have.  The CPU tests of these
# argument checks set it to "cpu" and replace the library with a recorder;
# no call ever computes on the host.
_DEVICE_TYPE = "cuda"


def _stream(stream, device=None):
    """The cudaStream_t handle of `stream` (default: the current stream).
    With `device`, the stream must belong to it and it must be the current
    device: the library launches on the current device only."""
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    if device is not None:
        if stream.device != device:
            raise ValueError(f"the stream is on {stream.device} but the tensors are on {device}; "
                             "select their device with torch.cuda.set_device")
        if device.type == "cuda" and torch.cuda.current_device() != device.index:
            raise ValueError(f"the tensors are on {device}, which is not the current device; "
                             "select it with torch.cuda.set_device")
    return ctypes.c_void_p(stream.cuda_stream)


def _need(t, shape, dtype, name, device=None):
    """t is a contiguous tensor of `shape` and `dtype` on the call's device."""
    import torch
    if not isinstance(t, torch.Tensor):
        raise TypeError(f"{name} must be a torch.Tensor")
    if t.device.type != _DEVICE_TYPE:
        raise ValueError(f"{name} must be a CUDA tensor")
    if device is not None and t.device != device:
        raise ValueError(f"{name} is on {t.device} but the call's tensors are on {device}")
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} has shape {tuple(t.shape)}, expected {tuple(shape)}")
    if t.dtype != dtype:
        raise ValueError(f"{name} has dtype {t.dtype}, expected {dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")


def _need_bytes(t, nbytes, name, device):
    """t is a contiguous uint8 buffer of at least `nbytes` bytes on `device`
    (a workspace, a packed field or the optimiser state)."""
    import torch
    _need(t, None, torch.uint8, name, device)
    if t.numel() < nbytes:
        raise ValueError(f"{name} holds {t.numel()} bytes, {nbytes} are needed")


def _field_ptrs(prob, EF, EA, field_type, device):
    """Check the per-wavelength field lists and return (n_lambda, EF
    pointer array, EA pointer array)."""
    import torch
    if len(EF) != len(EA):
        raise ValueError("EF and EA must have the same number of wavelengths")
    nl = len(EF)
    if nl > EPS_MAX_LAMBDA:
        raise ValueError(f"at most {EPS_MAX_LAMBDA} wavelengths per call")
    if field_type == EPS_FIELD_C64:
        for l in range(nl):
            _need(EF[l], (3, prob.nx, prob.ny, prob.nz), torch.complex64, f"EF[{l}]", device)
            _need(EA[l], (3, prob.nx, prob.ny, prob.nz), torch.complex64, f"EA[{l}]", device)
    else:
        nbytes = eps_packed_field_bytes(prob, field_type)
        for l in range(nl):
            _need_bytes(EF[l], nbytes, f"EF[{l}] (packed field)", device)
            _need_bytes(EA[l], nbytes, f"EA[{l}] (packed field)", device)
    ef = (ctypes.c_void_p * max(nl, 1))(*[t.data_ptr() for t in EF])
    ea = (ctypes.c_void_p * max(nl, 1))(*[t.data_ptr() for t in EA])
    return nl, ef, ea


def _scales(field_scales, nl):
    """The per-wavelength field scales as a float array, or None."""
    if field_scales is None:
        return None
    flat = [float(v) for v in _flatten(field_scales)]
    if len(flat) != 6 * nl:
        raise ValueError("field_scales must hold n_lambda x 2 x 3 values")
    return (ctypes.c_float * len(flat))(*flat)


def _eps_out(prob, eps_out, device):
    """(wanted, tensor or None) for an eps_out argument: a tensor, True to
    allocate one, or None / False for none."""
    import torch
    if eps_out is None or eps_out is False:
        return False, None
    shape = (3, prob.nx, prob.ny, prob.nz)
    if eps_out is True:
        eps_out = torch.empty(shape, dtype=torch.float32, device=device)
    _need(eps_out, shape, torch.float32, "eps_out", device)
    return True, eps_out


def eps_status_string(status: int) -> str:
    return lib().eps_status_string(status).decode()


def eps_workspace_size(prob: Problem, n_lambda: int = 1) -> int:
    n = ctypes.c_size_t(0)
    p = prob.c_struct()
    _check(lib().eps_workspace_size(ctypes.byref(p), n_lambda, ctypes.byref(n)),
           "eps_workspace_size")
    return n.value


def eps_forward(prob: Problem, C, eps=None, offdiag=None, stream=None):
    """eps_hat [3, nx, ny, nz] float32 (and the off-diagonal term when
    prob.flags has EPS_FLAG_OFFDIAG).  Returns eps, or (eps, offdiag)."""
    import torch
    _need(C, (prob.mx, prob.my), torch.float32, "C")
    dev = C.device
    shape = (3, prob.nx, prob.ny, prob.nz)
    if eps is None:
        eps = torch.empty(shape, dtype=torch.float32, device=dev)
    _need(eps, shape, torch.float32, "eps", dev)
    want_od = bool(prob.flags & EPS_FLAG_OFFDIAG)
    if want_od:
        od_shape = (4 if prob.flags & EPS_FLAG_NORMALS_3D else 2,) + shape[1:]
        if offdiag is None:
            offdiag = torch.empty(od_shape, dtype=torch.float32, device=dev)
        _need(offdiag, od_shape, torch.float32, "offdiag", dev)
    p = prob.c_struct()
    _check(lib().eps_forward(ctypes.byref(p), _ptr(C), _ptr(eps), _ptr(offdiag) if want_od else None,
                             _stream(stream, dev)), "eps_forward")
    return (eps, offdiag) if want_od else eps


def _workspace(prob, n_lambda, ws, device):
    import torch
    need = eps_workspace_size(prob, n_lambda)
    if ws is None:
        ws = torch.empty(max(need, 1), dtype=torch.uint8, device=device)
    _need_bytes(ws, 0, "ws", device)      # its size and alignment are checked by the library
    return ws


def eps_vjp(prob: Problem, C, EF, EA, scale: float = -2.0, dJdC=None, eps_out=None,
            field_type: int = EPS_FIELD_C64, field_scales=None, ws=None, stream=None):
    """Eq. 1 adjoint gradient dJ/dC [mx, my] from lists of forward / adjoint
    field tensors (complex64 [3, nx, ny, nz] for EPS_FIELD_C64, packed uint8
    buffers from eps_field_pack otherwise).  With eps_out (a tensor, or True
    to allocate one) the forward eps_hat is written by the same pass.
    Returns dJdC, or (dJdC, eps_out)."""
    import torch
    _need(C, (prob.mx, prob.my), torch.float32, "C")
    dev = C.device
    nl, ef, ea = _field_ptrs(prob, EF, EA, field_type, dev)
    fs = _scales(field_scales, nl)
    if dJdC is None:
        dJdC = torch.empty((prob.mx, prob.my), dtype=torch.float32, device=dev)
    _need(dJdC, (prob.mx, prob.my), torch.float32, "dJdC", dev)
    ret_eps, eps_out = _eps_out(prob, eps_out, dev)
    ws = _workspace(prob, nl, ws, dev)
    p = prob.c_struct()
    _check(lib().eps_vjp(ctypes.byref(p), _ptr(C), nl, field_type, ef, ea, fs, float(scale),
                         _ptr(dJdC), _ptr(eps_out), _ptr(ws), ws.numel(), _stream(stream, dev)),
           "eps_vjp")
    return (dJdC, eps_out) if ret_eps else dJdC


def eps_vjp_surrogate(prob: Problem, C, EF, EA, scale: float = -2.0, dJdC=None, eps_out=None,
                      S=None, field_type: int = EPS_FIELD_C64, field_scales=None, ws=None,
                      stream=None):
    """eps_vjp plus the Eq. 1 surrogate S = sum over the J-support voxels of
    eps_hat * scale Re(sum_l E_F,l E_A,l), whose gradient is dJ/dC.  S is a
    float64 0-d device tensor (allocated if not given).  Returns
    (dJdC, S) or, with eps_out, (dJdC, eps_out, S)."""
    import torch
    _need(C, (prob.mx, prob.my), torch.float32, "C")
    dev = C.device
    nl, ef, ea = _field_ptrs(prob, EF, EA, field_type, dev)
    fs = _scales(field_scales, nl)
    if dJdC is None:
        dJdC = torch.empty((prob.mx, prob.my), dtype=torch.float32, device=dev)
    _need(dJdC, (prob.mx, prob.my), torch.float32, "dJdC", dev)
    if S is None:
        S = torch.empty((), dtype=torch.float64, device=dev)
    _need(S, (), torch.float64, "S", dev)
    ret_eps, eps_out = _eps_out(prob, eps_out, dev)
    ws = _workspace(prob, nl, ws, dev)
    p = prob.c_struct()
    _check(lib().eps_vjp_surrogate(ctypes.byref(p), _ptr(C), nl, field_type, ef, ea, fs,
                                   float(scale), _ptr(dJdC), _ptr(eps_out), _ptr(S), _ptr(ws),
                                   ws.numel(), _stream(stream, dev)),
           "eps_vjp_surrogate")
    return (dJdC, eps_out, S) if ret_eps else (dJdC, S)


def _flatten(x):
    if hasattr(x, "tolist"):
        x = x.tolist()
    if isinstance(x, (list, tuple)):
        out = []
        for v in x:
            out.extend(_flatten(v))
        return out
    return [x]


def eps_vjp_real(prob: Problem, C, G, dJdC=None, ws=None, stream=None):
    """(d eps_hat / dC)^T G for a real float32 cotangent G [3, nx, ny, nz]."""
    import torch
    _need(C, (prob.mx, prob.my), torch.float32, "C")
    dev = C.device
    _need(G, (3, prob.nx, prob.ny, prob.nz), torch.float32, "G", dev)
    if dJdC is None:
        dJdC = torch.empty((prob.mx, prob.my), dtype=torch.float32, device=dev)
    _need(dJdC, (prob.mx, prob.my), torch.float32, "dJdC", dev)
    ws = _workspace(prob, 1, ws, dev)
    p = prob.c_struct()
    _check(lib().eps_vjp_real(ctypes.byref(p), _ptr(C), _ptr(G), _ptr(dJdC), _ptr(ws), ws.numel(),
                              _stream(stream, dev)), "eps_vjp_real")
    return dJdC


def eps_packed_field_bytes(prob: Problem, field_type: int) -> int:
    n = ctypes.c_size_t(0)
    p = prob.c_struct()
    _check(lib().eps_packed_field_bytes(ctypes.byref(p), field_type, ctypes.byref(n)),
           "eps_packed_field_bytes")
    return n.value


def eps_field_pack(prob: Problem, field_type: int, E, out=None, stream=None):
    """Pack one complex64 field [3, nx, ny, nz] into the reduced-precision
    buffer format eps_vjp accepts for EPS_FIELD_BF16X2_SCALED /
    EPS_FIELD_F16X2_SCALED (uint8 device tensor; see include/epschain.h)."""
    import torch
    _need(E, (3, prob.nx, prob.ny, prob.nz), torch.complex64, "E")
    dev = E.device
    nbytes = eps_packed_field_bytes(prob, field_type)
    if out is None:
        out = torch.empty(max(nbytes, 16), dtype=torch.uint8, device=dev)
    _need_bytes(out, nbytes, "out", dev)
    p = prob.c_struct()
    _check(lib().eps_field_pack(ctypes.byref(p), field_type, _ptr(E), _ptr(out), out.numel(),
                                _stream(stream, dev)), "eps_field_pack")
    return out


def _probs(probs):
    arr = (eps_problem_t * max(len(probs), 1))()
    for k, p in enumerate(probs):
        arr[k] = p.c_struct()
    return arr


def _ptrs(ts):
    return (ctypes.c_void_p * max(len(ts), 1))(*[None if t is None else t.data_ptr() for t in ts])


def eps_batched_workspace_size(probs, n_lambda: int = 1) -> int:
    n = ctypes.c_size_t(0)
    _check(lib().eps_batched_workspace_size(len(probs), _probs(probs), n_lambda, ctypes.byref(n)),
           "eps_batched_workspace_size")
    return n.value


def _batch_device(probs, Cs):
    """The device of a batch's controls, after checking that every region
    has its controls there."""
    import torch
    if len(probs) == 0:
        raise ValueError("a batch needs at least one region")
    if len(Cs) != len(probs):
        raise ValueError(f"{len(Cs)} control arrays for {len(probs)} regions")
    _need(Cs[0], (probs[0].mx, probs[0].my), torch.float32, "C[0]")
    dev = Cs[0].device
    for k, p in enumerate(probs):
        _need(Cs[k], (p.mx, p.my), torch.float32, f"C[{k}]", dev)
    return dev


def eps_forward_batched(probs, Cs, eps=None, stream=None):
    """eps_hat of every region in one call; returns the list of eps tensors
    (an empty batch is a no-op, as in the C call)."""
    import torch
    if len(probs) == 0 and len(Cs) == 0 and not eps:
        _check(lib().eps_forward_batched(0, _probs(probs), _ptrs([]), _ptrs([]), _stream(stream)),
               "eps_forward_batched")
        return []
    dev = _batch_device(probs, Cs)
    if eps is None:
        eps = [torch.empty((3, p.nx, p.ny, p.nz), dtype=torch.float32, device=dev) for p in probs]
    if len(eps) != len(probs):
        raise ValueError(f"{len(eps)} eps outputs for {len(probs)} regions")
    for k, (p, e) in enumerate(zip(probs, eps)):
        _need(e, (3, p.nx, p.ny, p.nz), torch.float32, f"eps[{k}]", dev)
    _check(lib().eps_forward_batched(len(probs), _probs(probs), _ptrs(Cs), _ptrs(eps),
                                     _stream(stream, dev)), "eps_forward_batched")
    return eps


class BatchedVjp:
    """eps_vjp_batched over a fixed set of regions with its arguments built
    once (and its workspace and outputs allocated once), so that the call can
    be repeated or captured in a CUDA graph.  EF[k] / EA[k] are lists of
    complex64 fields of region k (one per wavelength, the same number for
    every region)."""

    def __init__(self, probs, Cs, EF, EA, scale=-2.0, with_eps=True, ws=None):
        import torch
        dev = _batch_device(probs, Cs)
        n = len(probs)
        if len(EF) != n or len(EA) != n:
            raise ValueError(f"EF and EA must list the fields of each of the {n} regions")
        nl = len(EF[0])
        for k, p in enumerate(probs):
            if len(EF[k]) != nl or len(EA[k]) != nl:
                raise ValueError(f"region {k} does not have {nl} forward and adjoint fields")
            for l in range(nl):
                _need(EF[k][l], (3, p.nx, p.ny, p.nz), torch.complex64, f"EF[{k}][{l}]", dev)
                _need(EA[k][l], (3, p.nx, p.ny, p.nz), torch.complex64, f"EA[{k}][{l}]", dev)
        self._dev = dev
        self.dJdC = [torch.empty((p.mx, p.my), dtype=torch.float32, device=dev) for p in probs]
        self.eps = ([torch.empty((3, p.nx, p.ny, p.nz), dtype=torch.float32, device=dev)
                     for p in probs] if with_eps else None)
        need = eps_batched_workspace_size(probs, nl)
        self.ws = ws if ws is not None else torch.empty(max(need, 1), dtype=torch.uint8, device=dev)
        _need_bytes(self.ws, 0, "ws", dev)      # its size and alignment are checked by the library
        _stream(None, dev)                      # the batch's device is the current one
        self._keep = (Cs, EF, EA)
        self._p = _probs(probs)
        self._C = _ptrs(Cs)
        self._EF = _ptrs([t for k in range(n) for t in EF[k]])
        self._EA = _ptrs([t for k in range(n) for t in EA[k]])
        self._G = _ptrs(self.dJdC)
        self._E = _ptrs(self.eps) if with_eps else None
        self._args = (n, self._p, self._C, nl, EPS_FIELD_C64, self._EF, self._EA, None,
                      float(scale), self._G, self._E, _ptr(self.ws), self.ws.numel())
        self._fn = lib().eps_vjp_batched

    def __call__(self, stream=None):
        if stream is not None and stream.device != self._dev:
            raise ValueError(f"the stream is on {stream.device} but the batch is on {self._dev}")
        _check(self._fn(*self._args, _stream(stream)), "eps_vjp_batched")
        return self.dJdC, self.eps

    def set_tuning(self, **shapes):
        """Store launch shapes for this batch (eps_batched_set_tuning); keys are
        the eps_tuning_t fields multi, stencil_blocks_per_sm,
        scatter_blocks_per_sm, contract_blocks_per_sm, stage_components,
        defer_seeds, scatter_bulk_staging, scatter_tile_cols and
        concurrent_groups (defaults: the library's default shapes)."""
        r = eps_tuning_t()
        base = dict(multi=0, stencil_blocks_per_sm=3, scatter_blocks_per_sm=3,
                    contract_blocks_per_sm=3, stage_components=1, defer_seeds=0,
                    scatter_bulk_staging=1, scatter_tile_cols=32, concurrent_groups=0)
        base.update(shapes)
        for k, v in base.items():
            setattr(r, k, int(v))
        n, probs, nl = self._args[0], self._args[1], self._args[3]
        _check(lib().eps_batched_set_tuning(n, probs, nl, ctypes.byref(r)), "eps_batched_set_tuning")

    def autotune(self, reps: int = 5, stream=None) -> dict:
        """eps_autotune_batched on this batch: times candidate launch shapes,
        caches the fastest for later calls (and graph captures) of this batch
        and returns the choice.  Synchronises; call it before capturing."""
        r = eps_tuning_t()
        _check(lib().eps_autotune_batched(*self._args, int(reps), ctypes.byref(r),
                                          _stream(stream, self._dev)), "eps_autotune_batched")
        return {f: getattr(r, f) for f, _ in eps_tuning_t._fields_}


class eps_tuning_t(ctypes.Structure):
    _fields_ = [("multi", ctypes.c_int32), ("stencil_blocks_per_sm", ctypes.c_int32),
                ("scatter_blocks_per_sm", ctypes.c_int32), ("contract_blocks_per_sm", ctypes.c_int32),
                ("stage_components", ctypes.c_int32), ("defer_seeds", ctypes.c_int32),
                ("evaluations", ctypes.c_int32),
                ("default_ms", ctypes.c_float), ("tuned_ms", ctypes.c_float),
                ("scatter_bulk_staging", ctypes.c_int32), ("scatter_tile_cols", ctypes.c_int32),
                ("concurrent_groups", ctypes.c_int32)]


def eps_sync_status(stream=None):
    _check(lib().eps_sync_status(_stream(stream)), "eps_sync_status")


def eps_selftest_timeout(cycles: int, stream=None):
    """Launch the device-side timeout self-test (a bounded wait on a barrier
    nothing arrives at, `cycles` SM clock cycles long); the next
    eps_sync_status reports EPS_ERR_DEVICE_TIMEOUT."""
    _check(lib().eps_selftest_timeout(int(cycles), _stream(stream)), "eps_selftest_timeout")


def eps_selftest_bounds(stream=None):
    """Launch the debug-bounds self-test (a failing bounds check, no memory
    access); raises EpsError(EPS_ERR_UNSUPPORTED) on a release build."""
    _check(lib().eps_selftest_bounds(_stream(stream)), "eps_selftest_bounds")


def eps_set_l2_fetch_granularity(nbytes: int) -> int:
    """Set the current context's L2 fetch granularity hint; returns the
    previous value."""
    prev = ctypes.c_int32(0)
    _check(lib().eps_set_l2_fetch_granularity(int(nbytes), ctypes.byref(prev)),
           "eps_set_l2_fetch_granularity")
    return prev.value


def eps_profile_start():
    _check(lib().eps_profile_start(), "eps_profile_start")


def eps_launch_count() -> int:
    """Kernel launches the library has made in this process (host counter;
    the difference of two readings counts the calls in between)."""
    n = ctypes.c_uint64(0)
    _check(lib().eps_launch_count(ctypes.byref(n)), "eps_launch_count")
    return n.value


def eps_profile_stop(max_entries: int = 32):
    """{kernel name: (launches, total_ms)} for launches since eps_profile_start."""
    arr = (eps_profile_entry_t * max_entries)()
    n = ctypes.c_int32(0)
    _check(lib().eps_profile_stop(arr, max_entries, ctypes.byref(n)), "eps_profile_stop")
    return {arr[i].name.decode(): (arr[i].launches, arr[i].total_ms) for i in range(n.value)}


class PreparedVjp:
    """A fused forward + VJP call (eps_vjp) with its ctypes arguments built
    once, for launch loops where per-call marshalling would dominate.  The
    arguments are checked as eps_vjp checks them; the tensors passed in are
    kept alive by this object; calling it launches on `stream` (default: the
    current stream) and raises on a bad status."""

    def __init__(self, prob: Problem, C, EF, EA, dJdC, eps_out=None, ws=None, scale=-2.0,
                 field_type: int = EPS_FIELD_C64, field_scales=None):
        import torch
        _need(C, (prob.mx, prob.my), torch.float32, "C")
        dev = C.device
        nl, self._ef, self._ea = _field_ptrs(prob, EF, EA, field_type, dev)
        self._fs = _scales(field_scales, nl)
        _need(dJdC, (prob.mx, prob.my), torch.float32, "dJdC", dev)
        _, eps_out = _eps_out(prob, eps_out, dev)
        ws = _workspace(prob, nl, ws, dev)
        _stream(None, dev)                      # the tensors' device is the current one
        self._dev = dev
        self._keep = (C, list(EF), list(EA), dJdC, eps_out)
        self._ws = ws
        self._p = prob.c_struct()
        self._args = (ctypes.byref(self._p), _ptr(C), nl, field_type, self._ef, self._ea, self._fs,
                      float(scale), _ptr(dJdC), _ptr(eps_out), _ptr(ws), ws.numel())
        self._fn = lib().eps_vjp

    def __call__(self, stream=None):
        if stream is not None and stream.device != self._dev:
            raise ValueError(f"the stream is on {stream.device} but the tensors are on {self._dev}")
        _check(self._fn(*self._args, _stream(stream)), "eps_vjp")


# --------------------------------------------------------------- morphology

EPS_MORPH_DILATE, EPS_MORPH_ERODE = 0, 1
EPS_MORPH_MAX_OPS = 8
CLOSE_THEN_OPEN = (EPS_MORPH_DILATE, EPS_MORPH_ERODE, EPS_MORPH_ERODE, EPS_MORPH_DILATE)


class eps_morph_t(ctypes.Structure):
    _fields_ = [("alpha", ctypes.c_float), ("radius", ctypes.c_float), ("n_ops", ctypes.c_int32),
                ("ops", ctypes.c_int32 * EPS_MORPH_MAX_OPS)]


@dataclass(frozen=True)
class Morph:
    """Soft dilate / erode sequence of Eq. 4/5: alpha (App. B: 20), disk
    radius d/2 in subpixels, and the operations in order."""

    alpha: float = 20.0
    radius: float = 2.0
    ops: tuple = CLOSE_THEN_OPEN

    def c_struct(self) -> eps_morph_t:
        if len(self.ops) > EPS_MORPH_MAX_OPS:
            raise ValueError(f"at most {EPS_MORPH_MAX_OPS} operations")
        m = eps_morph_t()
        m.alpha = self.alpha
        m.radius = self.radius
        m.n_ops = len(self.ops)
        for k, op in enumerate(self.ops):
            m.ops[k] = int(op)
        return m


def eps_morph_workspace_size(prob: Problem, morph: Morph, n_lambda: int = 1) -> int:
    n = ctypes.c_size_t(0)
    p, m = prob.c_struct(), morph.c_struct()
    _check(lib().eps_morph_workspace_size(ctypes.byref(p), ctypes.byref(m), n_lambda,
                                          ctypes.byref(n)), "eps_morph_workspace_size")
    return n.value


def _morph_ws(prob, morph, ws, device):
    import torch
    need = eps_morph_workspace_size(prob, morph)
    if ws is None:
        ws = torch.empty(max(need, 1), dtype=torch.uint8, device=device)
    _need_bytes(ws, 0, "ws", device)      # its size and alignment are checked by the library
    return ws


def eps_forward_morph(prob: Problem, morph: Morph, C, eps=None, offdiag=None, ws=None, stream=None):
    """eps_hat of the chain with morphology (Eq. 2-6, then the Yee stage).
    Returns eps, or (eps, offdiag) when prob.flags has EPS_FLAG_OFFDIAG."""
    import torch
    _need(C, (prob.mx, prob.my), torch.float32, "C")
    dev = C.device
    shape = (3, prob.nx, prob.ny, prob.nz)
    if eps is None:
        eps = torch.empty(shape, dtype=torch.float32, device=dev)
    _need(eps, shape, torch.float32, "eps", dev)
    want_od = bool(prob.flags & EPS_FLAG_OFFDIAG)
    if want_od:
        if offdiag is None:
            offdiag = torch.empty((2,) + shape[1:], dtype=torch.float32, device=dev)
        _need(offdiag, (2,) + shape[1:], torch.float32, "offdiag", dev)
    ws = _morph_ws(prob, morph, ws, dev)
    p, m = prob.c_struct(), morph.c_struct()
    _check(lib().eps_forward_morph(ctypes.byref(p), ctypes.byref(m), _ptr(C), _ptr(eps),
                                   _ptr(offdiag) if want_od else None, _ptr(ws), ws.numel(),
                                   _stream(stream, dev)), "eps_forward_morph")
    return (eps, offdiag) if want_od else eps


def eps_vjp_morph(prob: Problem, morph: Morph, C, EF, EA, scale: float = -2.0, dJdC=None,
                  eps_out=None, field_scales=None, ws=None, stream=None):
    """Eq. 1 through the chain with morphology (complex64 fields).  Returns
    dJdC, or (dJdC, eps_out) when eps_out is given (True allocates it)."""
    import torch
    _need(C, (prob.mx, prob.my), torch.float32, "C")
    dev = C.device
    nl, ef, ea = _field_ptrs(prob, EF, EA, EPS_FIELD_C64, dev)
    fs = _scales(field_scales, nl)
    if dJdC is None:
        dJdC = torch.empty((prob.mx, prob.my), dtype=torch.float32, device=dev)
    _need(dJdC, (prob.mx, prob.my), torch.float32, "dJdC", dev)
    ret_eps, eps_out = _eps_out(prob, eps_out, dev)
    ws = _morph_ws(prob, morph, ws, dev)
    p, m = prob.c_struct(), morph.c_struct()
    _check(lib().eps_vjp_morph(ctypes.byref(p), ctypes.byref(m), _ptr(C), nl, EPS_FIELD_C64, ef, ea,
                               fs, float(scale), _ptr(dJdC), _ptr(eps_out), _ptr(ws), ws.numel(),
                               _stream(stream, dev)), "eps_vjp_morph")
    return (dJdC, eps_out) if ret_eps else dJdC


def eps_vjp_real_morph(prob: Problem, morph: Morph, C, G, dJdC=None, ws=None, stream=None):
    """(d eps_hat / dC)^T G through the chain with morphology."""
    import torch
    _need(C, (prob.mx, prob.my), torch.float32, "C")
    dev = C.device
    _need(G, (3, prob.nx, prob.ny, prob.nz), torch.float32, "G", dev)
    if dJdC is None:
        dJdC = torch.empty((prob.mx, prob.my), dtype=torch.float32, device=dev)
    _need(dJdC, (prob.mx, prob.my), torch.float32, "dJdC", dev)
    ws = _morph_ws(prob, morph, ws, dev)
    p, m = prob.c_struct(), morph.c_struct()
    _check(lib().eps_vjp_real_morph(ctypes.byref(p), ctypes.byref(m), _ptr(C), _ptr(G), _ptr(dJdC),
                                    _ptr(ws), ws.numel(), _stream(stream, dev)),
           "eps_vjp_real_morph")
    return dJdC


class PreparedVjpMorph:
    """eps_vjp_morph with its ctypes arguments built once (complex64 fields),
    checked as eps_vjp_morph checks them."""

    def __init__(self, prob: Problem, morph: Morph, C, EF, EA, dJdC, eps_out=None, ws=None,
                 scale=-2.0):
        import torch
        _need(C, (prob.mx, prob.my), torch.float32, "C")
        dev = C.device
        nl, self._ef, self._ea = _field_ptrs(prob, EF, EA, EPS_FIELD_C64, dev)
        _need(dJdC, (prob.mx, prob.my), torch.float32, "dJdC", dev)
        _, eps_out = _eps_out(prob, eps_out, dev)
        ws = _morph_ws(prob, morph, ws, dev)
        _stream(None, dev)                      # the tensors' device is the current one
        self._dev = dev
        self._keep = (C, list(EF), list(EA), dJdC, eps_out)
        self._ws = ws
        self._p, self._m = prob.c_struct(), morph.c_struct()
        self._args = (ctypes.byref(self._p), ctypes.byref(self._m), _ptr(C), nl, EPS_FIELD_C64,
                      self._ef, self._ea, None, float(scale), _ptr(dJdC), _ptr(eps_out), _ptr(ws),
                      ws.numel())
        self._fn = lib().eps_vjp_morph

    def __call__(self, stream=None):
        if stream is not None and stream.device != self._dev:
            raise ValueError(f"the stream is on {stream.device} but the tensors are on {self._dev}")
        _check(self._fn(*self._args, _stream(stream)), "eps_vjp_morph")


# ---------------------------------------------------------------- optimiser

class eps_opt_t(ctypes.Structure):
    _fields_ = [(n, ctypes.c_float) for n in ("lr", "b1", "b2", "adam_eps", "gray_tol", "gamma",
                                               "u0", "beta_min", "beta_max0")] + \
               [("n_iter", ctypes.c_int32)]


OPT_STATE_FIELDS = ("step", "beta", "beta_max", "t", "unbinarity", "gray", "gray_acc", "ticket")


@dataclass(frozen=True)
class OptParams:
    """Adam (Eq. 10-11) with the beta schedule and beta_max control (Eq.
    14-15); App. B defaults.  gray_tol: a subpixel with gray_tol < rho <
    1 - gray_tol counts as gray."""

    lr: float = 0.001
    b1: float = 0.9
    b2: float = 0.999
    adam_eps: float = 1e-8
    gray_tol: float = 0.05
    gamma: float = 0.95
    u0: float = 0.01
    beta_min: float = 10.0
    beta_max0: float = 100.0
    n_iter: int = 100

    def c_struct(self) -> eps_opt_t:
        o = eps_opt_t()
        for f in ("lr", "b1", "b2", "adam_eps", "gray_tol", "gamma", "u0", "beta_min", "beta_max0"):
            setattr(o, f, getattr(self, f))
        o.n_iter = self.n_iter
        return o


OPT_STATE_BYTES = 32


def eps_opt_init(opt: OptParams, state=None, device=None, stream=None):
    """Device optimiser state (a 32-byte uint8 tensor) set to iteration 0."""
    import torch
    if state is None:
        state = torch.zeros(OPT_STATE_BYTES, dtype=torch.uint8, device=device or "cuda")
    _need(state, (OPT_STATE_BYTES,), torch.uint8, "state")
    o = opt.c_struct()
    _check(lib().eps_opt_init(ctypes.byref(o), _ptr(state), _stream(stream, state.device)),
           "eps_opt_init")
    return state


def read_opt_state(state) -> dict:
    """The device state as a dict (copies 32 bytes to the host; synchronises)."""
    import struct
    b = bytes(state.cpu().numpy().tobytes())
    vals = struct.unpack("<i4f3I", b)
    return dict(zip(OPT_STATE_FIELDS, vals))


def eps_opt_step(prob: Problem, opt: OptParams, state, C, G, M, V, ws, morph=None, stream=None):
    """Iteration state.step + 1 in place on C, M, V; `ws` is the workspace of
    the VJP call (base chain, or morphology when `morph` is given) that
    evaluated C at beta = prob.beta."""
    import torch
    _need(C, (prob.mx, prob.my), torch.float32, "C")
    dev = C.device
    for name, t in (("G", G), ("M", M), ("V", V)):
        _need(t, (prob.mx, prob.my), torch.float32, name, dev)
    _need(state, (OPT_STATE_BYTES,), torch.uint8, "state", dev)
    _need_bytes(ws, 0, "ws", dev)      # its size and alignment are checked by the library
    p, o = prob.c_struct(), opt.c_struct()
    m = morph.c_struct() if morph is not None else None
    _check(lib().eps_opt_step(ctypes.byref(p), ctypes.byref(m) if m is not None else None,
                              ctypes.byref(o), _ptr(state), _ptr(C), _ptr(G), _ptr(M), _ptr(V),
                              _ptr(ws), ws.numel(), _stream(stream, dev)), "eps_opt_step")


# ------------------------------------------------------ coarse control grid

class eps_coarse_t(ctypes.Structure):
    _fields_ = [("ncx", ctypes.c_int32), ("ncy", ctypes.c_int32)]


@dataclass(frozen=True)
class Coarse:
    """Node grid of the coarse control variables (Eq. 2): ncx x ncy nodes
    spanning the design region edge to edge, hat basis."""

    ncx: int
    ncy: int

    def c_struct(self) -> eps_coarse_t:
        g = eps_coarse_t()
        g.ncx, g.ncy = self.ncx, self.ncy
        return g


def eps_coarse_workspace_size(prob: Problem, coarse: Coarse, n_lambda: int = 1) -> int:
    n = ctypes.c_size_t(0)
    p, g = prob.c_struct(), coarse.c_struct()
    _check(lib().eps_coarse_workspace_size(ctypes.byref(p), ctypes.byref(g), n_lambda,
                                           ctypes.byref(n)), "eps_coarse_workspace_size")
    return n.value


def _coarse_ws(prob, coarse, ws, device):
    import torch
    if ws is None:
        ws = torch.empty(max(eps_coarse_workspace_size(prob, coarse), 1), dtype=torch.uint8,
                         device=device)
    _need_bytes(ws, 0, "ws", device)      # its size and alignment are checked by the library
    return ws


def eps_forward_coarse(prob: Problem, coarse: Coarse, c, eps=None, ws=None, stream=None):
    """eps_hat [3, nx, ny, nz] from node values c [ncx, ncy]."""
    import torch
    _need(c, (coarse.ncx, coarse.ncy), torch.float32, "c")
    dev = c.device
    shape = (3, prob.nx, prob.ny, prob.nz)
    if eps is None:
        eps = torch.empty(shape, dtype=torch.float32, device=dev)
    _need(eps, shape, torch.float32, "eps", dev)
    if prob.flags & EPS_FLAG_OFFDIAG:
        raise ValueError("use the C entry point for the off-diagonal term with coarse controls")
    ws = _coarse_ws(prob, coarse, ws, dev)
    p, g = prob.c_struct(), coarse.c_struct()
    _check(lib().eps_forward_coarse(ctypes.byref(p), ctypes.byref(g), _ptr(c), _ptr(eps), None,
                                    _ptr(ws), ws.numel(), _stream(stream, dev)),
           "eps_forward_coarse")
    return eps


def eps_vjp_coarse(prob: Problem, coarse: Coarse, c, EF, EA, scale: float = -2.0, dJdc=None,
                   eps_out=None, ws=None, stream=None):
    """Eq. 1 with respect to the node values (complex64 fields).  Returns
    dJdc [ncx, ncy], or (dJdc, eps_out) when eps_out is given (True allocates)."""
    import torch
    _need(c, (coarse.ncx, coarse.ncy), torch.float32, "c")
    dev = c.device
    nl, ef, ea = _field_ptrs(prob, EF, EA, EPS_FIELD_C64, dev)
    if dJdc is None:
        dJdc = torch.empty((coarse.ncx, coarse.ncy), dtype=torch.float32, device=dev)
    _need(dJdc, (coarse.ncx, coarse.ncy), torch.float32, "dJdc", dev)
    ret_eps, eps_out = _eps_out(prob, eps_out, dev)
    ws = _coarse_ws(prob, coarse, ws, dev)
    p, g = prob.c_struct(), coarse.c_struct()
    _check(lib().eps_vjp_coarse(ctypes.byref(p), ctypes.byref(g), _ptr(c), nl, EPS_FIELD_C64, ef, ea,
                                None, float(scale), _ptr(dJdc), _ptr(eps_out), _ptr(ws), ws.numel(),
                                _stream(stream, dev)), "eps_vjp_coarse")
    return (dJdc, eps_out) if ret_eps else dJdc


def eps_vjp_real_coarse(prob: Problem, coarse: Coarse, c, G, dJdc=None, ws=None, stream=None):
    """(d eps_hat / dc)^T G with respect to the node values, for a real
    float32 cotangent G [3, nx, ny, nz]."""
    import torch
    _need(c, (coarse.ncx, coarse.ncy), torch.float32, "c")
    dev = c.device
    _need(G, (3, prob.nx, prob.ny, prob.nz), torch.float32, "G", dev)
    if dJdc is None:
        dJdc = torch.empty((coarse.ncx, coarse.ncy), dtype=torch.float32, device=dev)
    _need(dJdc, (coarse.ncx, coarse.ncy), torch.float32, "dJdc", dev)
    ws = _coarse_ws(prob, coarse, ws, dev)
    p, g = prob.c_struct(), coarse.c_struct()
    _check(lib().eps_vjp_real_coarse(ctypes.byref(p), ctypes.byref(g), _ptr(c), _ptr(G), _ptr(dJdc),
                                     _ptr(ws), ws.numel(), _stream(stream, dev)),
           "eps_vjp_real_coarse")
    return dJdc
