"""Host-side checks of the C ABI that need no GPU: the library loads, exports
every entry point the header declares, and rejects bad arguments on the
host before any CUDA call."""

import ctypes
import os
import re
import subprocess

import pytest

from paper_2505_03352_gb300 import epschain as ec

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    if not os.path.exists(ec.LIB_PATH):
        from paper_2505_03352_gb300 import build_lib
        build_lib.build()
    return ec.lib()


def declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if not fn.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", fn)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"\b(eps_[a-z0-9_]+)\s*\(", text):
            names.add(m.group(1))
    return names


def test_header_declares_the_boundary():
    names = declared_functions()
    for n in ("eps_forward", "eps_vjp", "eps_vjp_real", "eps_workspace_size",
              "eps_sync_status", "eps_status_string"):
        assert n in names


def test_library_exports_every_declared_symbol(L):
    out = subprocess.run(["nm", "-D", "--defined-only", ec.LIB_PATH], capture_output=True,
                         text=True, check=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if " T " in line}
    missing = declared_functions() - exported
    assert not missing, missing
    for n in declared_functions():
        assert hasattr(L, n)


def test_status_strings(L):
    for code, name in ec.STATUS_NAMES.items():
        assert ec.eps_status_string(code) == name
    assert ec.eps_status_string(99) == "EPS_ERR_UNKNOWN"


def prob(**kw):
    base = dict(mx=64, my=64, nz=16, radius=3.0, beta=8.0)
    base.update(kw)
    return ec.Problem(**base)


def test_workspace_size_layout(L):
    p = prob(mx=600, my=600, nz=24)
    n = ec.eps_workspace_size(p)
    w = 4 * 300 * 300 * 4          # Eq. 1 column sums
    seeds = 10 * 300 * 300 * 4     # adjoint seeds per Yee column
    sub = 600 * 600 * 4            # per-subpixel adjoint factors (two maps)
    al = lambda b: (b + 255) // 256 * 256
    assert n == al(w) + al(seeds) + 2 * al(sub)
    assert ec.eps_workspace_size(prob(mx=0)) == 0


@pytest.mark.parametrize("kw,status", [
    (dict(mx=63), ec.EpsError),
    (dict(sub=3), ec.EpsError),
    (dict(radius=0.0), ec.EpsError),
    (dict(radius=float("nan")), ec.EpsError),
    (dict(radius=12.5), ec.EpsError),
    (dict(nz=11), ec.EpsError),
    (dict(slab_k0=5, nz=16), ec.EpsError),
    (dict(bc=2), ec.EpsError),
    (dict(eps_clad=0.0), ec.EpsError),
    (dict(beta=float("inf")), ec.EpsError),
    (dict(flags=8), ec.EpsError),
])
def test_bad_problems_are_rejected_on_host(L, kw, status):
    with pytest.raises(status):
        ec.eps_workspace_size(prob(**kw))


def _codes(L, p, **kw):
    P = ctypes.byref(p.c_struct())
    n = ctypes.c_size_t()
    return L.eps_workspace_size(P, 1, ctypes.byref(n)), n.value


def test_status_codes_of_bad_problems(L):
    def code(**kw):
        return _codes(L, prob(**kw))[0]
    assert code(mx=63) == 2          # EPS_ERR_SHAPE
    assert code(sub=4) == 4          # EPS_ERR_UNSUPPORTED
    assert code(radius=12.5) == 4
    assert code(radius=-1.0) == 1    # EPS_ERR_INVALID_ARG
    assert code(nz=11) == 2
    assert code(bc=7) == 1


def test_entry_points_reject_null_pointers_before_launch(L):
    p = prob()
    P = ctypes.byref(p.c_struct())
    assert L.eps_forward(P, None, None, None, None) == 1
    assert L.eps_vjp_real(P, None, None, None, None, 0, None) == 1
    # bad field type and too many wavelengths are argument errors
    assert L.eps_vjp(P, None, 1, 9, None, None, None, -2.0, None, None, None, 0, None) == 1
    assert L.eps_vjp(P, None, 17, 0, None, None, None, -2.0, None, None, None, 0, None) == 1
    # non-finite scale
    assert L.eps_vjp(P, None, 1, 0, None, None, None, float("nan"), None, None, None, 0,
                     None) == 1


def test_workspace_too_small_is_reported(L):
    p = prob()
    P = ctypes.byref(p.c_struct())
    fake = ctypes.c_void_p(0x10000)   # never dereferenced: the check fails first
    arr = (ctypes.c_void_p * 1)(fake)
    st = L.eps_vjp(P, fake, 1, 0, arr, arr, None, -2.0, fake, None, fake, 16, None)
    assert st == 3   # EPS_ERR_WORKSPACE
    st = L.eps_vjp(P, fake, 1, 0, arr, arr, None, -2.0, fake, None, ctypes.c_void_p(0x10004),
                   1 << 30, None)
    assert st == 3   # misaligned workspace


def test_misaligned_field_pointer_is_rejected(L):
    p = prob()
    P = ctypes.byref(p.c_struct())
    fake = ctypes.c_void_p(0x10000)
    bad = (ctypes.c_void_p * 1)(ctypes.c_void_p(0x10008))
    st = L.eps_vjp(P, fake, 1, 0, bad, bad, None, -2.0, fake, None, fake, 1 << 30, None)
    assert st == 1


def test_odd_nz_rejected_for_complex_fields(L):
    p = prob(nz=15)
    P = ctypes.byref(p.c_struct())
    fake = ctypes.c_void_p(0x10000)
    arr = (ctypes.c_void_p * 1)(fake)
    st = L.eps_vjp(P, fake, 1, 0, arr, arr, None, -2.0, fake, None, fake, 1 << 30, None)
    assert st == 2


def test_binding_fails_loudly_without_library(monkeypatch, tmp_path):
    monkeypatch.setattr(ec, "_lib", None)
    monkeypatch.setattr(ec, "LIB_PATH", str(tmp_path / "missing.so"))
    with pytest.raises(RuntimeError):
        ec.lib()
