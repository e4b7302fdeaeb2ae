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
    epsc = 4 * 300 * 300 * 4       # per-column eps values for the Eq. 1 surrogate
    al = lambda b: (b + 255) // 256 * 256
    assert n == al(w) + al(seeds) + 2 * al(sub) + al(epsc)
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
    # the surrogate's value pointer: NULL or not 8-byte aligned
    fake = ctypes.c_void_p(0x10000)
    arr = (ctypes.c_void_p * 1)(fake)
    assert L.eps_vjp_surrogate(P, fake, 1, 0, arr, arr, None, -2.0, fake, None, None, fake,
                               1 << 30, None) == 1
    assert L.eps_vjp_surrogate(P, fake, 1, 0, arr, arr, None, -2.0, fake, None,
                               ctypes.c_void_p(0x10004), fake, 1 << 30, None) == 1


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


# ------------------------------------------------------------ morphology path

def test_morph_workspace_layout(L):
    p = prob(mx=600, my=600, nz=24)
    m = ec.Morph(alpha=20.0, radius=2.0)
    al = lambda b: (b + 255) // 256 * 256
    base = ec.eps_workspace_size(p)        # the Yee stage runs on rho_n with the same shapes
    maps = (len(m.ops) + 4) * al(600 * 600 * 4)   # rho_0..rho_n, P'(u), two adjoint maps
    assert ec.eps_morph_workspace_size(p, m) == maps + base
    assert ec.eps_morph_workspace_size(p, ec.Morph(ops=())) == 4 * al(600 * 600 * 4) + base
    assert ec.eps_morph_workspace_size(prob(mx=0), m) == 0


def _morph_code(L, p, m):
    n = ctypes.c_size_t()
    return L.eps_morph_workspace_size(ctypes.byref(p.c_struct()), ctypes.byref(m), 1,
                                      ctypes.byref(n))


def test_bad_morphology_is_rejected_on_host(L):
    p = prob()

    def code(alpha=20.0, radius=2.0, ops=(0, 1)):
        m = ec.eps_morph_t()
        m.alpha, m.radius, m.n_ops = alpha, radius, len(ops)
        for k, op in enumerate(ops[:8]):
            m.ops[k] = op
        return _morph_code(L, p, m)

    assert code() == 0
    assert code(alpha=0.0) == 1
    assert code(alpha=float("nan")) == 1
    assert code(alpha=61.0) == 1
    assert code(radius=-0.5) == 1
    assert code(radius=12.0) == 4        # disk larger than the built stencils
    assert code(radius=11.99) == 0
    assert code(ops=(0, 2)) == 1
    m = ec.eps_morph_t()
    m.alpha, m.radius, m.n_ops = 20.0, 2.0, 9
    assert _morph_code(L, p, m) == 1
    # the problem itself is validated first
    assert _morph_code(L, prob(mx=63), ec.Morph().c_struct()) == 2
    with pytest.raises(ValueError):
        ec.Morph(ops=(0,) * 9).c_struct()


def test_morph_entry_points_reject_bad_pointers_before_launch(L):
    p = prob()
    P = ctypes.byref(p.c_struct())
    M = ctypes.byref(ec.Morph().c_struct())
    fake = ctypes.c_void_p(0x10000)
    assert L.eps_forward_morph(P, M, None, None, None, fake, 1 << 30, None) == 1
    assert L.eps_forward_morph(P, M, fake, fake, None, fake, 16, None) == 3
    assert L.eps_vjp_real_morph(P, M, fake, None, fake, fake, 1 << 30, None) == 1
    arr = (ctypes.c_void_p * 1)(fake)
    assert L.eps_vjp_morph(P, M, fake, 1, 0, arr, arr, None, -2.0, fake, None, fake, 16,
                           None) == 3
    assert L.eps_vjp_morph(P, M, fake, 1, 0, arr, arr, None, -2.0, fake, None,
                           ctypes.c_void_p(0x10040), 1 << 30, None) == 3   # not 256-aligned
    assert L.eps_vjp_morph(P, M, fake, 1, 7, arr, arr, None, -2.0, fake, None, fake, 1 << 30,
                           None) == 1
    assert L.eps_vjp_morph(P, None, fake, 1, 0, arr, arr, None, -2.0, fake, None, fake, 1 << 30,
                           None) == 1


# ------------------------------------------------------------- optimiser step

def test_bad_optimiser_parameters_are_rejected_on_host(L):
    p = prob()
    fake = ctypes.c_void_p(0x10000)

    def code(**kw):
        o = ec.OptParams(**kw).c_struct()
        return L.eps_opt_step(ctypes.byref(p.c_struct()), None, ctypes.byref(o), fake, fake, fake,
                              fake, fake, fake, 16, None)

    assert code(lr=0.0) == 1
    assert code(b1=1.0) == 1
    assert code(b2=-0.1) == 1
    assert code(gray_tol=0.5) == 1
    assert code(gamma=1.0) == 1
    assert code(u0=0.0) == 1
    assert code(beta_min=0.0) == 1
    assert code(beta_max0=5.0) == 1          # below beta_min
    assert code(n_iter=0) == 1
    assert code(adam_eps=float("nan")) == 1
    assert code() == 3                         # valid parameters: the workspace is too small
    o = ec.OptParams().c_struct()
    assert L.eps_opt_init(ctypes.byref(o), None, None) == 1
    assert L.eps_opt_step(ctypes.byref(prob(beta=-1.0).c_struct()), None, ctypes.byref(o), fake,
                          fake, fake, fake, fake, fake, 1 << 30, None) == 1
    assert L.eps_opt_step(ctypes.byref(p.c_struct()), None, ctypes.byref(o), fake,
                          ctypes.c_void_p(0x10004), fake, fake, fake, fake, 1 << 30, None) == 1


# ------------------------------------------------------- coarse control grid

def test_coarse_workspace_and_validation(L):
    p = prob(mx=420, my=420, nz=24)
    al = lambda b: (b + 255) // 256 * 256
    base = ec.eps_workspace_size(p)
    assert ec.eps_coarse_workspace_size(p, ec.Coarse(36, 36)) == 2 * al(420 * 420 * 4) + base
    n = ctypes.c_size_t()
    P = ctypes.byref(p.c_struct())
    assert L.eps_coarse_workspace_size(P, ctypes.byref(ec.Coarse(1, 36).c_struct()), 1,
                                       ctypes.byref(n)) == 2
    assert L.eps_coarse_workspace_size(P, None, 1, ctypes.byref(n)) == 1
    fake = ctypes.c_void_p(0x10000)
    G = ctypes.byref(ec.Coarse(36, 36).c_struct())
    assert L.eps_forward_coarse(P, G, None, fake, None, fake, 1 << 30, None) == 1
    assert L.eps_forward_coarse(P, G, fake, fake, None, fake, 64, None) == 3
    arr = (ctypes.c_void_p * 1)(fake)
    assert L.eps_vjp_coarse(P, G, fake, 1, 0, arr, arr, None, -2.0, fake, None, fake, 64, None) == 3
    assert L.eps_vjp_real_coarse(P, G, fake, None, fake, fake, 1 << 30, None) == 1


def test_timeout_selftest_rejects_bad_limits_on_host(L):
    assert L.eps_selftest_timeout(0, None) == 1            # EPS_ERR_INVALID_ARG
    assert L.eps_selftest_timeout((1 << 31) + 1, None) == 1
    assert L.eps_selftest_timeout(-5, None) == 1


def test_debug_bounds_entry_is_declared_and_exported(L):
    # a release build answers the bounds self-test with EPS_ERR_UNSUPPORTED
    # before any launch
    assert L.eps_selftest_bounds(None) == 4               # EPS_ERR_UNSUPPORTED


def test_launch_counter_reads_without_a_launch(L):
    # a host-side counter: readable with no GPU, unchanged by calls that
    # return before any launch, and a null pointer is an argument error
    import ctypes
    a = ec.eps_launch_count()
    assert a >= 0
    assert L.eps_launch_count(None) == 1          # EPS_ERR_INVALID_ARG
    p = ec.Problem(mx=64, my=48, nz=16, radius=3.0, beta=8.0).c_struct()
    bad = ctypes.c_void_p(0)
    L.eps_forward(ctypes.byref(p), bad, bad, bad, None)   # rejected on the host
    assert ec.eps_launch_count() == a
