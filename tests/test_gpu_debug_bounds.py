"""The debug-bounds build (-DEPS_DEBUG_BOUNDS, libepschain_debug.so): every
checked global access tests its index against its buffer's extent and
records EPS_ERR_DEVICE_BOUNDS instead of leaving it.  A child process that
loads only that build runs the bounds self-test (the flag reaches the host)
and then every kernel family on edge-case shapes with no check firing; its
outputs equal the release build's bit for bit (the checks change no
arithmetic).  With compute-sanitizer closed on this pool, this is the
memory-safety evidence for the kernels' index arithmetic."""

import os
import subprocess
import sys
import textwrap

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = textwrap.dedent("""
    import sys
    sys.path.insert(0, {root!r})
    from paper_2505_03352_gb300 import epschain
    epschain.LIB_PATH = {lib!r}
    import numpy as np
    import torch
    import paper_2505_03352_gb300 as ec
    from tests import _bounds_cases
    ec.eps_sync_status()
    ec.eps_selftest_bounds()
    try:
        ec.eps_sync_status()
    except ec.EpsError as e:
        assert "EPS_ERR_DEVICE_BOUNDS" in str(e), e
    else:
        raise SystemExit("the bounds self-test did not reach the host")
    ec.eps_sync_status()          # reported once, then cleared
    out = _bounds_cases.run_cases(ec, torch)
    np.savez({path!r}, **out)
""")


@pytest.fixture(scope="module")
def debug_lib():
    from paper_2505_03352_gb300 import build_lib
    return build_lib.build(debug_bounds=True)


def test_release_build_has_no_bounds_checks():
    import paper_2505_03352_gb300 as ec
    with pytest.raises(ec.EpsError, match="EPS_ERR_UNSUPPORTED"):
        ec.eps_selftest_bounds()


def test_no_bounds_check_fires_and_results_equal_the_release_build(debug_lib, tmp_path):
    import torch

    import paper_2505_03352_gb300 as ec
    from tests import _bounds_cases
    path = str(tmp_path / "debug_bounds.npz")
    r = subprocess.run([sys.executable, "-c", CHILD.format(root=ROOT, lib=debug_lib, path=path)],
                       capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-3000:]
    dbg = np.load(path)
    rel = _bounds_cases.run_cases(ec, torch)
    assert set(dbg.files) == set(rel)
    differ = []
    for k, v in rel.items():
        assert np.all(np.isfinite(v)), k
        if not np.array_equal(dbg[k], v):
            differ.append((k, float(np.max(np.abs(dbg[k] - v)) / max(np.max(np.abs(v)), 1e-30))))
    assert not differ, differ
