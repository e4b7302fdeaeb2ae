"""Failure detection on the GPU without a fault: a bounded device-side wait
that nothing completes gives up, the host reads EPS_ERR_DEVICE_TIMEOUT
through eps_sync_status, the flag clears, and the context keeps working."""

import time

import numpy as np
import pytest

from oracle import epschain_oracle as orc

pytestmark = pytest.mark.gpu


def test_device_wait_gives_up_and_the_host_reads_the_timeout():
    import torch

    import paper_2505_03352_gb300 as ec
    ec.eps_sync_status()                        # start from a clean flag
    t0 = time.time()
    ec.eps_selftest_timeout(1 << 24)            # about 8 ms of SM clock
    with pytest.raises(ec.EpsError, match="EPS_ERR_DEVICE_TIMEOUT"):
        ec.eps_sync_status()
    assert time.time() - t0 < 30
    ec.eps_sync_status()                        # reported once, then cleared

    # the context still works: a fused call right after matches the oracle
    rng = np.random.default_rng(71)
    p = ec.Problem(mx=48, my=40, nz=16, radius=3.0, beta=8.0)
    o = orc.Problem(mx=48, my=40, nz=16, radius=3.0, beta=8.0)
    C = rng.random((48, 40), dtype=np.float32)
    shape = (3, p.nx, p.ny, p.nz)
    EF = (rng.standard_normal(shape) + 1j * rng.standard_normal(shape)).astype(np.complex64)
    EA = (rng.standard_normal(shape) + 1j * rng.standard_normal(shape)).astype(np.complex64)
    g = ec.eps_vjp(p, torch.from_numpy(C).cuda(), [torch.from_numpy(EF).cuda()],
                   [torch.from_numpy(EA).cuda()])
    ec.eps_sync_status()
    ref = orc.vjp_fields(o, C, [EF], [EA])
    assert np.max(np.abs(g.cpu().numpy() - ref)) <= 1e-4 * np.max(np.abs(ref))


def test_timeout_is_reported_after_later_work_on_the_stream():
    # the flag persists across later launches until the host reads it
    import torch

    import paper_2505_03352_gb300 as ec
    ec.eps_sync_status()
    ec.eps_selftest_timeout(1 << 20)
    p = ec.Problem(mx=32, my=32, nz=16, radius=2.0, beta=8.0)
    ec.eps_forward(p, torch.rand((32, 32), device="cuda"))
    with pytest.raises(ec.EpsError, match="EPS_ERR_DEVICE_TIMEOUT"):
        ec.eps_sync_status()
    ec.eps_sync_status()
