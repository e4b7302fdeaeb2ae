"""Process pool that times the FP64 oracle on every host core at once, for the
CPU-baseline leg of the benchmark.

TEST INFRASTRUCTURE, NOT PRODUCT CODE.  Only the test-suite, the smoke check
and the CPU-baseline leg of the benchmark may import this module.  It runs
the oracle as it stands: each worker draws the seeded inputs of the workload
itself (the whole problem, or a square window of it for workloads too large
for one host process), computes eps_hat and the Eq. 1 VJP `reps` times, and
reports its own elapsed time.  The workers start from a shared
barrier, so the timed parts overlap.  The pool uses the spawn start method,
which is safe after CUDA has been initialised in the parent.
"""

from __future__ import annotations

import multiprocessing as mp
import os
import sys
import time

_barrier = None


def _init(barrier):
    global _barrier
    _barrier = barrier


def _synth():
    """The seeded-input module, loaded from its file: importing it through
    its package would import torch in every worker."""
    import importlib.util
    path = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                        "paper_2505_03352_gb300", "synth.py")
    spec = importlib.util.spec_from_file_location("_timing_pool_synth", path)
    mod = importlib.util.module_from_spec(spec)
    sys.modules[spec.name] = mod          # dataclasses resolve the module by name
    spec.loader.exec_module(mod)
    return mod


def _worker(task):
    cfg, reps, window, index = task
    synth = _synth()

    from . import epschain_oracle as orc
    try:
        w = synth.WORKLOADS[cfg]
        if window:
            # a window of the given size (an int for a square) with the
            # workload's layout statistics, depth and wavelength count
            # (seeds offset per worker)
            import dataclasses
            wa, wb = (window, window) if isinstance(window, int) else tuple(window)
            w = dataclasses.replace(w, mx=wa, my=wb)
            C = synth.soi_layout(wa, wb, 1000 * (1000 + w.cfg) + index) \
                if w.layout == "soi" else synth.uniform_controls(wa, wb, 1000 + index)
            shape = synth.field_shape(w)
            EF = [synth.complex_field(shape, 1000 * (2000 + 10 * w.cfg + l) + index)
                  for l in range(w.n_lambda)]
            EA = [synth.complex_field(shape, 1000 * (3000 + 10 * w.cfg + l) + index)
                  for l in range(w.n_lambda)]
        else:
            C = synth.controls(w)
            EF, EA = synth.fields(w)
        p = orc.Problem(mx=w.mx, my=w.my, nz=w.nz, radius=w.radius, beta=w.beta)
    except BaseException:
        _barrier.abort()          # the other workers stop waiting at once
        raise
    _barrier.wait(timeout=120)
    t0 = time.perf_counter()
    for _ in range(reps):
        orc.eps_hat(p, C)
        orc.vjp_fields(p, C, EF, EA)
    return reps * w.voxels, time.perf_counter() - t0


def _mem_available_bytes():
    try:
        with open("/proc/meminfo") as f:
            for line in f:
                if line.startswith("MemAvailable:"):
                    return int(line.split()[1]) * 1024
    except OSError:
        pass
    return None


def default_workers(per_worker_bytes: int = 4 << 30, ceiling: int = 32) -> int:
    """One worker per core this process may run on, at most `ceiling`, and
    no more than the available memory holds at `per_worker_bytes` each (a
    whole cfg2 call of the oracle peaks near 1 GB)."""
    try:
        cores = len(os.sched_getaffinity(0))
    except (AttributeError, OSError):
        cores = os.cpu_count() or 1
    n = min(cores, ceiling)
    mem = _mem_available_bytes()
    if mem is not None:
        n = min(n, mem // per_worker_bytes)
    return max(1, int(n))


def all_cores(cfg: int, reps: int = 2, workers: int | None = None, window=0):
    """(voxels per second over all workers, workers, seconds): every worker
    runs `reps` forward + VJP calls of workload `cfg` (the whole problem, or
    a window of it when `window` is non-zero: an int for a square window of
    that many controls per side, or (mx, my)); the rate is the voxels of all
    workers over the slowest worker's time."""
    n = workers or default_workers()
    ctx = mp.get_context("spawn")
    barrier = ctx.Barrier(n)
    with ctx.Pool(n, initializer=_init, initargs=(barrier,)) as pool:
        res = pool.map(_worker, [(cfg, reps, window, i) for i in range(n)], chunksize=1)
    vox = sum(v for v, _ in res)
    slowest = max(t for _, t in res)
    return vox / slowest, n, slowest
