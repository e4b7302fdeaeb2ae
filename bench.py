"""Benchmark of the fused eps-chain forward + VJP (Eq. 1) on GB300.

One step = one fused forward + VJP call (eps_vjp with eps_out) on the
largest single-GPU workload: 3000 x 3000 controls, Yee grid 1500 x 1500 x 32
(R = 6, beta = 16, an 11-cell slab), eight wavelengths of complex64 E_F and
E_A (27.6 GB of fields resident on the device).  That is every stage of the
chain: filter, projection, mixing, dual-cell means, Sobel normals, Eq. 7,
the eps_hat write, the Eq. 1 field contraction and the adjoint scatter to
dJ/dC.  The 600 x 600 / 300 x 300 x 24 one-wavelength workload, the
three-wavelength differentiation form, the 64-region batch and the
BF16/FP16 field formats run afterwards as variants.

Timing: W warm-up steps, then exactly K steps.  Before every step a 256 MB
buffer is written and then read on the same stream (L2 flush that leaves no
dirty lines behind; the step's inputs are also far larger than L2); CUDA
events bracket each call and exclude the flush.  value = design voxels
(nx ny nz) per second of summed call time; with torchrun every rank runs its
own region (weak scaling) and the slowest rank's time is used.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--controls M]   (M x M-control crop of the workload: profiling captures)
"""

from __future__ import annotations

import argparse
import datetime as _dt
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "design voxels/s for fused eps-chain forward+VJP"
UNIT = "voxels/s"
L2_FLUSH_BYTES = 256 << 20
L2_FETCH_BYTES = 32
PROFILE_TRAFFIC = os.path.join(ROOT, "profiles", "traffic.json")
# the single-region contraction kernel and its copy/barrier helpers: a DRAM
# traffic record is used only while this file is unchanged
KERNEL_SOURCES = ["paper_2505_03352_gb300/csrc/epsc_contract_tma.cuh"]
PACKED_KERNEL_SOURCES = ["paper_2505_03352_gb300/csrc/epsc_pack.cuh"]


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=["cfg5", "cfg2"], default="cfg5",
                    help="workload of the main line: cfg5 (3000 x 3000 controls, 1500 x 1500 x 32, "
                         "8 wavelengths; the headline) or cfg2 (600 x 600, 300 x 300 x 24, "
                         "1 wavelength; for profiling captures of that size)")
    ap.add_argument("--controls", type=int, default=0,
                    help="crop the main workload to M x M controls (a smaller case of the same "
                         "kernels, for profiling captures); 0 = full size")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--variant-set",
                    default="cfg2,cfg3,cfg4,precision,morph,opt,coarse,normals3d,autograd",
                    help="comma-separated variants to run (cfg2, cfg3, cfg4, precision, morph, "
                         "opt, coarse, normals3d, autograd)")
    ap.add_argument("--no-variants", action="store_true",
                    help="skip every variant (cfg2, cfg3, batched cfg4, BF16/FP16 fields, ...)")
    args = ap.parse_args()
    if args.controls and (args.controls < 16 or args.controls % 2):
        ap.error("--controls must be an even number >= 16")
    return args


def main_workload(args):
    """The main line's workload: cfg5 (the headline) or cfg2, optionally
    cropped to M x M controls with the same depth, slab, filter and
    wavelength count."""
    import dataclasses

    from paper_2505_03352_gb300 import synth
    w = synth.WORKLOADS[5 if args.workload == "cfg5" else 2]
    if args.controls:
        m = args.controls
        w = dataclasses.replace(w, mx=m, my=m,
                                name=f"{w.name}_crop{m}x{m}")
    return w


def max_over_ranks(x: float, world: int, device=None) -> float:
    """Largest value of x over the ranks of the default process group (x on
    a single process)."""
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def link_floor(torch, dev, stream, h2d_bytes: int, d2h_bytes: int, reps: int = 10) -> dict:
    """The host link's copy rates, measured on plain pinned buffers of the
    step's own sizes, and the per-step time floor they set for the
    end-to-end loop: the two directions run concurrently across consecutive
    steps, so the floor is the slower direction's time."""
    def rate(nbytes: int, to_device: bool) -> float:
        host = torch.empty(nbytes, dtype=torch.uint8).pin_memory()
        devb = torch.empty(nbytes, dtype=torch.uint8, device=dev)
        dst, src = (devb, host) if to_device else (host, devb)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(stream):
            for _ in range(3):
                dst.copy_(src, non_blocking=True)
            e0.record(stream)
            for _ in range(reps):
                dst.copy_(src, non_blocking=True)
            e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / reps
        del host, devb
        return nbytes / (ms * 1e-3) / 1e9
    g_in = rate(h2d_bytes, True)
    g_out = rate(d2h_bytes, False)
    floor = max(h2d_bytes / (g_in * 1e9), d2h_bytes / (g_out * 1e9)) * 1e3
    return {"h2d_gbs": round(g_in, 1), "d2h_gbs": round(g_out, 1),
            "floor_ms_per_step": round(floor, 4),
            "note": "pinned-buffer copy rates of the step's byte counts; frac = floor / e2e ms per step"}


def weak_scaling_value(units_per_rank: float, world: int, steps: int, ms_total_max: float) -> float:
    """Whole-job throughput: every rank processes its own units each step,
    and the job takes as long as its slowest rank."""
    return world * units_per_rank * steps / (ms_total_max * 1e-3)


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


# ------------------------------------------------------------------ clocks

class ClockSampler:
    FIELDS = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    REASONS = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.samples = []
        self.proc = None
        self.thread = None

    def start(self, wait_s: float = 5.0):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-i", str(self.idx), "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return self
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()
        t0 = time.time()
        while not self.samples and time.time() - t0 < wait_s:
            time.sleep(0.05)
        return self

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 10:
                continue
            try:
                ts = _dt.datetime.strptime(parts[0], "%Y/%m/%d %H:%M:%S.%f").timestamp()
                sm = float(parts[2])
                smax = float(parts[3])
            except ValueError:
                continue
            flags = dict(zip(self.REASONS, [p.lower() == "active" for p in parts[6:10]]))
            self.samples.append((ts, sm, smax, flags))

    def stop(self):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self, t0: float, t1: float):
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        inside = [s for s in self.samples if t0 - 0.05 <= s[0] <= t1 + 0.15]
        use = inside or sorted(self.samples, key=lambda s: abs(s[0] - (t0 + t1) / 2))[:3]
        reasons = sorted({r for s in use for r, on in s[3].items() if on})
        return {"sm_mhz": statistics.median(s[1] for s in use),
                "sm_max_mhz": max(s[2] for s in use), "reasons": reasons,
                "samples": len(use), "in_timed_region": bool(inside)}


# ------------------------------------------------------------------ helpers

def kernel_hash(sources=None):
    h = hashlib.sha256()
    for rel in (KERNEL_SOURCES if sources is None else sources):
        with open(os.path.join(ROOT, rel), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def committed_traffic(workload: str, sources=None):
    """dram read+write bytes per launch of the dominant kernel (or of the
    kernel in `sources`) from the committed ncu summary, if it was taken on
    the current kernel source."""
    if not os.path.exists(PROFILE_TRAFFIC):
        return None
    with open(PROFILE_TRAFFIC) as f:
        d = json.load(f)
    ent = d.get(workload)
    if not ent or ent.get("kernel_hash") != kernel_hash(sources):
        return None
    return ent.get("bytes_per_launch")


def algorithmic_bytes(w, n_lambda):
    """Bytes one fused forward + VJP call must move: C read, dJ/dC write,
    eps_hat write and the J-support field planes (3 nk + 1 planes of E_F and
    E_A, 8 B each, per Yee column and wavelength)."""
    cols = w.nx * w.ny
    planes = 3 * w.slab_nk + 1
    return 8 * w.mx * w.my + 12 * cols * w.nz + cols * n_lambda * planes * 2 * 8


def contraction_bytes(w, n_lambda):
    """Algorithmic bytes of the Eq. 1 contraction kernel: the J-support field
    planes of E_F and E_A (544 B per Yee column and wavelength for complex64
    with an 11-plane slab) plus its four float32 column-sum maps."""
    cols = w.nx * w.ny
    planes = 3 * w.slab_nk + 1
    return cols * n_lambda * planes * 2 * 8 + 16 * cols


def _host(x):
    """numpy copy of an array that may live on the device."""
    import numpy as np
    return x.cpu().numpy() if hasattr(x, "cpu") else np.asarray(x)


def cpu_baseline(w, C, EF, EA, budget_s: float = 15.0, window: int = 0, max_windows: int = 12,
                 all_cores_reps: int = 2, keep: int = 0):
    """The FP64 oracle, as it stands, on a bounded sample of the workload:
    one thread, plus every host core at once (a spawned process per core,
    each running its own calls; reported under "all_cores").

    With window = 0 the sample is whole forward + VJP calls of the problem.
    Otherwise it is window x window-control windows of the workload's own
    inputs (C, E_F, E_A, which may be device tensors) at seeded positions,
    each solved by the oracle as a problem of its own; only the oracle's
    calls are timed, not the copies that cut the windows out.

    Returns (the cpu_baseline object, the oracle's results on the first
    `keep` windows as (a0, b0, window, dJ/dC, eps_hat)).  Those results are
    what the benchmark states every GPU result's error against; the oracle
    runs nowhere else in the GPU arm."""
    import numpy as np

    from oracle import epschain_oracle as orc
    whole = not window or window >= min(w.mx, w.my)
    reps = 0
    vox = 0
    dt = 0.0
    kept = []
    if whole:
        op = orc.Problem(mx=w.mx, my=w.my, nz=w.nz, radius=w.radius, beta=w.beta)
        Ch, EFh, EAh = _host(C), [_host(e) for e in EF], [_host(e) for e in EA]
        while reps < 20 and dt <= budget_s:
            t0 = time.perf_counter()
            e_ref = orc.eps_hat(op, Ch)
            g_ref = orc.vjp_fields(op, Ch, EFh, EAh)
            dt += time.perf_counter() - t0
            if not kept and keep > 0:
                kept.append((0, 0, 0, g_ref, e_ref))
            reps += 1
            vox += w.voxels
        sample = (f"{reps} full forward+VJP calls of {w.name} "
                  f"({len(EF)} wavelengths; numpy float64, single thread)")
    else:
        rng = np.random.default_rng(4242)
        Ch = _host(C)
        op = orc.Problem(mx=window, my=window, nz=w.nz, radius=w.radius, beta=w.beta)
        while reps < max_windows and dt <= budget_s:
            a0 = int(rng.integers(0, w.mx - window + 1)) // 2 * 2
            b0 = int(rng.integers(0, w.my - window + 1)) // 2 * 2
            Cw = np.ascontiguousarray(Ch[a0:a0 + window, b0:b0 + window])
            sl = (slice(None), slice(a0 // 2, (a0 + window) // 2),
                  slice(b0 // 2, (b0 + window) // 2), slice(None))
            EFw = [_host(e[sl]) for e in EF]
            EAw = [_host(e[sl]) for e in EA]
            t0 = time.perf_counter()
            e_ref = orc.eps_hat(op, Cw)
            g_ref = orc.vjp_fields(op, Cw, EFw, EAw)
            dt += time.perf_counter() - t0
            if len(kept) < keep:
                kept.append((a0, b0, window, g_ref, e_ref))
            reps += 1
            vox += op.nx * op.ny * op.nz
            del EFw, EAw
        sample = (f"{reps} windows of {window} x {window} controls ({window // 2} x {window // 2} x "
                  f"{w.nz} Yee cells, {len(EF)} wavelengths) cut from {w.name} at seeded positions, "
                  f"each a forward+VJP call of the oracle (numpy float64, single thread)")
    out = {"value": vox / dt, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample,
           "seconds": round(dt, 2)}
    if all_cores_reps > 0:
        try:
            from oracle import timing_pool
            size = (w.mx, w.my) if whole else (window, window)
            v, n, t = timing_pool.all_cores(w.cfg, reps=all_cores_reps, window=size)
            what = (f"{all_cores_reps} forward+VJP calls of a {size[0]} x {size[1]}-control problem "
                    f"with the statistics of {w.name} (own seeded inputs)")
            out["all_cores"] = {"value": v, "unit": UNIT, "cores": n, "seconds": round(t, 2),
                                "sample": f"{what} in each of {n} spawned processes, started together"}
        except Exception as e:          # the single-thread figure stands on its own
            out["all_cores"] = {"unavailable": f"{type(e).__name__}: {e}"[:200]}
    return out, kept


def oracle_errors(w, kept, g_dev, e_dev=None):
    """Worst errors of a GPU result against the oracle's window results
    (from the CPU-baseline leg): dJ/dC as max |diff| / max |oracle| and
    eps_hat as the largest elementwise relative difference, both over the
    windows' interiors.  The chain is local (eps_hat at a cell depends on C
    within R + 4 subpixels, dJ/dC on C and the fields within about 2R + 8),
    so inside a margin of 2 ceil(R) + 8 subpixels from a window edge that is
    not the region's edge the window problem equals the full one."""
    import math

    import numpy as np
    if not kept:
        return None
    margin = int(2 * math.ceil(w.radius)) + 8
    margin += margin % 2
    worst_g = worst_e = 0.0
    for a0, b0, win, g_ref, e_ref in kept:
        wa, wb = (win, win) if win else (w.mx, w.my)
        ia0 = margin if a0 > 0 else 0
        ib0 = margin if b0 > 0 else 0
        ia1 = wa - margin if a0 + wa < w.mx else wa
        ib1 = wb - margin if b0 + wb < w.my else wb
        gg = _host(g_dev[a0 + ia0:a0 + ia1, b0 + ib0:b0 + ib1]).astype(np.float64)
        rg = g_ref[ia0:ia1, ib0:ib1]
        worst_g = max(worst_g, float(np.max(np.abs(gg - rg)) / np.max(np.abs(rg))))
        if e_dev is not None:
            ge = _host(e_dev[:, (a0 + ia0) // 2:(a0 + ia1) // 2,
                             (b0 + ib0) // 2:(b0 + ib1) // 2, :]).astype(np.float64)
            re = e_ref[:, ia0 // 2:ia1 // 2, ib0 // 2:ib1 // 2, :]
            worst_e = max(worst_e, float(np.max(np.abs(ge - re) / np.abs(re))))
    out = {"dJdC_max_abs_err_over_max_abs_oracle": worst_g, "windows": len(kept)}
    if e_dev is not None:
        out["eps_hat_max_rel_err"] = worst_e
    return out


# ------------------------------------------------------------------ our arm

def main_inputs(torch, synth, w, dev):
    """Controls (host array and device copy) and the device field lists of
    the main workload.  Small workloads draw their fields on the host (the
    seeded numpy generator of the input module); the large ones on the
    device with seeded torch generators (seeds 2000 + 10 cfg + l for E_F and
    3000 + 10 cfg + l for E_A), since drawing 27.6 GB of normals on one host
    core would take minutes."""
    C = synth.controls(w)
    Cd = torch.from_numpy(C).to(dev)
    shape = (3, w.nx, w.ny, w.nz)
    if w.voxels * w.n_lambda * 16 <= (256 << 20):
        EF, EA = synth.fields(w)
        EFd = [torch.from_numpy(e).to(dev) for e in EF]
        EAd = [torch.from_numpy(e).to(dev) for e in EA]
        origin = "host numpy default_rng"
    else:
        EFd = _device_fields(torch, shape, w.n_lambda, 2000 + 10 * w.cfg, dev)
        EAd = _device_fields(torch, shape, w.n_lambda, 3000 + 10 * w.cfg, dev)
        origin = "device torch generators"
    return C, Cd, EFd, EAd, origin


def contraction_roofline(w, n_lambda, c_ms, peak, peak_kind, traffic):
    """Roofline of the Eq. 1 contraction: algorithmic bytes per launch over
    its event-timed duration, against the measured copy peak; with the DRAM
    bytes of the committed ncu capture (scaled to this launch), the DRAM
    fraction and the ceiling the field layout puts on the algorithmic one."""
    alg_c = contraction_bytes(w, n_lambda)
    achieved = alg_c / (c_ms * 1e-3) / 1e9 if c_ms > 0 else 0.0
    return {"bound": "hbm", "kernel": "eps_vjp_contract", "achieved": round(achieved, 1),
            "peak": peak, "unit": "GB/s", "frac": round(achieved / peak, 4),
            "traffic": traffic,
            # DRAM bytes actually moved (whole 32-byte sectors of the field
            # columns) per second against the peak, and the algorithmic
            # fraction the field layout allows at most
            "dram_frac": (round(traffic / (c_ms * 1e-3) / 1e9 / peak, 4)
                          if traffic and c_ms > 0 else None),
            "layout_ceiling_frac": round(alg_c / traffic, 4) if traffic else None,
            "peak_source": ("MEASURED_PEAKS.json hbm_gbs (of measured)" if peak_kind == "measured"
                            else "fallback 6.8 TB/s (of fallback)"),
            "algorithmic_bytes_per_launch": alg_c, "avg_launch_ms": round(c_ms, 5)}


def run_ours(args, rank, world, local):
    import torch

    import paper_2505_03352_gb300 as ec
    from paper_2505_03352_gb300 import synth

    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    w = main_workload(args)
    NL = w.n_lambda
    prob = ec.Problem(mx=w.mx, my=w.my, nz=w.nz, radius=w.radius, beta=w.beta)
    C, Cd, EFd, EAd, field_origin = main_inputs(torch, synth, w, dev)
    dJdC = torch.empty((w.mx, w.my), dtype=torch.float32, device=dev)
    eps = torch.empty((3, w.nx, w.ny, w.nz), dtype=torch.float32, device=dev)
    call = ec.PreparedVjp(prob, Cd, EFd, EAd, dJdC, eps_out=eps)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    flush_sink = torch.empty((), dtype=torch.float32, device=dev)
    # the field reads touch 32-byte sectors at the column pitch (library call)
    ec.eps_set_l2_fetch_granularity(L2_FETCH_BYTES)
    stream = torch.cuda.current_stream()

    def barrier():
        torch.cuda.synchronize()
        if world > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize()

    def flush_l2():
        # overwrite, then read back: the L2 ends up holding clean lines of an
        # unrelated buffer, so no write-back lands inside the next timed call
        flush.zero_()
        flush_sink.copy_(flush.sum())

    # warm-up (also fills the library's event pool)
    ec.eps_profile_start()
    for _ in range(max(args.warmup, 3)):
        flush_l2()
        call()
    torch.cuda.synchronize()
    ec.eps_profile_stop(64)
    ec.eps_sync_status()

    gpu_index = local
    vis = os.environ.get("CUDA_VISIBLE_DEVICES")
    if vis:
        ids = [v.strip() for v in vis.split(",")]
        if local < len(ids) and ids[local].isdigit():
            gpu_index = int(ids[local])
    sampler = ClockSampler(gpu_index).start() if rank == 0 else None

    K = args.steps
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(K)]
    barrier()
    launches0 = ec.eps_launch_count()
    t0 = time.time()
    for i in range(K):
        flush_l2()
        ev[i][0].record(stream)
        call()
        ev[i][1].record(stream)
    torch.cuda.synchronize()
    t1 = time.time()
    # the library's own kernel launches in the timed region (its host-side
    # counter; the L2 flushes are torch kernels and are not counted)
    timed_launches = ec.eps_launch_count() - launches0
    barrier()
    ec.eps_sync_status()
    step_ms = sorted(a.elapsed_time(b) for a, b in ev)
    ms_total = max_over_ranks(sum(step_ms), world, dev)
    time.sleep(0.25)
    clocks = None
    if sampler is not None:
        sampler.stop()
        clocks = sampler.summary(t0, t1)

    ms_step = ms_total / K
    value = weak_scaling_value(w.voxels, world, K, ms_total)

    # per-kernel durations: the same steps again with the library's event
    # pairs around every launch (kernels then run without launch overlap)
    KP = max(1, min(K, int(50.0 / max(ms_step, 1e-3))))
    ec.eps_profile_start()
    for _ in range(KP):
        flush_l2()
        call()
    torch.cuda.synchronize()
    prof = ec.eps_profile_stop(64)
    ec.eps_sync_status()

    # dominant kernel roofline: the Eq. 1 field contraction, timed per launch
    # by the library's events (profiling launches the kernels without overlap)
    peak, peak_kind = measured_peaks()
    kernels = {k: {"launches": n, "avg_ms": round(t / max(n, 1), 5)} for k, (n, t) in prof.items()}
    n_c, t_c = prof.get("eps_vjp_contract", (0, 0.0))
    c_ms = t_c / max(n_c, 1)
    call_alg = algorithmic_bytes(w, NL)
    roofline = contraction_roofline(w, NL, c_ms, peak, peak_kind, committed_traffic(w.name))
    roofline["whole_call"] = {"algorithmic_bytes": call_alg,
                              "achieved_gbs": round(call_alg / (ms_step * 1e-3) / 1e9, 1),
                              "frac": round(call_alg / (ms_step * 1e-3) / 1e9 / peak, 4)}
    roofline["kernels"] = kernels

    # the oracle on the host cores (rank 0, one GPU only): before the end to
    # end leg, whose pinned buffers hold the whole workload in host memory
    cpu = None
    kept = []
    accuracy = {"note": "not computed: the CPU-baseline leg (which runs the oracle) was skipped"}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        whole = w.voxels * NL <= 2_500_000
        cpu, kept = cpu_baseline(w, C, EFd, EAd, window=0 if whole else 384, keep=4)
        # dJ/dC and eps_hat of the timed calls (every call gives the same
        # result) against the oracle's results on the baseline's windows
        accuracy = oracle_errors(w, kept, dJdC, eps)
        accuracy["reference"] = ("FP64 oracle on the CPU-baseline windows' interiors "
                                 "(the windows of cpu_baseline.sample)")

    # end to end through the C ABI: every step copies its inputs from pinned
    # host memory to the device, makes the fused call and copies dJ/dC and
    # eps_hat back; all of it inside the timed region
    e2e = None
    if args.e2e_steps > 0:
        e2e = run_e2e(torch, ec, args, w, prob, C, Cd, EFd, EAd, dJdC, eps, call, stream, dev,
                      world, barrier)

    variants = None
    if rank == 0 and world == 1 and not args.no_variants:
        main = {"w": w, "C": C, "Cd": Cd, "EF": EFd, "EA": EAd, "dJdC": dJdC, "kept": kept} \
            if args.workload == "cfg5" and not args.controls else None
        del call, Cd, EFd, EAd, eps
        variants = run_variants(torch, ec, synth, dev, flush_l2,
                                set(args.variant_set.split(",")), main=main)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K,
            "warmup": args.warmup, "ms_per_step": round(ms_step, 5), "higher_is_better": True,
            "controls_per_s": round(world * w.mx * w.my / (ms_step * 1e-3), 1),
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": w.name, "controls": [w.mx, w.my],
                       "yee": [w.nx, w.ny, w.nz], "radius_px": w.radius, "beta": w.beta,
                       "eta": w.eta, "wavelengths": NL, "fields": "complex64",
                       "field_origin": field_origin,
                       "slab_planes": w.slab_nk, "bc": "clamp",
                       "l2": ("256 MB buffer written then read before every step, outside the "
                              "timed events; the step's inputs also exceed L2"),
                       "l2_fetch_granularity_bytes": L2_FETCH_BYTES,
                       "parallelism": f"replicas x{world}"},
            "step_ms": {"min": round(step_ms[0], 5), "median": round(step_ms[len(step_ms) // 2], 5),
                        "max": round(step_ms[-1], 5)},
            "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e,
            "accuracy_vs_fp64_oracle": accuracy,
            "gpu_launches": int(timed_launches),
            "variants": variants,
            "clocks": clocks,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def run_e2e(torch, ec, args, w, prob, C, Cd, EFd, EAd, dJdC, eps, call, stream, dev, world,
            barrier):
    """The fused call end to end through the C ABI, from pinned host memory.

    Each step copies C and every wavelength's E_F and E_A host -> device,
    calls eps_vjp, and copies dJ/dC and eps_hat device -> host, all inside
    the timed region.  Workloads whose fields fit twice in 8 GB run two
    streams with their own device buffers, so one step's copies overlap the
    other's compute; larger ones run the steps in sequence on one set of
    buffers (the host link, not the call, sets their time)."""
    hC = torch.from_numpy(C).pin_memory()
    hEF = [torch.empty(e.shape, dtype=e.dtype, pin_memory=True) for e in EFd]
    hEA = [torch.empty(e.shape, dtype=e.dtype, pin_memory=True) for e in EAd]
    for h, d in zip(hEF + hEA, EFd + EAd):
        h.copy_(d)
    h2d = hC.numel() * 4 + sum(t.numel() * 8 for t in hEF + hEA)
    d2h = dJdC.numel() * 4 + eps.numel() * 4
    two = 2 * (h2d + d2h) <= (8 << 30)
    streams = [stream, torch.cuda.Stream(device=dev)] if two else [stream]
    sets = []
    for k in range(len(streams)):
        if k == 0:
            bufs = (Cd, EFd, EAd, dJdC, eps, call)
        else:
            C2 = torch.empty_like(Cd)
            EF2 = [torch.empty_like(t) for t in EFd]
            EA2 = [torch.empty_like(t) for t in EAd]
            G2 = torch.empty_like(dJdC)
            E2 = torch.empty_like(eps)
            bufs = (C2, EF2, EA2, G2, E2, ec.PreparedVjp(prob, C2, EF2, EA2, G2, eps_out=E2))
        hG_k = torch.empty(tuple(dJdC.shape), dtype=torch.float32, pin_memory=True)
        hE_k = torch.empty(tuple(eps.shape), dtype=torch.float32, pin_memory=True)
        sets.append(bufs + (hG_k, hE_k))

    def e2e_step(i):
        C_, EF_, EA_, G_, E_, call_, hG_, hE_ = sets[i % len(sets)]
        st = streams[i % len(streams)]
        with torch.cuda.stream(st):
            C_.copy_(hC, non_blocking=True)
            for d, h in zip(EF_ + EA_, hEF + hEA):
                d.copy_(h, non_blocking=True)
            call_(st)
            hG_.copy_(G_, non_blocking=True)
            hE_.copy_(E_, non_blocking=True)

    for i in range(2 * len(streams)):
        e2e_step(i)
    barrier()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for st in streams[1:]:
        st.wait_event(e0)
    for i in range(args.e2e_steps):
        e2e_step(i)
    for st in streams[1:]:
        done = torch.cuda.Event()
        done.record(st)
        stream.wait_event(done)
    e1.record(stream)
    torch.cuda.synchronize()
    ec.eps_sync_status()
    ms = max_over_ranks(e0.elapsed_time(e1), world, dev)
    ms_e2e = ms / args.e2e_steps
    link = link_floor(torch, dev, stream, min(h2d, 2 << 30), min(d2h, 2 << 30))
    t_in, t_out = h2d / (link["h2d_gbs"] * 1e9), d2h / (link["d2h_gbs"] * 1e9)
    floor = (max(t_in, t_out) if two else t_in + t_out) * 1e3
    link["floor_ms_per_step"] = round(floor, 4)
    link["note"] = ("pinned-buffer copy rates (up to 2 GB per copy); floor = the slower direction "
                    "with two overlapping streams, else the sum of both directions")
    link["frac"] = round(floor / ms_e2e, 4)
    out = {"value": weak_scaling_value(w.voxels, world, args.e2e_steps, ms), "unit": UNIT,
           "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
           "ms_per_step": round(ms_e2e, 4), "steps": args.e2e_steps,
           "path": ("pinned host -> device copies, eps_vjp (C ABI), device -> host copies of "
                    "dJ/dC and eps_hat; " + ("two streams with double buffers, consecutive steps "
                                             "overlap" if two else "one stream, steps in sequence")),
           "link": link}
    torch.cuda.synchronize()
    del sets, hEF, hEA, hC
    return out


# ------------------------------------------------------------------ variants

def _timed(call, flush_l2, K, torch):
    """Mean milliseconds of `call` over K steps, L2 flushed before each."""
    stream = torch.cuda.current_stream()
    for _ in range(3):
        flush_l2()
        call()
    torch.cuda.synchronize()
    tot = 0.0
    for _ in range(K):
        flush_l2()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        call()
        b.record(stream)
        b.synchronize()
        tot += a.elapsed_time(b)
    return tot / K


def _timed_pipelined(call, flush_l2, K, torch):
    """Mean milliseconds of `call` over K steps, L2 flushed before each,
    with the host running ahead: every step is bracketed by its own events
    on the stream, but nothing synchronises between steps, so the host
    work of a step (Python, autograd bookkeeping, argument marshalling)
    overlaps the device work of the steps before it, as in a training loop
    that does not read results back every step."""
    stream = torch.cuda.current_stream()
    for _ in range(3):
        flush_l2()
        call()
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(K)]
    for a, b in ev:
        flush_l2()
        a.record(stream)
        call()
        b.record(stream)
    torch.cuda.synchronize()
    return sum(a.elapsed_time(b) for a, b in ev) / K


def _device_fields(torch, shape, n, seed, dev):
    g = torch.Generator(device=dev)
    out = []
    for l in range(n):
        g.manual_seed(seed + l)
        out.append(torch.randn(tuple(shape) + (2,), generator=g, device=dev).view(torch.complex64)[..., 0]
                   .contiguous())
    return out


def run_variants(torch, ec, synth, dev, flush_l2,
                 sel=("cfg2", "cfg3", "cfg4", "precision", "morph", "opt", "coarse", "normals3d",
                      "autograd"), main=None):
    """The other workloads and forms, each timed like the main workload (L2
    flushed before every call): the BF16/FP16 field formats on the main
    cfg5 inputs (precision), cfg2, the three-wavelength cfg3, the batched
    cfg4, the differentiation form through autograd, and the widened rows.
    `main` holds the main workload's device inputs and the oracle's window
    results when the main line ran the full cfg5 workload."""
    out = {}
    peak, _ = measured_peaks()

    if "precision" in sel:
        out["cfg5_precision_8wavelengths"] = run_precision_variant(torch, ec, synth, dev,
                                                                   flush_l2, main)
    if main is not None:
        main.clear()
        torch.cuda.empty_cache()

    if "cfg2" in sel:
        out["cfg2_fp32_1wavelength"] = run_cfg2_variant(torch, ec, synth, dev, flush_l2)

    if "cfg3" in sel:
        # cfg3: 2000 x 2000 controls, 1000 x 1000 x 32, three wavelengths
        w = synth.WORKLOADS[3]
        p = ec.Problem(mx=w.mx, my=w.my, nz=w.nz, radius=w.radius, beta=w.beta)
        C = torch.from_numpy(synth.controls(w)).to(dev)
        EF = _device_fields(torch, (3, w.nx, w.ny, w.nz), 3, 2030, dev)
        EA = _device_fields(torch, (3, w.nx, w.ny, w.nz), 3, 3030, dev)
        G = torch.empty((w.mx, w.my), device=dev)
        E = torch.empty((3, w.nx, w.ny, w.nz), device=dev)
        call = ec.PreparedVjp(p, C, EF, EA, G, eps_out=E)
        ms = _timed(call, flush_l2, 20, torch)
        alg = algorithmic_bytes(w, 3)
        out["cfg3_fp32_3wavelengths"] = {"workload": w.name, "value": w.voxels / (ms * 1e-3),
                                         "unit": UNIT, "ms_per_call": round(ms, 4),
                                         "controls_per_s": round(w.mx * w.my / (ms * 1e-3), 1),
                                         "whole_call_hbm_frac": round(alg / (ms * 1e-3) / 1e9 / peak, 4)}
        del C, EF, EA, G, E, call

    if "cfg4" in sel:
        # cfg4: 64 regions of uneven size, radius and beta; batched vs per region
        regs = synth.batched_regions()
        probs, Cs, EFs, EAs = [], [], [], []
        for r, rw in enumerate(regs):
            probs.append(ec.Problem(mx=rw.mx, my=rw.my, nz=rw.nz, radius=rw.radius, beta=rw.beta))
            Cs.append(torch.from_numpy(synth.soi_layout(rw.mx, rw.my, 1004 * 1000 + r)).to(dev))
            EFs.append(_device_fields(torch, (3, rw.nx, rw.ny, rw.nz), 1, 2040 * 1000 + r, dev))
            EAs.append(_device_fields(torch, (3, rw.nx, rw.ny, rw.nz), 1, 3040 * 1000 + r, dev))
        vox = sum(rw.voxels for rw in regs)
        bv = ec.BatchedVjp(probs, Cs, EFs, EAs)
        bv()
        torch.cuda.synchronize()
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph):
            bv()
        ms_default = _timed(graph.replay, flush_l2, 20, torch)
        # the project's autotuner picks the launch form and shapes for this
        # batch (cached by the library), then the graph is captured again
        tuning = bv.autotune(reps=3)
        del graph
        torch.cuda.synchronize()
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph):
            bv()
        ms_b = _timed(graph.replay, flush_l2, 20, torch)
        # the alternatives the tuner passed over, forced one at a time (no
        # graph; the tuner's pick is restored for anything after)
        keys = ("multi", "stencil_blocks_per_sm", "scatter_blocks_per_sm", "contract_blocks_per_sm",
                "stage_components", "defer_seeds", "scatter_bulk_staging", "scatter_tile_cols",
                "concurrent_groups")
        picked = {k: tuning.get(k, 0) for k in keys}
        alternatives = {}
        for name, change in (
                ("scatter_tile_cols", {"scatter_tile_cols": 64 if picked["scatter_tile_cols"] in (0, 32)
                                       else 32}),
                ("concurrent_groups", {"concurrent_groups": 1 - picked["concurrent_groups"]})):
            if picked["multi"]:
                continue
            bv.set_tuning(**dict(picked, **change))
            alternatives[name] = dict(change, ms_per_call=round(_timed(bv, flush_l2, 20, torch), 4))
        bv.set_tuning(**picked)
        singles = [ec.PreparedVjp(p, C, ef, ea, G, eps_out=E)
                   for p, C, ef, ea, G, E in zip(probs, Cs, EFs, EAs, bv.dJdC, bv.eps)]

        def per_region():
            for c in singles:
                c()

        ms_s = _timed(per_region, flush_l2, 20, torch)
        alg4 = sum(algorithmic_bytes(rw, 1) for rw in regs)
        out["cfg4_batched_64_regions"] = {
            "regions": len(regs), "voxels": vox, "value": vox / (ms_b * 1e-3), "unit": UNIT,
            "ms_per_call": round(ms_b, 4), "algorithmic_bytes": alg4,
            "whole_call_hbm_frac": round(alg4 / (ms_b * 1e-3) / 1e9 / peak, 4),
            "per_region_launches": {
                "value": vox / (ms_s * 1e-3), "ms_per_call": round(ms_s, 4)},
            "speedup_vs_per_region": round(ms_s / ms_b, 3),
            "default_shapes_ms_per_call": round(ms_default, 4), "autotuned": tuning,
            "alternatives": dict(alternatives, note=("the tuned shapes with one field changed, "
                                                     "timed without a graph")),
            "launch": ("one CUDA graph: 1 contraction + 1 persistent mixed-radius stencil and "
                       "1 scatter launch" if tuning["multi"] else
                       "one CUDA graph: 1 contraction + 1 stencil and 1 scatter launch per "
                       "radius group")}
        del bv, graph, singles, Cs, EFs, EAs

    if "morph" in sel:
        out["cfg2_morphology"] = run_morph_variant(torch, ec, synth, dev, flush_l2)
    if "opt" in sel:
        out["optimizer_step"] = run_opt_variant(torch, ec, synth, dev, flush_l2)
    if "coarse" in sel:
        out["coarse_controls"] = run_coarse_variant(torch, ec, synth, dev, flush_l2)
    if "normals3d" in sel:
        out["forward_tensor_cfg2"] = run_tensor_variant(torch, ec, synth, dev, flush_l2)
    if "autograd" in sel:
        out["autograd_cfg3"] = run_autograd_variant(torch, ec, synth, dev, flush_l2)
    return out


def run_precision_variant(torch, ec, synth, dev, flush_l2, main):
    """cfg5 with E_F and E_A stored as per-component-scaled BF16 and FP16
    complex pairs (the J-support planes only), FP32 accumulation.  Each
    format is timed like the main line; its packed contraction is timed per
    launch by the library's events; after the timed loops, its dJ/dC is
    compared with the FP64 oracle's on the CPU-baseline windows (the error
    against the oracle, quantisation included) and with the FP32 path's."""
    w = synth.WORKLOADS[5]
    p = ec.Problem(mx=w.mx, my=w.my, nz=w.nz, radius=w.radius, beta=w.beta)
    if main is not None:
        C, EF, EA, G32, kept = main["Cd"], main["EF"], main["EA"], main["dJdC"], main["kept"]
    else:
        C = torch.from_numpy(synth.controls(w)).to(dev)
        EF = _device_fields(torch, (3, w.nx, w.ny, w.nz), 8, 2050, dev)
        EA = _device_fields(torch, (3, w.nx, w.ny, w.nz), 8, 3050, dev)
        G32 = ec.eps_vjp(p, C, EF, EA)
        kept = []
    peak, _ = measured_peaks()
    G = torch.empty((w.mx, w.my), device=dev)
    E = torch.empty((3, w.nx, w.ny, w.nz), device=dev)
    g32_max = float(G32.abs().max())
    cols = w.nx * w.ny
    res = {"workload": w.name, "unit": UNIT}
    if kept:
        res["fp32"] = oracle_errors(w, kept, G32)
    for name, ft in (("bf16", ec.EPS_FIELD_BF16X2_SCALED), ("fp16", ec.EPS_FIELD_F16X2_SCALED)):
        PF = [ec.eps_field_pack(p, ft, e) for e in EF]
        PA = [ec.eps_field_pack(p, ft, e) for e in EA]
        call = ec.PreparedVjp(p, C, PF, PA, G, eps_out=E, field_type=ft)
        ms = _timed(call, flush_l2, 10, torch)
        ec.eps_profile_start()
        for _ in range(5):
            flush_l2()
            call()
        prof = ec.eps_profile_stop()
        ec.eps_sync_status()
        n_c, t_c = prof.get("eps_vjp_contract_packed", (0, 0.0))
        c_ms = t_c / max(n_c, 1)
        np_ = ec.eps_packed_field_bytes(p, ft) - 16
        c_bytes = 8 * 2 * np_ + 16 * cols            # packed planes read, W written
        c_alg = cols * 8 * (3 * w.slab_nk + 1) * 2 * 4 + 16 * cols
        alg = 8 * w.mx * w.my + 12 * cols * w.nz + cols * 8 * (3 * w.slab_nk + 1) * 2 * 4
        torch.cuda.synchronize()
        entry = {"value": w.voxels / (ms * 1e-3), "ms_per_call": round(ms, 4),
                 "algorithmic_bytes": alg,
                 "whole_call_hbm_frac": round(alg / (ms * 1e-3) / 1e9 / peak, 4),
                 "packed_contraction": {
                     "avg_launch_ms": round(c_ms, 5),
                     "bytes_moved_per_launch": c_bytes,
                     "gbs": round(c_bytes / (c_ms * 1e-3) / 1e9, 1) if c_ms > 0 else None,
                     "frac_of_copy_peak": (round(c_bytes / (c_ms * 1e-3) / 1e9 / peak, 4)
                                           if c_ms > 0 else None),
                     "algorithmic_frac": (round(c_alg / (c_ms * 1e-3) / 1e9 / peak, 4)
                                          if c_ms > 0 else None),
                     # ncu dram read + write bytes of one launch, committed
                     # (null if the kernel changed since, or not captured)
                     "traffic": committed_traffic(f"{w.name}_{name}", PACKED_KERNEL_SOURCES)},
                 "dJdC_max_dev_vs_fp32_path": (float((G - G32).abs().max()) / g32_max
                                               if g32_max > 0 else None),
                 "packed_bytes_per_field": ec.eps_packed_field_bytes(p, ft)}
        if kept:
            entry["vs_fp64_oracle"] = oracle_errors(w, kept, G)
        res[name] = entry
        del PF, PA, call
    res["parity"] = ("errors against the FP64 oracle on the CPU-baseline windows (vs_fp64_oracle), "
                     "computed after the timed loops; tests/test_gpu_large.py gates them")
    del G, E
    return res


def run_cfg2_variant(torch, ec, synth, dev, flush_l2):
    """600 x 600 controls, 300 x 300 x 24, one wavelength: the fused call
    and its contraction's roofline (a one-wave problem: launch and phase
    latency, not bandwidth, set its time)."""
    w = synth.WORKLOADS[2]
    p = ec.Problem(mx=w.mx, my=w.my, nz=w.nz, radius=w.radius, beta=w.beta)
    C = torch.from_numpy(synth.controls(w)).to(dev)
    EFh, EAh = synth.fields(w)
    EF = [torch.from_numpy(e).to(dev) for e in EFh]
    EA = [torch.from_numpy(e).to(dev) for e in EAh]
    G = torch.empty((w.mx, w.my), device=dev)
    E = torch.empty((3, w.nx, w.ny, w.nz), device=dev)
    call = ec.PreparedVjp(p, C, EF, EA, G, eps_out=E)
    ms = _timed(call, flush_l2, 500, torch)
    ec.eps_profile_start()
    for _ in range(200):
        flush_l2()
        call()
    prof = ec.eps_profile_stop()
    ec.eps_sync_status()
    peak, kind = measured_peaks()
    n_c, t_c = prof.get("eps_vjp_contract", (0, 0.0))
    alg = algorithmic_bytes(w, 1)
    return {"workload": w.name, "value": w.voxels / (ms * 1e-3), "unit": UNIT,
            "ms_per_call": round(ms, 5),
            "whole_call_hbm_frac": round(alg / (ms * 1e-3) / 1e9 / peak, 4),
            "contraction_roofline": contraction_roofline(w, 1, t_c / max(n_c, 1), peak, kind,
                                                         committed_traffic(w.name)),
            "kernel_us_avg": {k: round(v[1] / v[0] * 1e3, 2) for k, v in prof.items()}}


def run_autograd_variant(torch, ec, synth, dev, flush_l2):
    """The differentiation form at cfg3 (2000 x 2000 controls, 1000 x 1000 x
    32) through torch.autograd.Function, two ways:

    - adjoint (the configured form): S, eps_hat = EpsAdjoint(C; E_F, E_A)
      over three wavelengths of seeded complex64 fields, then S.backward().
      One fused library call computes eps_hat, dJ/dC and S; the backward
      scales the saved dJ/dC.  Algorithmic bytes as the fused call's.
    - chain: eps_hat = EpsChain(C) (eps_forward), then backward with a real
      cotangent G [3, nx, ny, nz] (eps_vjp_real), which recomputes the
      filtered density and projection from C.  Algorithmic bytes per Yee
      column: C read twice (16 B each), eps_hat written (12 nz), G read on
      its 3 nk + 1 support planes (4 B each) and dJ/dC written (16 B)."""
    w = synth.WORKLOADS[3]
    p = ec.Problem(mx=w.mx, my=w.my, nz=w.nz, radius=w.radius, beta=w.beta)
    Cp = torch.from_numpy(synth.controls(w)).to(dev).requires_grad_(True)
    peak, _ = measured_peaks()
    cols = w.nx * w.ny
    out = {"workload": w.name, "unit": UNIT}

    EF = _device_fields(torch, (3, w.nx, w.ny, w.nz), 3, 2030, dev)
    EA = _device_fields(torch, (3, w.nx, w.ny, w.nz), 3, 3030, dev)

    def functional_step():
        Cp.grad = None
        S, eps = ec.autograd.eps_adjoint(Cp, p, EF, EA, with_eps=True)
        S.backward()

    ms_functional = _timed(functional_step, flush_l2, 20, torch)
    # the fields stay fixed between two field solves: marshal them once
    surr = ec.autograd.AdjointSurrogate(p, EF, EA, with_eps=True)

    def adjoint_step():
        Cp.grad = None
        S, eps = surr(Cp)
        S.backward()

    ms = _timed(adjoint_step, flush_l2, 20, torch)
    ms_pipe = _timed_pipelined(adjoint_step, flush_l2, 20, torch)
    torch.cuda.synchronize()
    ec.eps_profile_start()
    for _ in range(10):
        flush_l2()
        adjoint_step()
    prof = ec.eps_profile_stop()
    ec.eps_sync_status()
    alg = algorithmic_bytes(w, 3)
    assert Cp.grad is not None and bool(torch.isfinite(Cp.grad).all())
    out["adjoint_3wavelengths"] = {
        "value": w.voxels / (ms * 1e-3), "ms_per_step": round(ms, 4),
        "step": ("S, eps = AdjointSurrogate(E_F, E_A over 3 wavelengths)(C); S.backward() "
                 "(EpsAdjoint with the fields marshalled once)"),
        "functional_form_ms_per_step": round(ms_functional, 4),
        "host_ahead_ms_per_step": round(ms_pipe, 4),
        "timing": ("ms_per_step: the host synchronises after every step, so its Python and "
                   "marshalling time counts; host_ahead_ms_per_step: no synchronisation between "
                   "steps (the host's work overlaps earlier steps' device work)"),
        "kernel_us_avg": {k: round(v[1] / v[0] * 1e3, 2) for k, v in prof.items()},
        "algorithmic_bytes": alg, "achieved_gbs": round(alg / (ms * 1e-3) / 1e9, 1),
        "hbm_frac": round(alg / (ms * 1e-3) / 1e9 / peak, 4)}
    del EF, EA, surr

    gen = torch.Generator(device=dev)
    gen.manual_seed(3303)
    G = torch.randn((3, w.nx, w.ny, w.nz), generator=gen, device=dev)

    def chain_step():
        Cp.grad = None
        eps = ec.autograd.eps_chain(Cp, p)
        eps.backward(G)

    ms = _timed(chain_step, flush_l2, 20, torch)
    torch.cuda.synchronize()
    ec.eps_profile_start()
    for _ in range(10):
        flush_l2()
        chain_step()
    prof = ec.eps_profile_stop()
    ec.eps_sync_status()
    alg = cols * (16 + 12 * w.nz + 16 + (3 * w.slab_nk + 1) * 4 + 16)
    assert Cp.grad is not None and bool(torch.isfinite(Cp.grad).all())
    out["chain_real_cotangent"] = {
        "value": w.voxels / (ms * 1e-3), "ms_per_step": round(ms, 4),
        "step": "eps = EpsChain(C); eps.backward(G)",
        "kernel_us_avg": {k: round(v[1] / v[0] * 1e3, 2) for k, v in prof.items()},
        "algorithmic_bytes": alg, "achieved_gbs": round(alg / (ms * 1e-3) / 1e9, 1),
        "hbm_frac": round(alg / (ms * 1e-3) / 1e9 / peak, 4)}
    return out


def run_tensor_variant(torch, ec, synth, dev, flush_l2):
    """cfg2 forward only: eps_hat alone, with the xy off-diagonal maps, and
    with 3-D face normals and the full off-diagonal output (4 maps).  The
    forward writes 12 nz B of eps_hat per column plus 4 nz B per
    off-diagonal map: an HBM-write-bound stencil."""
    import ctypes
    w = synth.WORKLOADS[2]
    C = torch.from_numpy(synth.controls(w)).to(dev)
    peak, _ = measured_peaks()
    cols = w.nx * w.ny
    eps = torch.empty((3, w.nx, w.ny, w.nz), device=dev)
    od = torch.empty((4, w.nx, w.ny, w.nz), device=dev)
    out = {"workload": w.name}
    for name, flags, n_od in (("eps_hat", 0, 0), ("eps_hat+xy", ec.EPS_FLAG_OFFDIAG, 2),
                              ("eps_hat+3d_normals+4_offdiag",
                               ec.EPS_FLAG_OFFDIAG | ec.EPS_FLAG_NORMALS_3D, 4)):
        p = ec.Problem(mx=w.mx, my=w.my, nz=w.nz, radius=w.radius, beta=w.beta, flags=flags)
        pc = p.c_struct()
        fn = ec.lib().eps_forward
        args = (ctypes.byref(pc), ctypes.c_void_p(C.data_ptr()), ctypes.c_void_p(eps.data_ptr()),
                ctypes.c_void_p(od.data_ptr()) if n_od else None)
        stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)

        def call():
            fn(*args, stream)

        ms = _timed(call, flush_l2, 100, torch)
        alg = cols * (16 + 4 * w.nz * (3 + n_od))
        gbs = alg / (ms * 1e-3) / 1e9
        out[name] = {"us_per_call": round(ms * 1e3, 2), "algorithmic_bytes": alg,
                     "achieved_gbs": round(gbs, 1), "hbm_frac": round(gbs / peak, 4)}
    ec.eps_sync_status()
    return out


def run_morph_variant(torch, ec, synth, dev, flush_l2):
    """cfg2 with morphological filtering (Eq. 3-6): closing then opening,
    alpha = 20 (App. B), disks of diameter 40 nm and 150 nm (radius 2 and
    7.5 subpixels at 10 nm).  The fused call is timed like the main
    workload; each map kernel is timed with the library's per-kernel events
    in a separate loop.  Its parity with the FP64 oracle on the full cfg2
    problem is the business of tests/test_gpu_morph.py."""
    w = synth.WORKLOADS[2]
    p = ec.Problem(mx=w.mx, my=w.my, nz=w.nz, radius=w.radius, beta=w.beta)
    Ch = synth.controls(w)
    C = torch.from_numpy(Ch).to(dev)
    EFh, EAh = synth.fields(w)
    EF = [torch.from_numpy(e).to(dev) for e in EFh]
    EA = [torch.from_numpy(e).to(dev) for e in EAh]
    G = torch.empty((w.mx, w.my), device=dev)
    E = torch.empty((3, w.nx, w.ny, w.nz), device=dev)
    base = ec.PreparedVjp(p, C, EF, EA, G, eps_out=E)
    ms_base = _timed(base, flush_l2, 50, torch)
    res = {"workload": w.name, "unit": UNIT, "alpha": 20.0, "ops": "dilate, erode, erode, dilate",
           "base_chain_ms_per_call": round(ms_base, 4)}
    for mr in (2.0, 7.5):
        m = ec.Morph(alpha=20.0, radius=mr)
        call = ec.PreparedVjpMorph(p, m, C, EF, EA, G, eps_out=E)
        ms = _timed(call, flush_l2, 50, torch)
        torch.cuda.synchronize()
        ec.eps_profile_start()
        for _ in range(20):
            flush_l2()
            call()
        prof = ec.eps_profile_stop()
        ec.eps_sync_status()
        kern = {k: round(v[1] / v[0] * 1e3, 2) for k, v in prof.items()}
        res[f"disk_radius_{mr:g}"] = {"value": w.voxels / (ms * 1e-3), "ms_per_call": round(ms, 4),
                                      "kernel_us_avg": kern}
    return res


def run_coarse_variant(torch, ec, synth, dev, flush_l2):
    """The paper's coarse parametrisation: a 210 x 210-cell design region
    (420 x 420 subpixels, nz = 24, cfg2 slab) driven by 36 x 36 control nodes
    (Eq. 2, hat basis), fused forward + VJP with one wavelength.  Its parity
    with the FP64 oracle is the business of tests/test_gpu_coarse.py."""
    import ctypes
    import numpy as np
    mx = my = 420
    nz, ncx, ncy = 24, 36, 36
    p = ec.Problem(mx=mx, my=my, nz=nz, radius=1.0, beta=16.0)
    g = ec.Coarse(ncx, ncy)
    ch = (0.5 + 0.35 * np.random.default_rng(1006).standard_normal((ncx, ncy))).astype(np.float32)
    c = torch.from_numpy(ch).to(dev)
    shape = (3, mx // 2, my // 2, nz)
    EFh, EAh = [synth.complex_field(shape, 2006)], [synth.complex_field(shape, 3006)]
    EF = [torch.from_numpy(e).to(dev) for e in EFh]
    EA = [torch.from_numpy(e).to(dev) for e in EAh]
    dc = torch.empty((ncx, ncy), device=dev)
    E = torch.empty(shape, device=dev)
    ws = torch.empty(ec.eps_coarse_workspace_size(p, g), dtype=torch.uint8, device=dev)
    pc, gc = p.c_struct(), g.c_struct()
    ef = (ctypes.c_void_p * 1)(EF[0].data_ptr())
    ea = (ctypes.c_void_p * 1)(EA[0].data_ptr())
    fn = ec.lib().eps_vjp_coarse
    args = (ctypes.byref(pc), ctypes.byref(gc), ctypes.c_void_p(c.data_ptr()), 1, 0, ef, ea, None,
            -2.0, ctypes.c_void_p(dc.data_ptr()), ctypes.c_void_p(E.data_ptr()),
            ctypes.c_void_p(ws.data_ptr()), ws.numel())
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)

    def call():
        fn(*args, stream)

    ms = _timed(call, flush_l2, 100, torch)
    ec.eps_profile_start()
    for _ in range(20):
        flush_l2()
        call()
    prof = ec.eps_profile_stop()
    ec.eps_sync_status()
    vox = (mx // 2) * (my // 2) * nz
    return {"workload": "210x210x24 cells, 36x36 control nodes, beta 16, 1 wavelength",
            "value": vox / (ms * 1e-3), "unit": UNIT, "ms_per_call": round(ms, 4),
            "kernel_us_avg": {k: round(v[1] / v[0] * 1e3, 2) for k, v in prof.items()}}


def run_opt_variant(torch, ec, synth, dev, flush_l2):
    """One on-device optimiser iteration (Adam + gray count + Eq. 14-15) on
    the cfg2 and cfg5 control grids, L2 flushed before each call: an
    HBM-bound elementwise kernel with 32 algorithmic bytes per control (C, M,
    V read and written, G and the VJP's per-subpixel factor read)."""
    import ctypes
    peak, _ = measured_peaks()
    out = {}
    for cfg in (2, 5):
        w = synth.WORKLOADS[cfg]
        p = ec.Problem(mx=w.mx, my=w.my, nz=w.nz, radius=w.radius, beta=w.beta)
        C = torch.from_numpy(synth.controls(w)).to(dev)
        EF = _device_fields(torch, (3, w.nx, w.ny, w.nz), 1, 2000 + 10 * cfg, dev)
        EA = _device_fields(torch, (3, w.nx, w.ny, w.nz), 1, 3000 + 10 * cfg, dev)
        ws = torch.empty(ec.eps_workspace_size(p), dtype=torch.uint8, device=dev)
        G = ec.eps_vjp(p, C, EF, EA, ws=ws)      # fills the workspace for the gray count
        del EF, EA
        M, V = torch.zeros_like(C), torch.zeros_like(C)
        # tiny steps keep the design (and so the VJP workspace) meaningful
        opt = ec.OptParams(lr=1e-9, beta_min=w.beta, beta_max0=w.beta, n_iter=1 << 30)
        state = ec.eps_opt_init(opt)
        pc, oc = p.c_struct(), opt.c_struct()
        fn = ec.lib().eps_opt_step
        args = (ctypes.byref(pc), None, ctypes.byref(oc), ctypes.c_void_p(state.data_ptr()),
                ctypes.c_void_p(C.data_ptr()), ctypes.c_void_p(G.data_ptr()),
                ctypes.c_void_p(M.data_ptr()), ctypes.c_void_p(V.data_ptr()),
                ctypes.c_void_p(ws.data_ptr()), ws.numel())
        stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)

        def call():
            fn(*args, stream)

        ms = _timed(call, flush_l2, 100, torch)
        ec.eps_sync_status()
        st = ec.read_opt_state(state)
        alg = 32 * w.mx * w.my
        gbs = alg / (ms * 1e-3) / 1e9
        out[w.name] = {"controls": w.mx * w.my, "us_per_call": round(ms * 1e3, 2),
                       "algorithmic_bytes": alg, "achieved_gbs": round(gbs, 1),
                       "hbm_frac": round(gbs / peak, 4), "gray_fraction": round(st["unbinarity"], 5)}
        del C, ws, G, M, V
    return out


# ------------------------------------------------------------ reference arm

def run_reference(args, rank, world):
    """The FP64 oracle, as it stands, on the host cores (rank 0 only), on
    the main line's workload: whole calls when the workload is small enough,
    else one window x window-control window of it per step (the window's own
    seeded inputs with the workload's layout statistics, depth, filter and
    wavelength count), sized so that warm-up + steps take about two
    minutes."""
    if rank != 0:
        return
    import dataclasses

    from oracle import epschain_oracle as orc
    from paper_2505_03352_gb300 import synth
    w = main_workload(args)

    def inputs(win, index):
        ww = w if win >= min(w.mx, w.my) else dataclasses.replace(w, mx=win, my=win)
        C = synth.soi_layout(ww.mx, ww.my, 1000 * (1000 + w.cfg) + index)
        shape = synth.field_shape(ww)
        EF = [synth.complex_field(shape, 1000 * (2000 + 10 * w.cfg + l) + index)
              for l in range(w.n_lambda)]
        EA = [synth.complex_field(shape, 1000 * (3000 + 10 * w.cfg + l) + index)
              for l in range(w.n_lambda)]
        return ww, C, EF, EA

    def step(ww, C, EF, EA):
        p = orc.Problem(mx=ww.mx, my=ww.my, nz=ww.nz, radius=ww.radius, beta=ww.beta)
        t0 = time.perf_counter()
        orc.eps_hat(p, C)
        orc.vjp_fields(p, C, EF, EA)
        return ww.voxels, time.perf_counter() - t0

    # one 384 x 384-control window per step (about a second of oracle work
    # at cfg5), smaller if warm-up + steps would not fit in about two minutes
    win = min(w.mx, w.my, 384)
    _, t = step(*inputs(win, 0))
    budget = 120.0 / max(args.steps + args.warmup, 1)
    while win > 64 and t > budget:
        win = max(64, win // 2 // 2 * 2)
        _, t = step(*inputs(win, 0))
    for i in range(args.warmup):
        step(*inputs(win, 1 + i))
    vox = 0
    dt = 0.0
    for i in range(args.steps):
        v, t = step(*inputs(win, 1 + args.warmup + i))
        vox += v
        dt += t
    value = vox / dt
    whole = win >= min(w.mx, w.my)
    sample = (f"whole {w.name} problem per step" if whole else
              f"one {win} x {win}-control window ({win // 2} x {win // 2} x {w.nz} Yee cells, "
              f"{w.n_lambda} wavelengths) with the statistics of {w.name} per step, own seeded inputs")
    sample += "; numpy float64, single thread; input generation outside the timed part"
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(dt / max(args.steps, 1) * 1e3, 3), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": w.name, "controls": [w.mx, w.my], "yee": [w.nx, w.ny, w.nz],
                   "radius_px": w.radius, "beta": w.beta, "wavelengths": w.n_lambda,
                   "fields": "complex64", "parallelism": "host cores"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    rank, world, local = dist_env()
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    run_ours(args, rank, world, local)


if __name__ == "__main__":
    main()
