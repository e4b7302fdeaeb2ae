"""Host-side pieces of the benchmark, without a GPU: the algorithmic byte
counts against the per-column figures of the measurement plan (C read 16 B,
dJ/dC write 16 B, eps_hat write 12 nz B, 544 B of J-support field planes per
wavelength), the committed ncu traffic used only for the kernel source it
was taken on, the roofline peak, and the reference arm's JSON line."""

import json
import os
import subprocess
import sys

import numpy as np
import pytest

import bench
from paper_2505_03352_gb300 import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.mark.parametrize("cfg,nl,per_column", [(2, 1, 864), (3, 3, 2048), (5, 8, 4768)])
def test_algorithmic_bytes_per_column(cfg, nl, per_column):
    w = synth.WORKLOADS[cfg]
    cols = w.nx * w.ny
    assert bench.algorithmic_bytes(w, nl) == per_column * cols


def test_cfg2_call_and_contraction_bytes():
    w = synth.WORKLOADS[2]
    assert bench.algorithmic_bytes(w, 1) == 77_760_000
    assert bench.contraction_bytes(w, 1) == 50_400_000      # 544 + 16 B per column


def test_committed_traffic_needs_the_current_kernel_source(monkeypatch):
    w = synth.WORKLOADS[2]
    with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
        rec = json.load(f)[w.name]
    monkeypatch.setattr(bench, "kernel_hash", lambda sources=None: rec["kernel_hash"])
    assert bench.committed_traffic(w.name) == rec["bytes_per_launch"]
    assert rec["bytes_per_launch"] == rec["dram_read_bytes"] + rec["dram_write_bytes"]
    monkeypatch.setattr(bench, "kernel_hash", lambda sources=None: "0" * 16)
    assert bench.committed_traffic(w.name) is None
    assert bench.committed_traffic("no such workload") is None


def test_packed_traffic_record_is_keyed_by_the_packed_kernel_source(monkeypatch):
    # the precision variant's record hashes the packed contraction's own
    # source, not the FP32 contraction's
    name = synth.WORKLOADS[5].name + "_bf16"
    with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
        rec = json.load(f)[name]
    assert rec["kernel_files"] == bench.PACKED_KERNEL_SOURCES
    assert rec["bytes_per_launch"] == rec["dram_read_bytes"] + rec["dram_write_bytes"]
    seen = []

    def fake_hash(sources=None):
        seen.append(sources)
        return rec["kernel_hash"] if sources == bench.PACKED_KERNEL_SOURCES else "0" * 16

    monkeypatch.setattr(bench, "kernel_hash", fake_hash)
    assert bench.committed_traffic(name, bench.PACKED_KERNEL_SOURCES) == rec["bytes_per_launch"]
    assert bench.committed_traffic(name) is None
    assert seen == [bench.PACKED_KERNEL_SOURCES, None]


def test_measured_peak_is_the_driver_copy_rate():
    peak, kind = bench.measured_peaks()
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            assert peak == pytest.approx(json.load(f)["hbm_gbs"])
        assert kind == "measured"
    else:
        assert (peak, kind) == (6800.0, "fallback")


def test_reference_arm_prints_one_json_line():
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1",
                        "--warmup", "1"], cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC and d["unit"] == bench.UNIT
    assert d["value"] > 0 and d["higher_is_better"] is True
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}


def test_cpu_baseline_times_the_oracle_on_a_bounded_sample():
    w = synth.WORKLOADS[1]
    C = synth.controls(w)
    EF, EA = synth.fields(w)
    cpu, kept = bench.cpu_baseline(w, C, EF, EA, budget_s=0.5, keep=1)
    assert cpu["kind"] == "oracle" and cpu["cores"] == 1 and cpu["unit"] == bench.UNIT
    assert cpu["value"] > 0 and 0 < cpu["seconds"] < 60
    assert w.name in cpu["sample"]
    # the kept result is the oracle's own: the error of the oracle against
    # itself is zero, and a perturbed copy shows its perturbation
    (a0, b0, win, g_ref, e_ref), = kept
    err = bench.oracle_errors(w, kept, g_ref.astype(np.float32), e_ref.astype(np.float32))
    assert err["dJdC_max_abs_err_over_max_abs_oracle"] < 1e-6
    assert err["eps_hat_max_rel_err"] < 1e-6
    bumped = g_ref.copy()
    bumped[3, 5] += 0.01 * np.max(np.abs(g_ref))
    assert abs(bench.oracle_errors(w, kept, bumped)["dJdC_max_abs_err_over_max_abs_oracle"]
               - 0.01) < 1e-9
    allc = cpu["all_cores"]
    from oracle import timing_pool
    assert allc["cores"] == timing_pool.default_workers() and allc["value"] > 0, allc
    assert 1 <= timing_pool.default_workers() <= 32
    assert timing_pool.default_workers(per_worker_bytes=1 << 50) == 1     # memory caps the pool


def test_cpu_baseline_windows_and_their_interiors():
    # window mode: seeded windows of a larger problem, and the error helper
    # compares only window interiors (a margin of 2 ceil(R) + 8 subpixels
    # from every window edge inside the region)
    import dataclasses
    w = dataclasses.replace(synth.WORKLOADS[2], mx=160, my=160, name="cfg2_crop160")
    C = synth.controls(w)
    EF, EA = synth.fields(w, 1)
    cpu, kept = bench.cpu_baseline(w, C, EF, EA, budget_s=0.2, window=64, max_windows=2,
                                   all_cores_reps=0, keep=2)
    assert "windows of 64 x 64 controls" in cpu["sample"] and len(kept) >= 1
    from oracle import epschain_oracle as orc
    op = orc.Problem(mx=w.mx, my=w.my, nz=w.nz, radius=w.radius, beta=w.beta)
    g_full = orc.vjp_fields(op, C, EF, EA)
    e_full = orc.eps_hat(op, C)
    err = bench.oracle_errors(w, kept, g_full, e_full)
    assert err["dJdC_max_abs_err_over_max_abs_oracle"] < 1e-12
    assert err["eps_hat_max_rel_err"] < 1e-12


def test_gpu_arm_runs_end_to_end_on_a_stand_in_device():
    # bench.py's GPU arm, every variant included, driven on the CPU with
    # torch.cuda and the library stubbed (tests/_bench_stand_in.py): its host
    # logic must produce the one JSON line with every key of the contract
    r = subprocess.run([sys.executable, os.path.join(ROOT, "tests", "_bench_stand_in.py")],
                       cwd=ROOT, capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-3000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
              "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config", "roofline",
              "cpu_baseline", "e2e", "gpu_launches", "clocks"):
        assert k in d, k
    assert d["metric"] == bench.METRIC and d["unit"] == bench.UNIT and d["n_gpus"] == 1
    assert {"bound", "achieved", "peak", "unit", "frac", "traffic"} <= set(d["roofline"])
    rf = d["roofline"]
    if rf["traffic"]:                       # the committed capture matches the kernel source
        assert rf["layout_ceiling_frac"] == round(rf["algorithmic_bytes_per_launch"]
                                                  / rf["traffic"], 4)
        assert rf["dram_frac"] > 0
    assert d["config"]["workload"] == synth.WORKLOADS[5].name and d["config"]["wavelengths"] == 8
    assert {"value", "unit", "cores", "kind", "sample"} <= set(d["cpu_baseline"])
    assert d["e2e"]["h2d_bytes_per_step"] > 0 and d["e2e"]["d2h_bytes_per_step"] > 0
    assert d["gpu_launches"] > 0
    assert "dJdC_max_abs_err_over_max_abs_oracle" in d["accuracy_vs_fp64_oracle"]
    c5 = d["variants"]["cfg5_precision_8wavelengths"]
    for ft in ("bf16", "fp16"):
        assert "dJdC_max_dev_vs_fp32_path" in c5[ft] and "vs_fp64_oracle" in c5[ft]
        assert "packed_contraction" in c5[ft]
    assert "dJdC_max_abs_err_over_max_abs_oracle" in c5["fp32"]
    assert set(d["variants"]) >= {"cfg2_fp32_1wavelength", "cfg3_fp32_3wavelengths",
                                  "cfg4_batched_64_regions", "cfg5_precision_8wavelengths",
                                  "cfg2_morphology", "optimizer_step", "coarse_controls",
                                  "forward_tensor_cfg2", "autograd_cfg3"}
