"""Throughput benchmark of the lattice Boltzmann Bona-Masso step on GB300.

Default workload: 3D gauge wave along x on the D3Q19 lattice, 256^3 cells,
FP32 storage and arithmetic, A = 0.1, ping-pong streaming, 1000 steps
(the 3D configuration's 256^3 FP32 case). One "step" is one full lattice
Boltzmann time step over the whole lattice (moment pass + fused
collide-and-stream kernel). Metric: lattice updates/s in Mcell*var/s
(cells x 16 fields x steps / s).

Workload "batched": the ensemble configuration, 512 independent 1D/2D
gauge-wave runs (seed 150502037; N uniform in 64..4096 for 1D and 64..512
for 2D, tau uniform in [0.51, 2], A log-uniform in [1e-3, 0.1], FP32
deviation storage) advanced by one persistent cooperative launch per step.
There one "step" is one launch in which every run advances one crossing
time (N of its steps), so 10 steps are the configuration's 10 crossings; the
runs are re-initialised after the warm-up launches.

Prints one JSON line (rank 0). Under torchrun each rank runs an independent
replica of the workload on its own GPU (the path has no exchange step), so
scaling is weak and value = units of all ranks / max time over ranks.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl lbnr|reference]
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1505_02037_gb300 import workloads as W  # noqa: E402

WORKLOADS = {
    # name: (vset, N, storage, direction, A[, wave, streaming, shift, shift field amplitude])
    "gauge3d-256-f32": (3, 256, "f32", "x", 0.1),
    "gauge3d-256-dev_bf16": (3, 256, "dev_bf16", "x", 0.1),
    "gauge3d-256-dev_f16": (3, 256, "dev_f16", "x", 0.1),
    "gauge3d-256-dev_f32": (3, 256, "dev_f32", "x", 0.1),
    "gauge3d-256-f64": (3, 256, "f64", "x", 0.1),
    "gauge3d-128-f64": (3, 128, "f64", "x", 0.1),
    "gauge3d-128-f64-diag": (3, 128, "f64", "xyz", 0.1),
    # the largest configuration's lattice: 384^3, one 68.9 GB buffer, in place
    "linear3d-384-dev_f32-aa": (3, 384, "dev_f32", "xyz", 1e-6, "linear", "aa"),
    # constant shift beta = (0.1, 0.05, -0.05): the shift-carrying launch form
    # (larger shifts raise the scheme's amplification factor; this one keeps
    # the 256^3 run stable at tau = 4.5)
    "gauge3d-256-f32-shift": (3, 256, "f32", "x", 0.1, "gauge", "auto", (0.1, 0.05, -0.05)),
    # plus a static divergence-free shear field of amplitude 0.02 (every B
    # term); A = 0.01, as the sheared coordinates stretch the metric over
    # the run's 3.9 crossing times
    "gauge3d-256-f32-shiftfield": (3, 256, "f32", "x", 0.01, "gauge", "auto",
                                   (0.05, 0.02, -0.02), 0.02),
}


def workload(name):
    t = WORKLOADS[name]
    vset, N, storage, direction, A = t[:5]
    wave = t[5] if len(t) > 5 else "gauge"
    streaming = t[6] if len(t) > 6 else "auto"
    return vset, N, storage, direction, A, wave, streaming


def shift_of(name):
    t = WORKLOADS.get(name, ())
    return t[7] if len(t) > 7 else None


def shift_field_of(name, shape, dx):
    t = WORKLOADS.get(name, ())
    if len(t) <= 8:
        return None
    return W.shear_shift3(shape, dx, t[8])


def fields_for(wave, shape, dx, A, direction, beta=None):
    if wave == "linear":
        return W.linear_wave(shape, dx, A, direction=direction, beta=beta)
    return W.gauge_wave(shape, dx, A, direction=direction, beta=beta)


BYTES = {"f64": 8, "f32": 4, "dev_f32": 4, "dev_bf16": 2, "dev_f16": 2}
DTYPE = {"f64": "f64", "f32": "f32", "dev_f32": "f32", "dev_bf16": "f32 (bf16 storage)",
         "dev_f16": "f32 (f16 storage)"}


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=None,
                   help="default 1000 (10 for the batched workload)")
    p.add_argument("--warmup", type=int, default=None,
                   help="default 10 (3 for the batched workload)")
    p.add_argument("--impl", default="lbnr", choices=["lbnr", "reference"])
    p.add_argument("--workload", default="gauge3d-256-f32",
                   choices=sorted(WORKLOADS) + ["batched", "gauge3d-256-f32-ad"])
    p.add_argument("--tau", type=float, default=4.5)
    p.add_argument("--profile-steps", type=int, default=20)
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--launches-per-crossing", type=int, default=8,
                   help="batched workload: launches per crossing time (each run advances N / this "
                        "many steps per launch, and the blocks are re-planned between launches)")
    p.add_argument("--deriv", default="sync", choices=["sync", "lag"],
                   help="time level of A and D for the batched workload (lag: one pass and "
                        "one team barrier per step)")
    p.add_argument("--no-modes", action="store_true",
                   help="skip the same-run LAG record and the one-crossing precision records")
    p.add_argument("--variant", default=None,
                   help="collide launch form by name (default: the autotuner's choice)")
    a = p.parse_args()
    batched = a.workload == "batched"
    if a.steps is None:
        a.steps = 10 if batched else 1000
    if a.warmup is None:
        a.warmup = 3 if batched else 10
    return a


def over_ranks(elapsed, units, world, device):
    """Whole-job totals of a timed region: the largest elapsed time over
    ranks and the sum of the units every rank processed (one all-reduce
    each; a no-op on one rank). Returns (elapsed_max, units_sum)."""
    import torch
    t = torch.tensor([float(elapsed)], dtype=torch.float64, device=device)
    u = torch.tensor([float(units)], dtype=torch.float64, device=device)
    if world > 1:
        import torch.distributed as dist
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), float(u.item())


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0}, "fallback"


class ClockSampler:
    """nvidia-smi samples during the timed region (SM clock, reasons)."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.samples = []
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 9:
                self.samples.append(parts)

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(s[1]) for s in self.samples if s[1].replace(".", "").isdigit()]
        mx = [float(s[2]) for s in self.samples if s[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for s in self.samples for i in range(4)
                          if s[5 + i].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(self.samples)}


from paper_1505_02037_gb300.traffic_table import (  # noqa: E402
    AD_SOURCES, BATCH_SOURCES, COLLIDE_SOURCES, source_hash)


def _traffic_entry(kernel_key, files):
    """The traffic table's entry for kernel_key if it was written by the
    capture script for the current kernel sources (else None): an entry whose
    hash differs, or that carries a hand-written note instead of a capture
    hash, is not trusted."""
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
            e = json.load(f).get(kernel_key)
    except OSError:
        return None
    if not e or "sources_note" in e or e.get("source_hash") != source_hash(files):
        return None
    return e


def profile_entry(kernel_key, field):
    """A per-cell figure from the committed ncu summaries, if it was taken on
    the current kernel sources (else None)."""
    e = _traffic_entry(kernel_key, COLLIDE_SOURCES)
    return None if e is None else e.get(field)


def traffic_for(kernel_key, cells, files=COLLIDE_SOURCES):
    """DRAM bytes per launch from the committed ncu summary, if it was taken
    on the current kernel sources (else None)."""
    e = _traffic_entry(kernel_key, files)
    return None if e is None else e["dram_bytes_per_cell"] * cells


def cpu_baseline(vset, storage, direction, A, tau, wave="gauge", seconds=12.0, beta=None,
                 field_fn=None):
    """The FP64 oracle as it stands, on this host's cores, on a bounded sample
    of the same workload (a 48^3 periodic piece of the same wave, same tau)."""
    from oracle import oracle as O
    n = 48
    shape = (n, n, n) if vset == 3 else (n, n, 1)
    o = O.Oracle(vset, shape, tau, 1 / n, slicing=0 if wave == "linear" else 1, shift=beta,
                 shift_field=field_fn(shape, 1 / n) if field_fn else None)
    f = o.init(fields_for(wave, shape, 1 / n, A, direction, beta))
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    steps, t0 = 0, time.perf_counter()
    while True:
        f = o.step(f)
        steps += 1
        el = time.perf_counter() - t0
        if el > seconds or steps >= 1000:
            break
    cells = n ** 3 if vset == 3 else n * n
    return {"value": cells * 16 * steps / el / 1e6, "unit": "Mcell*var/s", "cores": cores,
            "kind": "oracle",
            "sample": f"FP64 oracle, D3Q19 {n}^3 periodic {wave} wave (A={A}, tau={tau}), "
                      f"{steps} steps in {el:.1f} s on {cores} host threads"}


def workload_config(args, streaming_name="ping-pong"):
    vset, N, storage, direction, A, wave, _ = workload(args.workload)
    beta = shift_of(args.workload)
    return {
        "workload": f"3D {wave} wave along {direction}, D3Q19 {N}^3 periodic, "
                    f"{storage} storage, A={A}, tau={args.tau}, {streaming_name} streaming"
                    + (f", constant shift beta={beta}" if beta else "")
                    + (f", static shear shift field of amplitude {WORKLOADS[args.workload][8]}"
                       if len(WORKLOADS[args.workload]) > 8 else ""),
        "workload_key": args.workload, "cells": N ** 3, "fields": 16, "velocities": 19,
        "tau_note": "tau=0.6 of the configuration is linearly unstable for this scheme "
                    "(blows up near step 100 at any N and A); cost per step does not "
                    "depend on tau",
    }


def run_reference(args):
    """Reference arm: the FP64 oracle timed on the host cores, each step a
    bounded sample (one oracle step on a 24^3 piece of the workload)."""
    vset, N, storage, direction, A, wave, _ = workload(args.workload)
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from oracle import oracle as O
    n = 24
    beta = shift_of(args.workload)
    o = O.Oracle(vset, (n, n, n), args.tau, 1 / n, slicing=0 if wave == "linear" else 1,
                 shift=beta, shift_field=shift_field_of(args.workload, (n, n, n), 1 / n))
    f = o.init(fields_for(wave, (n, n, n), 1 / n, A, direction, beta))
    for _ in range(args.warmup):
        f = o.step(f)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        f = o.step(f)
    el = time.perf_counter() - t0
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    value = n ** 3 * 16 * args.steps / el / 1e6
    sample = (f"each step: one FP64 oracle step of a {n}^3 periodic piece of the workload "
              f"on {cores} host threads")
    line = {"impl": "reference", "metric": "lattice updates/s", "value": value,
            "unit": "Mcell*var/s", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": el / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": workload_config(args),
            "cpu_baseline": {"value": value, "unit": "Mcell*var/s", "cores": cores,
                             "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "Mcell*var/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# Batched ensemble
# ---------------------------------------------------------------------------
ENSEMBLE_SEED = 150502037


# FP64 flops per cell of the D3Q19 FP64 collide (dadd + dmul + 2 dfma thread
# instructions per cell, counted by ncu on the 64^3 gauge wave); used when
# the traffic table holds no count taken on the current sources
FP64_FLOPS_PER_CELL = 2948.0
FP64_FLOPS_SOURCE = ("ncu counts of the FP64 collide (64^3 gauge wave), last taken on the "
                     "tile-blocked layout; the traffic table holds none for these sources")

E2E_REPEATS = 3


def median_of(fn, repeats=E2E_REPEATS):
    """Median of `repeats` wall times from fn() (host-to-device bandwidth
    from pinned memory varies from one copy to the next)."""
    return statistics.median(fn() for _ in range(repeats))


def batched_config(world_rank_seed_note="", sub=8):
    return {
        "workload": "ensemble of 512 independent gauge-wave runs (seed 150502037): 1D D1Q3 "
                    "N~U{64..4096} or 2D D2Q9 NxN, N~U{64..512} (x-aligned for even run id, "
                    "(1,1) diagonal for odd), tau~U[0.51,2.0], A~logU[1e-3,0.1], 10 crossing "
                    "times (10 N steps) per run, FP32 deviation storage, one persistent "
                    "cooperative launch per step (graph-captured)" + world_rank_seed_note,
        "workload_key": "batched", "runs": 512, "fields": 16,
        "step": f"every run advances one crossing time: {sub} launches of ceil(N/{sub}) steps "
                "each, the work re-planned over the live runs before each launch; 10 steps = the "
                "whole configuration from t = 0",
        "tau_note": "every tau in [0.51, 2] is linearly unstable for this scheme; a run whose "
                    "moments turn non-finite stops at that step and only the steps actually "
                    "taken are counted",
    }


def oracle_rate_on_ensemble(specs, seconds):
    """FP64 oracle throughput (Mcell*var/s) on the first runs of the ensemble,
    50 steps each (initialisation not timed), for about `seconds`."""
    from oracle import oracle as O
    units, timed, used = 0, 0.0, 0
    for r in specs:
        o = O.Oracle(r["vset"], r["shape"], r["tau"], r["dx"])
        f = o.init(W.ensemble_fields(r))
        n = min(r["steps"], 50)
        ts = time.perf_counter()
        try:
            o.run(f, n)
        except FloatingPointError:
            pass
        timed += time.perf_counter() - ts
        units += r["shape"][0] * r["shape"][1] * 16 * n
        used += 1
        if timed > seconds:
            break
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    return units / timed / 1e6, cores, (
        f"FP64 oracle on the first {used} runs of the ensemble, {50} steps each "
        f"(initialisation untimed), {timed:.1f} s on {cores} host threads")


def run_reference_batched(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    specs = W.ensemble(seed=ENSEMBLE_SEED)
    per_step = 20.0 / max(args.steps + args.warmup, 1)
    for _ in range(args.warmup):
        oracle_rate_on_ensemble(specs, per_step)
    vals = []
    for _ in range(args.steps):
        rate, cores, sample = oracle_rate_on_ensemble(specs, per_step)
        vals.append(rate)
    value = statistics.median(vals)
    units_per_step = sum(r["shape"][0] * r["shape"][1] * 16 * r["N"] for r in specs)
    line = {"impl": "reference", "metric": "lattice updates/s", "value": value,
            "unit": "Mcell*var/s", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": units_per_step / (value * 1e6) * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": batched_config(),
            "cpu_baseline": {"value": value, "unit": "Mcell*var/s", "cores": cores,
                             "kind": "oracle", "sample": "each step: " + sample},
            "e2e": {"value": value, "unit": "Mcell*var/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# The 37-field scheme (independently evolved A_k and D_kij)
# ---------------------------------------------------------------------------
AD_N, AD_A, AD_NF = 256, 0.1, 37


def ad_config(args):
    return {"workload": f"3D gauge wave along x, D3Q19 {AD_N}^3 periodic, the 37-field scheme "
                        f"(A_k and D_kij evolved), f32 storage, A={AD_A}, tau={args.tau}, "
                        "ping-pong streaming",
            "workload_key": args.workload, "cells": AD_N ** 3, "fields": AD_NF, "velocities": 19,
            "unit_note": "a lattice update is one of the 37 variables of one cell"}


def ad_oracle_rate(args, n, steps=None, seconds=12.0):
    from oracle import oracle as O
    o = O.Oracle(3, (n, n, n), args.tau, 1 / n)
    f = o.ad_init(W.gauge_wave((n, n, n), 1 / n, AD_A))
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    done, t0 = 0, time.perf_counter()
    while True:
        f = o.ad_step(f)
        done += 1
        el = time.perf_counter() - t0
        if (steps is not None and done >= steps) or (steps is None and (el > seconds or done >= 1000)):
            break
    return n ** 3 * AD_NF * done / el / 1e6, done, el, cores


def run_reference_ad(args):
    """Reference arm for the 37-field workload: the FP64 oracle on a 24^3
    piece, one oracle step per step."""
    if int(os.environ.get("RANK", "0")) != 0:
        return
    n = 24
    ad_oracle_rate(args, n, steps=args.warmup)
    value, done, el, cores = ad_oracle_rate(args, n, steps=args.steps)
    sample = (f"each step: one FP64 oracle step of the 37-field scheme on a {n}^3 periodic piece "
              f"of the workload on {cores} host threads")
    line = {"impl": "reference", "metric": "lattice updates/s", "value": value,
            "unit": "Mcell*var/s", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": el / done * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": ad_config(args),
            "cpu_baseline": {"value": value, "unit": "Mcell*var/s", "cores": cores,
                             "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "Mcell*var/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main_ad(args):
    """The 37-field scheme on 256^3 D3Q19, FP32 storage: one fused kernel per
    step (no stencil pass), timed like the main workload."""
    import torch
    import torch.distributed as dist
    from paper_1505_02037_gb300 import lbnr
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    N = AD_N
    shape, cells = (N, N, N), N ** 3
    fields = W.gauge_wave(shape, 1 / N, AD_A).reshape(16, cells)
    stream = torch.cuda.Stream(device=dev)
    lat = lbnr.ADLattice(3, shape, args.tau, 1 / N, storage="f32", stream=stream)
    lat.init(fields)
    # the launch form: each timed over a few steps, the fastest kept
    tuning = {}
    for form, name in enumerate(lat.forms):
        lat.set_form(form)
        lat.step(1)
        tuning[name] = lat.step_timed(4) / 4
    best = min(tuning, key=tuning.get)
    lat.set_form(lat.forms.index(best))
    lat.init(fields)

    def barrier():
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
            torch.cuda.synchronize()

    lat.step(args.warmup)
    barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        barrier()
        e0.record(stream)
        lat.step(args.steps)
        e1.record(stream)
        barrier()
    ms = e0.elapsed_time(e1)
    ms_max, units_all = over_ranks(ms, cells * AD_NF * args.steps, world, dev)
    finite = True
    try:
        lat.status()
    except lbnr.NonFiniteError:
        finite = False
    # the kernel alone: events around each launch on the lattice's stream
    kms = lat.step_timed(args.profile_steps) / args.profile_steps
    alg = cells * 2 * AD_NF * 19 * 4  # every distribution read once and written once
    peaks, peak_kind = measured_peaks()
    peak = float(peaks["hbm_gbs"])
    achieved = alg / (kms * 1e-3) / 1e9
    tkey = f"k_ad_collide:gauge3d-256-f32-ad:{best}"
    line = {
        "metric": "lattice updates/s", "value": units_all / (ms_max * 1e-3) / 1e6,
        "unit": "Mcell*var/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms_max / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": dict(ad_config(args),
                       l2=f"inputs larger than L2 ({2 * AD_NF * 19 * 4 * cells / 1e9:.1f} GB of "
                          "distributions)",
                       state_finite_after_run=finite,
                       parallelism="replicas" if world > 1 else "single GPU"),
        "roofline": {"bound": "hbm", "kernel": "k_ad_collide (37-field collide-and-stream)",
                     "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                     "peak_source": f"hbm_gbs of {peak_kind}",
                     "algorithmic_bytes_per_cell": alg / cells, "avg_launch_ms": kms,
                     "traffic": traffic_for(tkey, cells, AD_SOURCES)},
        "gpu_launches": args.steps, "launch_form": f"37-field, {best}",
        "autotune_ms_per_collide": tuning,
        "clocks": clk.summary(),
    }
    if not args.no_e2e:
        hf = torch.from_numpy(fields.copy()).pin_memory()
        k = args.steps

        def once():
            barrier()
            t0 = time.perf_counter()
            lat.init(hf.numpy())
            lat.step(k)
            try:
                lat.moments()
            except lbnr.NonFiniteError:
                pass
            barrier()
            return time.perf_counter() - t0

        el, u = over_ranks(median_of(once), cells * AD_NF * k, world, dev)
        line["e2e"] = {"value": u / el / 1e6, "unit": "Mcell*var/s",
                       "h2d_bytes_per_step": hf.numel() * 8 / k,
                       "d2h_bytes_per_step": AD_NF * cells * 8 / k, "steps_per_transfer": k,
                       "repeats": E2E_REPEATS, "statistic": "median wall time"}
    lat.close()
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        value, done, el, cores = ad_oracle_rate(args, 48)
        line["cpu_baseline"] = {"value": value, "unit": "Mcell*var/s", "cores": cores,
                                "kind": "oracle",
                                "sample": f"FP64 oracle, 37-field scheme, D3Q19 48^3 periodic gauge "
                                          f"wave (A={AD_A}, tau={args.tau}), {done} steps in "
                                          f"{el:.1f} s on {cores} host threads"}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def main_batched(args):
    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    from paper_1505_02037_gb300 import autotune, lbnr

    # each rank its own ensemble (independent problems; rank 0 = the seed above)
    specs = W.ensemble(seed=ENSEMBLE_SEED + rank)
    sub = args.launches_per_crossing  # launches per crossing time
    for r in specs:
        r["steps_total"] = r["steps"]
        r["steps"] = -(-r["N"] // sub)
    cells = [r["shape"][0] * r["shape"][1] for r in specs]
    offs = np.concatenate([[0], np.cumsum(cells)]) * 16
    host = torch.empty(int(offs[-1]), dtype=torch.float64).pin_memory()
    hnp = host.numpy()
    for i, r in enumerate(specs):
        hnp[offs[i]:offs[i + 1]] = W.ensemble_fields(r).reshape(-1)
    b = lbnr.Batch(specs, storage="dev_f32", replan=True, deriv_mode=args.deriv)

    def init_all():
        for i in range(len(specs)):
            lbnr.lbnr_batch_init(b.b, i, host[offs[i]:offs[i + 1]])

    def barrier():
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
            torch.cuda.synchronize()

    init_all()
    tuning = autotune.tune_batch(b, trial_steps=16, reset=init_all)
    init_all()
    for _ in range(args.warmup):
        for _ in range(sub):
            b.run()
    b.status()
    init_all()
    plan0 = b.plan()  # the plan the timed region starts from (every run live)
    barrier()
    stream = b.stream
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        barrier()
        e0.record(stream)
        for _ in range(args.steps * sub):
            b.run()
        e1.record(stream)
        barrier()
    ms = e0.elapsed_time(e1)
    rc, per = b.status()
    taken = np.array([b.steps_done(i) for i in range(len(specs))], dtype=np.int64)
    units = float(sum(c * 16 * t for c, t in zip(cells, taken)))
    ms_max, units_all = over_ranks(ms, units, world, dev)
    qs = [3 if r["vset"] == 1 else 9 for r in specs]
    # distributions in and out, and the stencil planes (read once under SYNC;
    # read and written under LAG)
    aux_b = 14 * 4 if args.deriv == "lag" else 7 * 4
    alg = float(sum(c * t * (2 * 16 * q * 4 + aux_b) for c, t, q in zip(cells, taken, qs)))
    peaks, peak_kind = measured_peaks()
    peak = float(peaks["hbm_gbs"])
    achieved = alg / (ms * 1e-3) / 1e9
    plan = b.plan()
    nonfinite = sum(1 for x in per if x == -4)
    value = units_all / (ms_max * 1e-3) / 1e6
    line = {
        "metric": "lattice updates/s", "value": value, "unit": "Mcell*var/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms_max / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32 (f32 deviation storage)", "data": "synthetic",
        "config": dict(batched_config(sub=sub), l2="inputs larger than L2 (%.1f GB of distributions)"
                       % (sum(c * 16 * q * 4 * 2 for c, q in zip(cells, qs)) / 1e9),
                       parallelism="one ensemble per GPU" if world > 1 else "single GPU",
                       cell_steps_taken=int(taken @ np.array(cells)),
                       cell_steps_configured=int(sum(c * r["steps_total"]
                                                     for c, r in zip(cells, specs))),
                       runs_nonfinite=nonfinite, runs_timed_out=sum(1 for x in per if x == -5),
                       deriv_mode=args.deriv),
        "roofline": {"bound": "hbm", "kernel": "k_batch (persistent ensemble kernel)",
                     "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "peak_source": f"hbm_gbs of {peak_kind}",
                     "algorithmic_bytes_per_cell_step": "2*16*Q*4 + 7*4 (LAG: 14*4), Q = 3 or 9",
                     "avg_launch_ms": ms / (args.steps * sub),
                     # per-cell-step DRAM bytes of the same kernel on 16 D2Q9
                     # 256^2 runs, scaled to this run's cell-steps per launch
                     "traffic": traffic_for(f"k_batch:batched:{args.deriv}",
                                            float(taken @ np.array(cells)) / (args.steps * sub),
                                            BATCH_SOURCES)},
        "gpu_launches": args.steps * sub,
        "launch_form": f"block {plan['block']} x grid {plan['grid']}, "
                       f"graph={'yes' if plan['graphed'] else 'no'}, "
                       f"{sum(1 for x in plan0['teams'] if x > 1)} runs on teams at the start",
        "autotune_ms_per_trial": {f"{k[0]}x{k[1]}": v for k, v in tuning.items()},
        "clocks": clk.summary(),
    }
    if not args.no_e2e:
        # through the public API from pinned host fields: init every run,
        # K launches, read back every run's status and step count
        def once():
            barrier()
            t0 = time.perf_counter()
            init_all()
            for _ in range(args.steps * sub):
                b.run()
            b.status()
            barrier()
            return time.perf_counter() - t0

        el = median_of(once)
        taken2 = np.array([b.steps_done(i) for i in range(len(specs))], dtype=np.int64)
        u2 = float(sum(c * 16 * t for c, t in zip(cells, taken2)))
        el, u2 = over_ranks(el, u2, world, dev)
        line["e2e"] = {"value": u2 / el / 1e6, "unit": "Mcell*var/s",
                       "h2d_bytes_per_step": host.numel() * 8 / args.steps,
                       "d2h_bytes_per_step": len(specs) * (4 + 8) / args.steps,
                       "repeats": E2E_REPEATS, "statistic": "median wall time"}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        rate, cores, sample = oracle_rate_on_ensemble(specs, 12.0)
        line["cpu_baseline"] = {"value": rate, "unit": "Mcell*var/s", "cores": cores,
                                "kind": "oracle", "sample": sample}
    if rank == 0:
        print(json.dumps(line), flush=True)
    b.close()
    if world > 1:
        dist.destroy_process_group()


def timed_steps(lat, n):
    """Milliseconds of n steps of lat (graph launches) by CUDA events on the
    lattice's stream, synchronised on both sides."""
    import torch
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(lat.stream)
    lat.step(n)
    e1.record(lat.stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1)


def deriv_mode_records(args, line, fields, sync_ms, sync_col_ms, sync_aux_ms, vset, N, storage,
                       wave, streaming):
    """The same workload in the LAG derivative mode (reading R17): the collide
    kernel writes the next step's stencil planes itself, so a step is one
    kernel. Timed like the main run (same steps after the same warm-up)."""
    from paper_1505_02037_gb300 import autotune, lbnr
    lat = lbnr.Lattice(vset, (N, N, N), args.tau, 1 / N, storage=storage,
                       slicing=lbnr.LBNR_GEODESIC if wave == "linear" else lbnr.LBNR_HARMONIC,
                       streaming={"auto": lbnr.LBNR_STREAM_AUTO, "aa": lbnr.LBNR_STREAM_AA}[streaming],
                       deriv_mode="lag")
    lat.init(fields)
    tuning = autotune.tune(lat)
    lat.step(args.warmup)
    ms = timed_steps(lat, args.steps) / args.steps
    _, col = lat.step_timed(args.profile_steps)
    col /= args.profile_steps
    cells = N ** 3
    s = BYTES[storage]
    cb = 8 if storage == "f64" else 4
    alg = cells * (2 * 16 * 19 * s + 14 * cb)  # f in + f out + lagged planes read and written
    peak = line["roofline"].get("peak") if line["roofline"]["bound"] == "hbm" else \
        line["roofline"]["hbm"]["peak"]
    out = {
        "sync": {"ms_per_step": sync_ms, "value": cells * 16 / (sync_ms * 1e-3) / 1e6,
                 "kernels_per_step": 2, "k_aux_ms": sync_aux_ms, "k_collide_ms": sync_col_ms},
        "lag": {"ms_per_step": ms, "value": cells * 16 / (ms * 1e-3) / 1e6, "kernels_per_step": 1,
                "k_collide_ms": col, "launch_form": lat.variants[lat.variant],
                "collide_hbm_frac": alg / (col * 1e-3) / 1e9 / peak,
                "algorithmic_bytes_per_cell": alg / cells,
                "traffic": traffic_for(f"k_collide:{args.workload}-lag:{lat.variants[lat.variant]}",
                                       cells),
                "autotune_ms_per_collide": tuning},
        "note": "LAG takes A and D from the previous step's corrected alpha and gamma (the paper "
                "is silent on the time level); both are first order",
    }
    lat.close()
    return out


def precision_records(args, N, device_index):
    """FP64 against FP32 storage against FP32 deviation storage on the same
    GPU in the same run: the x-aligned gauge wave with A = 0.01 on N^3 over one
    crossing time (N steps) at tau = args.tau; for each, throughput and the
    error against the closed-form solution at t = 1 (max over fields and cells,
    relative to A), and the reduced forms' distance from the FP64 run."""
    from paper_1505_02037_gb300 import autotune, lbnr
    A, steps, cells = 0.01, N, N ** 3
    fields = W.gauge_wave((N, N, N), 1 / N, A).reshape(16, cells)
    exact = W.gauge_wave((N, 1, 1), 1 / N, A, t=steps / N).reshape(16, 1, N)
    out, ref = {}, None
    for storage in ("f64", "f32", "dev_f32"):
        lat = lbnr.Lattice(3, (N, N, N), args.tau, 1 / N, storage=storage)
        lat.init(fields)
        autotune.tune(lat)
        lat.init(fields)
        ms = timed_steps(lat, steps)
        finite = True
        try:
            m = lat.moments().reshape(16, N * N, N)
        except lbnr.NonFiniteError:
            finite, m = False, None
        rec = {"value": cells * 16 * steps / (ms * 1e-3) / 1e6, "ms_per_step": ms / steps,
               "launch_form": lat.variants[lat.variant], "finite": finite}
        if storage == "f64":
            # the FP64 step is bound by the FP64 pipe: its collide kernel's
            # flops (ncu count per cell) against the rate measured here
            flops = profile_entry(f"k_collide:gauge3d-{N}-f64:{rec['launch_form']}",
                                  "fp64_flops_per_cell")
            source = "ncu counts on the current sources (profiles/traffic.json)"
            if flops is None:
                flops, source = FP64_FLOPS_PER_CELL, FP64_FLOPS_SOURCE
            _, col = lat.step_timed(4)
            peak = lbnr.lbnr_fp64_fma_rate(lat.stream)
            rec["collide_ms"] = col / 4
            rec["fp64_peak_tflops_measured"] = peak
            ach = flops * cells / (col / 4 * 1e-3) / 1e12
            rec["alu"] = {"flops_per_cell": flops, "flops_source": source, "achieved_tflops": ach,
                          "frac": ach / peak}
        if finite:
            rec["err_vs_analytic"] = float(np.abs(m - exact).max() / A)
            if ref is None:
                ref = m
            else:
                rec["err_vs_fp64"] = float(np.abs(m - ref).max() / A)
        lat.close()
        out[storage] = rec
    out["speedup_vs_fp64"] = {k: out[k]["value"] / out["f64"]["value"] for k in ("f32", "dev_f32")}
    out["workload"] = (f"3D gauge wave along x, D3Q19 {N}^3, A={A}, tau={args.tau}, "
                       f"{steps} steps (one crossing time), ping-pong; errors relative to A")
    return out


def main():
    args = parse()
    if args.workload == "batched":
        return run_reference_batched(args) if args.impl == "reference" else main_batched(args)
    if args.workload == "gauge3d-256-f32-ad":
        return run_reference_ad(args) if args.impl == "reference" else main_ad(args)
    if args.impl == "reference":
        return run_reference(args)
    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    from paper_1505_02037_gb300 import lbnr

    vset, N, storage, direction, A, wave, streaming = workload(args.workload)
    shape = (N, N, N)
    cells = N ** 3
    Q = 19
    beta = shift_of(args.workload)
    fields = fields_for(wave, shape, 1 / N, A, direction, beta).reshape(16, cells)
    lat = lbnr.Lattice(vset, shape, args.tau, 1 / N, storage=storage,
                       slicing=lbnr.LBNR_GEODESIC if wave == "linear" else lbnr.LBNR_HARMONIC,
                       streaming={"auto": lbnr.LBNR_STREAM_AUTO,
                                  "aa": lbnr.LBNR_STREAM_AA}[streaming])
    if beta:
        lat.set_shift(beta)
    sfield = shift_field_of(args.workload, shape, 1 / N)
    if sfield is not None:
        lat.set_shift_field(sfield)
        del sfield
    lat.init(fields)

    def barrier():
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
            torch.cuda.synchronize()

    # warm-up: the autotuner's trial steps, then graph capture
    from paper_1505_02037_gb300 import autotune
    if beta:
        tuning = {}  # one launch form carries the shift terms
    elif args.variant:
        lat.set_variant(lat.variants.index(args.variant))
        tuning = {}
    else:
        tuning = autotune.tune(lat)
    form = ("P1-reread-shiftfield" if len(WORKLOADS[args.workload]) > 8
            else "P1-reread-shift" if beta else lat.variants[lat.variant])
    lat.step(args.warmup)
    barrier()
    stream = lat.stream
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        barrier()
        e0.record(stream)
        lat.step(args.steps)
        e1.record(stream)
        barrier()
    ms = e0.elapsed_time(e1)
    ms_max, units_all = over_ranks(ms, cells * 16 * args.steps, world, dev)
    finite = True
    try:
        lat.status()
    except lbnr.NonFiniteError:
        finite = False

    # constraint monitor (FP64 moments, corrections, H/M/C norms and the 16
    # lattice sums), a call made every m steps outside the step itself
    lat.constraints()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(3):
        lat.constraints()
    monitor_ms = (time.perf_counter() - t0) / 3 * 1e3

    # per-kernel durations (same steps, one launch at a time, events around each)
    ms_aux, ms_col = lat.step_timed(args.profile_steps)
    col_ms = ms_col / args.profile_steps
    aux_ms = ms_aux / args.profile_steps
    s = BYTES[storage]
    cbytes = 8 if storage == "f64" else 4
    alg_collide = cells * (2 * 16 * Q * s + 7 * cbytes)  # f in + f out + stencil planes once
    alg_aux = cells * (7 * Q * s + 7 * cbytes)
    peaks, peak_kind = measured_peaks()
    # burst figure: the kernel is timed as one launch of a few milliseconds
    peak = float(peaks["hbm_gbs"])
    achieved = alg_collide / (col_ms * 1e-3) / 1e9
    tkey = f"k_collide:{args.workload}:{form}"
    traffic = traffic_for(tkey, cells)
    hbm_roofline = {"bound": "hbm", "kernel": "k_collide (fused collide-and-stream)",
                    "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                    "peak_source": f"hbm_gbs of {peak_kind}",
                    "algorithmic_bytes_per_cell": alg_collide / cells,
                    "avg_launch_ms": col_ms, "traffic": traffic}
    roofline = hbm_roofline
    flops = profile_entry(tkey, "fp64_flops_per_cell") if storage == "f64" else None
    flops_source = "ncu counts on the current sources (profiles/traffic.json)"
    if storage == "f64" and flops is None:
        flops, flops_source = FP64_FLOPS_PER_CELL, FP64_FLOPS_SOURCE
    if flops is not None:
        # FP64 is bound by the FP64 pipe: its peak is the rate a register
        # FMA-chain kernel sustains on this GPU, measured here
        fp64_peak = lbnr.lbnr_fp64_fma_rate(lat.stream)
        ach = flops * cells / (col_ms * 1e-3) / 1e12
        roofline = {"bound": "alu", "kernel": "k_collide (fused collide-and-stream, FP64)",
                    "achieved": ach, "peak": fp64_peak, "unit": "TFLOP/s", "frac": ach / fp64_peak,
                    "peak_source": "measured in this run: FP64 FMA chains at full occupancy "
                                   "(lbnr_fp64_fma_rate)",
                    "flops_per_cell": flops, "flops_source": flops_source,
                    "avg_launch_ms": col_ms, "traffic": traffic, "hbm": hbm_roofline}

    value = units_all / (ms_max * 1e-3) / 1e6
    line = {
        "metric": "lattice updates/s", "value": value, "unit": "Mcell*var/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms_max / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": DTYPE[storage], "data": "synthetic",
        "config": dict(
            workload_config(args, "ping-pong" if lat.streaming == 1 else "AA in-place"),
            l2=f"inputs larger than L2 ({lat.workspace.numel() / 1e9:.1f} GB working set)",
            state_finite_after_run=finite,
            parallelism="replicas" if world > 1 else "single GPU"),
        "roofline": roofline,
        "kernels_ms_per_step": {"k_aux": aux_ms, "k_collide": col_ms,
                                "k_aux_frac_of_peak": alg_aux / (aux_ms * 1e-3) / 1e9 / peak},
        "step_algorithmic_hbm_frac": (alg_collide + alg_aux) / (ms_max / args.steps * 1e-3)
                                     / 1e9 / peak,
        "constraint_monitor_ms_per_call": monitor_ms,
        "gpu_launches": 2 * args.steps,
        "launch_form": form,
        "autotune_ms_per_collide": tuning,
        "clocks": clk.summary(),
    }

    if not args.no_e2e:
        # End to end through the public API with host buffers: pinned host
        # fields -> lbnr_init -> lbnr_step(K) -> lbnr_moments into pinned host.
        hf = torch.from_numpy(fields.copy()).pin_memory()
        hout = torch.empty((16, cells), dtype=torch.float64).pin_memory()
        k = args.steps

        def once():
            barrier()
            t0 = time.perf_counter()
            lat.init(hf)
            lat.step(k)
            try:
                lat.moments(hout)
            except lbnr.NonFiniteError:
                pass
            barrier()
            return time.perf_counter() - t0

        el, u_e2e = over_ranks(median_of(once), cells * 16 * k, world, dev)
        line["e2e"] = {"value": u_e2e / el / 1e6, "unit": "Mcell*var/s",
                       "h2d_bytes_per_step": hf.numel() * 8 / k,
                       "d2h_bytes_per_step": hout.numel() * 8 / k,
                       "steps_per_transfer": k, "repeats": E2E_REPEATS,
                       "statistic": "median wall time"}

    if not args.no_modes and not beta and len(WORKLOADS[args.workload]) <= 8:
        lat.close()
        del lat
        line["deriv_modes"] = deriv_mode_records(args, line, fields, ms_max / args.steps, col_ms,
                                                 aux_ms, vset, N, storage, wave, streaming)
        if storage in ("f32", "dev_f32") and wave == "gauge" and direction == "x":
            line["precision_one_crossing"] = precision_records(args, N, local)

    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(
            vset, storage, direction, A, args.tau, wave, beta=beta,
            field_fn=(lambda sh, dx: shift_field_of(args.workload, sh, dx))
            if len(WORKLOADS[args.workload]) > 8 else None)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
