#!/usr/bin/env python
"""Benchmark: guiding-centre particle-steps/s on GB300 (one JSON line on rank 0).

Workload: the perturbed Parker wind on a 256x128x256 FP32 grid (eps = 0.1, 8 modes) with
three ensembles of 10^6 electrons at 81 keV injected at r = 0.28 AU, 24 deg latitude,
lambda = 0.1, 0.5 and 1.0 AU (the three runs batched in one context). A bench step is one
gc_advance of PUSH_STEPS guiding-centre steps of every particle (dt = 0.5 s) with the
snapshot tallies armed (every 100 steps) and the cell sort every 1000 steps. The FP32
path (double-float accumulators) is the timed path; the plain FP64 path is measured on
the same workload for comparison. Inputs (268 MB grid, ~520 MB particle state) exceed
the 129 MB L2, so no flush is needed between steps.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
from __future__ import annotations

import argparse
import dataclasses
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2403_06706_gb300 import synth  # noqa: E402

LAUNCH = dict(block=128, steps_per_launch=1000, sort_every=1000)
PUSH_STEPS = 1000
TALLY = dict(cadence=100, n_mu=32, n_E=32, n_r=64, n_age=32, E_lo_keV=5.0, E_hi_keV=600.0,
             r_lo_au=0.1, r_hi_au=2.5, age_max_s=86400.0, rwin_lo_au=0.9, rwin_hi_au=1.1,
             age_young_s=1200.0)
METRIC = "GC particle-steps/s on 1 GB300: plain FP64 vs FP32/neural-field at stated error"
UNIT = "particle-steps/s"
# FP32 work one particle-step of the FP32 path executes: two field evaluations (gather 236
# + right-hand side 228 flop each, the directional derivatives of Eqs. 1-2 all taken along
# v_par b + v_E) plus predictor, corrector, free path and shell test (71 flop) and the five
# double-float accumulations (4 additions each); FMA = 2 flop, sqrt / rcp / div / atan2 /
# floor = 1 each. The FP64 path accumulates with one addition each. The method's nominal
# work for the same step is larger: about 2.0 kflop in the natural formulation (8-corner
# weights for value and gradient of 8 channels, full Jacobians), 3400 flop as the FP64
# oracle's plain definitions execute it (oracle/opcount.cpp). The roofline's `achieved`
# takes the method's algorithmic figure, 2.0 kflop per particle-step; the fraction of the
# executed count and the issue ceiling are reported beside it.
FLOP_PER_PSTEP = 2 * (236 + 228) + 71 + 5 * 4
FLOP_PER_PSTEP_FP64 = 2 * (236 + 228) + 71 + 5
FLOP_PER_PSTEP_NOMINAL = 2000
# FP32 peak from the unit counts (152 SMs x 128 FP32 lanes x 2 flop x 2.07 GHz), reported
# beside the measured one (gc_fma_peak)
FP32_PEAK_DERIVED_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12
FP64_PEAK_NOMINAL_TFLOPS = 1.25  # nominal dense FP64 of a GB300
# ncu counters of the push kernels (DRAM bytes of one launch, thread instructions per
# particle-step, FP64 pipe activity), with the sha256 of the kernel sources they were taken on
COUNTERS_FILE = os.path.join(ROOT, "profiles", "push_counters.txt")
COUNTER_SOURCES = ("gc_push.cu", "gc_device.cuh", "gc_internal.h", "unit_circle_table.h")
SM_REASONS = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
# Neural field: tensor-core work of one evaluation with its Jacobian (value + 3 tangent
# rows through three 256 x 256 layers and the 256 x 8 output layer, FMA = 2 flop)
NEURAL_FLOP_PER_EVAL = 3 * 4 * 256 * 256 * 2 + 4 * 256 * 8 * 2
# the neural path is timed over a steady window of NEURAL_TIMED_CALLS calls of
# NEURAL_STEPS_PER_CALL push steps (10^3 steps) after one warm-up call; the large workload's
# network push over LARGE_CALLS calls of LARGE_NEURAL_STEPS
NEURAL_STEPS_PER_CALL = 100
NEURAL_TIMED_CALLS = 10
LARGE_NEURAL_STEPS = 10
# SIREN parameters: BF16 hidden and output weights (3 x 256 x 256 + 8 x 256), FP32 first-layer
# weights and biases (256 x 3 + 4 x 256 + 8)
NETWORK_BYTES = 2 * (3 * 65536 + 2048) + 4 * (768 + 4 * 256 + 8)
# timed advance calls per path on the large workload (after one warm-up call)
LARGE_CALLS = 2


def push_counters() -> dict:
    """The ncu counters of the push kernels, or {"stale": True, ...} without them when the
    kernel sources have changed since they were taken."""
    import hashlib

    vals, h = {}, hashlib.sha256()
    for name in COUNTER_SOURCES:
        with open(os.path.join(ROOT, "paper_2403_06706_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    try:
        for line in open(COUNTERS_FILE):
            parts = line.split("#", 1)[0].split()
            if len(parts) == 2:
                vals[parts[0]] = parts[1]
    except OSError:
        return {"stale": True, "reason": "no counters file"}
    if vals.get("kernel_sources_sha256") != h.hexdigest():
        return {"stale": True, "reason": "kernel sources changed since the ncu capture"}
    out = {"stale": False}
    for k, v in vals.items():
        if k != "kernel_sources_sha256":
            out[k] = float(v)
    return out


def workload(n_per_lambda: int = 1_000_000):
    return synth.c2_perturbed(n_per_lambda=n_per_lambda)


def config_dict(wl, n_per_rank):
    return {
        "workload": wl.name,
        "grid": f"{wl.wind.n_r}x{wl.wind.n_th}x{wl.wind.n_ph}x8 f32, r {wl.wind.r_min_au}-{wl.wind.r_max_au} AU",
        "perturbation": {"eps": wl.wind.eps, "modes": wl.wind.n_modes},
        "particles_per_gpu": n_per_rank,
        "lambda_au": [e.lam_au for e in wl.ensembles],
        "energy_keV": 81.0,
        "dt_s": wl.dt,
        "push_steps_per_step": PUSH_STEPS,
        "tally_cadence": TALLY["cadence"],
        "sort_every": LAUNCH["sort_every"],
        "l2": "inputs larger than L2 (268 MB grid, ~520 MB particle state per GPU); no flush",
    }


class ClockSampler:
    """nvidia-smi clock / throttle samples of one GPU while the timed region runs."""

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def __enter__(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             + ",".join("clocks_event_reasons." + r for r in SM_REASONS))
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={q}", "--format=csv,noheader,nounits",
                                          "-lms", "200", "-i", str(self.index)],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (FileNotFoundError, OSError):
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if self.proc is None or not self.path or not os.path.exists(self.path):
            return None
        sm, mx, reasons = [], [], set()
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 5 + len(SM_REASONS):
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for name, v in zip(SM_REASONS, parts[5:5 + len(SM_REASONS)]):
                if v.lower() == "active":
                    reasons.add(name)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def _oracle_setup(wl, nodes, n_per_ens):
    """The FP64 oracle's field, parameters, ensembles and the injected state of the first
    n_per_ens ids of every ensemble of `wl` (the ids the GPU path gives them)."""
    import oracle
    from oracle import AU

    f = oracle.grid_field(nodes, wl.wind.r_min_au * AU, wl.wind.r_max_au * AU)
    p = oracle.params(seed=wl.seed)
    oe = [oracle.ensemble(r0_au=e.r0_au, lat_deg=e.lat_deg, lon_deg=e.lon_deg, E0_keV=e.E0_keV,
                          lam_au=e.lam_au, r_in_au=e.r_in, r_out_au=e.r_out_au, energy_law=e.energy_law,
                          E_lo_keV=e.E_lo_keV, E_hi_keV=e.E_hi_keV, E_index=e.E_index, mu_law=e.mu_law,
                          scatter_law=e.scatter_law)
          for e in wl.ensembles]
    first = np.cumsum([0] + [e.count for e in wl.ensembles])[:-1]
    parts = []
    for k, f0 in enumerate(first):
        counts = [0] * len(oe)
        counts[k] = min(n_per_ens, wl.ensembles[k].count)
        parts.append(oracle.inject(f, p, oe, counts, id0=int(f0), dt=wl.dt))
    st = oracle.StateArrays({k: np.concatenate([q[k] for q in parts], axis=-1) for k in parts[0].arrays})
    return f, p, oe, st


def _oracle_run(wl, nodes, n_per_ens, cores, seconds=None, n_steps=None, pilot_steps=50):
    """Advance the first n_per_ens ids of every ensemble of `wl` with the FP64 oracle on
    `cores` threads: `n_steps` steps from injection, or, after a pilot of `pilot_steps`, as
    many as take about `seconds`. Returns (particles, timed steps, wall seconds)."""
    import oracle

    f, p, oe, st = _oracle_setup(wl, nodes, n_per_ens)
    k0 = 0
    if n_steps is None:
        t0 = time.perf_counter()
        oracle.advance(f, p, oe, st, 0.0, 0, wl.dt, pilot_steps, n_threads=cores)
        pilot = time.perf_counter() - t0
        k0 = pilot_steps
        n_steps = int(max(pilot_steps, min(40000, pilot_steps * seconds / max(pilot, 1e-3))))
    t0 = time.perf_counter()
    oracle.advance(f, p, oe, st, k0 * wl.dt, k0, wl.dt, n_steps, n_threads=cores)
    return st.n, n_steps, time.perf_counter() - t0


def cpu_baseline(wl, nodes, seconds=10.0):
    """The FP64 oracle as it stands, on the host cores: the first 4096 ids of every
    ensemble of the workload, advanced for about `seconds` after 50 steps from injection; the
    same sample on one core; and the plain 64x32x64 FP64 workload (4096 electrons, 3600
    steps) in full on all cores, and for about five seconds on one core."""
    cores = os.cpu_count() or 1
    n, k, el = _oracle_run(wl, nodes, 4096, cores, seconds=seconds)
    out = {"value": n * k / el, "unit": UNIT, "cores": cores, "kind": "oracle",
           "sample": f"{n} particles (first 4096 ids of each lambda ensemble) x {k} "
                     f"steps after 50 from injection, FP64 oracle on the same FP32 grid values, "
                     f"{el:.1f} s wall"}
    n, k, el = _oracle_run(wl, nodes, 4096, 1, seconds=seconds / 2)
    out["single_core"] = {"value": n * k / el, "unit": UNIT, "cores": 1,
                          "sample": f"the same {n} particles x {k} steps after 50, {el:.1f} s wall"}
    w1 = synth.c1_plain_fp64()
    nodes1 = synth.wind_grid(w1.wind, dtype=np.float64)
    n, k, el = _oracle_run(w1, nodes1, w1.n_particles, cores, n_steps=w1.n_steps)
    n1, k1, el1 = _oracle_run(w1, nodes1, w1.n_particles, 1, seconds=5.0)
    out["plain_fp64_workload"] = {
        "workload": w1.name, "value": n * k / el, "unit": UNIT, "cores": cores,
        "sample": f"in full: {n} particles x {k} steps from injection, {el:.1f} s wall",
        "single_core": {"value": n1 * k1 / el1, "unit": UNIT, "cores": 1,
                        "sample": f"{n1} particles x {k1} steps after 50 from injection, {el1:.1f} s wall"}}
    return out


def run_reference(args, rank, world):
    """Reference arm: the FP64 oracle timed on the host cores (rank 0 only)."""
    if rank != 0:
        return
    import oracle

    wl = workload()
    nodes = synth.wind_grid(wl.wind, dtype=np.float32)
    f, p, oe, st = _oracle_setup(wl, nodes, 512)
    cores = os.cpu_count() or 1
    ref_steps = 2000  # push steps per bench step of this arm
    t, k = 0.0, 0
    for _ in range(args.warmup):
        oracle.advance(f, p, oe, st, t, k, wl.dt, ref_steps, n_threads=cores)
        t += ref_steps * wl.dt
        k += ref_steps
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.advance(f, p, oe, st, t, k, wl.dt, ref_steps, n_threads=cores)
        t += ref_steps * wl.dt
        k += ref_steps
    el = time.perf_counter() - t0
    value = st.n * ref_steps * args.steps / el
    sample = (f"{st.n} particles (first 512 ids of each lambda ensemble) x {ref_steps} steps per "
              f"bench step, FP64 oracle, {cores} host threads")
    config = config_dict(wl, sum(e.count for e in wl.ensembles))
    config["timed_sample"] = {"particles": st.n, "push_steps_per_step": ref_steps,
                              "ids": "the first 512 of each lambda ensemble"}
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": el / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": config,
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def _fit_siren(c, w, X, schedule):
    """Train the context's SIREN on X["n_samples"] uniform-in-volume samples of its loaded
    grid with the given (epochs, Adam step) schedule; returns the per-epoch losses and the
    seconds taken."""
    import torch

    xs = torch.from_numpy(synth.siren_samples(X["n_samples"], w)).to("cuda")
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    losses = [c.field_fit(xs, n_epochs=ep, batch=X["batch"], lr=lr) for ep, lr in schedule]
    torch.cuda.synchronize()
    t_fit = time.perf_counter() - t0
    del xs
    return np.concatenate(losses), t_fit


def _siren_error(c, w):
    """RMS error of the network against the grid interpolant on 2^20 held-out points, relative
    to the RMS of the (scaled) channel groups B, E and |B|."""
    import torch

    xv = torch.from_numpy(synth.siren_samples(1 << 20, w, seed=1)).to("cuda")
    y = torch.empty((xv.shape[0], 8), device="cuda")
    t = torch.empty((xv.shape[0], 8), device="cuda")
    c.siren_eval(xv, y)
    c.field_targets(xv, t)
    torch.cuda.synchronize()
    d = (y - t).double()
    return {g: float(torch.sqrt((d[:, sl] ** 2).mean() / (t[:, sl].double() ** 2).mean()))
            for g, sl in (("B", slice(0, 3)), ("E", slice(3, 6)), ("absB", slice(6, 7)))}


def _training_dict(X, schedule, loss, t_fit):
    n_ep = sum(ep for ep, _ in schedule)
    return {"samples": X["n_samples"], "epochs": n_ep, "batch": X["batch"],
            "schedule": [[ep, lr] for ep, lr in schedule],
            "seconds": t_fit, "samples_per_s": X["n_samples"] * n_ep / t_fit,
            "loss_first_epoch": float(loss[0]) if len(loss) else None,
            "loss_last_epoch": float(loss[-1]) if len(loss) else None}


def _timed_calls(c, stream, dt, n_steps, n_calls):
    """Device milliseconds of n_calls advance calls of n_steps each (CUDA events on the
    context's stream)."""
    import torch

    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(n_calls):
        c.advance(dt, n_steps)
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1)


def neural_bench(args, nodes, local, stream, rank):
    """The neural-field path: train the SIREN on samples of the grid interpolant, measure its
    field error against the grid, then time the split-step push with the network as the
    field source (10^7 electrons)."""
    from paper_2403_06706_gb300 import gcpush, shard

    wn = synth.c4_neural(args.neural_particles)
    X = wn.extra
    epochs = X["epochs"] if args.neural_epochs is None else args.neural_epochs
    w = wn.wind
    c = gcpush.Context(precision=gcpush.PREC_FP32_MIXED, device=local, stream=stream, seed=wn.seed, dt_init=wn.dt,
                       id_base=shard.id_base(rank, wn.n_particles))
    c.field_load(nodes, w.r_min_au, w.r_max_au)
    c.siren_set(synth.siren_init(seed=0), omega0=X["omega0"], r_max_au=w.r_max_au, B_scale=w.B1,
                E_scale=w.B1 * w.u_sw)
    schedule = X["schedule"] if args.neural_epochs is None else ((epochs, X["lr"]),)
    loss, t_fit = _fit_siren(c, w, X, schedule)
    err = _siren_error(c, w)
    # push with the network as the field source
    c.field_select(gcpush.FIELD_SIREN)
    c.inject(list(wn.ensembles))
    c.advance(wn.dt, NEURAL_STEPS_PER_CALL)
    s0 = c.stats()
    ms = _timed_calls(c, stream, wn.dt, NEURAL_STEPS_PER_CALL, NEURAL_TIMED_CALLS)
    s1 = c.stats()
    n = wn.n_particles
    evals = s1["field_evals"] - s0["field_evals"]
    fms = s1["field_ms"] - s0["field_ms"]
    achieved = NEURAL_FLOP_PER_EVAL * evals / (fms / 1e3) / 1e12
    peaks = _measured_peaks()
    peak = peaks.get("bf16_tflops_sustained")
    c.close()
    return {
        "workload": wn.name, "particles": n,
        "value": n * NEURAL_STEPS_PER_CALL * NEURAL_TIMED_CALLS / (ms / 1e3),
        "unit": UNIT, "ms_per_step": ms / (NEURAL_TIMED_CALLS * NEURAL_STEPS_PER_CALL),
        "push_steps": NEURAL_TIMED_CALLS * NEURAL_STEPS_PER_CALL, "warmup_push_steps": NEURAL_STEPS_PER_CALL,
        "roofline": {"bound": "tensor", "kernel": "siren_eval_kernel", "achieved": achieved,
                     "peak": peak, "unit": "TFLOP/s", "frac": (achieved / peak) if peak else None,
                     "peak_basis": "measured bf16 cuBLAS, sustained (MEASURED_PEAKS.json)",
                     "flop_per_eval": NEURAL_FLOP_PER_EVAL, "evals": evals,
                     "eval_share_of_step": fms / ms},
        "training": _training_dict(X, schedule, loss, t_fit),
        "field_rel_rms_vs_grid": err,
        "footprint_bytes": {"network_bf16": NETWORK_BYTES, "grid_f32": int(nodes.nbytes)},
    }


def large_bench(args, local, stream, rank):
    """The large workload, grid against network: the 512x256x512 FP32 grid (2.15 GB; eps 0.2,
    16 modes), 3x10^7 electrons with an E^-3 spectrum on [20, 500] keV, lambda 0.3 AU, tallies
    of pitch x energy x r on 64 x 64 x 128 bins, pushed once with the inline grid gather and
    once with a SIREN trained on this grid (the neural workload's schedule) as the field
    source. Reports both rates, the network's field error against the grid and the two
    footprints (the smoothness side of the comparison is tests/test_gpu_gain.py)."""
    from paper_2403_06706_gb300 import gcpush, shard

    wl = synth.c5_large(args.large_particles)
    w = wl.wind
    X = synth.c4_neural().extra
    t0 = time.perf_counter()
    nodes = synth.wind_grid(w, dtype=np.float32)
    t_synth = time.perf_counter() - t0
    tally = dict(cadence=100, n_mu=64, n_E=64, n_r=128, E_lo_keV=5.0, E_hi_keV=600.0,
                 r_lo_au=w.r_min_au, r_hi_au=w.r_max_au)
    n = wl.n_particles
    out = {"workload": wl.name, "particles": n, "grid_synthesis_s": t_synth}

    def context():
        c = gcpush.Context(precision=gcpush.PREC_FP32_MIXED, device=local, stream=stream, seed=wl.seed,
                           dt_init=wl.dt, id_base=shard.id_base(rank, n))
        c.field_load(nodes, w.r_min_au, w.r_max_au)
        return c

    # the grid path: one warm-up launch, then LARGE_CALLS launches of PUSH_STEPS
    c = context()
    c.inject(list(wl.ensembles))
    c.set_launch(**LAUNCH)
    c.tally_arm(**tally)
    c.advance(wl.dt, PUSH_STEPS)
    ms = _timed_calls(c, stream, wl.dt, PUSH_STEPS, LARGE_CALLS)
    t = c.tally_read()
    out["grid"] = {"value": n * PUSH_STEPS * LARGE_CALLS / (ms / 1e3), "unit": UNIT,
                   "push_steps": PUSH_STEPS * LARGE_CALLS, "warmup_push_steps": PUSH_STEPS,
                   "tally_samples": int(t["n_seen"][0]), "tally_out_of_range": int(t["n_seen"][1])}
    c.close()

    # the neural path: the network trained on this grid, then the split-step push
    c = context()
    c.siren_set(synth.siren_init(seed=0), omega0=X["omega0"], r_max_au=w.r_max_au, B_scale=w.B1,
                E_scale=w.B1 * w.u_sw)
    loss, t_fit = _fit_siren(c, w, X, X["schedule"])
    err = _siren_error(c, w)
    c.field_select(gcpush.FIELD_SIREN)
    c.inject(list(wl.ensembles))
    c.tally_arm(**dict(tally, cadence=LARGE_NEURAL_STEPS))
    c.advance(wl.dt, LARGE_NEURAL_STEPS)
    ms = _timed_calls(c, stream, wl.dt, LARGE_NEURAL_STEPS, LARGE_CALLS)
    t = c.tally_read()
    out["neural"] = {"value": n * LARGE_NEURAL_STEPS * LARGE_CALLS / (ms / 1e3), "unit": UNIT,
                     "push_steps": LARGE_NEURAL_STEPS * LARGE_CALLS,
                     "warmup_push_steps": LARGE_NEURAL_STEPS,
                     "tally_samples": int(t["n_seen"][0]), "tally_out_of_range": int(t["n_seen"][1]),
                     "training": _training_dict(X, X["schedule"], loss, t_fit),
                     "field_rel_rms_vs_grid": err}
    c.close()
    out["grid_over_neural"] = out["grid"]["value"] / out["neural"]["value"]
    out["footprint_bytes"] = {"network_bf16": NETWORK_BYTES, "grid_f32": int(nodes.nbytes)}
    return out


def _measured_peaks() -> dict:
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except OSError:
        return {}


def _max_over_ranks(x: float, dist) -> float:
    if dist is None:
        return x
    import torch

    t = torch.tensor([x], device="cuda")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def e2e_sharded(args, wl, nodes, local, rank, n_rank, world, dist, pinned, k_steps):
    """End-to-end throughput through the public API with the rank's particles split over
    args.e2e_shards contexts, each on its own stream and driven by its own host thread:
    every step each shard copies its state in from pinned host memory (gc_particles_set),
    advances PUSH_STEPS steps (gc_advance) and copies its state and tallies out
    (gc_particles_get, gc_tally). The library releases the GIL in every call, so one
    shard's copies run while the others push."""
    import threading

    import torch

    from paper_2403_06706_gb300 import gcpush, shard

    K = max(1, args.e2e_shards)
    ctxs, hosts, tally_bytes = [], [], 0
    first = shard.id_base(rank, n_rank)
    for k in range(K):
        ens = [dataclasses.replace(e, count=e.count // K + (1 if k < e.count % K else 0)) for e in wl.ensembles]
        c = gcpush.Context(precision=gcpush.PREC_FP32_MIXED, device=local, stream=torch.cuda.Stream(),
                           seed=wl.seed, dt_init=wl.dt, id_base=first)
        first += sum(e.count for e in ens)
        c.field_load(nodes, wl.wind.r_min_au, wl.wind.r_max_au)
        c.inject(ens)
        c.set_launch(**LAUNCH)
        c.tally_arm(**TALLY)
        c.advance(wl.dt, PUSH_STEPS)
        h = gcpush.state_buffers(c.n, alloc=pinned)
        c.get_state(out=h)
        c.set_state(h)
        tally_bytes += sum(v.nbytes for v in c.tally_read().values())
        ctxs.append(c)
        hosts.append(h)
    assert sum(c.n for c in ctxs) == n_rank
    start = threading.Barrier(K + 1)
    errors = []

    def work(k):
        c, h = ctxs[k], hosts[k]
        try:
            start.wait()
            for _ in range(k_steps):
                c.set_state(h)
                c.advance(wl.dt, PUSH_STEPS)
                c.get_state(out=h)
                c.tally_read()
        except Exception as e:  # reported after the join
            errors.append(e)

    threads = [threading.Thread(target=work, args=(k,)) for k in range(K)]
    for t in threads:
        t.start()
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    t0 = time.perf_counter()
    start.wait()
    for t in threads:
        t.join()
    torch.cuda.synchronize()
    el = _max_over_ranks(time.perf_counter() - t0, dist)
    if errors:
        raise errors[0]
    nb = sum(gcpush.state_nbytes(h) for h in hosts)
    for c in ctxs:
        c.close()
    return {"value": world * n_rank * PUSH_STEPS * k_steps / el, "unit": UNIT,
            "h2d_bytes_per_step": nb, "d2h_bytes_per_step": nb + tally_bytes, "steps": k_steps,
            "contexts": K, "host_threads": K,
            "api": "per context: gc_particles_set (pinned host) + gc_advance + gc_particles_get + gc_tally"}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=("ours", "reference"))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--e2e-shards", type=int, default=4,
                    help="contexts (streams, host threads) the end-to-end population is split over")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--no-neural", action="store_true")
    ap.add_argument("--no-variants", action="store_true")
    ap.add_argument("--neural-particles", type=int, default=10_000_000)
    ap.add_argument("--neural-epochs", type=int, default=None)
    ap.add_argument("--no-large", action="store_true",
                    help="skip the large workload (512x256x512 grid against the network)")
    ap.add_argument("--large-particles", type=int, default=30_000_000)
    ap.add_argument("--particles", type=int, default=3_000_000,
                    help="particles per GPU (split over the three lambda ensembles); smaller "
                         "values are for profiler captures")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return run_reference(args, rank, world)

    import torch

    from paper_2403_06706_gb300 import gcpush, shard

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    gcpush.build()
    fp32_peak, fp64_peak = gcpush.fma_peak(local)
    counters = push_counters()
    wl = workload(args.particles // 3)
    n_rank = wl.n_particles
    nodes = synth.wind_grid(wl.wind, dtype=np.float32)
    stream = torch.cuda.current_stream()

    def barrier():
        if dist is not None:
            dist.barrier()

    # ---------------- device-resident FP32 path ---------------------------------------
    ctx = gcpush.Context(precision=gcpush.PREC_FP32_MIXED, device=local, stream=stream, seed=wl.seed,
                         dt_init=wl.dt, id_base=shard.id_base(rank, n_rank))
    ctx.field_load(nodes, wl.wind.r_min_au, wl.wind.r_max_au)
    ctx.inject(list(wl.ensembles))
    ctx.set_launch(**LAUNCH)
    ctx.tally_arm(**TALLY)
    for _ in range(args.warmup):
        ctx.advance(wl.dt, PUSH_STEPS)
    torch.cuda.synchronize()
    s0 = ctx.stats()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        barrier()
        torch.cuda.synchronize()
        ev0.record(stream)
        for _ in range(args.steps):
            ctx.advance(wl.dt, PUSH_STEPS)
        ev1.record(stream)
        torch.cuda.synchronize()
        barrier()
    el_ms = ev0.elapsed_time(ev1)
    s1 = ctx.stats()
    if dist is not None:
        t = torch.tensor([el_ms], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        el_ms = float(t.item())
    value = world * n_rank * PUSH_STEPS * args.steps / (el_ms / 1e3)
    launches = s1["push_launches"] - s0["push_launches"]
    push_ms = (s1["push_ms"] - s0["push_ms"]) / max(launches, 1)
    steps_per_launch = PUSH_STEPS * args.steps / max(launches, 1)
    pstep_rate = n_rank * steps_per_launch / (push_ms / 1e3)  # particle-steps/s of one launch
    achieved = FLOP_PER_PSTEP_NOMINAL * pstep_rate / 1e12
    executed = FLOP_PER_PSTEP * pstep_rate / 1e12
    fresh = not counters["stale"]
    same_shape = fresh and (n_rank, round(steps_per_launch)) == (counters.get("push_fp32.launch_particles"),
                                                                   counters.get("push_fp32.launch_steps"))
    instr = counters.get("push_fp32.thread_instr_per_particle_step") if fresh else None
    issue_ceiling = 152 * 4 * 32 * 2.07e9 / instr if instr else None
    roofline = {"bound": "alu", "achieved": achieved, "peak": fp32_peak, "unit": "TFLOP/s",
                "frac": achieved / fp32_peak,
                "traffic": int(counters["push_fp32.dram_bytes_per_launch"]) if same_shape else None,
                "kernel": "push_kernel<float>", "launch_ms": push_ms,
                "flop_per_particle_step": FLOP_PER_PSTEP_NOMINAL,
                "flop_basis": "the method's algorithmic work per particle-step (two field evaluations "
                              "with 8-corner value and gradient weights of 8 channels and full "
                              "Jacobians, the right-hand side, predictor and corrector)",
                "executed": {"flop_per_particle_step": FLOP_PER_PSTEP, "achieved": executed,
                             "frac": executed / fp32_peak},
                "issue": {"thread_instr_per_particle_step": instr, "ceiling_particle_steps_per_s": issue_ceiling,
                          "frac": pstep_rate / issue_ceiling if issue_ceiling else None},
                "peak_basis": "measured: gc_fma_peak (independent FP32 FMA chains on every SM, best of 10 "
                              "launches, CUDA events), taken just before the timed region",
                "peak_derived": FP32_PEAK_DERIVED_TFLOPS,
                "frac_of_derived": achieved / FP32_PEAK_DERIVED_TFLOPS,
                "counters": "profiles/push_counters.txt" + (" (stale: sources changed since the ncu capture; "
                                                             "traffic and issue left null)" if not fresh else ""),
                "push_share_of_step": (s1["push_ms"] - s0["push_ms"]) / el_ms}
    gpu_launches = s1["kernel_launches"] - s0["kernel_launches"]
    clocks = clk.summary()

    # ---------------- end to end through host buffers ---------------------------------
    e2e = None
    if not args.no_e2e:
        pinned = lambda shape, dt: torch.empty(shape, dtype={np.float64: torch.float64,
                                                              np.uint32: torch.int32}[dt],
                                               pin_memory=True).numpy().view(dt)
        k_e2e = max(1, min(args.steps, 3))
        # one context: copy in, advance, copy out, one call after the other
        host = gcpush.state_buffers(ctx.n, alloc=pinned)
        ctx.get_state(out=host)
        barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(k_e2e):
            ctx.set_state(host)
            ctx.advance(wl.dt, PUSH_STEPS)
            ctx.get_state(out=host)
            ctx.tally_read()
        torch.cuda.synchronize()
        el1 = _max_over_ranks(time.perf_counter() - t0, dist)
        single = {"value": world * n_rank * PUSH_STEPS * k_e2e / el1, "unit": UNIT, "contexts": 1}
        # the same population split over contexts on their own streams, one host thread each:
        # one shard's copies overlap the others' pushes
        e2e = e2e_sharded(args, wl, nodes, local, rank, n_rank, world, dist, pinned, k_e2e)
        e2e["single_context"] = single
    ctx.close()

    # ---------------- plain FP64 path on the same workload ----------------------------
    fp64 = None
    if not args.no_fp64:
        c64 = gcpush.Context(precision=gcpush.PREC_FP64, device=local, stream=stream, seed=wl.seed,
                             dt_init=wl.dt, id_base=shard.id_base(rank, n_rank))
        c64.field_load(nodes, wl.wind.r_min_au, wl.wind.r_max_au)
        c64.inject(list(wl.ensembles))
        c64.set_launch(**LAUNCH)
        n64 = 40
        c64.advance(wl.dt, n64)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        c64.advance(wl.dt, n64)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        v64 = world * n_rank * n64 / (ms / 1e3)
        a64 = FLOP_PER_PSTEP_FP64 * v64 / world / 1e12
        fp64 = {"value": v64, "unit": UNIT, "push_steps": n64,
                "note": "same workload, FP64 grid and arithmetic; timed after the same start-up",
                "roofline": {"bound": "fp64", "achieved": a64, "peak": fp64_peak, "unit": "TFLOP/s",
                             "frac": a64 / fp64_peak, "flop_per_particle_step": FLOP_PER_PSTEP_FP64,
                             "flop_basis": "executed (the nominal 2.0 kflop would exceed the FP64 peak: "
                                           "this kernel runs the regrouped right-hand side too)",
                             "peak_basis": "measured: gc_fma_peak (independent FP64 FMA chains on every SM)",
                             "peak_nominal": FP64_PEAK_NOMINAL_TFLOPS,
                             "fp64_pipe_active_ncu": counters.get("push_fp64.fp64_pipe_active") if fresh else None}}
        c64.close()

    # ---------------- 64 uneven ensembles, graph replay, autotuned launch shape -------------
    batched = None
    if not args.no_batched:
        wb = synth.c3_batched()
        cb = gcpush.Context(precision=gcpush.PREC_FP32_MIXED, device=local, stream=stream, seed=wb.seed,
                            dt_init=wb.dt, id_base=shard.id_base(rank, wb.n_particles))
        cb.field_load(nodes, wb.wind.r_min_au, wb.wind.r_max_au)
        cb.inject(list(wb.ensembles))
        cb.tally_arm(**TALLY)
        cb.advance(wb.dt, 1000)  # spread the ensembles out before tuning
        choice = cb.autotune(wb.dt, trial_steps=200)
        cb.set_graph(True)
        nb_steps = 500
        for _ in range(2):
            cb.advance(wb.dt, nb_steps)
        torch.cuda.synchronize()
        b0 = torch.cuda.Event(enable_timing=True)
        b1 = torch.cuda.Event(enable_timing=True)
        b0.record(stream)
        for _ in range(args.steps):
            cb.advance(wb.dt, nb_steps)
        b1.record(stream)
        torch.cuda.synchronize()
        bms = b0.elapsed_time(b1)
        batched = {"workload": wb.name, "ensembles": len(wb.ensembles), "particles": wb.n_particles,
                   "value": world * wb.n_particles * nb_steps * args.steps / (bms / 1e3), "unit": UNIT,
                   "push_steps_per_call": nb_steps, "graph": True, "autotune": choice}
        cb.close()

    # ---------------- method variants on the same workload (Sect. 3.2, Sect. 2.2) -------------
    variants = None
    if not args.no_variants:
        variants = {}
        nodes_tf = nodes.copy()
        nodes_tf[..., 7] = synth.potential_of(wl.wind, 500.0)[None, None, :].astype(nodes.dtype)
        # a time-dependent field: the wind turning faster and stronger (5e5 m/s, 4.2 nT at
        # 1 AU, another perturbation) over the variant's whole run, two snapshots blended in time
        nodes_t1 = synth.wind_grid(dataclasses.replace(wl.wind, B1=4.2e-9, u_sw=5.0e5, seed=wl.wind.seed + 1),
                                   dtype=nodes.dtype)
        window = (0.0, 3 * PUSH_STEPS * wl.dt)
        for name, opt, grid, ideal, grid1 in (("wind_frame_collisions", {"wind_u": 4.0e5}, nodes, True, None),
                                              ("two_fluid_field", {}, nodes_tf, 2, None),
                                              ("time_dependent_field", {}, nodes, True, nodes_t1)):
            cv = gcpush.Context(precision=gcpush.PREC_FP32_MIXED, device=local, stream=stream, seed=wl.seed,
                                dt_init=wl.dt, id_base=shard.id_base(rank, n_rank), **opt)
            cv.field_load(grid, wl.wind.r_min_au, wl.wind.r_max_au, ideal=ideal)
            if grid1 is not None:
                cv.field_load_next(grid1, *window)
            cv.inject(list(wl.ensembles))
            cv.set_launch(**LAUNCH)
            cv.tally_arm(**TALLY)
            cv.advance(wl.dt, PUSH_STEPS)
            torch.cuda.synchronize()
            v0 = torch.cuda.Event(enable_timing=True)
            v1 = torch.cuda.Event(enable_timing=True)
            v0.record(stream)
            for _ in range(2):
                cv.advance(wl.dt, PUSH_STEPS)
            v1.record(stream)
            torch.cuda.synchronize()
            variants[name] = {"value": world * n_rank * PUSH_STEPS * 2 / (v0.elapsed_time(v1) / 1e3),
                              "unit": UNIT, "push_steps": 2 * PUSH_STEPS,
                              "collisions": cv.stats()["collisions"]}
            cv.close()

    neural = None
    if not args.no_neural:
        neural = neural_bench(args, nodes, local, stream, rank)

    large = None
    if not args.no_large:
        large = large_bench(args, local, stream, rank)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(wl, nodes)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": el_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic (seeded Parker + solenoidal perturbation grid; injected electrons)",
            "config": config_dict(wl, n_rank),
            "parallelism": f"particles sharded by id, {world} GPU(s), no data-path collective",
            "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": gpu_launches,
            "clocks": clocks, "fp64_plain": fp64, "batched": batched, "variants": variants,
            "neural": neural, "large": large,
            "accuracy": "FP32 path within 1e-4 of the FP64 oracle over the first 1e3 steps; "
                        "FP64 path within 1e-9 (tests/test_gpu_parity.py, tests/test_gpu_fullsize.py)",
        }
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
