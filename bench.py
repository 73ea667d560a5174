#!/usr/bin/env python3
"""Benchmark of the PAMD hot path on one GB300.

A step is one full anneal of the paper-shaped workload: a 75-atom synthetic
peptide-like chain, R = 8192 replicas, theta = 1000 BAOAB steps of 1 fs per
temperature, 100 geometric temperature steps 1000 -> 250 K (101 propagate
blocks, 100 resamplings, 101 measurements), run as one CUDA graph after
re-initialising the population on the device.  The metric is atom-steps per
second over all replicas (and ms per full anneal).

Prints one JSON line.  ``--impl reference`` times the FP64 CPU oracle on a
bounded sample of the same workload instead.
"""
from __future__ import annotations

import argparse
import ctypes
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOADS = {
    "c2": dict(
        workload="paper-shaped plain PAMD: 75-atom chain, R=8192, theta=1000, dt=1 fs, "
                 "100 geometric temperature steps 1000->250 K",
        n_atoms=75, gen_seed=1, R=8192, theta=1000, K=100, T0=1000.0, TK=250.0, dt=0.001,
        gamma=1.0, seed=12345),
    "c3": dict(
        workload="batched uneven anneals: 16 chains N~U{20..200} (seed 7), R=4096 each, "
                 "theta=500, dt=1 fs, 50 geometric temperature steps 800->300 K, one persistent "
                 "launch per temperature step",
        n_atoms=0, gen_seed=1, R=4096, theta=500, K=50, T0=800.0, TK=300.0, dt=0.001,
        gamma=1.0, seed=12345, batch=16),
    "c1": dict(
        workload="plain PAMD: 22-atom chain, R=256, theta=100, dt=1 fs, "
                 "20 geometric temperature steps 1000->300 K",
        n_atoms=22, gen_seed=1, R=256, theta=100, K=20, T0=1000.0, TK=300.0, dt=0.001,
        gamma=1.0, seed=12345),
    "c5": dict(
        workload="learned surrogate: 75-atom chain, R=65536, theta=1000, dt=1 fs, 100 geometric "
                 "temperature steps 1000->250 K; MLP 2775 inverse distances -> 512 -> 512 -> 1 "
                 "(SiLU, BF16 tensor cores, FP32 accumulation) trained on ~2M exact samples from "
                 "runs shaped like the 75-atom R=8192 workload",
        n_atoms=75, gen_seed=1, R=65536, theta=1000, K=100, T0=1000.0, TK=250.0, dt=0.001,
        gamma=1.0, seed=12345, hidden=512),
}

METRIC = "atom-steps/sec over all replicas (full anneal)"
UNIT = "atom-steps/s"

# Algorithmic floating-point work per replica-step of the propagate kernel
# (forces-only steps, Newton's third law): the nominal 40 flop per nonbonded
# pair of the method's work model W(N), 30 per bond, 60 per angle, 120 per
# dihedral, 20 per atom for the integrator and noise.  FLOP_PAIR_KERNEL is
# the count of the kernel's own pair arithmetic (fma = 2, rsqrt = 1), reported
# beside it.
FLOP_PAIR, FLOP_BOND, FLOP_ANGLE, FLOP_DIH, FLOP_ATOM = 40, 30, 60, 120, 20
FLOP_PAIR_KERNEL = 36

# FP32 peak of one GB300 from unit counts: 152 SMs x 128 FP32 lanes x 2 flop
# (FMA) x 2.07 GHz.  Reported beside the measured peak (pamd_fp32_peak).
FP32_PEAK_DERIVED_TFLOPS = 152 * 128 * 2 * 2.070e9 / 1e12

# dram bytes (read + write) of one propagate launch from the ncu capture in
# profiles/, keyed by the hash of the kernel source it was taken on; the value
# is dropped automatically when the kernel source changes.
NCU_TRAFFIC = {
    # ncu capture of this kernel (75-atom chain, R = 8192, theta = 100):
    # dram__bytes_read.sum 15.05 MB + dram__bytes_write.sum 0 (the written
    # state stays in L2 until after the kernel); the state moves once per
    # launch whatever theta is
    "82c42a4517bd10bf": 15045632,
    # the same capture after the pair-parameter table: 15.30 MB read, 0 written
    "c465a4813deb4e22": 15304704,
    # after the bonded terms moved to reciprocal square roots and the O-step
    # noise to the hardware sine/cosine: 15.09 MB read, 0 written
    "226d5425bfeba8c3": 15087360,
    # after the Lennard-Jones force moved to s6 (2 eps s6 - eps): 15.09 MB read
    "62276454e318c196": 15088128,
    # 5 atoms per lane in 128-thread blocks (the shape the tuner now picks,
    # 15 x 5, two replicas per warp): 15.27 MB read, 0 written, 4.85 ms cold
    "534aba4b3a6abf48": 15266304,
    # packed FP32x2 kernel (propagate_x2_kernel<5>, 15 x 5 shape): 15.12 MB
    # read, 768 B written per theta = 100 launch
    "938d23f1e613472b": 15118336,
    # after the fast hardware logarithm in the O-step noise (hash now covers
    # the device helpers): 15.38 MB read, 16 KB written
    "95216bfda12f5b00": 15393792,
    # after the masked t = 1 tile moved out of the ring loop: 15.28 MB read,
    # 4 KB written
    "652d5224e640d87d": 15279616,
    # the same kernel after the scalar kernel's tile loop changed in the
    # shared header: 15.45 MB read, 4 KB written
    "fdf32df449bee016": 15451136,
    # after the own block's excluded pairs were left out by position: 15.24 MB
    # read, 10 KB written
    "f6b1bb8fe2572c72": 15246080,
    # after the t = 1 tile's masks became compile-time constants: 15.18 MB
    # read, 26 KB written
    "3be35c0f8ab35a11": 15205120,
}


def flop_per_replica_step(n, flop_pair=FLOP_PAIR):
    pairs = n * (n - 1) // 2 - max(2 * n - 3, 0)
    return (flop_pair * pairs + FLOP_BOND * max(n - 1, 0) + FLOP_ANGLE * max(n - 2, 0)
            + FLOP_DIH * max(n - 3, 0) + FLOP_ATOM * n)


def measured_fp32_peak(pamd, iters=20000, reps=100):
    """FP32 FMA throughput measured on this GPU, scalar and packed FP32x2
    forms (include/pamd_bench.h); the larger is the roofline's peak."""
    scalar = pamd.pamd_fp32_peak(False, iters, reps)
    packed = pamd.pamd_fp32_peak(True, iters, reps)
    return {"ffma_tflops": scalar["tflops"], "ffma2_tflops": packed["tflops"],
            "peak_tflops": max(scalar["tflops"], packed["tflops"]),
            "timed_s": (scalar["ms"] + packed["ms"]) / 1e3}


def kernel_source_hash(packed=False):
    """Hash of the source of the timed propagate kernel (the packed kernel
    includes the scalar kernel's header; both include the device helpers)."""
    names = ["pamd_device.cuh", "propagate_impl.cuh"] + (["propagate_x2_impl.cuh"] if packed else [])
    h = hashlib.sha256()
    for n in names:
        h.update(open(os.path.join(ROOT, "paper_1806_06016_gb300", "csrc", n), "rb").read())
    return h.hexdigest()[:16]


def batch_sizes(w):
    import pamd_inputs as pi
    return pi.batched_chain_sizes(w["batch"])


def atom_steps(w, replicas):
    n = sum(batch_sizes(w)) if w.get("batch") else w["n_atoms"]
    return n * replicas * w["theta"] * (w["K"] + 1)


# ----------------------------------------------------------------- clocks

class ClockSampler:
    """nvidia-smi samples (200 ms) while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-i", str(self.index)],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.thread.join(timeout=5)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for name, val in zip(names, parts[5:9]):
                if val.lower() == "active":
                    reasons.add(name)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax),
                "reasons": sorted(reasons), "samples": len(sm)}


# ----------------------------------------------------------------- CPU legs

def oracle_sample(w, reps=512, theta=100):
    """The FP64 oracle on a bounded sample of the workload: `reps` replicas of
    the same chain, two temperatures (theta steps each, one resampling)."""
    import numpy as np

    import oracle
    import pamd_inputs as pi
    top = pi.make_chain(w["n_atoms"], w["gen_seed"])
    ratio = (w["TK"] / w["T0"]) ** (1.0 / w["K"])
    temps = np.array([w["T0"], w["T0"] * ratio])
    cores = os.cpu_count() or 1
    t0 = time.perf_counter()
    oracle.anneal(top, reps, temps, theta, w["dt"], w["gamma"], w["seed"], n_threads=cores)
    dt = time.perf_counter() - t0
    units = w["n_atoms"] * reps * theta * 2
    sample = (f"{reps} replicas of the {w['n_atoms']}-atom chain, theta={theta}, "
              f"2 temperatures (1 resampling), {units:.3g} atom-steps, FP64, {cores} threads")
    return units / dt, dt, cores, sample


def run_reference(args, w):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle
    oracle.build()
    for _ in range(args.warmup):
        oracle_sample(w)
    times, rates = [], []
    for _ in range(args.steps):
        rate, dt, cores, sample = oracle_sample(w)
        times.append(dt)
        rates.append(rate)
    value = sum(w["n_atoms"] * 512 * 100 * 2 for _ in times) / sum(times)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * statistics.mean(times),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": config_of(w, args),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def config_of(w, args):
    return {"workload": w["workload"], "n_atoms": w["n_atoms"],
            "replicas_per_gpu": (getattr(args, "replicas", 0) or w["R"]) * w.get("batch", 1),
            "theta": w["theta"], "temperature_steps": w["K"], "T_first_K": w["T0"],
            "T_last_K": w["TK"], "dt_fs": w["dt"] * 1e3, "gamma_per_ps": w["gamma"],
            "precision": "FP32 forces/integration, FP64 energies/weights/lnQ",
            "parallelism": "one GPU",
            "l2": "flushed (512 MB write) between timed steps"}


# ----------------------------------------------------------------- GPU leg

def run_gpu(args, w):
    import numpy as np
    import torch

    import pamd_inputs as pi
    from paper_1806_06016_gb300 import build as pbuild
    from paper_1806_06016_gb300 import pamd

    torch.cuda.set_device(0)
    dev = torch.cuda.current_device()
    pbuild.build()
    pamd.load()

    temps = pi.geometric_schedule(w["T0"], w["TK"], w["K"])
    R, theta, dt = args.replicas or w["R"], w["theta"], w["dt"]
    seed = w["seed"]
    # the library launches on this stream; the timing events are recorded on it
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    if w.get("batch"):
        sizes = batch_sizes(w)
        tops = [pi.make_chain(n, m + 1) for m, n in enumerate(sizes)]
        top = tops[int(np.argmax(sizes))]
        # per-molecule launch shapes by measurement among the batched kernel's shapes (untimed)
        ctx = pamd.pamd_init_batch(tops, [R] * len(tops), [temps[0]] * len(tops), seed,
                                   pamd.torch_options(gamma_per_ps=w["gamma"], autotune=1))
        pop = pamd.Population.__new__(pamd.Population)
        pop.ctx, pop.top, pop.R = ctx, top, R * len(tops)
        tune = {"per_molecule": [pamd.pamd_info(pamd.pamd_batch_sub(ctx, m)) for m in range(len(tops))]}
    else:
        top = pi.make_chain(w["n_atoms"], w["gen_seed"])
        pop = pamd.Population(top, R, temps[0], seed, pamd.torch_options(gamma_per_ps=w["gamma"]))
        tune = pamd.pamd_autotune(pop.ctx, 50)   # launch shape by measurement (untimed)
    flush = torch.empty(512 * 1024 * 1024, dtype=torch.uint8, device="cuda")

    def one_anneal():
        pamd.pamd_reset(pop.ctx, temps[0], seed)
        pamd.pamd_anneal(pop.ctx, temps, theta, dt)

    for _ in range(args.warmup):
        one_anneal()
    torch.cuda.synchronize()

    sampler = ClockSampler(dev)
    torch.cuda.synchronize()
    sampler.start()
    launches0 = pamd.pamd_launch_count(pop.ctx)
    elapsed_ms = 0.0
    for _ in range(args.steps):
        flush.zero_()
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        one_anneal()
        ev1.record(stream)
        ev1.synchronize()
        elapsed_ms += ev0.elapsed_time(ev1)
    torch.cuda.synchronize()
    launches = pamd.pamd_launch_count(pop.ctx) - launches0
    clocks = sampler.stop()
    total_units = atom_steps(w, R) * args.steps
    if w.get("batch"):
        # one batched launch advances all molecules; no single-kernel roofline
        pop.close()
        line = {"metric": METRIC, "value": total_units / (elapsed_ms / 1e3), "unit": UNIT,
                "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": elapsed_ms / args.steps, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": dict(config_of(w, args), launch_shape=tune, atoms=batch_sizes(w)),
                "gpu_launches": int(launches), "clocks": clocks}
        print(json.dumps(line), flush=True)
        return
    value = total_units / (elapsed_ms / 1e3)

    # dominant kernel: the persistent propagate launch, timed alone in the
    # same shape (theta steps over all R replicas) with events on its stream
    pamd.pamd_reset(pop.ctx, temps[0], seed)
    prop_ms = []
    for _ in range(3):
        flush.zero_()
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        pamd.pamd_propagate(pop.ctx, theta, dt, temps[0])
        ev1.record(stream)
        ev1.synchronize()
        prop_ms.append(ev0.elapsed_time(ev1))
    prop_avg = statistics.mean(prop_ms)
    flops = flop_per_replica_step(w["n_atoms"]) * R * theta
    flops36 = flop_per_replica_step(w["n_atoms"], FLOP_PAIR_KERNEL) * R * theta
    achieved = flops / (prop_avg / 1e3) / 1e12
    shape = tune if isinstance(tune, dict) else {}
    traffic = NCU_TRAFFIC.get(kernel_source_hash(shape.get("pair_arith") == 2))
    peak = measured_fp32_peak(pamd)
    roofline = {"bound": "alu", "achieved": achieved, "peak": peak["peak_tflops"], "unit": "TFLOP/s",
                "frac": achieved / peak["peak_tflops"], "traffic": traffic,
                "kernel": "propagate_x2_kernel" if shape.get("pair_arith") == 2 else "propagate_kernel",
                "launch_ms": prop_avg, "flop_per_launch": flops,
                "flop_model": f"W(N) with {FLOP_PAIR} flop per nonbonded pair",
                "frac_kernel_count": flops36 / (prop_avg / 1e3) / 1e12 / peak["peak_tflops"],
                "flop_model_kernel_count": f"W(N) with {FLOP_PAIR_KERNEL} flop per pair (the kernel's own count)",
                "peak_basis": "measured: pamd_fp32_peak, FMA chains filling every SM, larger of "
                              "FFMA and packed FFMA2, event-timed in this run",
                "peak_measured": peak,
                "peak_derived_tflops": FP32_PEAK_DERIVED_TFLOPS,
                "frac_of_derived": achieved / FP32_PEAK_DERIVED_TFLOPS}

    # end to end through the C-ABI with host buffers: upload the initial
    # population, run the anneal, read the per-temperature observables back
    rng = np.random.default_rng(seed)
    x_host = np.repeat((top.x0 - top.x0.mean(0))[None], R, axis=0)
    v_host = rng.normal(0.0, math.sqrt(0.008314462618 * temps[0] / 12.0), (R, w["n_atoms"], 3))
    fam_host = np.arange(R, dtype=np.int32)
    e2e_steps = max(1, min(args.steps, 2))
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        pamd.pamd_set_state(pop.ctx, x_host, v_host, None, fam_host)
        pamd.pamd_set_counters(pop.ctx, 0, 0, 0.0)
        obs = pamd.pamd_anneal(pop.ctx, temps, theta, dt)
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    np_ = (w["n_atoms"] + 3) // 4 * 4
    h2d = R * 6 * np_ * 4 + R * 4 + 8
    d2h = (w["K"] + 1) * ctypes.sizeof(pamd.PamdObs) + 48
    e2e = {"value": atom_steps(w, R) * e2e_steps / e2e_s, "unit": UNIT,
           "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
           "final_e_pot_kJmol": obs[-1]["e_pot"], "final_sum_lnQ": obs[-1]["sum_lnQ"]}
    pop.close()

    cpu = None
    if not args.no_cpu_baseline:
        rate, dt_s, cores, sample = oracle_sample(w)
        cpu = {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample}
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": elapsed_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": dict(config_of(w, args), launch_shape=tune), "roofline": roofline,
        "cpu_baseline": cpu, "e2e": e2e,
        "gpu_launches": int(launches), "clocks": clocks,
    }
    print(json.dumps(line), flush=True)


def run_kernel(args, w):
    """Propagate launches only (theta steps over all R replicas), for
    profiling and launch-shape sweeps.  Prints one JSON line."""
    import torch

    import pamd_inputs as pi
    from paper_1806_06016_gb300 import build as pbuild
    from paper_1806_06016_gb300 import pamd

    torch.cuda.set_device(0)
    pbuild.build()
    top = pi.make_chain(w["n_atoms"], w["gen_seed"])
    theta = args.theta or w["theta"]
    R = args.replicas or w["R"]
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    opts = pamd.torch_options(gamma_per_ps=w["gamma"], lanes_per_replica=args.lanes,
                              warps_per_block=args.warps, replicas_per_lane=args.rpl,
                              pair_arith=args.pairs,
                              precision=1 if args.fp64 else 0)
    pop = pamd.Population(top, R, w["T0"], w["seed"], opts)
    if args.autotune:
        pop.autotune(50)
    info = pop.info()
    shape = pamd.pamd_get_shape(pop.ctx) if not args.fp64 else None
    for _ in range(args.warmup):
        pamd.pamd_propagate(pop.ctx, theta, w["dt"], w["T0"])
    torch.cuda.synchronize()
    ms = []
    for _ in range(args.steps):
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        pamd.pamd_propagate(pop.ctx, theta, w["dt"], w["T0"])
        ev1.record(stream)
        ev1.synchronize()
        ms.append(ev0.elapsed_time(ev1))
    pop.close()
    avg = statistics.mean(ms)
    flops = flop_per_replica_step(w["n_atoms"]) * R * theta
    achieved = flops / (avg / 1e3) / 1e12
    peak = FP32_PEAK_DERIVED_TFLOPS
    print(json.dumps({"mode": "kernel", "n_atoms": w["n_atoms"], "replicas": R, "theta": theta,
                      "launch": info, "shape": shape,
                      "rpl": args.rpl, "fp64": args.fp64, "ms": avg, "atom_steps_per_s": w["n_atoms"] * R * theta / (avg / 1e3),
                      "achieved_tflops": achieved, "frac_of_derived_peak": achieved / peak}), flush=True)


def run_fp32peak(args):
    """The FP32 peak that the force kernel's roofline divides by: FMA chains
    filling every SM, scalar and packed, timed for about a second each with
    the clocks sampled meanwhile.  Prints one JSON line."""
    import torch

    from paper_1806_06016_gb300 import build as pbuild
    from paper_1806_06016_gb300 import pamd
    torch.cuda.set_device(0)
    pbuild.build()
    pamd.load()
    pamd.pamd_fp32_peak(False, 2000, 5)  # warm-up
    sampler = ClockSampler(0)
    sampler.start()
    peak = measured_fp32_peak(pamd, iters=20000, reps=max(1, args.steps) * 80)
    clocks = sampler.stop()
    print(json.dumps({"mode": "fp32peak", **peak, "derived_tflops": FP32_PEAK_DERIVED_TFLOPS,
                      "clocks": clocks}), flush=True)


def run_control(args):
    """Resampling on and off (the measured-temperature and lowest-temperature
    energy comparison of the paper's Figs. 2 and 4) on the 75-atom chain: the
    paper's eight temperatures 700 ... 200 K and R = 10000 replicas, PA with
    theta = 1000 and 4375 and the resampling-off anneal with theta = 4375, each
    started from the same population equilibrated at 700 K.  Prints one JSON
    line."""
    import numpy as np
    import torch

    import pamd_inputs as pi
    from paper_1806_06016_gb300 import build as pbuild
    from paper_1806_06016_gb300 import pamd

    torch.cuda.set_device(0)
    pbuild.build()
    N, dt, seed = 75, 0.001, 12345
    R = args.replicas or 10000
    theta_eq = args.theta or 20000
    temps = np.array([700.0, 585.0, 489.0, 409.0, 342.0, 286.0, 239.0, 200.0])
    top = pi.make_chain(N, 1)
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    # one equilibrated population at T0, copied into every run
    with pamd.Population(top, R, temps[0], seed, pamd.torch_options()) as pop:
        pop.propagate(theta_eq, dt, temps[0])
        x0, v0, _, _ = pop.state()
    runs = {}
    for name, theta, resample in (("pa_theta1000", 1000, True), ("pa_theta4375", 4375, True),
                                  ("anneal_theta4375", 4375, False)):
        with pamd.Population(top, R, temps[0], seed + 1, pamd.torch_options()) as pop:
            pop.set_state(x0, v0)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            obs = pop.anneal(temps, theta, dt, resample=resample)
            wall = time.perf_counter() - t0
            _, _, E, fam = pop.state()
        runs[name] = {
            "theta": theta, "resample": resample, "wall_s": wall,
            "atom_steps_per_s": N * R * theta * len(temps) / wall,
            "T_m": [o["t_meas"] for o in obs],
            "e_pot": [o["e_pot"] for o in obs], "e_pot_se": [o["e_pot_se"] for o in obs],
            "rg": [o["rg"] for o in obs], "n_families": [o["n_families"] for o in obs],
            "sum_lnQ": [o["sum_lnQ"] for o in obs],
            "E_final": E,
        }
    out = {"mode": "control", "n_atoms": N, "replicas": R, "dt_ps": dt, "theta_equilibration": theta_eq,
           "T_K": temps.tolist()}
    for name, r in runs.items():
        E = r.pop("E_final")
        q = np.quantile(E, [0.05, 0.25, 0.5, 0.75, 0.95])
        r["E_final_quantiles_5_25_50_75_95"] = [float(v) for v in q]
        r["T_m_minus_T_max_K"] = float(np.max(np.abs(np.array(r["T_m"]) - temps)))
        out[name] = r
    # lowest temperature: PA vs anneal, mean difference in combined family-binned errors
    a, b = out["pa_theta4375"], out["anneal_theta4375"]
    d = b["e_pot"][-1] - a["e_pot"][-1]
    out["anneal_minus_pa_e_pot_200K"] = {"kJmol": d, "combined_se": float(np.hypot(a["e_pot_se"][-1], b["e_pot_se"][-1]))}
    if not args.no_cpu_baseline:
        # the oracle on a bounded sample of the same runs: 128 replicas,
        # theta = 100 at each of the eight temperatures, resampling off
        import oracle
        oracle.build()
        cores = os.cpu_count() or 1
        t0 = time.perf_counter()
        oracle.anneal(top, 128, temps, 100, dt, 1.0, seed, resample=False, n_threads=cores)
        t_or = time.perf_counter() - t0
        units = N * 128 * 100 * len(temps)
        out["cpu_baseline"] = {"value": units / t_or, "unit": UNIT, "cores": cores, "kind": "oracle",
                               "sample": f"128 replicas, theta=100 at the 8 temperatures, resampling off, "
                                         f"{units:.3g} atom-steps, FP64, {cores} threads"}
    print(json.dumps(out), flush=True)


def run_wham(args):
    """WHAM refinement of the free energies (free-energy paragraph).  (1) The
    75-atom R = 8192 anneal (theta = 1000, 100 steps 1000 -> 250 K) records its
    energies at all 101 temperatures; WHAM seeded with the running sum of ln Q
    refines ln Z(T_i) and reweights <E> to the midpoints of the schedule.  (2)
    Synthetic energies shaped like the R = 2^20 anneal (61 temperatures x 2^20
    samples, 512 MB): the histogram pass alone (no sweeps) and with 100 sweeps,
    each call timed on the host (it synchronises).  Prints one JSON line."""
    import numpy as np
    import torch

    import pamd_inputs as pi
    from paper_1806_06016_gb300 import build as pbuild
    from paper_1806_06016_gb300 import pamd

    torch.cuda.set_device(0)
    pbuild.build()
    w = WORKLOADS["c2"]
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    sh = stream.cuda_stream
    out = {"mode": "wham"}
    R = args.replicas or w["R"]
    temps = pi.geometric_schedule(w["T0"], w["TK"], w["K"])
    top = pi.make_chain(w["n_atoms"], w["gen_seed"])
    rec = torch.empty((len(temps), R), dtype=torch.float64, device="cuda")
    with pamd.Population(top, R, temps[0], w["seed"], pamd.torch_options()) as pop:
        pamd.pamd_record_energies(pop.ctx, rec.data_ptr(), len(temps))
        obs = pop.anneal(temps, w["theta"], w["dt"])
    z = np.array([o["sum_lnQ"] for o in obs])
    mids = np.sqrt(temps[1:] * temps[:-1])
    t0 = time.perf_counter()
    g = pamd.pamd_wham(rec.data_ptr(), len(temps), R, temps, 2000, lnZ_init=z, max_iter=2000, tol=1e-10,
                       T_eval=mids, stream=sh)
    dt_call = time.perf_counter() - t0
    e_pa = np.array([o["e_pot"] for o in obs])
    # the PA means at neighbouring temperatures bracket the reweighted midpoint values
    between = np.mean((g["e_mean_eval"] - e_pa[1:]) * (g["e_mean_eval"] - e_pa[:-1]) <= 0)
    out["anneal"] = {
        "workload": w["workload"], "n_bins": 2000, "sweeps": g["iterations"], "last_change": g["max_delta"],
        "call_s": dt_call,
        "lnZ_wham_minus_sum_lnQ_max_abs": float(np.max(np.abs(g["lnZ"] - (z - z[0])))),
        "lnZ_final": {"wham": float(g["lnZ"][-1]), "sum_lnQ": float(z[-1] - z[0])},
        "midpoint_e_mean_between_neighbours_fraction": float(between),
    }
    if not args.no_cpu_baseline:
        # the oracle on the same recorded energies, same bins, start values and stopping rule
        from oracle import wham as owham
        E_host = rec.cpu().numpy()
        t0 = time.perf_counter()
        o = owham.wham(E_host, temps, 2000, lnZ_init=z, max_iter=2000, tol=1e-10, T_eval=mids)
        t_or = time.perf_counter() - t0
        out["cpu_baseline"] = {"value": t_or, "unit": "s per WHAM call", "cores": 1, "kind": "oracle",
                               "sample": f"the same {len(temps)} x {R} energies, 2000 bins, "
                                         f"{o['iterations']} sweeps (numpy FP64)",
                               "lnZ_max_abs_diff_vs_gpu": float(np.max(np.abs(o["lnZ"] - g["lnZ"])))}
    # synthetic large set: Gaussian energies whose mean and width follow the
    # 75-atom chain's (mean from the PA run, width sqrt(k_B T^2 C_v) ~ 10 kJ/mol)
    K4, R4 = 60, 1 << 20
    t4 = pi.geometric_schedule(1000.0, 250.0, K4)
    mean4 = np.ascontiguousarray(np.interp(t4[::-1], temps[::-1], e_pa[::-1])[::-1])
    gen = torch.Generator(device="cuda").manual_seed(1)
    E4 = torch.randn((K4 + 1, R4), dtype=torch.float64, device="cuda", generator=gen)
    E4.mul_(torch.from_numpy(0.04 * t4).cuda()[:, None]).add_(torch.from_numpy(mean4).cuda()[:, None])
    torch.cuda.synchronize()
    times = {}
    for name, iters in (("histograms_only", 0), ("sweeps_100", 100)):
        ts = []
        for _ in range(max(3, args.steps)):
            t0 = time.perf_counter()
            pamd.pamd_wham(E4.data_ptr(), K4 + 1, R4, t4, 4096, max_iter=iters, tol=0.0, stream=sh)
            ts.append(time.perf_counter() - t0)
        times[name] = statistics.median(ts)
    nbytes = 8 * (K4 + 1) * R4
    out["large"] = {"temperatures": K4 + 1, "samples_per_temperature": R4, "bytes": nbytes, "n_bins": 4096,
                    "call_s": times,
                    "histogram_call_GBps": nbytes / times["histograms_only"] / 1e9,
                    "sweep_ms": 1e3 * (times["sweeps_100"] - times["histograms_only"]) / 100}
    print(json.dumps(out), flush=True)


def run_adaptive(args):
    """Temperature schedules from the overlap condition and the resampling
    rules on the 75-atom R = 8192 workload (theta = 1000, 1000 -> 250 K): the
    geometric 100-step schedule with multinomial, systematic, nearest-integer
    and Poisson resampling (the last two with a fluctuating population), and
    adaptive schedules for two overlap targets; plus the cost
    of one overlap step at R = 8192 and R = 2^20.  Prints one JSON line."""
    import numpy as np
    import torch

    import pamd_inputs as pi
    from paper_1806_06016_gb300 import build as pbuild
    from paper_1806_06016_gb300 import pamd

    torch.cuda.set_device(0)
    pbuild.build()
    w = WORKLOADS["c2"]
    R = args.replicas or w["R"]
    top = pi.make_chain(w["n_atoms"], w["gen_seed"])
    temps = pi.geometric_schedule(w["T0"], w["TK"], w["K"])
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    out = {"mode": "adaptive", "workload": w["workload"], "replicas": R}

    def summary(obs, wall, temps_used):
        return {"temperatures": len(temps_used), "wall_s": wall,
                "atom_steps_per_s": w["n_atoms"] * R * w["theta"] * len(temps_used) / wall,
                "e_pot_final": obs[-1]["e_pot"], "e_pot_se_final": obs[-1]["e_pot_se"],
                "rg_final": obs[-1]["rg"], "sum_lnQ_final": obs[-1]["sum_lnQ"],
                "families_final": obs[-1]["n_families"],
                "T_first_steps": [float(t) for t in temps_used[:6]]}

    for rule, name in ((pamd.PAMD_RESAMPLE_MULTINOMIAL, "geometric_multinomial"),
                       (pamd.PAMD_RESAMPLE_SYSTEMATIC, "geometric_systematic"),
                       (pamd.PAMD_RESAMPLE_NEAREST, "geometric_nearest_integer"),
                       (pamd.PAMD_RESAMPLE_POISSON, "geometric_poisson")):
        with pamd.Population(top, R, temps[0], w["seed"], pamd.torch_options(resample_rule=rule)) as pop:
            pop.anneal(temps, w["theta"], w["dt"])  # graph capture and warm-up
            pop.reset(temps[0], w["seed"])
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            obs = pop.anneal(temps, w["theta"], w["dt"])
            out[name] = summary(obs, time.perf_counter() - t0, temps)
            sizes = [o["R_live"] for o in obs]
            out[name]["population_size"] = {"min": min(sizes), "max": max(sizes),
                                            "mean": float(np.mean(sizes)), "final": sizes[-1]}
    for alpha in (0.5, 0.8):
        with pamd.Population(top, R, temps[0], w["seed"], pamd.torch_options()) as pop:
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            obs, used = pamd.pamd_anneal_adaptive(pop.ctx, w["T0"], w["TK"], alpha, w["theta"], w["dt"], 400)
            out[f"adaptive_alpha{alpha}"] = summary(obs, time.perf_counter() - t0, used)
    # one overlap step (the search alone: 2 + 2 x 4 launches and one synchronisation)
    gen = torch.Generator(device="cuda").manual_seed(3)
    for n in (R, 1 << 20):
        E = torch.randn(n, dtype=torch.float64, device="cuda", generator=gen).mul_(40.0).sub_(2000.0)
        pamd.pamd_overlap_temperature(E.data_ptr(), n, 1000.0, 250.0, 0.5, stream.cuda_stream)
        ts = []
        for _ in range(20):
            t0 = time.perf_counter()
            pamd.pamd_overlap_temperature(E.data_ptr(), n, 1000.0, 250.0, 0.5, stream.cuda_stream)
            ts.append(time.perf_counter() - t0)
        out[f"overlap_step_ms_R{n}"] = 1e3 * statistics.median(ts)
        if n == R and not args.no_cpu_baseline:
            # the oracle's FP64 overlap root on the same energies
            from oracle import adaptive as oadapt
            E_host = E.cpu().numpy()
            t0 = time.perf_counter()
            T_or, _ = oadapt.next_temperature(E_host, 1000.0, 250.0, 0.5)
            t_or = time.perf_counter() - t0
            T_gpu, _ = pamd.pamd_overlap_temperature(E.data_ptr(), n, 1000.0, 250.0, 0.5, stream.cuda_stream)
            out["cpu_baseline"] = {"value": 1e3 * t_or, "unit": "ms per overlap step", "cores": 1,
                                   "kind": "oracle",
                                   "sample": f"the same {n} energies, Brent root in FP64 (numpy)",
                                   "T_next": {"oracle": T_or, "gpu": T_gpu}}
    print(json.dumps(out), flush=True)


def run_precision(args):
    """Large-population precision study (75-atom chain, 60 geometric steps
    1000 -> 250 K, theta = 200): the mixed FP32/FP64 path against the all-FP64
    GPU path at the same seeds, the mixed path's force error against the FP64
    path on the same configurations, and the
    resampling throughput at R = 2^20.  Prints one JSON line."""
    import numpy as np
    import torch

    import pamd_inputs as pi
    from paper_1806_06016_gb300 import build as pbuild
    from paper_1806_06016_gb300 import pamd

    torch.cuda.set_device(0)
    pbuild.build()
    N, theta, K, dt, seed = 75, 200, 60, 0.001, 12345
    R = args.replicas or 2048
    top = pi.make_chain(N, 1)
    temps = pi.geometric_schedule(1000.0, 250.0, K)
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    out = {"mode": "precision", "n_atoms": N, "replicas": R, "theta": theta, "temperature_steps": K}

    def anneal(precision, sd):
        o = pamd.torch_options(precision=precision)
        pop = pamd.Population(top, R, temps[0], sd, o)
        if precision == 0:
            pop.autotune(20)
            # warm-up anneal (graph capture); the FP64 anneal runs for tens of
            # seconds, where the capture is negligible
            pop.anneal(temps, theta, dt)
            pop.reset(temps[0], sd)
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        obs = pop.anneal(temps, theta, dt)
        ev1.record(stream)
        ev1.synchronize()
        x, _, _, _ = pop.state()
        f, _ = pop.forces()
        pop.close()
        return obs, ev0.elapsed_time(ev1), x, f

    # independent anneals (different seeds) of each mode: the two modes are
    # compared through the spread of their run means, since FP32 rounding
    # makes even same-seed runs independent realisations
    seeds = [seed + 1000 * s_ for s_ in range(args.seeds)]
    runs = {0: [], 1: []}
    for prec in (0, 1):
        for s_ in seeds[: (args.seeds if prec == 0 else max(2, args.seeds // 2))]:
            runs[prec].append(anneal(prec, s_))
    obs32, ms32, x32, f32 = runs[0][0]
    obs64, ms64, x64, f64 = runs[1][0]

    def stat(prec, key):
        a = np.array([[o[key] for o in r[0]] for r in runs[prec]])
        return a.mean(0), a.std(0, ddof=1) / math.sqrt(a.shape[0]), a
    e32, s32, _ = stat(0, "e_pot"); e64, s64, _ = stat(1, "e_pot")
    g32, q32, _ = stat(0, "rg"); g64, q64, _ = stat(1, "rg")
    f32q, _, _ = stat(0, "sum_lnQ"); f64q, _, _ = stat(1, "sum_lnQ")
    comb = np.sqrt(s32 ** 2 + s64 ** 2)
    out["seeds"] = {"mixed": len(runs[0]), "fp64": len(runs[1])}
    out["e_bias_kJmol"] = [float(v) for v in (e32 - e64)[::10]]
    out["e_se_kJmol"] = [float(v) for v in comb[::10]]
    out["T_K"] = [float(v) for v in temps[::10]]
    out["e_bias_in_se_max"] = float(np.max(np.abs(e32 - e64) / comb))
    out["rg_bias_in_se_max"] = float(np.max(np.abs(g32 - g64) / np.sqrt(q32 ** 2 + q64 ** 2)))
    out["sum_lnQ_final"] = {"mixed": float(f32q[-1]), "fp64": float(f64q[-1])}
    out["anneal_ms"] = {"mixed": ms32, "fp64": ms64}
    out["families_final"] = {"mixed": [r[0][-1]["n_families"] for r in runs[0]],
                             "fp64": [r[0][-1]["n_families"] for r in runs[1]]}
    # force error of the mixed path on its final configurations, against the
    # all-FP64 GPU path evaluated on the same configurations (that path is held
    # to the FP64 oracle at 1e-10 by the parity tests)
    ref = pamd.Population(top, R, temps[0], seed, pamd.torch_options(precision=1))
    ref.set_state(x32, np.zeros_like(x32))
    f_ref, _ = ref.forces()
    ref.close()
    out["force_rel_rmse_vs_fp64_gpu"] = {
        "mixed": math.sqrt(float(np.sum((f32 - f_ref) ** 2)) / float(np.sum(f_ref ** 2)))}
    # resampling at R = 2^20: whole chain (weights, scans, counts, gather)
    big = 1 << 20
    pop = pamd.Population(top, big, 1000.0, seed, pamd.torch_options())
    pamd.pamd_propagate(pop.ctx, 2, dt, 1000.0)
    flush = torch.empty(512 * 1024 * 1024, dtype=torch.uint8, device="cuda")
    ms = []
    for i in range(4):
        flush.zero_()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        pamd.pamd_resample(pop.ctx, 1000.0 - 5 * i, 995.0 - 5 * i, want_copies=False)
        ev1.record(stream)
        ev1.synchronize()
        ms.append(ev0.elapsed_time(ev1))
    pop.close()
    gather_bytes = 2 * big * 6 * ((N + 3) // 4 * 4) * 4
    chain_ms = statistics.mean(ms[1:])
    out["resample_R2p20"] = {"chain_ms": chain_ms, "gather_bytes": gather_bytes,
                             "gather_GBps_lower_bound": gather_bytes / (chain_ms / 1e3) / 1e9}
    if args.replicas == 0:
        # the whole schedule in mixed precision at the full population R = 2^20
        # (the all-FP64 path would take hours there); its <E>(T) against the
        # FP64 runs above, in combined standard errors
        with pamd.Population(top, big, temps[0], seed, pamd.torch_options()) as pop:
            pop.autotune(20)
            pop.anneal(temps[:2], theta, dt)  # graph of a short schedule: warms up the kernels
            pop.reset(temps[0], seed)
            ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            ev0.record(stream)
            obs = pop.anneal(temps, theta, dt)
            ev1.record(stream)
            ev1.synchronize()
            t_ms = ev0.elapsed_time(ev1)
        e_big = np.array([o["e_pot"] for o in obs]); s_big = np.array([o["e_pot_se"] for o in obs])
        comb_big = np.sqrt(s_big ** 2 + s64 ** 2)
        out["mixed_R2p20"] = {
            "anneal_s": t_ms / 1e3, "atom_steps_per_s": N * big * theta * (K + 1) / (t_ms / 1e3),
            "e_pot_kJmol": [float(v) for v in e_big[::10]], "e_pot_se_kJmol": [float(v) for v in s_big[::10]],
            "e_minus_fp64_R2048_in_se_max": float(np.max(np.abs(e_big - e64) / comb_big)),
            "e_minus_mixed_R2048_in_se_max": float(np.max(np.abs(e_big - e32) / np.sqrt(s_big ** 2 + s32 ** 2))),
            "e_fp64_R2048_kJmol": [float(v) for v in e64[::10]],
            "e_mixed_R2048_kJmol": [float(v) for v in e32[::10]],
            "sum_lnQ_final": obs[-1]["sum_lnQ"], "families_final": obs[-1]["n_families"],
            "rg_final": obs[-1]["rg"]}
    print(json.dumps(out), flush=True)


def run_resample(args):
    """Resampling of a large population (75-atom chain, R = 2^20 by default):
    the whole chain (weights, scans, copy counts, gather) timed with events
    on its stream, and the gather's algorithmic bytes (state read + written,
    2 x 6 Np x 4 B per replica).  Prints one JSON line."""
    import torch

    import pamd_inputs as pi
    from paper_1806_06016_gb300 import build as pbuild
    from paper_1806_06016_gb300 import pamd

    torch.cuda.set_device(0)
    pbuild.build()
    N = 75
    R = args.replicas or (1 << 20)
    top = pi.make_chain(N, 1)
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    pop = pamd.Population(top, R, 1000.0, 12345, pamd.torch_options())
    pamd.pamd_propagate(pop.ctx, 2, 0.001, 1000.0)
    flush = torch.empty(512 * 1024 * 1024, dtype=torch.uint8, device="cuda")
    ms = []
    for i in range(args.warmup + args.steps):
        flush.zero_()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        pamd.pamd_resample(pop.ctx, 1000.0 - 2 * i, 998.0 - 2 * i, want_copies=False)
        ev1.record(stream)
        ev1.synchronize()
        if i >= args.warmup:
            ms.append(ev0.elapsed_time(ev1))
    pop.close()
    gather_bytes = 2 * R * 6 * ((N + 3) // 4 * 4) * 4
    chain = statistics.mean(ms)
    print(json.dumps({"mode": "resample", "n_atoms": N, "replicas": R, "chain_ms": chain,
                      "gather_bytes": gather_bytes,
                      "chain_GBps": gather_bytes / (chain / 1e3) / 1e9}), flush=True)


def gemm_shapes(M, n_atoms=75, hidden=512):
    """The four tensor-core products of one surrogate force evaluation of M
    configurations: (name, rows, cols, depth)."""
    P = n_atoms * (n_atoms - 1) // 2
    Pp = (P + 7) // 8 * 8
    return [("layer1 a.W1^T", M, hidden, Pp), ("layer2 h1.W2^T", M, hidden, hidden),
            ("backward d2.W2", M, hidden, hidden), ("backward d1.W1", M, Pp, hidden)]


def time_gemms(torch, S, stream, M, reps=10, n_atoms=75, hidden=512):
    """Device time (ms) of each surrogate GEMM shape: mean of `reps` back-to-back
    launches between CUDA events on the launch stream (after 2 warm-ups)."""
    res = []
    g = torch.Generator(device="cuda").manual_seed(0)
    for name, m, n, k in gemm_shapes(M, n_atoms, hidden):
        A = torch.randn(m, k, generator=g, device="cuda").to(torch.bfloat16)
        B = torch.randn(n, k, generator=g, device="cuda").to(torch.bfloat16)
        S.gemm_bf16_time(A, B, 2)
        t = S.gemm_bf16_time(A, B, reps)
        flop = 2.0 * m * n * k
        res.append({"gemm": name, "M": m, "N": n, "K": k, "ms": t, "tflops": flop / (t / 1e3) / 1e12})
        del A, B
    return res


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        return {}


def run_gemm(args):
    """The surrogate's four GEMM shapes at M = R (65536 by default), each
    timed alone with events on its stream.  Prints one JSON line."""
    import torch

    from paper_1806_06016_gb300 import build as pbuild
    from paper_1806_06016_gb300 import surrogate as S

    torch.cuda.set_device(0)
    pbuild.build()
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    M = args.replicas or 65536
    res = time_gemms(torch, S, stream, M, reps=max(3, args.steps))
    peak = measured_peaks().get("bf16_tflops")
    for r in res:
        r["frac_of_measured_bf16"] = r["tflops"] / peak if peak else None
    print(json.dumps({"mode": "gemm", "M": M, "gemms": res, "bf16_peak_tflops": peak}), flush=True)


def run_surrogate_kernel(args):
    """Surrogate-driven propagate launches only: a randomly initialised model
    (identity normalisation fitted to the start geometry) drives R replicas
    of the 75-atom chain for theta steps per pamd_propagate call, timed with
    events on the population's stream.  Prints one JSON line (ms per MD step
    and the effective tensor throughput of the four GEMMs per step)."""
    import numpy as np
    import torch

    import pamd_inputs as pi
    from paper_1806_06016_gb300 import build as pbuild
    from paper_1806_06016_gb300 import pamd
    from paper_1806_06016_gb300 import surrogate as S

    torch.cuda.set_device(0)
    pbuild.build()
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    w = WORKLOADS["c5"]
    N, R = w["n_atoms"], args.replicas or w["R"]
    theta = args.theta or 20
    top = pi.make_chain(N, w["gen_seed"])
    x = torch.from_numpy(pi.perturbed_positions(top, 4096, 0.01, 3).astype(np.float32)).cuda()
    model = S.MLP(N, w["hidden"], seed=7)
    model.fit_normalization(x, torch.linspace(-1.0, 1.0, 4096, dtype=torch.float64, device="cuda"))
    pop = pamd.Population(top, R, 300.0, w["seed"], pamd.torch_options())
    S.attach(pop.ctx, model)
    for _ in range(args.warmup):
        pamd.pamd_propagate(pop.ctx, theta, w["dt"], 300.0)
    torch.cuda.synchronize()
    def timed(call):
        ms = []
        for _ in range(args.steps):
            ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            ev0.record(stream)
            call()
            ev1.record(stream)
            ev1.synchronize()
            ms.append(ev0.elapsed_time(ev1))
        return statistics.mean(ms)

    ms = timed(lambda: pamd.pamd_propagate(pop.ctx, theta, w["dt"], 300.0))
    # the same theta steps inside a one-temperature anneal: one CUDA graph
    # whose MD loop is a WHILE node (plus the observables)
    pamd.pamd_anneal(pop.ctx, [300.0], theta, w["dt"])
    torch.cuda.synchronize()
    ms_graph = timed(lambda: pamd.pamd_anneal(pop.ctx, [300.0], theta, w["dt"]))
    pop.close()
    model.close()
    per_step = ms / (theta + 1)
    flop = sum(2.0 * m * n * k for _, m, n, k in gemm_shapes(R, N, w["hidden"]))
    print(json.dumps({"mode": "surrogate_kernel", "replicas": R, "theta": theta,
                      "ms_per_launch": ms, "ms_per_force_evaluation": per_step,
                      "graph_ms_per_anneal": ms_graph,
                      "graph_ms_per_force_evaluation": ms_graph / (theta + 1),
                      "gemm_tflops_effective": flop / (per_step / 1e3) / 1e12,
                      "atom_steps_per_s": N * R * theta / (ms / 1e3)}), flush=True)


def run_surrogate(args, w):
    """Learned-surrogate workload: harvest exact data, train, compare.

    1. Training data: exact anneals shaped like the 75-atom R = 8192
       workload (theta = 1000, 100 geometric steps 1000 -> 250 K), each
       population recorded with its exact energies and forces after every
       temperature block; the first ``--harvest-runs`` runs (different seeds)
       are training data (2^21 samples drawn), one more run is held out.
    2. Training: force matching (lam = 1) with Adam on the GPU kernels.
    3. Held-out energy and force errors against the exact force field.
    4. Full anneals at R = 65536 with the exact force field and with the
       surrogate: time (CUDA events on the anneal stream) and the per-
       temperature <E> and <R_g> of the two.
    Prints one JSON line; its value is the surrogate anneal's atom-steps/s.
    """
    import numpy as np
    import torch

    import pamd_inputs as pi
    from paper_1806_06016_gb300 import build as pbuild
    from paper_1806_06016_gb300 import pamd
    from paper_1806_06016_gb300 import surrogate as S

    torch.cuda.set_device(0)
    pbuild.build()
    pamd.load()
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    N, theta, dt = w["n_atoms"], w["theta"], w["dt"]
    R = args.replicas or w["R"]
    K = args.temps or w["K"]
    temps = pi.geometric_schedule(w["T0"], w["TK"], K)
    top = pi.make_chain(N, w["gen_seed"])
    out = {"mode": "surrogate", "config": dict(config_of(w, args), replicas_per_gpu=R,
                                               temperature_steps=K, hidden=w["hidden"])}
    # 1. data
    t0 = time.perf_counter()
    temps_h = pi.geometric_schedule(1000.0, 250.0, 100)
    runs = [S.harvest(top, 8192, temps_h, 1000, dt, 1000 + r, pamd.torch_options())
            for r in range(args.harvest_runs + 1)]
    harvest_s = time.perf_counter() - t0
    x_tr = np.concatenate([r[0] for r in runs[:-1]])
    E_tr = np.concatenate([r[1] for r in runs[:-1]])
    F_tr = np.concatenate([r[2] for r in runs[:-1]])
    rng = np.random.default_rng(0)
    n_train = min(len(x_tr), args.train_samples)
    pick = rng.choice(len(x_tr), n_train, replace=False)
    x_tr, E_tr, F_tr = x_tr[pick], E_tr[pick], F_tr[pick]
    x_te, E_te, F_te = runs[-1]
    sel = rng.choice(len(x_te), min(len(x_te), 65536), replace=False)
    x_te, E_te, F_te = x_te[sel], E_te[sel], F_te[sel]
    del runs
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    xt, Et, Ft = dev(x_tr), dev(E_tr), dev(F_tr)
    out["training_data"] = {"train_samples": int(n_train), "test_samples": int(len(x_te)),
                   "harvest_runs": args.harvest_runs, "harvest_s": harvest_s,
                   "E_train_mean_sd": [float(E_tr.mean()), float(E_tr.std())],
                   "F_train_rms": float(np.sqrt(np.mean(F_tr.astype(np.float64) ** 2)))}
    # 2. training
    model = S.MLP(N, w["hidden"], seed=7)
    model.fit_normalization(xt[:262144], Et[:262144])
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    hist = model.train(xt, Et, Ft, epochs=args.epochs, batch=args.batch, lam=1.0, lr=1e-3,
                       lr_final=1e-5, report_every=500)
    torch.cuda.synchronize()
    train_s = time.perf_counter() - t0
    steps = args.epochs * (n_train // args.batch)
    out["training"] = {"epochs": args.epochs, "batch": args.batch, "steps": steps, "s": train_s,
                       "samples_per_s": steps * args.batch / train_s,
                       "loss": [[int(a), float(b)] for a, b in hist]}
    xe = dev(x_te)

    def held_out():
        Ep, Fp = model.energy_forces(xe)
        Ep, Fp = Ep.cpu().numpy(), Fp.cpu().numpy().astype(np.float64)
        return {"force_rmse_kJmol_nm": float(np.sqrt(np.mean((Fp - F_te) ** 2))),
                "force_rel_rmse": float(np.sqrt(np.mean((Fp - F_te) ** 2) /
                                                np.mean(F_te.astype(np.float64) ** 2))),
                "energy_rmse_kJmol": float(np.sqrt(np.mean((Ep - E_te) ** 2))),
                "energy_sd_kJmol": float(E_te.std())}

    out["held_out_after_training"] = held_out()
    # 2b. refinement rounds: the configurations a surrogate-driven anneal of the
    # same shape visits (theta = 500), labelled by the exact force field, are
    # added to the training set and the model is trained further
    out["refinement"] = []
    for r in range(args.refine_rounds):
        t0 = time.perf_counter()
        xr, Er, Fr = S.harvest(top, 8192, temps_h, 500, dt, 2000 + r, pamd.torch_options(), model=model)
        harvest_r = time.perf_counter() - t0
        rg_end = float(np.mean(np.sqrt(np.mean(np.sum(
            (xr[-8192:] - xr[-8192:].mean(1, keepdims=True)) ** 2, axis=2), axis=1))))
        # configurations the surrogate reaches far outside the physical range
        # (overlapping atoms: exact energies up to 1e11 kJ/mol) would swamp the
        # loss; keep those within 6 SD of the training energies and 5x the
        # training force RMS.  (Clipping their labels instead, which breaks the
        # energy-force consistency of the data, made the network diverge.)
        f_rms = np.sqrt(np.mean(Fr.astype(np.float64) ** 2, axis=(1, 2)))
        keep = (Er <= E_tr.mean() + 6.0 * E_tr.std()) & (f_rms <= 5.0 * np.sqrt(np.mean(F_tr.astype(np.float64) ** 2)))
        xr, Er, Fr = xr[keep], Er[keep], Fr[keep]
        xt = torch.cat([xt, dev(xr)])
        Et = torch.cat([Et, dev(Er)])
        Ft = torch.cat([Ft, dev(Fr)])
        t0 = time.perf_counter()
        hist_r = model.train(xt, Et, Ft, epochs=args.refine_epochs, batch=args.batch, lam=1.0,
                             lr=3e-4, lr_final=1e-5, seed=r + 1, report_every=2000)
        torch.cuda.synchronize()
        out["refinement"].append({"round": r + 1, "added_samples": int(len(xr)),
                                  "discarded_samples": int((~keep).sum()),
                                  "surrogate_rg_at_250K_before": rg_end,
                                  "exact_E_mean_of_added": float(Er.mean()),
                                  "harvest_s": harvest_r, "train_s": time.perf_counter() - t0,
                                  "loss_last": float(hist_r[-1][1]) if hist_r else None,
                                  "held_out": held_out()})
    out["held_out"] = held_out()
    model_params = {k: (np.asarray(v, dtype=np.float64) if isinstance(v, np.ndarray) else float(v))
                    for k, v in model.get_params().items()}
    del xe, xt, Et, Ft
    # 4. anneals
    gemms = time_gemms(torch, S, stream, R)
    flush = torch.empty(512 * 1024 * 1024, dtype=torch.uint8, device="cuda")
    Np = (N + 3) // 4 * 4
    rng_h = np.random.default_rng(w["seed"])
    x_host = np.repeat((top.x0 - top.x0.mean(0))[None], R, axis=0)
    v_host = rng_h.normal(0.0, math.sqrt(0.008314462618 * temps[0] / 12.0), (R, N, 3))
    fam_host = np.arange(R, dtype=np.int32)

    def anneal(with_model):
        pop = pamd.Population(top, R, temps[0], w["seed"], pamd.torch_options(gamma_per_ps=w["gamma"]))
        if with_model:
            S.attach(pop.ctx, model)
        else:
            pop.autotune(50)
        # warm-up: short anneals at the first two temperatures
        for _ in range(args.warmup):
            pamd.pamd_anneal(pop.ctx, temps[:2], min(theta, 50), dt)
        per_eval = None
        if with_model:
            # one force evaluation (features, four GEMMs, step kernel): theta = 20 launch
            ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            ev0.record(stream)
            pamd.pamd_propagate(pop.ctx, 20, dt, temps[0])
            ev1.record(stream)
            ev1.synchronize()
            per_eval = ev0.elapsed_time(ev1) / 21
        torch.cuda.synchronize()
        flush.zero_()
        torch.cuda.synchronize()
        l0 = pamd.pamd_launch_count(pop.ctx)
        # end to end through the C-ABI: the start population from host memory,
        # the anneal, the per-temperature observables back to the host
        t0 = time.perf_counter()
        pamd.pamd_set_state(pop.ctx, x_host, v_host, None, fam_host)
        pamd.pamd_set_counters(pop.ctx, 0, 0, 0.0)
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        obs = pamd.pamd_anneal(pop.ctx, temps, theta, dt)
        ev1.record(stream)
        ev1.synchronize()
        wall = time.perf_counter() - t0
        launches = pamd.pamd_launch_count(pop.ctx) - l0
        pop.close()
        return obs, ev0.elapsed_time(ev1), wall, launches, per_eval

    sampler = ClockSampler(torch.cuda.current_device())
    sampler.start()
    obs_x, ms_x, wall_x, l_x, _ = anneal(False)
    obs_s, ms_s, wall_s, l_s, per_eval = anneal(True)
    clocks = sampler.stop()
    model.close()

    def cmp(key, se):
        a = np.array([o[key] for o in obs_s]); b = np.array([o[key] for o in obs_x])
        s = np.sqrt(np.array([o[se] for o in obs_s]) ** 2 + np.array([o[se] for o in obs_x]) ** 2)
        return {"max_abs": float(np.max(np.abs(a - b))), "max_in_se": float(np.max(np.abs(a - b) / s)),
                "mean_abs": float(np.mean(np.abs(a - b))),
                "T_K": [float(t) for t in temps[::10]], "surrogate": [float(v) for v in a[::10]],
                "exact": [float(v) for v in b[::10]]}

    units = N * R * theta * (K + 1)
    out["anneal"] = {"exact_ms": ms_x, "surrogate_ms": ms_s, "speedup_surrogate_over_exact": ms_x / ms_s,
                     "exact_atom_steps_per_s": units / (ms_x / 1e3),
                     "surrogate_atom_steps_per_s": units / (ms_s / 1e3),
                     "launches": {"exact": int(l_x), "surrogate": int(l_s)},
                     "e_pot": cmp("e_pot", "e_pot_se"), "rg": cmp("rg", "rg_se"),
                     "sum_lnQ_final": {"surrogate": obs_s[-1]["sum_lnQ"], "exact": obs_x[-1]["sum_lnQ"]}}
    out["gemms"] = gemms
    # per force evaluation: four GEMMs (event-timed alone) and the step kernel
    # (the rest of the event-timed evaluation)
    gemm_ms = sum(r["ms"] for r in gemms)
    step_ms = max(per_eval - gemm_ms, 1e-6)
    # algorithmic bytes of one step-kernel launch: de/da row read (FP32), the
    # feature row written (BF16), the replica state read and written
    step_bytes = R * (padded_pairs(N) * (4 + 2) + 2 * 6 * Np * 4)
    hbm = measured_peaks().get("hbm_gbs")
    bf16 = measured_peaks().get("bf16_tflops_sustained")
    top_g = max(gemms, key=lambda r: r["ms"])
    out["force_evaluation_ms"] = {"total": per_eval, "gemms": gemm_ms, "step_kernel": step_ms}
    out["roofline"] = {"bound": "hbm", "achieved": step_bytes / (step_ms / 1e3) / 1e9, "peak": hbm,
                       "unit": "GB/s", "frac": step_bytes / (step_ms / 1e3) / 1e9 / hbm if hbm else None,
                       "traffic": None, "kernel": "mlp_step_kernel (largest time share)",
                       "bytes_per_launch": step_bytes,
                       "launch_ms_basis": "event-timed force evaluation minus the event-timed GEMMs",
                       "peak_basis": "measured copy bandwidth (MEASURED_PEAKS.json)"}
    out["roofline_gemm"] = {"bound": "tensor", "achieved": top_g["tflops"], "peak": bf16, "unit": "TFLOP/s",
                            "frac": top_g["tflops"] / bf16 if bf16 else None, "traffic": None,
                            "kernel": "gemm_bf16_kernel " + top_g["gemm"],
                            "peak_basis": "measured sustained cuBLAS bf16 (MEASURED_PEAKS.json)"}
    h2d = R * 6 * Np * 4 + R * 4
    d2h = (K + 1) * ctypes.sizeof(pamd.PamdObs)
    out.update({"metric": METRIC, "value": units / (ms_s / 1e3), "unit": UNIT, "n_gpus": 1, "steps": 1,
                "warmup": args.warmup, "ms_per_step": ms_s, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "bf16 tensor cores / f32", "data": "synthetic",
                "e2e": {"value": units / wall_s, "unit": UNIT, "h2d_bytes_per_step": h2d,
                        "d2h_bytes_per_step": d2h},
                "gpu_launches": int(l_s), "clocks": clocks})
    if not args.no_cpu_baseline:
        out["cpu_baseline"] = surrogate_oracle_sample(top, model_params, temps[0], dt, w)
    print(json.dumps(out), flush=True)


def padded_pairs(n):
    """Pairs of an n-atom molecule rounded up to a multiple of 8 (row length
    of the feature and de/da matrices)."""
    P = n * (n - 1) // 2
    return (P + 7) // 8 * 8


def surrogate_oracle_sample(top, params, T, dt, w, reps=16, steps=10):
    """The FP64 oracle of the surrogate dynamics (oracle/mlp.py) on a bounded
    sample: `reps` replicas for `steps` BAOAB steps, single thread."""
    import numpy as np

    from oracle import mlp as omlp
    rng = np.random.default_rng(1)
    x0 = np.repeat((top.x0 - top.x0.mean(0))[None], reps, axis=0)
    v0 = rng.normal(0.0, math.sqrt(0.008314462618 * T / 12.0), x0.shape)
    t0 = time.perf_counter()
    omlp.propagate(params, x0, v0, top.mass, steps, dt, T, w["gamma"], 5, 0)
    dt_s = time.perf_counter() - t0
    return {"value": top.n_atoms * reps * steps / dt_s, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"{reps} replicas x {steps} surrogate BAOAB steps (FP64 numpy, trained weights)"}


def main():
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="c2")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--mode", choices=["anneal", "kernel", "precision", "resample", "gemm", "surrogate",
                                       "surrogate_kernel", "control", "wham", "adaptive", "fp32peak"],
                    default="anneal")
    ap.add_argument("--theta", type=int, default=0,
                    help="kernel mode: steps per launch; control mode: equilibration steps at 700 K")
    ap.add_argument("--replicas", type=int, default=0,
                    help="population size (per molecule for the batched workload); default: the workload's")
    ap.add_argument("--lanes", type=int, default=0, help="kernel mode: lanes per replica")
    ap.add_argument("--warps", type=int, default=0, help="kernel mode: warps per block")
    ap.add_argument("--autotune", action="store_true", help="kernel mode: tune the launch shape")
    ap.add_argument("--rpl", type=int, default=0, help="kernel mode: replicas per lane group (1, 2)")
    ap.add_argument("--pairs", type=int, default=0,
                    help="kernel mode: pair arithmetic (0 auto, 1 scalar, 2 packed FP32x2)")
    ap.add_argument("--fp64", action="store_true", help="kernel mode: all-FP64 propagate")
    ap.add_argument("--seeds", type=int, default=8, help="precision mode: independent anneals")
    ap.add_argument("--temps", type=int, default=0, help="surrogate mode: temperature steps")
    ap.add_argument("--harvest-runs", type=int, default=3, help="surrogate mode: exact training runs")
    ap.add_argument("--train-samples", type=int, default=1 << 21, help="surrogate mode")
    ap.add_argument("--epochs", type=int, default=40, help="surrogate mode: training epochs")
    ap.add_argument("--batch", type=int, default=2048, help="surrogate mode: minibatch")
    ap.add_argument("--refine-rounds", type=int, default=2,
                    help="surrogate mode: rounds of exact labels for surrogate-visited states")
    ap.add_argument("--refine-epochs", type=int, default=8, help="surrogate mode: epochs per round")
    args = ap.parse_args()
    w = WORKLOADS[args.workload]
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if args.impl == "ours" and (args.gpus != 1 or world > 1):
        # every population runs on a single GPU: no sharding, no collectives
        if int(os.environ.get("RANK", "0")) == 0:
            print(json.dumps({"metric": METRIC, "unit": UNIT, "n_gpus": max(args.gpus, world),
                              "unavailable": "one GPU only: a population is never split across GPUs"}),
                  flush=True)
        return
    if args.mode == "kernel":
        run_kernel(args, w)
    elif args.mode == "fp32peak":
        run_fp32peak(args)
    elif args.mode == "precision":
        run_precision(args)
    elif args.mode == "control":
        run_control(args)
    elif args.mode == "wham":
        run_wham(args)
    elif args.mode == "adaptive":
        run_adaptive(args)
    elif args.mode == "resample":
        run_resample(args)
    elif args.mode == "gemm":
        run_gemm(args)
    elif args.mode == "surrogate_kernel":
        run_surrogate_kernel(args)
    elif args.mode == "surrogate" or args.workload == "c5":
        run_surrogate(args, WORKLOADS["c5"])
    elif args.impl == "reference":
        run_reference(args, w)
    else:
        run_gpu(args, w)


if __name__ == "__main__":
    main()
