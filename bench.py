"""Throughput benchmark of the neutrino geodesic hot path on GB300.

One benchmark step is one whole pass of the hot path over one workload:
pre-initial sampling and momentum transform, n_steps leapfrog steps (each a
field build at the new scale factor plus one fused particle pass), and the
delta-f weighted CIC deposit.  The metric is particle-steps per second
(species x particles x leapfrog steps / time).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun (N > 1) every rank runs an independent replica of the
workload (its own seed) with no data-path collective; rank 0 prints one JSON
line with the whole-job aggregate.  --impl reference times the CPU oracle on
the host cores on a bounded sample of the same workload.
"""
import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2207_14256_gb300 import inputs as I  # noqa: E402

METRIC = "neutrino particle-steps/s at 256^3 vs plain FP64 GPU form; served p99 latency"
UNIT = "particle-steps/s"
WORKLOAD = "c3_3x256"
# Algorithmic bytes of the method per unit of work, by precision setting (0 FP64; 1, 2 FP32/BF16
# grids with the FP64 state; 3, 4 the split state with FP32/BF16 grids): a particle-step reads
# and writes x and q at FP64 and reads q0 at FP32 (108 B; 120 B with q0 at FP64), and a kick
# reads the seven gradient fields of every cell once (28 B per cell at FP32, 14 B at BF16, 56 B
# at FP64).
PARTICLE_STEP_BYTES = {0: 120, 1: 108, 2: 108, 3: 108, 4: 108}
GRID_READ_BYTES_PER_CELL = {0: 56, 1: 28, 2: 14, 3: 28, 4: 14}
FORM_NAMES = {0: "FP64 grids and state", 1: "FP32 grids, FP64 state", 2: "BF16 grids, FP64 state",
              3: "FP32 grids, split state (fixed-point x, FP32 q0 + dq)",
              4: "BF16 grids, split state (fixed-point x, FP32 q0 + dq)"}
# FP64-pipe instructions of the FP64-state pass (k_push_wide), counted in its source: a drift
# takes 18 (|q|^2 3, v = 1 + |q|^2 / (m a_c)^2 1, the inverse square root 4, t 1, five FP64
# terms of the polynomial 5, D 1, x += q D 3) and a kick 12 (argument 1, first-order inverse
# square root 3, one FP64 term of each of two polynomials 2, K_phi 1, K_psi 2, q += dq 3);
# |q0|^2 takes 3 per particle and pass.  Conversions run on the integer pipe.  ncu's count of
# FP64-pipe instructions (profiles/) checks these figures.
WIDE_FP64_PER_STEP = 30
WIDE_FP64_PER_PASS = 3

# FP64-pipe instructions per particle-step of the plain FP64 pass (k_push_f64), from ncu
# (sm__inst_executed_pipe_fp64.sum x 32 / particle-steps of the launch, 128^3 particles, one step
# per pass; profiles/), for its FP64-pipe roofline.  Dropped if the sources changed.
PLAIN_FP64 = {"per_particle_step": 19136512 * 32 / 128 ** 3,
              "sources_sha256": "a61bc5ef3323c092:256bffcc5979e4f1:55a2ba5a6a8ebd0f"}

# DRAM bytes per particle-step of the pass, from ncu (dram__bytes_read.sum + dram__bytes_write.sum,
# mean over the 50 passes of a one-species 256^3 run of the bench's schedule;
# profiles/), by precision setting.  A launch's traffic is this times the particle-steps it
# processes (the species are sorted one after the other, so each reads the grid on its own).
# Valid only for the kernel sources they were measured on: their hash is checked and the figure
# dropped if they changed.
PUSH_TRAFFIC = {1: {"bytes_per_particle_step": (10.827e9 + 0.795e9) / (256 ** 3 * 8),
                    "sources_sha256": "a61bc5ef3323c092:256bffcc5979e4f1:55a2ba5a6a8ebd0f"},
                3: {"bytes_per_particle_step": (3.433e9 + 0.402e9) / (256 ** 3 * 4),
                    "sources_sha256": "a61bc5ef3323c092:256bffcc5979e4f1:55a2ba5a6a8ebd0f"}}
PUSH_SOURCES = ("k_particles.cu", "fdf_internal.cuh", "device_math.cuh")


def push_sources_hash():
    """Hash of the pass kernels' sources with comments and blank space removed, so that only a
    change of the code itself drops the ncu figures measured on it."""
    import hashlib
    import re

    d = os.path.join(ROOT, "paper_2207_14256_gb300", "csrc")
    parts = []
    for f in PUSH_SOURCES:
        src = open(os.path.join(d, f)).read()
        src = re.sub(r"/\*.*?\*/", " ", src, flags=re.S)
        src = re.sub(r"//[^\n]*", " ", src)
        parts.append(hashlib.sha256(" ".join(src.split()).encode()).hexdigest()[:16])
    return ":".join(parts)


def describe(p):
    return ("%d species x %d^3 particles on a %d^3 grid, box %g Mpc, m = %s eV, %d steps in log a from z = %g "
            "to %g, %s" % (p["n_species"], round(p["n_part"] ** (1 / 3)), p["n_grid"], p["box"],
                           "/".join("%g" % m for m in p["m_ev"]), p["n_steps"], p["z_start"], p["z_end"],
                           FORM_NAMES[p["precision"]]))


# ----------------------------------------------------------------------------------------------
class Clocks:
    """nvidia-smi samples during the timed region."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in self.lines:
            f = [x.strip() for x in l.split(",")]
            if len(f) < 7:
                continue
            try:
                sm.append(float(f[0]))
                smax = float(f[1])
            except ValueError:
                continue
            for n, v in zip(names, f[3:7]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": smax, "samples": len(sm),
                "reasons": sorted(reasons)}


def peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        return {}


# ----------------------------------------------------------------------------------------------
def rank_params(workload, rank, n_species=0, precision=-1):
    """The workload of one replica: every rank runs the same shapes with its own seed."""
    p = I.config(workload, seed=I.config(workload)["seed"] + 1000 * rank)
    if n_species:
        p["n_species"] = n_species
        p["m_ev"] = (p["m_ev"] * 4)[:n_species]
    if precision >= 0:
        p["precision"] = precision
    return p


def max_over_ranks(dist, values, device):
    """Element-wise maximum of a list of floats over all ranks (the slowest rank's times)."""
    if dist is None:
        return [float(v) for v in values]
    import torch

    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(v) for v in t]


def whole_job_value(world, units_per_rank, seconds):
    """Units all ranks processed divided by the (max-over-ranks) time."""
    return world * units_per_rank / seconds


def run_once(fdf, ctx, p, out_dev):
    fdf.fdf_sample(ctx)
    fdf.fdf_step(ctx, p["n_steps"])
    fdf.fdf_deposit(ctx, -1, fdf.FDF_Q_W_EPS, out_dev)


def run_graph_once(fdf, ctx, p, out_dev):
    """The same run through fdf_run_graph: sample + steps replayed as one recorded CUDA graph."""
    fdf.fdf_run_graph(ctx, p["n_steps"])
    fdf.fdf_deposit(ctx, -1, fdf.FDF_Q_W_EPS, out_dev)


def time_form(fdf, torch, P, T, stream, p, dep, runs, warmup, barrier):
    """ms per whole run (fdf_run_graph replays + deposit, CUDA events on the context's
    stream) and the per-kernel times of one instrumented run after them."""
    ctx = fdf.fdf_create(P, T, stream)
    try:
        with torch.cuda.stream(stream):
            for _ in range(warmup):
                run_graph_once(fdf, ctx, p, dep)
            barrier()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(runs):
                run_graph_once(fdf, ctx, p, dep)
            e1.record(stream)
            barrier()
            ms = e0.elapsed_time(e1) / runs
            fdf.fdf_timing(ctx, True)
            run_once(fdf, ctx, p, dep)
            barrier()
            ktimes = {k: fdf.fdf_kernel_time(ctx, v) for k, v in fdf.KERNEL_CLASSES.items()}
            fdf.fdf_timing(ctx, False)
    finally:
        fdf.fdf_destroy(ctx)
    return ms, ktimes


def hbm_roofline(p, ktimes, hbm):
    """The particle pass against HBM: the method's algorithmic bytes per launch (108 B per
    particle-step: x and q read and written in FP64, q0 read in FP32; + 28 B per cell per kick
    for the seven FP32 gradient fields) over its mean launch time."""
    prec = p["precision"]
    push_ms, push_n = ktimes["push"]
    push_avg = push_ms / max(push_n, 1)
    n_total = p["n_species"] * p["n_part"]
    N3 = p["n_grid"] ** 3
    # a run takes n_steps particle-steps per particle and n_steps + 1 grid reads (the opening
    # half kick and one merged kick per step), over push_n launches
    alg = (p["n_steps"] * n_total * PARTICLE_STEP_BYTES[prec] +
           (p["n_steps"] + 1) * N3 * GRID_READ_BYTES_PER_CELL[prec]) / max(push_n, 1)
    achieved = alg / (push_avg / 1e3) / 1e9
    tr = PUSH_TRAFFIC.get(prec)
    return {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
            "frac": achieved / hbm if hbm else None,
            "traffic": (tr["bytes_per_particle_step"] * n_total * p["n_steps"] / max(push_n, 1)
                        if tr and push_sources_hash() == tr["sources_sha256"] else None),
            "traffic_note": "ncu DRAM bytes per particle-step of the pass (one-species 256^3 run, the headline's "
                            "schedule; profiles/) times the launch's particle-steps; null when the kernel sources "
                            "changed since the capture",
            "peak_source": "measured (MEASURED_PEAKS.json hbm_gbs)" if hbm else "fallback 6800",
            "algorithmic_bytes_per_launch": alg, "avg_launch_ms": push_avg,
            "steps_per_launch": p["n_steps"] / max(push_n, 1),
            "per_unit": "%d B per particle-step + %d B per cell per kick" % (PARTICLE_STEP_BYTES[prec],
                                                                           GRID_READ_BYTES_PER_CELL[prec])}


def fp64_roofline(p, ktimes, dfma_per_s):
    """The FP64-state pass against the FP64 pipe: FP64-pipe instructions per launch (counted
    in k_push_wide's source) over its mean launch time, against the measured DFMA issue rate."""
    push_ms, push_n = ktimes["push"]
    push_avg = push_ms / max(push_n, 1)
    n_total = p["n_species"] * p["n_part"]
    ops = (WIDE_FP64_PER_STEP * p["n_steps"] * n_total + WIDE_FP64_PER_PASS * n_total * push_n) / max(push_n, 1)
    achieved = ops / (push_avg / 1e3) / 1e9
    peak = dfma_per_s / 1e9 if dfma_per_s else None
    return {"bound": "alu", "pipe": "fp64", "achieved": achieved, "peak": peak,
            "unit": "G FP64-pipe instructions/s", "frac": achieved / peak if peak else None,
            "peak_source": "measured in this run: fdf_pipe_rates (dependent DFMA chains on every SM, CUDA events)",
            "per_unit": "%d FP64-pipe instructions per particle-step + %d per particle per pass (k_push_wide's "
                        "source; ncu's count in profiles/)" % (WIDE_FP64_PER_STEP, WIDE_FP64_PER_PASS),
            "instructions_per_launch": ops, "avg_launch_ms": push_avg}


def bench_ours(args, rank, world, dist):
    import torch

    from paper_2207_14256_gb300 import fdf

    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    p = rank_params(args.workload, rank, args.n_species, args.precision)
    tables = I.transfer_tables(p)
    stream = torch.cuda.Stream(device=dev)
    P = fdf.make_params(p)
    T, keep = fdf.make_tables(tables)
    # the schedule knobs (re-sort distance, bucket size, steps per pass) from the autotuner
    tune = None
    if args.schedule:
        for k, v in json.loads(args.schedule).items():
            setattr(P, k, int(v))
        tune = {"knobs": fdf.knobs(P), "source": "--schedule"}
    elif not args.no_tune:
        P, tune_ms, tune_trials = fdf.fdf_tune(P, T, stream)
        tune = {"knobs": fdf.knobs(P), "best_run_ms": tune_ms, "timed_runs": tune_trials}
    N = p["n_grid"]
    dep = torch.zeros((N, N, N), dtype=torch.float64, device=dev)
    units = p["n_species"] * p["n_part"] * p["n_steps"]
    # the issue rates of the FP64 pipe (the denominator of the FP64-state pass's roofline),
    # the FP32 pipe and FP64 <-> FP32 conversions on this GPU
    d_rate, f_rate, c_rate = fdf.fdf_pipe_rates(stream)
    pipes = {"dfma_per_s": d_rate, "fp64_tflops": 2 * d_rate / 1e12, "ffma_per_s": f_rate,
             "cvt_round_trips_per_s": c_rate,
             "note": "fdf_pipe_rates: best of five launches of 64 warps per SM running 8 independent chains "
                     "per thread; a conversion round trip is FP64 -> FP32 -> FP64"}

    def barrier():
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()

    ctx = fdf.fdf_create(P, T, stream)
    try:
        with torch.cuda.stream(stream):
            # the first warm-up run records the run's graph; the timed runs replay it
            for _ in range(args.warmup):
                run_graph_once(fdf, ctx, p, dep)
            barrier()
            clocks = Clocks(dev.index)
            clocks.start()
            l0 = fdf.fdf_launch_count(ctx)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            barrier()
            e0.record(stream)
            for _ in range(args.steps):
                run_graph_once(fdf, ctx, p, dep)
            e1.record(stream)
            barrier()
            ms = e0.elapsed_time(e1)
            launches = fdf.fdf_launch_count(ctx) - l0
            clk = clocks.stop()
            # Per-kernel times from one more run, made with the sequential calls and an
            # event pair around every launch (fdf_timing).  The events cost about 10 ms
            # per run, so they stay out of the timed region above.
            fdf.fdf_timing(ctx, True)
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
            ev[0].record(stream)
            fdf.fdf_sample(ctx)
            ev[1].record(stream)
            fdf.fdf_step(ctx, p["n_steps"])
            ev[2].record(stream)
            fdf.fdf_deposit(ctx, -1, fdf.FDF_Q_W_EPS, dep)
            ev[3].record(stream)
            barrier()
            inst_ms = ev[0].elapsed_time(ev[3])
            phases = {"sample_ms": ev[0].elapsed_time(ev[1]), "steps_ms": ev[1].elapsed_time(ev[2]),
                      "deposit_ms": ev[2].elapsed_time(ev[3])}
            ktimes = {k: fdf.fdf_kernel_time(ctx, v) for k, v in fdf.KERNEL_CLASSES.items()}
            fdf.fdf_timing(ctx, False)
            # host time to enqueue the steps of one run while the device works through
            # them: the most a captured graph of the run could save
            fdf.fdf_sample(ctx)
            h0 = time.perf_counter()
            fdf.fdf_step(ctx, p["n_steps"])
            host_ms = (time.perf_counter() - h0) * 1e3
            barrier()
    finally:
        fdf.fdf_destroy(ctx)

    # end to end through the C-ABI with host buffers: tables uploaded by fdf_create,
    # every species' x, q, w read back into pinned host memory, every step
    np_ = p["n_part"]
    hx = torch.empty((3, np_), dtype=torch.float64, pin_memory=True)
    hq = torch.empty((3, np_), dtype=torch.float64, pin_memory=True)
    hw = torch.empty((np_,), dtype=torch.float64, pin_memory=True)
    e2e_steps = max(1, min(args.steps, 3))
    # one device arena for the contexts of every step, as a long-lived caller would hold
    # (fdf_create carves it; no cudaMalloc/cudaFree per step)
    arena = torch.empty(fdf.fdf_footprint(P), dtype=torch.uint8, device=dev)
    barrier()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        c2 = fdf.fdf_create(P, T, stream, arena)
        try:
            fdf.fdf_sample(c2)
            fdf.fdf_step(c2, p["n_steps"])
            for s in range(p["n_species"]):
                fdf.fdf_get(c2, s, hx, hq, hw)
        finally:
            fdf.fdf_destroy(c2)
    barrier()
    e2e_s = time.perf_counter() - t0
    del arena
    tab_bytes = sum(np.asarray(tables[k]).nbytes for k in ("lnk", "lna", "T_psi", "T_phi", "dTphi_dlna", "cdf_t",
                                                         "cdf_F"))

    # the plain FP64 form on the same workload (one warm-up, one timed run)
    plain = None
    if not args.no_plain:
        p64 = dict(p, precision=I.PREC_F64)
        P64 = fdf.make_params(p64)
        c3 = fdf.fdf_create(P64, T, stream)
        try:
            with torch.cuda.stream(stream):
                run_once(fdf, c3, p64, dep)
                barrier()
                f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                fdf.fdf_timing(c3, True)
                f0.record(stream)
                run_once(fdf, c3, p64, dep)
                f1.record(stream)
                barrier()
                pms = f0.elapsed_time(f1)
                push64 = fdf.fdf_kernel_time(c3, fdf.FDF_K_PUSH)
        finally:
            fdf.fdf_destroy(c3)
        plain = {"value": units / (pms / 1e3), "ms_per_step": pms, "push_ms_per_launch": push64[0] / push64[1],
                 "push_launches": push64[1]}
        if push_sources_hash() == PLAIN_FP64["sources_sha256"]:
            # the plain pass against the FP64 pipe: ncu's FP64 instructions per particle-step
            ops = PLAIN_FP64["per_particle_step"] * p["n_species"] * p["n_part"] * p["n_steps"] / push64[1]
            ach = ops / (push64[0] / push64[1] / 1e3) / 1e9
            plain["roofline_fp64"] = {"bound": "alu", "pipe": "fp64", "achieved": ach, "peak": d_rate / 1e9,
                                      "unit": "G FP64-pipe instructions/s", "frac": ach / (d_rate / 1e9),
                                      "per_unit": "%.0f FP64-pipe instructions per particle-step (ncu)"
                                                  % PLAIN_FP64["per_particle_step"]}

    # the paper's super-steps (Sec. 2.1: fields built only where the transfer functions
    # changed by more than 1%, interpolated in between), same workload and schedule
    superstep = None
    if not args.no_superstep:
        Pss = fdf.make_params(dict(p, superstep_tol=0.01))
        for k, v in fdf.knobs(P).items():
            setattr(Pss, k, v)
        c4 = fdf.fdf_create(Pss, T, stream)
        try:
            with torch.cuda.stream(stream):
                run_once(fdf, c4, p, dep)
                barrier()
                s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                s0.record(stream)
                for _ in range(2):
                    run_once(fdf, c4, p, dep)
                s1.record(stream)
                barrier()
                sms = s0.elapsed_time(s1) / 2
                built = fdf.fdf_supersteps(c4, p["n_steps"])[1]
        finally:
            fdf.fdf_destroy(c4)
        superstep = {"value": units / (sms / 1e3), "ms_per_step": sms, "superstep_tol": 0.01,
                     "transforms_per_run": built, "steps_per_run": p["n_steps"] + 1,
                     "note": "the same workload with the paper's super-steps (not the headline: the headline builds "
                             "every step's fields by transform)"}

    # the split-state form (fixed-point positions, FP32 q0 + dq) on the same workload with
    # its own tuned schedule (the headline's with --schedule or --no-tune): not the
    # configured precision, reported beside it
    split = None
    if not args.no_split:
        psp = dict(p, precision=I.PREC_F32_FIXED)
        Psp = fdf.make_params(psp)
        if args.schedule or args.no_tune:
            for k, v in fdf.knobs(P).items():
                if k not in ("n_gl", "pass_blocks", "gather_tile"):
                    setattr(Psp, k, v)
        else:
            Psp, _, _ = fdf.fdf_tune(Psp, T, stream)
        sms, skt = time_form(fdf, torch, Psp, T, stream, psp, dep, 2, 1, barrier)
        split = {"value": units / (sms / 1e3), "ms_per_step": sms, "precision": FORM_NAMES[psp["precision"]],
                 "schedule": fdf.knobs(Psp),
                 "kernels": {k: {"ms_per_step": v[0], "launches_per_step": v[1]} for k, v in skt.items()},
                 "roofline_hbm": hbm_roofline(psp, skt, peaks().get("hbm_gbs"))}

    # the reduced-precision workload (BF16 gradient grids, FP64 state; 512^3 particles on 256^3, 300 steps)
    c4 = None
    if not args.no_c4:
        p4 = rank_params("c4_512_bf16", rank)
        P4 = fdf.make_params(p4)
        for k, v in fdf.knobs(P).items():
            if k != "n_gl":
                setattr(P4, k, v)
        T4, keep4 = fdf.make_tables(I.transfer_tables(p4))
        N4 = p4["n_grid"]
        dep4 = torch.zeros((N4, N4, N4), dtype=torch.float64, device=dev)
        ms4, kt4 = time_form(fdf, torch, P4, T4, stream, p4, dep4, 1, 1, barrier)
        units4 = p4["n_species"] * p4["n_part"] * p4["n_steps"]
        c4 = {"workload": "c4_512_bf16", "description": describe(p4), "value": units4 / (ms4 / 1e3),
              "ms_per_step": ms4, "schedule": fdf.knobs(P4),
              "kernels": {k: {"ms_per_step": v[0], "launches_per_step": v[1]} for k, v in kt4.items()},
              "roofline_hbm": hbm_roofline(p4, kt4, peaks().get("hbm_gbs"))}
        del dep4

    return dict(p=p, ms=ms, units=units, launches=launches, ktimes=ktimes, inst_ms=inst_ms, phases=phases,
                clocks=clk, e2e_s=e2e_s, pipes=pipes,
                tune=tune, host_ms=host_ms, superstep=superstep, split=split, c4=c4,
                e2e_steps=e2e_steps, tab_bytes=tab_bytes, d2h=p["n_species"] * np_ * 7 * 8, plain=plain)


# ----------------------------------------------------------------------------------------------
SERVED_BUDGET = 180 * 10 ** 9     # bytes of HBM the served stream may hold
SERVED_ARRIVAL_SEED = 5


def served_requests(n_req):
    """The served stream's requests: request i draws its shapes from seed 1000 + i."""
    reqs = []
    for i in range(n_req):
        r = np.random.default_rng(1000 + i)
        N = int(r.choice([64, 128, 256]))
        side = int(r.choice([64, 128, 256, 512]))
        ns = int(r.integers(1, 4))
        masses = [float(m) for m in r.uniform(0.02, 0.3, size=ns)]
        steps = int(r.integers(100, 301))
        reqs.append(I.config("c2_128", box=1000.0, n_part=side ** 3, n_grid=N, n_species=ns, m_ev=masses,
                             n_steps=steps, seed=1000 + i, precision=I.PREC_F32))
    return reqs


def serve(fdf, reqs, tables, arrivals, max_active, slice_steps, merge=False):
    """Submit request i at arrivals[i] seconds (server clock), release each as it
    finishes; returns per-request latencies and the span from first submit to last done."""
    srv = fdf.Server(SERVED_BUDGET, max_active=max_active, slice_steps=slice_steps, merge=merge)
    try:
        t_start = srv.clock()
        ids, infos = [], {}
        i = 0
        while len(infos) < len(reqs):
            now = srv.clock() - t_start
            while i < len(reqs) and arrivals[i] <= now:
                ids.append(srv.submit(reqs[i], tables))
                i += 1
            wait_ms = 50 if i >= len(reqs) else max(0, min(50, int((arrivals[i] - now) * 1e3)))
            rid = srv.wait(wait_ms)
            while rid is not None:
                info = srv.info(rid)
                if info.status != fdf.FDF_REQ_DONE:
                    raise RuntimeError("request %d failed: %s" % (rid, info.message.decode()))
                infos[rid] = (info.t_submit, info.t_admit, info.t_done, info.particle_steps)
                srv.release(rid)
                rid = srv.wait(0)
    finally:
        srv.close()
    lat = np.array([infos[r][2] - infos[r][0] for r in ids])
    span = max(v[2] for v in infos.values()) - min(v[0] for v in infos.values())
    work = sum(v[3] for v in infos.values())
    return lat, span, work


def bench_served(n_req=64, load=0.8, max_active=8, slice_steps=8, merge=False):
    """The served stream: first all requests at once (the batched capacity), then
    Poisson arrivals at `load` times that capacity; p50/p99 latency of the second.
    merge: the server steps the requests' passes in merged launches."""
    from paper_2207_14256_gb300 import fdf

    reqs = served_requests(n_req)
    tables = I.transfer_tables(reqs[0])
    lat0, span0, work = serve(fdf, reqs, tables, [0.0] * n_req, max_active, slice_steps, merge)
    capacity = work / span0
    mean_service = work / n_req / capacity
    rate = load / mean_service
    gaps = np.random.default_rng(SERVED_ARRIVAL_SEED).exponential(1.0 / rate, size=n_req)
    arrivals = np.cumsum(gaps) - gaps[0]
    lat, span, work = serve(fdf, reqs, tables, arrivals, max_active, slice_steps, merge)
    return {"requests": n_req, "merged_passes": merge,
            "p50_s": float(np.percentile(lat, 50)), "p99_s": float(np.percentile(lat, 99)),
            "max_s": float(lat.max()), "value": work / span, "unit": UNIT,
            "capacity": capacity, "offered_load": load, "arrival_rate_per_s": rate,
            "saturated_p50_s": float(np.percentile(lat0, 50)), "saturated_p99_s": float(np.percentile(lat0, 99)),
            "budget_bytes": SERVED_BUDGET, "max_active": max_active, "slice_steps": slice_steps,
            "note": ("requests: grid 64/128/256, 64^3..512^3 particles per species, 1-3 species, m U(0.02, 0.3) eV, "
                     "100-300 steps, box 1000 Mpc, FP32 grids and FP64 state (request i from seed 1000 + i); %s; "
                     "Poisson arrivals (seed 5) at %.0f%% of the capacity measured with every request queued at "
                     "once; latency = submit to results resident on the device"
                     % ("one merged launch per round steps a pass of every running request" if merge else
                        "each request launches its own passes on its own streams", 100 * load))}


# ----------------------------------------------------------------------------------------------
def cpu_baseline(workload, budget_s=25.0):
    """The oracle as it stands, on the host cores, on a bounded sample of the workload:
    one field build at full grid size plus one leapfrog step of a particle subset,
    extrapolated to the whole workload (grids per step + particles per step)."""
    import oracle

    p = I.config(workload)
    tables = I.transfer_tables(p)
    o = oracle.Oracle(p, tables)
    threads = oracle.num_threads()
    t0 = time.perf_counter()
    R = o.noise()
    t_noise = time.perf_counter() - t0
    t0 = time.perf_counter()
    o.fields(o.lna(p["n_steps"] // 2), 0x7F, R)
    t_grid = time.perf_counter() - t0
    m = 1 << 16
    gidx = np.arange(m)
    frozen = np.zeros((8, p["n_grid"], p["n_grid"], p["n_grid"]))
    ic = o.initial(gidx, frozen=frozen)
    k = p["n_steps"] // 2
    t0 = time.perf_counter()
    o.integrate(gidx, ic["x"], ic["q"], ic["q0"], k, k + 2, frozen=frozen)
    t_part = (time.perf_counter() - t0) / (2 * m)
    n_total = p["n_species"] * p["n_part"]
    t_step = t_grid + n_total * t_part
    value = n_total / t_step
    sample = ("oracle: one %d^3 field build (%.2f s) + two leapfrog steps of %d particles (%.2f us/particle-step, "
              "frozen fields), extrapolated to %d particles x %d steps; noise field once (%.2f s, excluded)"
              % (p["n_grid"], t_grid, m, t_part * 1e6, n_total, p["n_steps"], t_noise))
    return {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle", "sample": sample,
            "seconds_per_leapfrog_step": t_step}


def line_base(args, world):
    return {"metric": METRIC, "unit": UNIT, "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "data": "synthetic"}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=WORKLOAD)
    ap.add_argument("--no-plain", action="store_true", help="skip the plain FP64 comparison")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU baseline")
    ap.add_argument("--no-served", action="store_true", help="skip the served stream")
    ap.add_argument("--no-tune", action="store_true", help="use the automatic schedule knobs")
    ap.add_argument("--no-superstep", action="store_true", help="skip the super-step variant")
    ap.add_argument("--no-split", action="store_true", help="skip the split-state form")
    ap.add_argument("--no-c4", action="store_true", help="skip the reduced-precision workload")
    ap.add_argument("--schedule", default="", help='schedule knobs as JSON, e.g. {"sort_tile": 1} (no tuning)')
    ap.add_argument("--served-requests", type=int, default=64)
    ap.add_argument("--served-merged", action="store_true",
                    help="also run the served stream with merged pass launches across requests")
    ap.add_argument("--precision", type=int, default=-1,
                    help="override the workload's precision setting (FDF_PREC_*: 0 FP64, 1/2 FP32/BF16 grids with "
                         "the FP64 state, 3/4 the split state)")
    ap.add_argument("--n-species", type=int, default=0,
                    help="override the species count (smaller device footprint for profiler captures)")
    args = ap.parse_args()

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    p = I.config(args.workload)

    if args.impl == "reference":
        # the CPU oracle: rank 0 alone works, other ranks exit without work
        if rank != 0:
            return
        steps = []
        for _ in range(args.warmup + args.steps):
            steps.append(cpu_baseline(args.workload))
        timed = steps[args.warmup:]
        v = float(np.median([s["value"] for s in timed]))
        cb = dict(timed[0], value=v)
        out = line_base(args, world)
        out.update({"impl": "reference", "value": v,
                    "ms_per_step": float(np.median([s["seconds_per_leapfrog_step"] for s in timed])) * 1e3 *
                    p["n_steps"], "dtype": "f64",
                    "config": {"workload": args.workload, "description": describe(p),
                               "l2": "inputs larger than L2 (host run)"},
                    "cpu_baseline": cb, "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0,
                                                "d2h_bytes_per_step": 0}})
        print(json.dumps(out))
        return

    dist = None
    if world > 1:
        import torch
        import torch.distributed as td

        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", 0)))
        td.init_process_group("nccl")
        dist = td
    r = bench_ours(args, rank, world, dist)
    ms = r["ms"]
    e2e_s = r["e2e_s"] / r["e2e_steps"]
    ms, e2e_s = max_over_ranks(dist, [ms, e2e_s], "cuda")
    ms_per_step = ms / args.steps
    value = whole_job_value(world, r["units"], ms_per_step / 1e3)
    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return

    pk = peaks()
    hbm = pk.get("hbm_gbs")
    prec = r["p"]["precision"]
    kname = {0: "k_push_f64", 1: "k_push_wide", 2: "k_push_wide", 3: "k_push_split", 4: "k_push_split"}[prec]
    kname += " (fused drift + wrap + gather + kick over a pass of leapfrog steps)"
    timing = "CUDA events around every launch of one run on the context's stream, right after the timed region"
    roof_hbm = dict(hbm_roofline(r["p"], r["ktimes"], hbm), kernel=kname, launch_timing=timing)
    if prec in (1, 2):
        # the FP64-state pass is bound by the FP64 pipe: that is its roofline
        roof = dict(fp64_roofline(r["p"], r["ktimes"], r["pipes"]["dfma_per_s"]), kernel=kname, launch_timing=timing)
    else:
        roof = roof_hbm
    n_total = r["p"]["n_species"] * r["p"]["n_part"]
    per_run = {k: {"ms_per_step": v[0], "launches_per_step": v[1]} for k, v in r["ktimes"].items()}
    per_run["note"] = ("one instrumented run after the timed region (sequential calls, an event pair per launch: "
                       "%.1f ms for the run)" % r["inst_ms"])
    out = line_base(args, world)
    out.update({
        "value": value, "ms_per_step": ms_per_step, "dtype": "f64 state, f32 grids",
        "config": {"workload": args.workload, "description": describe(r["p"]),
                   "l2": "inputs larger than L2 (%.1f GB particle state: x, q FP64, q0 FP32)" % (n_total * 60 / 1e9),
                   "parallelism": "replicas" if world > 1 else "single",
                   "schedule": r["tune"] or "automatic",
                   "timed_call": "fdf_run_graph (sample + steps replayed as one recorded CUDA graph) + fdf_deposit "
                                 "per step"},
        "roofline": roof,
        "roofline_hbm": roof_hbm,
        "pipe_rates": r["pipes"],
        "e2e": {"value": whole_job_value(world, r["units"], e2e_s), "unit": UNIT, "h2d_bytes_per_step": r["tab_bytes"],
                "d2h_bytes_per_step": r["d2h"],
                "note": "fdf_create on a caller-held device arena (table upload) + sample + steps + fdf_get of "
                        "x, q and w of every species into pinned host memory + fdf_destroy, per step"},
        "gpu_launches": r["launches"],
        "host_enqueue_ms_per_step": r["host_ms"],
        "phases": dict(r["phases"], steps_only_value=whole_job_value(world, r["units"], r["phases"]["steps_ms"] / 1e3),
                       note="the instrumented run's phases: fdf_sample (sampling, the first grid build, the "
                            "momentum transform, the first sort), fdf_step(n_steps) and fdf_deposit; "
                            "steps_only_value = particle-steps / steps_ms"),
        "kernels": per_run,
        "clocks": r["clocks"],
    })
    if r["superstep"]:
        out["superstep"] = dict(r["superstep"], value=world * r["superstep"]["value"])
    if r["plain"]:
        out["plain_f64"] = dict(r["plain"], value=world * r["plain"]["value"],
                                note="the plain FP64 form (FP64 grids, FFT, state and arithmetic), same workload")
        out["speedup_vs_plain_f64"] = value / out["plain_f64"]["value"]
    if r["split"]:
        out["split_state"] = dict(r["split"], value=world * r["split"]["value"],
                                  note="the split-state form (FDF_PREC_F32_FIXED) on the same workload, its own "
                                       "tuned schedule: positions as 32-bit fixed point, momenta as FP32 q0 + dq, "
                                       "float-float drift and FP32 kick integrals; not the configured precision")
    if r["c4"]:
        out["c4"] = dict(r["c4"], value=world * r["c4"]["value"],
                         note="the reduced-precision workload, timed as the headline (graph replays + deposit)")
    if not args.no_served and world == 1:
        out["served"] = bench_served(args.served_requests)
        if args.served_merged:
            out["served_merged"] = bench_served(args.served_requests, merge=True)
    if not args.no_cpu and world == 1:
        out["cpu_baseline"] = cpu_baseline(args.workload)
    print(json.dumps(out))
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
