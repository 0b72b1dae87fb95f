#!/usr/bin/env python
"""Throughput of the implicit-depletant HPMC hot path on one or more GB300s.

Metric: colloid trial moves/s (whole job), with depletant insertions/s (drawn
and evaluated) alongside, at fixed (phi_c, q, eta_r).

Workload: 16384 hard spheres, phi_c = 0.30, depletant size ratio q = 0.15,
reservoir packing fraction eta_r in {0.1, 0.2, 0.3, 0.4} (four independent
systems), translation step tuned (untimed) to ~30% acceptance, n_trial = 0,
FP32 + certified-margin form (``--precision fp64`` for the plain FP64 form).
One step = one checkerboard sweep of each of the four systems (4 x 16384
trial moves), run as one batch of four independent replicas.  Synthetic,
seeded inputs (fcc start, melted during tuning).

Timing: W untimed warm-up steps, then K steps each bracketed by CUDA events on
the launching stream, with a 256 MB buffer written between steps to flush L2
(the working set itself is L2-resident).  Multi-GPU (torchrun): every rank
runs its own replicas (weak scaling); barrier + max over ranks.

``--impl reference`` times the CPU oracle (oracle/) on this host on a bounded
sample of the same workload: it is the reference arm of this repository.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

ETAS = (0.1, 0.2, 0.3, 0.4)
N, PHI, Q = 16384, 0.30, 0.15
WORKLOAD = "spheres_16384_phi0.30_q0.15_eta0.1-0.4"
# Translation steps giving ~30% acceptance at each eta_r (from the untimed
# tuner on the GPU); the reference arm uses them as fixed values.
D_MAX_TUNED = {0.1: 0.0160, 0.2: 0.0080, 0.3: 0.0053, 0.4: 0.0040}
ACC_TARGET = 0.30

# Algorithmic ALU lane-operations (roofline):
#  lens kernel, per depletant drawn: 6/pi attempts x (Philox4x32-10: 40,
#  point in the cube + ball test: 11) + old-pose test (8); per move: move and
#  Poisson Philox (2 x 40), proposal and cell check (20), Poisson search (12)
OPS_PER_DEP = 6.0 / math.pi * (40.0 + 11.0) + 8.0
OPS_PER_MOVE_LENS = 2 * 40.0 + 20.0 + 12.0
#  colour-phase kernel, per move: proposal and cell check (20), ~25 neighbour
#  candidates x 8 (overlap test)
OPS_PER_MOVE_PHASE = 20.0 + 25 * 8.0
#  FP64 plain form (one kernel): everything above per evaluated depletant
OPS_PER_MOVE = 2 * 40.0 + 20.0 + 12.0 + 25 * 8.0
ISSUE_LANES_PER_SM = 128        # 4 SM sub-partitions x 32 lanes, one instruction / clock
BYTES_PER_MOVE = 2 * 32 + 16 + 2 * 4   # pos (double4) read + cell-local copy + cell list ids
# DRAM bytes (read + write) per launch from one ncu capture of the current kernel
# build on the four-state-point 16384-sphere batch, in the timed steps' conditions
# (ncu --cache-control none; the mean over the 8 phases of a sweep that starts
# after the 256 MB L2 flush; profiles/k_phase_sphere_fp32_*.md).
MEASURED_TRAFFIC = {"k_phase_sphere_fp32": 5.44e6, "k_lens_sphere_fp32": 11.88e6}


def _dist():
    from paper_1508_07077_gb300 import replicas
    return replicas.world()


class ClockSampler:
    """nvidia-smi clock / throttle samples during the timed region."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.QUERY,
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *exc):
        self.lines = []
        if self.proc is not None:
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [ln for ln in out.splitlines() if ln.strip()]
        return False

    def summary(self):
        sms, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sms.append(float(f[1]))
                smax = float(f[2])
            except ValueError:
                continue
            for name, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        if not sms:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sms), "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sms)}


def cpu_oracle_rate(systems, d_max, sweeps, first_sweep=0, v0_mode=0, soft_eps=0.0):
    """Moves/s and insertions/s of the serial oracle on this host (1 core)."""
    from oracle import oracle as O
    O.build()
    t0 = time.perf_counter()
    moves = drawn = evaluated = 0
    for s in systems:
        _, _, c, _ = O.run(s.pos, s.L, q=s.q, n_r=s.n_r, d_max=d_max[s.extra["eta_r"]],
                           seed=s.seed, replica=s.replica, n_sweeps=sweeps, sweep0=first_sweep,
                           v0_mode=v0_mode, soft_eps=soft_eps)
        moves += c["moves"]
        drawn += c["dep_drawn"]
        evaluated += c["dep_evaluated"]
    dt = time.perf_counter() - t0
    return moves / dt, drawn / dt, evaluated / dt, dt, moves


def run_reference(args, ws, rank):
    from paper_1508_07077_gb300 import workloads as W
    if rank != 0:
        return
    systems = [W.spheres_16384(eta, seed=1) for eta in ETAS]
    for s in systems:
        s.extra["eta_r"] = round(s.extra["eta_r"], 1)
    # each step: one sweep of one of the four systems (bounded CPU sample)
    times, moves = [], 0
    drawn = evaluated = 0
    from oracle import oracle as O
    O.build()
    pos = {s.extra["eta_r"]: s.pos.copy() for s in systems}
    for step in range(args.warmup + args.steps):
        s = systems[step % len(systems)]
        eta = s.extra["eta_r"]
        t0 = time.perf_counter()
        p, _, c, _ = O.run(pos[eta], s.L, q=s.q, n_r=s.n_r, d_max=D_MAX_TUNED[eta], seed=1,
                           n_sweeps=1, sweep0=step // len(systems),
                           v0_mode=1 if args.v0 == "shell" else 0)
        dt = time.perf_counter() - t0
        pos[eta] = p
        if step >= args.warmup:
            times.append(dt)
            moves += c["moves"]
            drawn += c["dep_drawn"]
            evaluated += c["dep_evaluated"]
    total = sum(times)
    value = moves / total
    line = {
        "impl": "reference", "metric": "colloid trial moves/s", "value": value,
        "unit": "moves/s", "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * total / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "form": "serial CPU oracle", "v0": args.v0,
                   "step": "one sweep of one of the four eta_r systems (16384 moves)"},
        "insertions_drawn_per_s": drawn / total,
        "insertions_evaluated_per_s": evaluated / total,
        "cpu_baseline": {"value": value, "unit": "moves/s", "cores": 1, "kind": "oracle",
                         "sample": "%d sweeps x 16384 spheres, eta_r cycling 0.1..0.4"
                                   % args.steps},
        "e2e": {"value": value, "unit": "moves/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))


def tune_batch(ctx, hpmc, d0, ns, rounds=12, sweeps=15):
    """Untimed: melt the lattice starts and tune each replica's d_max to ~30%
    acceptance (per-replica counters)."""
    d = list(d0)
    for _ in range(rounds):
        for r, dr in enumerate(d):
            hpmc.hpmc_set_replica_moves(ctx, r, dr, 0.0, 1.0)
        hpmc.hpmc_reset_counters(ctx)
        hpmc.hpmc_sweep(ctx, sweeps)
        for r, n in enumerate(ns):
            _, _, cnt = hpmc.hpmc_get_replica(ctx, r, n)
            acc = cnt["accept"] / max(1, cnt["moves"])
            d[r] = d[r] * min(2.0, max(0.5, (acc + 0.02) / (ACC_TARGET + 0.02)))
    for r, dr in enumerate(d):
        hpmc.hpmc_set_replica_moves(ctx, r, dr, 0.0, 1.0)
    return d


def run_batched(args, ws, rank, local):
    """128 independent sphere replicas (N log-uniform in [500, 20000], phi_c
    U[0.1, 0.45], q in {0.1, 0.15, 0.2}, eta_r U[0.05, 0.4]) as one batch, vs the
    same replicas one at a time (each in its own context, one stream)."""
    import torch
    import torch.distributed as dist
    from paper_1508_07077_gb300 import build, hpmc, replicas as R, workloads as W

    if ws > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    try:
        hpmc.load()
    except ImportError:
        build.build()
        hpmc.load()
    prec = hpmc.HPMC_FP32_RECHECK if args.precision == "fp32" else hpmc.HPMC_FP64
    stream = torch.cuda.current_stream()
    reps = W.batched_replicas(128, seed=1)
    descs = [{"n": s.n, "box_l": s.L, "pos": s.pos, "q": s.q, "n_r": s.n_r, "n_trial": 0,
              "d_max": 0.01, "replica": R.replica_ids(128, rank)[k]}
             for k, s in enumerate(reps)]
    ctx = hpmc.hpmc_init_batch(descs, seed=1, precision=prec, device=local)
    ns = [s.n for s in reps]
    dtuned = tune_batch(ctx, hpmc, [0.01] * len(reps), ns, rounds=8, sweeps=10)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    for _ in range(args.warmup):
        hpmc.hpmc_sweep(ctx, 1, stream)
    hpmc.hpmc_reset_counters(ctx)
    torch.cuda.synchronize()
    if ws > 1:
        dist.barrier()
    a = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    b = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    with ClockSampler(local) as clk:
        for k in range(args.steps):
            flush.zero_()
            a[k].record(stream)
            hpmc.hpmc_sweep(ctx, 1, stream)
            b[k].record(stream)
        torch.cuda.synchronize()
    if ws > 1:
        dist.barrier()
    ms = sum(x.elapsed_time(y) for x, y in zip(a, b))
    _, cnt = hpmc.hpmc_get_state(ctx)
    # end to end through the C ABI with host buffers (pinned), copies timed
    host_pos = torch.empty((sum(ns), 3), dtype=torch.float64).pin_memory().numpy()
    sweep_e, _ = hpmc.hpmc_get_state(ctx, host_pos)
    e2e_steps = max(3, min(args.steps, 50) // 2)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for k in range(e2e_steps):
        hpmc.hpmc_set_state(ctx, host_pos, None, sweep_e + k, stream)
        hpmc.hpmc_sweep(ctx, 1, stream)
        hpmc.hpmc_get_state(ctx, host_pos, None, stream)
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    # one at a time
    allpos = np.empty((sum(ns), 3))
    sweep_now, _ = hpmc.hpmc_get_state(ctx, allpos)
    singles, off = [], 0
    for k, s in enumerate(reps):
        smp = hpmc.Sampler(allpos[off:off + s.n].copy(), s.L, q=s.q, n_r=s.n_r,
                           d_max=dtuned[k], seed=1, replica=descs[k]["replica"],
                           precision=prec, device=local)
        smp.sweep(1)
        singles.append(smp)
        off += s.n
    torch.cuda.synchronize()
    seq_steps = min(args.steps, 10)
    sa = [torch.cuda.Event(enable_timing=True) for _ in range(seq_steps)]
    sb = [torch.cuda.Event(enable_timing=True) for _ in range(seq_steps)]
    for k in range(seq_steps):
        flush.zero_()
        sa[k].record(stream)
        for smp in singles:
            smp.sweep(1, stream)
        sb[k].record(stream)
    torch.cuda.synchronize()
    seq_ms = sum(x.elapsed_time(y) for x, y in zip(sa, sb))
    for smp in singles:
        smp.close()
    # whole job: every rank's units over the slowest rank's time
    ms, seq_ms, e2e_s = R.reduce_max([ms, seq_ms, e2e_s], "cuda")
    moves_all, drawn_all, eval_all = R.reduce_sum(
        [cnt["moves"], cnt["dep_drawn"], cnt["dep_evaluated"]], "cuda")
    if rank == 0:
        value = moves_all / (ms * 1e-3)
        line = {
            "metric": "colloid trial moves/s", "value": value, "unit": "moves/s",
            "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32" if prec == 1 else "f64", "data": "synthetic",
            "config": {"workload": "batched_128_spheres_N500-20000",
                       "replicas": len(reps), "colloids": sum(ns),
                       "step": "1 sweep of every replica, one batch (one set of launches)",
                       "l2": "flushed between steps (256 MB write)"},
            "one_at_a_time_moves_per_s": ws * seq_steps * sum(ns) / (seq_ms * 1e-3),
            "e2e": {"value": ws * e2e_steps * sum(ns) / e2e_s, "unit": "moves/s",
                    "h2d_bytes_per_step": int(host_pos.nbytes),
                    "d2h_bytes_per_step": int(host_pos.nbytes)},
            "insertions_drawn_per_s": drawn_all / (ms * 1e-3),
            "insertions_evaluated_per_s": eval_all / (ms * 1e-3),
            "acceptance": cnt["accept"] / max(1, cnt["moves"]),
            "gpu_launches": args.steps * (1 + (1 if prec == 1 else 0) + 8),
            "clocks": clk.summary(),
        }
        print(json.dumps(line))
    hpmc.hpmc_destroy(ctx)
    if ws > 1:
        dist.destroy_process_group()


# Gibbs exchange kernel, per attempt of a depletant or CB-trial stream:
# Philox (40) + ball test (11) + ~6 colloids within reach x 8 (point test).
OPS_PER_GIBBS_TRIAL = 40.0 + 11.0 + 6 * 8.0


def run_gibbs(args, ws, rank, local):
    """Gibbs-ensemble coexistence runs (Sec. IV.B): 152 pairs (one CTA per
    pair) of two boxes of 512 spheres at phi_c = 0.12, q = 0.8, eta_r from
    0.80 to 1.00 across the pairs (a scan through coexistence), n_trial =
    100.  One step = 1 sweep of every box + 100 exchange attempts per pair.
    (512 per box: with q = 0.8 the cell width must exceed 1.8, and 256
    spheres would leave cells too wide for the cell-bin capacity.)"""
    import torch
    import torch.distributed as dist
    from paper_1508_07077_gb300 import build, hpmc, replicas as R, workloads as W

    if ws > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    try:
        hpmc.load()
    except ImportError:
        build.build()
        hpmc.load()
    prec = hpmc.HPMC_FP32_RECHECK if args.precision == "fp32" else hpmc.HPMC_FP64
    stream = torch.cuda.current_stream()
    n_pairs, N, phi, q, n_trial, n_ex = 152, 512, 0.12, 0.8, 100, 100
    etas = np.linspace(0.80, 1.00, n_pairs)
    base = rank * 2 * n_pairs
    boxes = []
    for p, eta in enumerate(etas):
        a = W.make_system("gibbs0", W.SPHERE, N, phi, q, float(eta), seed=1, replica=base + 2 * p)
        b = W.make_system("gibbs1", W.SPHERE, N, phi, q, float(eta), seed=1,
                          replica=base + 2 * p + 1)
        boxes.append((a, b))
    pairs = [((a.pos, a.L), (b.pos, b.L), {"q": q, "n_r": a.n_r, "n_trial": n_trial,
                                           "d_max": 0.15}) for a, b in boxes]
    gp = hpmc.GibbsPairs(pairs, seed=1, precision=prec, device=local, replica0=base)
    if args.warps != 1:
        hpmc.hpmc_set_launch(gp.ctx, args.warps, 1)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    for _ in range(args.warmup):
        gp.cycle(1, n_ex, stream)
    g0 = [hpmc.hpmc_get_gibbs(gp.ctx, p)[1] for p in range(n_pairs)]
    hpmc.hpmc_reset_counters(gp.ctx)
    torch.cuda.synchronize()
    if ws > 1:
        dist.barrier()
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(args.steps)]
    with ClockSampler(local) as clk:
        for k in range(args.steps):
            flush.zero_()
            ev[k][0].record(stream)
            hpmc.hpmc_sweep(gp.ctx, 1, stream)
            ev[k][1].record(stream)
            hpmc.hpmc_gibbs_exchange(gp.ctx, n_ex, stream)
            ev[k][2].record(stream)
        torch.cuda.synchronize()
    if ws > 1:
        dist.barrier()
    sweep_ms = sum(e[0].elapsed_time(e[1]) for e in ev)
    ex_ms = sum(e[1].elapsed_time(e[2]) for e in ev)
    ms = sweep_ms + ex_ms
    _, cnt = hpmc.hpmc_get_state(gp.ctx)
    g1 = [hpmc.hpmc_get_gibbs(gp.ctx, p)[1] for p in range(n_pairs)]
    gd = {k: sum(b[k] - a[k] for a, b in zip(g0, g1)) for k in g1[0]}
    live = hpmc.hpmc_get_live(gp.ctx, 2 * n_pairs)
    # end to end through the C ABI with host buffers (pinned), copies timed:
    # every box's slots uploaded (and checked), one sweep and the exchanges,
    # the slots and counters read back
    n_slots = sum(rep["n"] for rep in gp.reps)
    host_pos = torch.empty((n_slots, 3), dtype=torch.float64).pin_memory().numpy()
    sweep_now, _ = hpmc.hpmc_get_state(gp.ctx, host_pos)
    e2e_steps = max(3, min(args.steps, 20) // 2)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for k in range(e2e_steps):
        hpmc.hpmc_set_state(gp.ctx, host_pos, None, sweep_now + k, stream)
        gp.cycle(1, n_ex, stream)
        hpmc.hpmc_get_state(gp.ctx, host_pos, None, stream)
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    # the replica counters hold the sweeps' blocking depletants too: the
    # exchange's own rate per attempt from two more steps (untimed), the
    # counters read between the sweep and the exchanges
    ex_blk = 0
    for _ in range(2):
        hpmc.hpmc_sweep(gp.ctx, 1, stream)
        _, c_a = hpmc.hpmc_get_state(gp.ctx, None, None, stream)
        hpmc.hpmc_gibbs_exchange(gp.ctx, n_ex, stream)
        _, c_b = hpmc.hpmc_get_state(gp.ctx, None, None, stream)
        ex_blk += c_b["dep_blocking"] - c_a["dep_blocking"]
    blk_per_attempt = ex_blk / (2.0 * n_ex * n_pairs)
    gp.close()
    ms, ex_ms, e2e_s = R.reduce_max([ms, ex_ms, e2e_s], "cuda")
    attempts_all, moves_all, blocking_all = R.reduce_sum(
        [gd["attempts"], cnt["moves"], blk_per_attempt * gd["attempts"]], "cuda")
    if rank == 0:
        clocks = clk.summary()
        sms = torch.cuda.get_device_properties(local).multi_processor_count
        peak = sms * ISSUE_LANES_PER_SM * 2070.0e6 / 1e12
        # exchange kernel: depletant streams and 2 n_trial - 1 CB trials per
        # blocking depletant of an exchange, 6/pi attempts per point in the ball
        trials = 6.0 / math.pi * (gd["dep_drawn"] + blocking_all * (2 * n_trial - 1))
        achieved = OPS_PER_GIBBS_TRIAL * trials / (ex_ms * 1e-3) / 1e12
        line = {
            "metric": "Gibbs exchange attempts/s", "value": attempts_all / (ms * 1e-3),
            "unit": "attempts/s", "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32" if prec == 1 else "f64", "data": "synthetic",
            "config": {"workload": "gibbs_152_pairs_2x512_spheres_phi0.12_q0.8_eta0.8-1.0",
                       "n_trial": n_trial, "exchanges_per_pair_per_step": n_ex,
                       "step": "1 sweep of every box + 100 exchange attempts per pair",
                       "l2": "flushed between steps (256 MB write)"},
            "colloid_moves_per_s": moves_all / (ms * 1e-3),
            "exchange_ms_per_step": ex_ms / args.steps,
            "sweep_ms_per_step": sweep_ms / args.steps,
            "exchange_acceptance": gd["accept"] / max(1, gd["attempts"]),
            "exchange_outcomes": gd,
            "exchange_blocking_per_attempt": blk_per_attempt,
            "e2e": {"value": ws * e2e_steps * n_ex * n_pairs / e2e_s, "unit": "attempts/s",
                    "h2d_bytes_per_step": int(host_pos.nbytes),
                    "d2h_bytes_per_step": int(host_pos.nbytes)},
            "box_populations": {"min": min(live), "max": max(live)},
            "gpu_launches": args.steps * (1 + (1 if prec == 1 else 0) + 8 + 1),
            "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "Tops/s",
                         "frac": achieved / peak, "traffic": None, "kernel": "k_gibbs_exchange",
                         "peak_basis": "%d SMs x 128 lanes x 2070 MHz (issue rate)" % sms},
            "clocks": clocks,
        }
        if not args.no_cpu_baseline:
            from oracle import oracle as O
            O.build()
            a, b = boxes[0]
            t0 = time.perf_counter()
            _, _, _, _, g = O.gibbs_run(a.pos, b.pos, a.L, b.L, q=q, n_r=a.n_r, n_trial=n_trial,
                                        d_max=(0.15, 0.15), seed=1, replicas=(base, base + 1),
                                        n_cycles=args.cpu_cycles_gibbs, sweeps_per_cycle=1,
                                        ex_per_cycle=n_ex)
            dt = time.perf_counter() - t0
            line["cpu_baseline"] = {
                "value": g["attempts"] / dt, "unit": "attempts/s", "cores": 1, "kind": "oracle",
                "sample": "%d steps of pair 0 (eta_r 0.80) from the start (%d attempts, "
                          "%.1f s)" % (args.cpu_cycles_gibbs, g["attempts"], dt)}
        print(json.dumps(line))
    if ws > 1:
        dist.destroy_process_group()


# Anisotropic lens kernel, per depletant drawn: the sphere work plus the two
# body-frame tests (rotation 15 + shape test 15 lane-ops), the old-pose one
# for the ~55% that overlap the new pose; per move: two frames (2 x 20) more.
OPS_PER_DEP_ANISO = 6.0 / math.pi * (40.0 + 11.0) + 30.0 + 0.55 * 30.0
OPS_PER_MOVE_LENS_ANISO = 2 * 40.0 + 20.0 + 12.0 + 40.0
# Phase kernel, per move: ~25 candidates x 8 (bounding test) and ~4 near
# candidates through the FP32 portal refinement (~20 steps x 80 lane-ops).
OPS_PER_MOVE_PHASE_ANISO = 25 * 8.0 + 4 * 20 * 80.0


def run_shape(args, ws, rank, local):
    """One anisotropic system: 32768 hemispheres (phi_c 0.25, q 0.10, eta_r
    0.30) or 65536 discoids (phi_c 0.30, q 0.10, eta_r 0.25), translation and
    rotation moves (a_max 0.2 rad, p_translate 0.5), d_max tuned to ~30%
    acceptance, warps per colloid and cell size from the autotuner."""
    import torch
    import torch.distributed as dist
    from paper_1508_07077_gb300 import build, hpmc, replicas as R, workloads as W

    if ws > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    try:
        hpmc.load()
    except ImportError:
        build.build()
        hpmc.load()
    prec = hpmc.HPMC_FP32_RECHECK if args.precision == "fp32" else hpmc.HPMC_FP64
    sysf = W.hemispheres_32768 if args.workload == "hemispheres" else W.discoids_65536
    s = sysf(seed=1)
    stream = torch.cuda.current_stream()
    smp = hpmc.Sampler(s.pos, s.L, quat=s.quat, shape=s.shape, shape_params=s.shape_params,
                       q=s.q, n_r=s.n_r, d_max=0.02, a_max=s.a_max, p_translate=s.p_translate,
                       seed=1, replica=R.replica_ids(1, rank)[0], precision=prec,
                       device=local)
    ctx = smp.ctx
    d = 0.02
    for _ in range(10 if not args.no_tune else 0):
        hpmc.hpmc_set_moves(ctx, d, s.a_max, s.p_translate)
        hpmc.hpmc_reset_counters(ctx)
        hpmc.hpmc_sweep(ctx, 10)
        _, cnt = hpmc.hpmc_get_state(ctx)
        acc = cnt["accept"] / max(1, cnt["moves"])
        d = min(0.1, d * min(2.0, max(0.5, (acc + 0.02) / (ACC_TARGET + 0.02))))
    hpmc.hpmc_set_moves(ctx, d, s.a_max, s.p_translate)
    nc_auto = int(s.L / (1.0 + s.q)) & ~1
    cells = (0, nc_auto - 2) if nc_auto > 4 else (0,)
    warps, ncell, tuned_ms = hpmc.hpmc_autotune(ctx, warps=(1, 2, 4), cells=cells, n_sweeps=3)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    for _ in range(args.warmup):
        hpmc.hpmc_sweep(ctx, 1, stream)
    hpmc.hpmc_reset_counters(ctx)
    torch.cuda.synchronize()
    if ws > 1:
        dist.barrier()
    a = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    b = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    with ClockSampler(local) as clk:
        for k in range(args.steps):
            flush.zero_()
            a[k].record(stream)
            hpmc.hpmc_sweep(ctx, 1, stream)
            b[k].record(stream)
        torch.cuda.synchronize()
    if ws > 1:
        dist.barrier()
    ms = sum(x.elapsed_time(y) for x, y in zip(a, b))
    _, cnt = hpmc.hpmc_get_state(ctx)
    # per-kernel times (kernels launched one by one, events around each)
    hpmc.hpmc_set_timing(ctx, 1)
    hpmc.hpmc_reset_counters(ctx)
    tsweeps = min(args.steps, 10)
    hpmc.hpmc_sweep(ctx, tsweeps, stream)
    kern_ms, kern_n = hpmc.hpmc_get_timing(ctx)
    _, tc = hpmc.hpmc_get_state(ctx)
    hpmc.hpmc_set_timing(ctx, 0)
    # end to end through the C ABI with host buffers
    host_pos = torch.empty((s.n, 3), dtype=torch.float64).pin_memory().numpy()
    host_q = torch.empty((s.n, 4), dtype=torch.float64).pin_memory().numpy()
    sweep_now, _ = hpmc.hpmc_get_state(ctx, host_pos, host_q)
    e2e_steps = max(3, min(args.steps, 20) // 2)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for k in range(e2e_steps):
        hpmc.hpmc_set_state(ctx, host_pos, host_q, sweep_now + k, stream)
        hpmc.hpmc_sweep(ctx, 1, stream)
        hpmc.hpmc_get_state(ctx, host_pos, host_q, stream)
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    ms, e2e_s = R.reduce_max([ms, e2e_s], "cuda")
    moves_all, drawn_all, eval_all = R.reduce_sum(
        [cnt["moves"], cnt["dep_drawn"], cnt["dep_evaluated"]], "cuda")
    if rank == 0:
        sms = torch.cuda.get_device_properties(local).multi_processor_count
        peak = sms * ISSUE_LANES_PER_SM * 2070.0e6 / 1e12
        cand = {}
        if kern_n[2]:
            lens_ops = (OPS_PER_DEP_ANISO * tc["dep_drawn"] + OPS_PER_MOVE_LENS_ANISO * tc["moves"])
            cand["k_lens_aniso_fp32"] = (kern_ms[2], lens_ops / (kern_ms[2] * 1e-3) / 1e12)
        ph_ops = OPS_PER_MOVE_PHASE_ANISO * tc["moves"]
        ph_name = "k_phase_aniso_fp32" if prec == 1 else "k_phase_aniso_fp64"
        cand[ph_name] = (kern_ms[1], ph_ops / (kern_ms[1] * 1e-3) / 1e12)
        dominant = max(cand, key=lambda k: cand[k][0])
        achieved = cand[dominant][1]
        line = {
            "metric": "colloid trial moves/s", "value": moves_all / (ms * 1e-3),
            "unit": "moves/s", "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32" if prec == 1 else "f64", "data": "synthetic",
            "config": {"workload": s.name + "_phi%.2f_q%.2f_eta%.2f" % (
                           s.extra["phi_c"], s.q, s.extra["eta_r"]),
                       "form": "FP32+FP64 recheck" if prec == 1 else "FP64",
                       "n_trial": 0, "a_max": s.a_max, "p_translate": s.p_translate,
                       "d_max": round(d, 5), "step": "1 sweep (%d moves)" % s.n,
                       "autotuned": {"warps_per_colloid": warps, "n_cell": ncell,
                                     "ms_per_sweep": tuned_ms},
                       "l2": "flushed between steps (256 MB write)"},
            "insertions_drawn_per_s": drawn_all / (ms * 1e-3),
            "insertions_evaluated_per_s": eval_all / (ms * 1e-3),
            "acceptance": cnt["accept"] / max(1, cnt["moves"]),
            "translate_fraction": cnt["translate"] / max(1, cnt["moves"]),
            "fp64_rechecks_per_move": cnt["rechecks"] / max(1, cnt["moves"]),
            "gpu_launches": args.steps * (1 + (2 if prec == 1 else 0) + 8),
            "kernels": {"phase_ms_per_sweep": kern_ms[1] / tsweeps,
                        "lens_ms_per_sweep": kern_ms[2] / tsweeps,
                        "cells_ms_per_sweep": kern_ms[0] / tsweeps,
                        "achieved_tops": {k: v[1] for k, v in cand.items()}},
            "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "Tops/s",
                         "frac": achieved / peak, "traffic": None, "kernel": dominant,
                         "peak_basis": "%d SMs x 128 lanes x 2070 MHz (issue rate)" % sms},
            "clocks": clk.summary(),
            "e2e": {"value": ws * e2e_steps * s.n / e2e_s, "unit": "moves/s",
                    "h2d_bytes_per_step": s.n * 7 * 8, "d2h_bytes_per_step": s.n * 7 * 8 + 128},
        }
        if not args.no_cpu_baseline:
            from oracle import oracle as O
            O.build()
            pos, quat, _, _ = smp.state(with_quat=True)
            t0 = time.perf_counter()
            _, _, oc, _ = O.run(pos, s.L, shape=s.shape, shape_params=s.shape_params, quat=quat,
                                q=s.q, n_r=s.n_r, d_max=d, a_max=s.a_max,
                                p_translate=s.p_translate, seed=1, n_cell=ncell,
                                n_sweeps=args.cpu_sweeps_shape, sweep0=sweep_now + e2e_steps)
            dt = time.perf_counter() - t0
            line["cpu_baseline"] = {"value": oc["moves"] / dt, "unit": "moves/s", "cores": 1,
                                    "kind": "oracle",
                                    "sample": "%d sweeps of the system (%d moves, %.1f s)"
                                              % (args.cpu_sweeps_shape, oc["moves"], dt)}
        print(json.dumps(line))
    smp.close()
    if ws > 1:
        dist.destroy_process_group()


def run_ours(args, ws, rank, local):
    import torch
    import torch.distributed as dist
    from paper_1508_07077_gb300 import build, hpmc, replicas as R, workloads as W

    if ws > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    try:
        hpmc.load()
    except ImportError:
        build.build()
        hpmc.load()
    prec = hpmc.HPMC_FP32_RECHECK if args.precision == "fp32" else hpmc.HPMC_FP64
    stream = torch.cuda.current_stream()

    # the four state points as one batch (independent replicas, one set of
    # launches per sweep); this rank's replicas are keyed by its rank
    systems = [W.spheres_16384(eta, seed=1) for eta in ETAS]
    etas = [round(s.extra["eta_r"], 1) for s in systems]
    descs = [{"n": s.n, "box_l": s.L, "pos": s.pos, "q": s.q, "n_r": s.n_r, "n_trial": 0,
              "d_max": D_MAX_TUNED[e], "replica": R.replica_ids(len(systems), rank)[k]}
             for k, (s, e) in enumerate(zip(systems, etas))]
    ctx = hpmc.hpmc_init_batch(descs, seed=1, precision=prec, device=local)
    hpmc.hpmc_set_launch(ctx, args.warps, args.ilp)
    if args.v0 == "shell":
        hpmc.hpmc_set_v0(ctx, hpmc.HPMC_V0_SHELL)
    if args.soft > 0.0:
        hpmc.hpmc_set_soft(ctx, args.soft)
    ns = [s.n for s in systems]
    d0 = [D_MAX_TUNED[e] for e in etas]
    dtuned = d0 if args.no_tune else tune_batch(ctx, hpmc, d0, ns)
    dmax = dict(zip(etas, dtuned))
    torch.cuda.synchronize()

    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")

    def step():
        hpmc.hpmc_sweep(ctx, 1, stream)

    for _ in range(args.warmup):
        step()
    hpmc.hpmc_reset_counters(ctx)
    torch.cuda.synchronize()
    if ws > 1:
        dist.barrier()

    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    with ClockSampler(local) as clk:
        time.sleep(0.25)
        for k in range(args.steps):
            flush.zero_()
            starts[k].record(stream)
            step()
            ends[k].record(stream)
        torch.cuda.synchronize()
    if ws > 1:
        dist.barrier()
    ms = sum(a.elapsed_time(b) for a, b in zip(starts, ends))
    _, cnt = hpmc.hpmc_get_state(ctx)
    moves, drawn, evaluated = cnt["moves"], cnt["dep_drawn"], cnt["dep_evaluated"]
    rechecks, accept = cnt["rechecks"], cnt["accept"]

    # per-kernel durations (events around each launch, kernels launched one by one)
    hpmc.hpmc_reset_counters(ctx)
    hpmc.hpmc_set_timing(ctx, True)
    timing_steps = min(args.steps, 50)
    for k in range(timing_steps):
        flush.zero_()
        step()
    kern_ms, kern_n = hpmc.hpmc_get_timing(ctx)
    hpmc.hpmc_set_timing(ctx, False)
    _, tc = hpmc.hpmc_get_state(ctx)
    t_moves, t_eval, t_drawn = tc["moves"], tc["dep_evaluated"], tc["dep_drawn"]

    # the same batch with the shell-restricted V_0 (Sec. III.C remark), same
    # step sizes: reported beside the headline, which keeps the circumsphere
    shell = None
    if args.v0 == "circumsphere" and not args.no_shell and args.soft == 0.0:
        hpmc.hpmc_set_v0(ctx, hpmc.HPMC_V0_SHELL)
        for _ in range(args.warmup):
            step()
        hpmc.hpmc_reset_counters(ctx)
        torch.cuda.synchronize()
        sh_a = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
        sh_b = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
        for k in range(args.steps):
            flush.zero_()
            sh_a[k].record(stream)
            step()
            sh_b[k].record(stream)
        torch.cuda.synchronize()
        sh_ms = sum(a.elapsed_time(b) for a, b in zip(sh_a, sh_b))
        _, sc = hpmc.hpmc_get_state(ctx)
        hpmc.hpmc_reset_counters(ctx)
        hpmc.hpmc_set_timing(ctx, True)
        for k in range(timing_steps):
            flush.zero_()
            step()
        sk_ms, sk_n = hpmc.hpmc_get_timing(ctx)
        hpmc.hpmc_set_timing(ctx, False)
        hpmc.hpmc_set_v0(ctx, hpmc.HPMC_V0_CIRCUMSPHERE)
        sh_ms = R.reduce_max([sh_ms], "cuda")[0]
        sh_moves, sh_drawn = R.reduce_sum([sc["moves"], sc["dep_drawn"]], "cuda")
        shell = {"value": sh_moves / (sh_ms * 1e-3), "unit": "moves/s",
                 "ms_per_step": sh_ms / args.steps, "steps": args.steps,
                 "insertions_drawn_per_s": sh_drawn / (sh_ms * 1e-3),
                 "acceptance": sc["accept"] / max(1, sc["moves"]),
                 "fp64_rechecks_per_move": sc["rechecks"] / max(1, sc["moves"]),
                 "lens_ms_per_launch": sk_ms[2] / max(1, sk_n[2]),
                 "phase_ms_per_launch": sk_ms[1] / max(1, sk_n[1]),
                 "note": "V_0 = the excluded-volume shell of the move's level; same "
                         "acceptance probabilities, fewer depletants per move"}

    # the same four systems one at a time (separate contexts, one stream)
    allpos = np.empty((sum(ns), 3))
    sweep_now, _ = hpmc.hpmc_get_state(ctx, allpos)
    singles = []
    off = 0
    for k, s in enumerate(systems):
        smp = hpmc.Sampler(allpos[off:off + s.n].copy(), s.L, q=s.q, n_r=s.n_r,
                           d_max=dtuned[k], seed=1, replica=descs[k]["replica"],
                           precision=prec, warps=args.warps, ilp=args.ilp, device=local,
                           soft_eps=args.soft)
        hpmc.hpmc_set_state(smp.ctx, allpos[off:off + s.n].copy(), None, sweep_now)
        smp.sweep(1)
        singles.append(smp)
        off += s.n
    torch.cuda.synchronize()
    seq_steps = min(args.steps, 50)
    sa = [torch.cuda.Event(enable_timing=True) for _ in range(seq_steps)]
    sb = [torch.cuda.Event(enable_timing=True) for _ in range(seq_steps)]
    for k in range(seq_steps):
        flush.zero_()
        sa[k].record(stream)
        for smp in singles:
            smp.sweep(1, stream)
        sb[k].record(stream)
    torch.cuda.synchronize()
    seq_ms = sum(a.elapsed_time(b) for a, b in zip(sa, sb))
    for smp in singles:
        smp.close()

    # end to end through the C ABI with host buffers (pinned), copies timed
    host_pos = torch.empty((sum(ns), 3), dtype=torch.float64).pin_memory().numpy()
    sweep_now, _ = hpmc.hpmc_get_state(ctx, host_pos)
    torch.cuda.synchronize()
    e2e_steps = max(3, min(args.steps, 200) // 2)
    t0 = time.perf_counter()
    for k in range(e2e_steps):
        hpmc.hpmc_set_state(ctx, host_pos, None, sweep_now + k, stream)
        hpmc.hpmc_sweep(ctx, 1, stream)
        hpmc.hpmc_get_state(ctx, host_pos, None, stream)
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0

    # max over ranks
    ms, e2e_s, seq_ms = R.reduce_max([ms, e2e_s, seq_ms], "cuda")
    moves_all, drawn_all, eval_all = R.reduce_sum([moves, drawn, evaluated], "cuda")

    if rank == 0:
        clocks = clk.summary()
        sms = torch.cuda.get_device_properties(local).multi_processor_count
        phase_launch_ms = kern_ms[1] / max(1, kern_n[1])
        lens_launch_ms = kern_ms[2] / max(1, kern_n[2])
        f_peak = 2070.0e6
        peak = sms * ISSUE_LANES_PER_SM * f_peak / 1e12
        if kern_n[2]:
            lens_ops = (OPS_PER_DEP * t_drawn + OPS_PER_MOVE_LENS * t_moves) / kern_n[2]
            phase_ops = OPS_PER_MOVE_PHASE * t_moves / max(1, kern_n[1])
            cand = {"k_lens_sphere_fp32": (kern_ms[2], lens_ops / (lens_launch_ms * 1e-3) / 1e12),
                    "k_phase_sphere_fp32": (kern_ms[1],
                                            phase_ops / (phase_launch_ms * 1e-3) / 1e12)}
        else:
            ops = (OPS_PER_DEP * t_eval + OPS_PER_MOVE * t_moves) / max(1, kern_n[1])
            cand = {"k_phase_sphere_fp64": (kern_ms[1], ops / (phase_launch_ms * 1e-3) / 1e12)}
        dominant = max(cand, key=lambda k: cand[k][0])
        achieved = cand[dominant][1]
        bytes_per_launch = BYTES_PER_MOVE * t_moves / max(1, kern_n[1])
        value = moves_all / (ms * 1e-3)
        e2e_moves = ws * e2e_steps * sum(ns)
        line = {
            "metric": "colloid trial moves/s", "value": value, "unit": "moves/s",
            "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32" if prec == 1 else "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "form": "FP32+FP64 recheck" if prec == 1 else "FP64",
                       "v0": args.v0,
                       "colloid_depletant": ("Hertz eps=%g kT" % args.soft) if args.soft else "hard",
                       "n_trial": 0, "step": "1 sweep of each of 4 systems (65536 moves)",
                       "schedule": "4 systems as one batch (one set of launches per sweep)",
                       "d_max": {str(k): round(v, 5) for k, v in dmax.items()},
                       "l2": "flushed between steps (256 MB write)",
                       "warps_per_colloid": args.warps, "attempts_per_thread": args.ilp},
            "one_at_a_time_moves_per_s": ws * seq_steps * sum(ns) / (seq_ms * 1e-3),
            "insertions_drawn_per_s": drawn_all / (ms * 1e-3),
            "insertions_evaluated_per_s": eval_all / (ms * 1e-3),
            "acceptance": accept / max(1, moves),
            "fp64_rechecks_per_move": rechecks / max(1, moves),
            "gpu_launches": args.steps * (1 + (1 if prec == 1 else 0) + 8),
            "kernels": {"phase_ms_per_launch": phase_launch_ms,
                        "lens_ms_per_launch": lens_launch_ms,
                        "cells_ms_per_sweep": kern_ms[0] / max(1, kern_n[0]),
                        "share": {"cells": kern_ms[0] / max(1e-9, sum(kern_ms)),
                                  "phase": kern_ms[1] / max(1e-9, sum(kern_ms)),
                                  "lens": kern_ms[2] / max(1e-9, sum(kern_ms))},
                        "achieved_tops": {k: v[1] for k, v in cand.items()}},
            "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "Tops/s",
                         "frac": achieved / peak,
                         "traffic": MEASURED_TRAFFIC.get(dominant), "kernel": dominant,
                         "peak_basis": "%d SMs x 128 lanes x 2070 MHz (issue rate)" % sms,
                         "hbm_achieved_gbs": bytes_per_launch / (phase_launch_ms * 1e-3) / 1e9},
            "clocks": clocks,
            "e2e": {"value": e2e_moves / e2e_s, "unit": "moves/s",
                    "h2d_bytes_per_step": sum(ns) * 3 * 8,
                    "d2h_bytes_per_step": sum(ns) * 3 * 8 + 8 * 16},
        }
        if shell is not None:
            line["shell_v0"] = shell
        if not args.no_cpu_baseline:
            # the oracle on the host on a bounded sample of the same workload
            for s in systems:
                s.extra["eta_r"] = round(s.extra["eta_r"], 1)
            mv, dr, ev, dt, nm = cpu_oracle_rate(systems, dmax, args.cpu_sweeps,
                                                 v0_mode=1 if args.v0 == "shell" else 0,
                                                 soft_eps=args.soft)
            line["cpu_baseline"] = {
                "value": mv, "unit": "moves/s", "cores": 1, "kind": "oracle",
                "sample": "%d sweep(s) of each of the 4 systems from the fcc start "
                          "(%d moves, %.1f s)" % (args.cpu_sweeps, nm, dt),
                "insertions_evaluated_per_s": ev}
        print(json.dumps(line))
    hpmc.hpmc_destroy(ctx)
    if ws > 1:
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--precision", choices=("fp32", "fp64"), default="fp32")
    ap.add_argument("--warps", type=int, default=1)
    ap.add_argument("--ilp", type=int, default=1)
    ap.add_argument("--no-tune", action="store_true")
    ap.add_argument("--workload", choices=("spheres_16384", "batched", "hemispheres", "discoids",
                                           "gibbs"),
                    default="spheres_16384",
                    help="spheres_16384: the headline four-state-point workload; batched: "
                         "128 replicas of uneven size and state point; hemispheres / "
                         "discoids: 32768 hemispheres or 65536 discoids with rotations; "
                         "gibbs: 152 Gibbs-ensemble pairs (exchange attempts/s)")
    ap.add_argument("--cpu-cycles-gibbs", type=int, default=40)
    ap.add_argument("--v0", choices=("circumsphere", "shell"), default="circumsphere",
                    help="depletant region V_0 of the spheres workload: the new pose's "
                         "circumsphere (the paper's; default, with a shell measurement "
                         "alongside) or the excluded-volume shell of the move")
    ap.add_argument("--soft", type=float, default=0.0,
                    help="Hertz colloid-depletant interaction of this strength (kT), "
                         "in either form")
    ap.add_argument("--no-shell", action="store_true",
                    help="skip the shell-V_0 measurement beside the headline")
    ap.add_argument("--cpu-sweeps-shape", type=int, default=3)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-sweeps", type=int, default=40)
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    ws, rank, local = _dist()
    if args.impl == "reference":
        run_reference(args, ws, rank)
    elif args.workload == "batched":
        run_batched(args, ws, rank, local)
    elif args.workload in ("hemispheres", "discoids"):
        run_shape(args, ws, rank, local)
    elif args.workload == "gibbs":
        run_gibbs(args, ws, rank, local)
    else:
        run_ours(args, ws, rank, local)


if __name__ == "__main__":
    main()
