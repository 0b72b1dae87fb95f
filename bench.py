#!/usr/bin/env python
"""Throughput of the implicit-depletant HPMC hot path on one or more GB300s.

Metric: colloid trial moves/s (whole job), with depletant insertions/s (drawn
and evaluated) alongside, at fixed state points (phi_c, q, eta_r).

Headline workload (default, ``--workload batched``): 128 independent
hard-sphere replicas, N log-uniform in [500, 20000] (sum 621288 colloids),
phi_c U[0.1, 0.45], q in {0.1, 0.15, 0.2}, eta_r U[0.05, 0.4], all from one
seed, in one batch (one set of launches per sweep, recorded as a CUDA graph),
FP32 certified form with FP64 re-checks, n_trial = 0.  A step is one
checkerboard sweep of every replica.  Before timing, a fixed step-size
procedure runs (from the fcc starts, TUNE_ROUNDS rounds of TUNE_SWEEPS
sweeps, each replica's d_max scaled from its own acceptance counters towards
30%), then W warm-up sweeps.  The procedure uses only trajectory counters, so
any implementation of the method that reproduces the trajectories (the CPU
oracle does, bit for bit) arrives at the same step sizes and the same start.

Beside the headline, on the same JSON line (N = 1): the same replicas one at
a time, the 4 x 16384-sphere workload (FP32 form, shell V_0, plain FP64 form),
32768 hemispheres and 65536 discoids with rotations.

Timing: W untimed warm-up steps, then the K-step loop bracketed by CUDA
events on the launching stream with a 256 MB buffer written between steps
(L2 flush); the K-step loop is repeated until the timed region has lasted
at least a second (``repeats``), so that the clock sampler sees the load.
Multi-GPU (torchrun): every rank runs its own 128 replicas (weak scaling);
barrier + max over ranks.

``--impl reference`` times the CPU oracle (oracle/) on this host's cores on
the same workload, after the same step-size procedure: the reference arm of
this repository.
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
from concurrent.futures import ThreadPoolExecutor

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

ACC_TARGET = 0.30
TUNE_ROUNDS, TUNE_SWEEPS, D_START = 8, 5, 0.01
N_REPLICAS = 128
BATCHED = "batched_128_spheres_N500-20000_phi0.10-0.45_q0.10-0.20_eta0.05-0.40"

# Algorithmic ALU lane-operations per unit of work (the method's required
# arithmetic, counted from its operations, not from what a kernel skips):
#  Philox4x32-10 with the round keys precomputed: 10 rounds x (two 32x32
#  multiplies giving both halves of the product, two three-input XORs)
OPS_PHILOX = 40.0
#  an attempt of a one-point stream (CB trials, the Gibbs exchange): one
#  Philox call, three coordinates from the words (3 x 3) and the ball test
#  (3 FMA-type ops + compare): 13 more
OPS_ATTEMPT = OPS_PHILOX + 13.0
#  an attempt of a move's paired depletant stream: half a Philox call (two
#  points per call), the same coordinates and ball test
OPS_ATTEMPT_PAIRED = 0.5 * OPS_PHILOX + 13.0
#  an accepted point: the new- and old-pose tests (difference, squared length,
#  compare)
OPS_DEP = 8.0
#  per move in the lens kernel: the move and Poisson draws (one Philox
#  evaluation: lanes draw different counters), the proposal and its cell
#  test, the Poisson table search
OPS_MOVE_LENS = OPS_PHILOX + 20.0 + 12.0
#  per move in the colour phases: cell test, ~25 neighbour-pair tests (8
#  ops), the lens points against the neighbours near the move (~5 x 8)
OPS_MOVE_PHASE = 20.0 + 25 * 8.0 + 5 * 8.0
#  mean attempts per point of the ball: the cube-to-ball volume ratio
ATTEMPTS_PER_POINT = 6.0 / math.pi
#  FP64 form: FP64 instructions per attempt (coordinates 3 x 2, ball test 5)
#  and per accepted point (the pose tests, 2 x 5)
FP64_PER_ATTEMPT, FP64_PER_DEP = 11.0, 10.0
# Algorithmic HBM bytes per move: the FP64 pose read and written (2 x 32),
# the FP32 cell-relative copy (16), the cell-list entries (2 x 4)
BYTES_PER_MOVE = 2 * 32 + 16 + 2 * 4
# DRAM bytes (read + write) per launch of the headline's dominant kernel from
# the committed ncu capture of the current build (profiles/), keyed by
# (kernel, replicas, schedule): the mean over the 16 colour-phase launches of
# two timed sweeps of the 128-replica batch (L2 flushed before each step, ncu
# without cache control), or None for other cases.
MEASURED_TRAFFIC: dict = {("colour_phases", 128, 0): 44.0e6}
# The same without the flush buffer's write-back: the first phase after the
# flush writes back the flush's dirty lines (18.0 MB against 2.5 MB for the
# other phases); with its writes taken as the others' mean.
MEASURED_TRAFFIC_NO_WRITEBACK: dict = {("colour_phases", 128, 0): 42.0e6}


def _dist():
    from paper_1508_07077_gb300 import replicas
    return replicas.world()


def cpu_model() -> str:
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.lower().startswith("model name"):
                return ln.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        with open("/proc/cpuinfo") as f:
            for ln in f:
                if ln.lower().startswith("model name"):
                    return ln.split(":", 1)[1].strip()
    except OSError:
        pass
    return "unknown"


class ClockSampler:
    """nvidia-smi clock / throttle samples during the timed region."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

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


# --- the step-size procedure (identical on every implementation) -------------

def cell_width(L: float, q: float) -> float:
    """Width of the largest even checkerboard grid with cells >= 1 + q."""
    nc = int(L / (1.0 + q))
    nc -= nc & 1
    return L / nc


def tune_update(d: float, accept: int, moves: int, w: float) -> float:
    """One round of the step-size rule: scale towards 30% acceptance (at most
    a factor 2 either way), kept in [1e-4, w / 4]."""
    acc = accept / max(1, moves)
    d = d * min(2.0, max(0.5, (acc + 0.02) / (ACC_TARGET + 0.02)))
    return min(max(d, 1e-4), 0.25 * w)


def batched_workload(rank: int = 0, count: int = N_REPLICAS):
    """The batch (its first `count` replicas: a smaller case of the same
    workload, for profiler captures)."""
    from paper_1508_07077_gb300 import replicas as R, workloads as W
    reps = W.batched_replicas(N_REPLICAS, seed=1)[:count]
    keys = R.replica_ids(N_REPLICAS, rank)[:count]
    widths = [cell_width(s.L, s.q) for s in reps]
    return reps, keys, widths


# --- CPU oracle legs ------------------------------------------------------------

class OracleBatch:
    """The batch's replicas advanced by the CPU oracle, one replica per task on a
    pool of host threads (replicas are independent; the oracle's C code runs
    without the interpreter lock), or serially on one core."""

    def __init__(self, reps, keys, cores):
        from oracle import oracle as O
        O.build()
        self.O = O
        self.reps, self.keys, self.cores = reps, keys, cores
        self.pos = [s.pos.copy() for s in reps]
        self.sweep = 0

    def run(self, d, n_sweeps, cores=None):
        """n_sweeps sweeps of every replica with step sizes d; returns the
        per-replica counters."""
        cores = self.cores if cores is None else cores
        s0 = self.sweep

        def one(r):
            s = self.reps[r]
            p, _, c, _ = self.O.run(self.pos[r], s.L, q=s.q, n_r=s.n_r, d_max=d[r], seed=1,
                                    replica=self.keys[r], sweep0=s0, n_sweeps=n_sweeps)
            return p, c

        order = sorted(range(len(self.reps)), key=lambda r: -self.reps[r].n)
        if cores > 1:
            with ThreadPoolExecutor(max_workers=cores) as ex:
                res = dict(zip(order, ex.map(one, order)))
        else:
            res = {r: one(r) for r in order}
        self.sweep += n_sweeps
        cnts = []
        for r in range(len(self.reps)):
            self.pos[r] = res[r][0]
            cnts.append(res[r][1])
        return cnts

    def tune(self, widths):
        d = [D_START] * len(self.reps)
        for _ in range(TUNE_ROUNDS):
            cnts = self.run(d, TUNE_SWEEPS)
            d = [tune_update(d[r], c["accept"], c["moves"], widths[r]) for r, c in enumerate(cnts)]
        return d


def cpu_baseline_batched(d_gpu, warmup, rank, count=N_REPLICAS):
    """The oracle on this host: the step-size procedure and the warm-up sweeps
    on all cores, then one sweep of every replica on all cores (timed, 3
    times) and the same first sweep on one core (timed); the one-core and
    all-core results must be identical."""
    reps, keys, widths = batched_workload(rank, count)
    cores = os.cpu_count() or 1
    ob = OracleBatch(reps, keys, cores)
    t0 = time.perf_counter()
    d = ob.tune(widths)
    ob.run(d, warmup)
    prep_s = time.perf_counter() - t0
    start = [p.copy() for p in ob.pos]
    t0 = time.perf_counter()
    c_all = ob.run(d, 1)
    t_first = time.perf_counter() - t0
    after_first = [p.copy() for p in ob.pos]
    t0 = time.perf_counter()
    ob.run(d, 2)
    t_all = t_first + (time.perf_counter() - t0)
    moves_all = 3 * sum(s.n for s in reps)
    # one core, the same first sweep from the same state
    ob.pos, ob.sweep = start, ob.sweep - 3
    t0 = time.perf_counter()
    c_one = ob.run(d, 1, cores=1)
    t_one = time.perf_counter() - t0
    identical = all(np.array_equal(a, b) for a, b in zip(ob.pos, after_first)) and all(
        a == b for a, b in zip(c_all, c_one))
    moves_one = sum(c["moves"] for c in c_one)
    drawn = sum(c["dep_drawn"] for c in c_one)
    return {
        "value": moves_all / t_all, "unit": "moves/s", "cores": cores, "kind": "oracle",
        "cpu": cpu_model(),
        "sample": "the headline workload after the same step-size procedure and %d warm-up "
                  "sweeps (%.1f s on %d cores): 3 sweeps of every replica on %d cores "
                  "(%d moves, %.1f s), the first of them again on 1 core"
                  % (warmup, prep_s, cores, cores, moves_all, t_all),
        "one_core": {"value": moves_one / t_one, "unit": "moves/s", "cores": 1,
                     "seconds": t_one, "insertions_drawn_per_s": drawn / t_one},
        "one_core_equals_all_cores": bool(identical),
        "step_sizes_equal_gpu": bool(d_gpu is not None and np.array_equal(np.array(d),
                                                                          np.array(d_gpu))),
    }


def run_reference(args, ws, rank):
    """--impl reference: the oracle on this host's cores, same workload, same
    step-size procedure and warm-up, K timed steps of one sweep of every
    replica (replicas on a pool of threads)."""
    if rank != 0:
        return
    if args.workload != "batched":
        print(json.dumps({"impl": "reference", "unavailable":
                          "the reference arm covers the headline workload (batched) only"}))
        return
    reps, keys, widths = batched_workload(0, args.replicas)
    cores = os.cpu_count() or 1
    ob = OracleBatch(reps, keys, cores)
    d = ob.tune(widths)
    ob.run(d, args.warmup)
    times, moves, drawn, evaluated = [], 0, 0, 0
    for _ in range(args.steps):
        t0 = time.perf_counter()
        cnts = ob.run(d, 1)
        times.append(time.perf_counter() - t0)
        moves += sum(c["moves"] for c in cnts)
        drawn += sum(c["dep_drawn"] for c in cnts)
        evaluated += sum(c["dep_evaluated"] for c in cnts)
    total = sum(times)
    value = moves / total
    line = {
        "impl": "reference", "metric": "colloid trial moves/s", "value": value,
        "unit": "moves/s", "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * total / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": batched_config(args.replicas, sum(s.n for s in reps)),
        "insertions_drawn_per_s": drawn / total,
        "insertions_evaluated_per_s": evaluated / total,
        "cpu_baseline": {"value": value, "unit": "moves/s", "cores": cores, "kind": "oracle",
                         "cpu": cpu_model(),
                         "sample": "%d steps, each one sweep of every replica (%d moves), "
                                   "replicas on %d threads" % (args.steps, moves, cores)},
        "e2e": {"value": value, "unit": "moves/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))


def batched_config(count: int = N_REPLICAS, colloids: int = 621288):
    name = BATCHED if count == N_REPLICAS else BATCHED + "_first%d" % count
    return {"workload": name, "replicas": count, "colloids": colloids,
            "form": "FP32+FP64 recheck", "n_trial": 0,
            "step": "1 sweep of every replica (%d moves), one batch" % colloids,
            "start": "fcc starts, %d rounds x %d sweeps of the step-size rule (d_max from %g "
                     "towards 30%% acceptance, per replica), then the warm-up sweeps"
                     % (TUNE_ROUNDS, TUNE_SWEEPS, D_START),
            "l2": "flushed between steps (256 MB write)"}


# --- GPU helpers ---------------------------------------------------------------

def load_lib():
    from paper_1508_07077_gb300 import build, hpmc
    try:
        hpmc.load()
    except ImportError:
        build.build()
        hpmc.load()
    return hpmc


def timed_steps(step, K, stream, flush, min_ms=0.0, ws=1):
    """K steps bracketed by CUDA events (L2 flushed before each); the K-step
    loop is repeated until min_ms of timed time (the same count on every
    rank).  Returns (total ms, repeats)."""
    import torch
    import torch.distributed as dist

    def one():
        a = [torch.cuda.Event(enable_timing=True) for _ in range(K)]
        b = [torch.cuda.Event(enable_timing=True) for _ in range(K)]
        torch.cuda.synchronize()
        if ws > 1:
            dist.barrier()
        # an NVTX range over the timed launches, so that a profiler can be
        # limited to them (ncu --nvtx --nvtx-include "timed steps/")
        torch.cuda.nvtx.range_push("timed steps")
        for k in range(K):
            flush.zero_()
            a[k].record(stream)
            step()
            b[k].record(stream)
        torch.cuda.nvtx.range_pop()
        torch.cuda.synchronize()
        if ws > 1:
            dist.barrier()
        return sum(x.elapsed_time(y) for x, y in zip(a, b))

    from paper_1508_07077_gb300 import replicas as R
    first = one()
    reps = 1 if first >= min_ms else int(math.ceil(min_ms / max(first, 1e-3)))
    reps = int(R.reduce_max([reps], "cuda")[0]) if ws > 1 else reps
    total = first
    for _ in range(reps - 1):
        total += one()
    return total, reps


def kernel_times(hpmc, ctx, step, flush, n):
    """Per-kernel milliseconds over n steps (kernels launched one by one with
    events around them): (ms per kind, launches per kind, counters)."""
    hpmc.hpmc_reset_counters(ctx)
    hpmc.hpmc_set_timing(ctx, True)
    for _ in range(n):
        flush.zero_()
        step()
    km, kn = hpmc.hpmc_get_timing(ctx)
    hpmc.hpmc_set_timing(ctx, False)
    _, tc = hpmc.hpmc_get_state(ctx)
    return km, kn, tc


def lens_ops(tc):
    """Algorithmic lane-ops of the lens kernel for counters tc."""
    attempts = ATTEMPTS_PER_POINT * tc["dep_drawn"]
    return OPS_ATTEMPT_PAIRED * attempts + OPS_DEP * tc["dep_drawn"] + OPS_MOVE_LENS * tc["moves"]


def fp32_rooflines(km, kn, tc, pk):
    """Per-kernel achieved lane-ops/s and fractions of the measured ceilings
    (FP32 form): the lens kernel against the measured Philox-pipe ceiling
    (round-key Philox calls/s x 40 lane-ops), the colour phases against the
    measured FP32 issue ceiling (FFMA/s)."""
    out = {}
    philox_peak = pk["philox_rk_calls_per_s"] * OPS_PHILOX / 1e12
    fp32_peak = pk["ffma_per_s"] / 1e12
    if kn[2]:
        a = lens_ops(tc) / (km[2] * 1e-3) / 1e12
        # the generator's own share: one call per two attempts and one per move
        calls = 0.5 * ATTEMPTS_PER_POINT * tc["dep_drawn"] + tc["moves"]
        calls_rate = calls / (km[2] * 1e-3)
        out["k_lens_sphere_fp32"] = {"ms": km[2], "achieved": a, "peak": philox_peak,
                                     "frac": a / philox_peak,
                                     "peak_basis": "measured Philox4x32-10 (round keys) calls/s "
                                                   "x 40 lane-ops",
                                     "depletants_drawn_per_s": tc["dep_drawn"] / (km[2] * 1e-3),
                                     "philox_calls_per_s": calls_rate,
                                     "philox_frac_of_measured": calls_rate /
                                     pk["philox_rk_calls_per_s"]}
    if kn[1]:
        a = OPS_MOVE_PHASE * tc["moves"] / (km[1] * 1e-3) / 1e12
        out["colour_phases"] = {"ms": km[1], "achieved": a, "peak": fp32_peak,
                                "frac": a / fp32_peak,
                                "hbm_gbs": BYTES_PER_MOVE * tc["moves"] / (km[1] * 1e-3) / 1e9,
                                "peak_basis": "measured FP32 FMA/s (lane-ops)"}
    return out


# --- headline: 128 batched replicas -----------------------------------------------

def run_batched(args, ws, rank, local):
    import torch
    import torch.distributed as dist
    from paper_1508_07077_gb300 import peaks, replicas as R

    if ws > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    hpmc = load_lib()
    pk = peaks.measure()
    stream = torch.cuda.current_stream()
    reps, keys, widths = batched_workload(rank, args.replicas)
    ns = [s.n for s in reps]
    n_all = sum(ns)
    descs = [{"n": s.n, "box_l": s.L, "pos": s.pos, "q": s.q, "n_r": s.n_r, "n_trial": 0,
              "d_max": D_START, "replica": keys[k]} for k, s in enumerate(reps)]
    ctx = hpmc.hpmc_init_batch(descs, seed=1, precision=hpmc.HPMC_FP32_RECHECK, device=local)
    hpmc.hpmc_set_launch(ctx, 1, args.schedule)
    # the step-size procedure (the same rule the oracle legs replay)
    d = [D_START] * len(reps)
    for _ in range(TUNE_ROUNDS):
        for r, dr in enumerate(d):
            hpmc.hpmc_set_replica_moves(ctx, r, dr, 0.0, 1.0)
        hpmc.hpmc_reset_counters(ctx)
        hpmc.hpmc_sweep(ctx, TUNE_SWEEPS, stream)
        cnts = [hpmc.hpmc_get_replica(ctx, r, n)[2] for r, n in enumerate(ns)]
        d = [tune_update(d[r], c["accept"], c["moves"], widths[r]) for r, c in enumerate(cnts)]
    for r, dr in enumerate(d):
        hpmc.hpmc_set_replica_moves(ctx, r, dr, 0.0, 1.0)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")

    def step():
        hpmc.hpmc_sweep(ctx, 1, stream)

    for _ in range(args.warmup):
        step()
    hpmc.hpmc_reset_counters(ctx)
    with ClockSampler(local) as clk:
        ms, repeats = timed_steps(step, args.steps, stream, flush, min_ms=1000.0, ws=ws)
    _, cnt = hpmc.hpmc_get_state(ctx)
    km, kn, tc = kernel_times(hpmc, ctx, step, flush, min(args.steps, 20))
    # end to end through the C ABI with host (pinned) buffers: every step uploads
    # all positions (checked), sweeps, and reads all positions and counters back
    host_pos = torch.empty((n_all, 3), dtype=torch.float64).pin_memory().numpy()
    sweep_now, _ = hpmc.hpmc_get_state(ctx, host_pos)
    e2e_steps = max(3, min(args.steps, 50) // 2)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for k in range(e2e_steps):
        hpmc.hpmc_set_state(ctx, host_pos, None, sweep_now + k, stream)
        hpmc.hpmc_sweep(ctx, 1, stream)
        hpmc.hpmc_get_state(ctx, host_pos, None, stream)
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    # the other schedule of the colour phases, same state (context)
    other = None
    if not args.no_extras:
        hpmc.hpmc_set_launch(ctx, 1, 1 - args.schedule)
        for _ in range(3):
            step()
        o_ms, _ = timed_steps(step, args.steps, stream, flush)
        other = {"schedule": "eight launches per sweep" if args.schedule == 1
                 else "one persistent launch per sweep",
                 "value": args.steps * n_all / (o_ms * 1e-3), "ms_per_step": o_ms / args.steps}
        hpmc.hpmc_set_launch(ctx, 1, args.schedule)
    # the same replicas one at a time (each in its own context, one stream)
    seq = None
    if not args.no_extras:
        allpos = np.empty((n_all, 3))
        sweep_now, _ = hpmc.hpmc_get_state(ctx, allpos)
        singles, off = [], 0
        for k, s in enumerate(reps):
            smp = hpmc.Sampler(allpos[off:off + s.n].copy(), s.L, q=s.q, n_r=s.n_r, d_max=d[k],
                               seed=1, replica=keys[k], precision=hpmc.HPMC_FP32_RECHECK,
                               schedule=args.schedule, device=local)
            smp.sweep(1)
            singles.append(smp)
            off += s.n

        def seq_step():
            for smp in singles:
                smp.sweep(1, stream)

        seq_ms, _ = timed_steps(seq_step, min(args.steps, 10), stream, flush)
        for smp in singles:
            smp.close()
        seq = min(args.steps, 10) * n_all / (seq_ms * 1e-3)
    hpmc.hpmc_destroy(ctx)

    ms, e2e_s = R.reduce_max([ms, e2e_s], "cuda")
    moves_all, drawn_all, eval_all = R.reduce_sum(
        [cnt["moves"], cnt["dep_drawn"], cnt["dep_evaluated"]], "cuda")
    line = None
    if rank == 0:
        roof = fp32_rooflines(km, kn, tc, pk)
        dominant = max(roof, key=lambda k: roof[k]["ms"])
        dom = roof[dominant]
        value = moves_all / (ms * 1e-3)
        # kind 0 is the cell-list pair of launches (bins, task order)
        launches_per_step = (2 * kn[0] + kn[1] + kn[2]) / max(1, min(args.steps, 20))
        line = {
            "metric": "colloid trial moves/s", "value": value, "unit": "moves/s",
            "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms / (args.steps * repeats), "repeats": repeats,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": dict(batched_config(args.replicas, n_all), schedule="persistent colour phases"
                           if args.schedule == 1 else "eight phase launches per sweep",
                           timed_region="the K-step loop repeated %d times (>= 1 s)" % repeats),
            "insertions_drawn_per_s": drawn_all / (ms * 1e-3),
            "insertions_evaluated_per_s": eval_all / (ms * 1e-3),
            "acceptance": cnt["accept"] / max(1, cnt["moves"]),
            "fp64_rechecks_per_move": cnt["rechecks"] / max(1, cnt["moves"]),
            "step_sizes": {"min": min(d), "median": statistics.median(d), "max": max(d)},
            "gpu_launches": int(round(launches_per_step * args.steps * repeats)),
            "kernels": {"cells_ms_per_step": km[0] / max(1, min(args.steps, 20)),
                        "lens_ms_per_step": km[2] / max(1, min(args.steps, 20)),
                        "phases_ms_per_step": km[1] / max(1, min(args.steps, 20)),
                        "share": {"cells": km[0] / sum(km), "lens": km[2] / sum(km),
                                  "phases": km[1] / sum(km)},
                        "rooflines": roof},
            "roofline": {"bound": "alu", "achieved": dom["achieved"], "peak": dom["peak"],
                         "unit": "Tops/s", "frac": dom["frac"],
                         "traffic": MEASURED_TRAFFIC.get((dominant, args.replicas, args.schedule)),
                         "traffic_without_flush_writeback":
                             MEASURED_TRAFFIC_NO_WRITEBACK.get((dominant, args.replicas, args.schedule)),
                         "traffic_algorithmic": BYTES_PER_MOVE * n_all / 8.0
                         if dominant == "colour_phases" else None,
                         "kernel": dominant,
                         "peak_basis": dom["peak_basis"] + " (of measured)"},
            "pipe_peaks_measured": pk,
            "clocks": clk.summary(),
            "e2e": {"value": ws * e2e_steps * n_all / e2e_s, "unit": "moves/s",
                    "h2d_bytes_per_step": int(host_pos.nbytes),
                    "d2h_bytes_per_step": int(host_pos.nbytes) + 8 * 16},
        }
        if other is not None:
            line["other_schedule"] = other
        if seq is not None:
            line["one_at_a_time_moves_per_s"] = seq
    if ws > 1:
        dist.destroy_process_group()
    return line, d


# --- extras: the single-system workloads ------------------------------------------

def spheres_16384(args, local, pk):
    """The four 16384-sphere state points (phi_c 0.30, q 0.15, eta_r 0.1..0.4)
    as one batch: FP32 form (and its shell V_0), plain FP64 form; oracle on all
    cores for 2 sweeps from the same tuned state."""
    import torch
    from paper_1508_07077_gb300 import workloads as W
    hpmc = load_lib()
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    etas = (0.1, 0.2, 0.3, 0.4)
    systems = [W.spheres_16384(eta, seed=1) for eta in etas]
    widths = [cell_width(s.L, s.q) for s in systems]
    out = {"workload": "spheres_16384_phi0.30_q0.15_eta0.1-0.4 (4 x 16384, one batch)"}
    K = min(args.steps, 20)
    for prec in (1, 0):
        descs = [{"n": s.n, "box_l": s.L, "pos": s.pos, "q": s.q, "n_r": s.n_r,
                  "d_max": D_START, "replica": k} for k, s in enumerate(systems)]
        ctx = hpmc.hpmc_init_batch(descs, seed=1, precision=prec, device=local)
        d = [D_START] * 4
        for _ in range(TUNE_ROUNDS):
            for r, dr in enumerate(d):
                hpmc.hpmc_set_replica_moves(ctx, r, dr, 0.0, 1.0)
            hpmc.hpmc_reset_counters(ctx)
            hpmc.hpmc_sweep(ctx, TUNE_SWEEPS, stream)
            cnts = [hpmc.hpmc_get_replica(ctx, r, s.n)[2] for r, s in enumerate(systems)]
            d = [tune_update(d[r], c["accept"], c["moves"], widths[r])
                 for r, c in enumerate(cnts)]
        for r, dr in enumerate(d):
            hpmc.hpmc_set_replica_moves(ctx, r, dr, 0.0, 1.0)

        def step():
            hpmc.hpmc_sweep(ctx, 1, stream)

        for _ in range(3):
            step()
        hpmc.hpmc_reset_counters(ctx)
        ms, _ = timed_steps(step, K, stream, flush)
        _, cnt = hpmc.hpmc_get_state(ctx)
        km, kn, tc = kernel_times(hpmc, ctx, step, flush, K)
        res = {"value": cnt["moves"] / (ms * 1e-3), "unit": "moves/s", "ms_per_step": ms / K,
               "insertions_drawn_per_s": cnt["dep_drawn"] / (ms * 1e-3),
               "acceptance": cnt["accept"] / max(1, cnt["moves"]),
               "d_max": [round(x, 5) for x in d],
               "kernel_ms_per_step": {"cells": km[0] / K, "phases": km[1] / K, "lens": km[2] / K}}
        if prec == 1:
            res["fp64_rechecks_per_move"] = cnt["rechecks"] / max(1, cnt["moves"])
            res["rooflines"] = fp32_rooflines(km, kn, tc, pk)
            hpmc.hpmc_set_v0(ctx, hpmc.HPMC_V0_SHELL)
            for _ in range(3):
                step()
            hpmc.hpmc_reset_counters(ctx)
            sms, _ = timed_steps(step, K, stream, flush)
            _, sc = hpmc.hpmc_get_state(ctx)
            res["shell_v0"] = {"value": sc["moves"] / (sms * 1e-3), "ms_per_step": sms / K,
                               "insertions_drawn_per_s": sc["dep_drawn"] / (sms * 1e-3),
                               "acceptance": sc["accept"] / max(1, sc["moves"])}
            hpmc.hpmc_set_v0(ctx, hpmc.HPMC_V0_CIRCUMSPHERE)
            # the soft (Hertz, eps = 10 kT) colloid-depletant interaction,
            # same systems and steps
            hpmc.hpmc_set_soft(ctx, 10.0)
            for _ in range(3):
                step()
            hpmc.hpmc_reset_counters(ctx)
            fms, _ = timed_steps(step, K, stream, flush)
            _, fc = hpmc.hpmc_get_state(ctx)
            res["soft_eps10"] = {"value": fc["moves"] / (fms * 1e-3), "ms_per_step": fms / K,
                                 "acceptance": fc["accept"] / max(1, fc["moves"]),
                                 "fp64_rechecks_per_move": fc["rechecks"] / max(1, fc["moves"])}
            hpmc.hpmc_set_soft(ctx, 0.0)
            out["fp32"] = res
            # the oracle on all cores (cells of a colour phase on threads), 2
            # sweeps of each system from the fcc start at the starting step size
            if not args.no_cpu_baseline:
                from oracle import oracle as O
                O.build()
                cores = os.cpu_count() or 1
                t0 = time.perf_counter()
                moves = 0
                for k, s in enumerate(systems):
                    _, _, c, _ = O.run(s.pos, s.L, q=s.q, n_r=s.n_r, d_max=D_START, seed=1,
                                       replica=k, n_sweeps=2, threads=cores)
                    moves += c["moves"]
                dt = time.perf_counter() - t0
                out["cpu_oracle_all_cores"] = {"value": moves / dt, "unit": "moves/s",
                                               "cores": cores,
                                               "sample": "2 sweeps of each system from the "
                                                         "fcc start at d_max %g" % D_START}
        else:
            fp64_peak = pk["dfma_per_s"] / 1e12
            ops = (FP64_PER_ATTEMPT * ATTEMPTS_PER_POINT + FP64_PER_DEP) * tc["dep_evaluated"]
            a = ops / (km[1] * 1e-3) / 1e12
            res["roofline_fp64"] = {"kernel": "k_phase_sphere_fp64", "achieved": a,
                                    "peak": fp64_peak, "unit": "T FP64 inst/s",
                                    "frac": a / fp64_peak,
                                    "peak_basis": "measured FP64 FMA/s (instructions)"}
            out["fp64"] = res
        hpmc.hpmc_destroy(ctx)
    return out


def shape_system(args, local, kind, pk):
    """32768 hemispheres or 65536 discoids with rotations (a_max 0.2 rad,
    p_translate 0.5), step size tuned, warps per colloid and cell count from
    the autotuner, FP32 form."""
    import torch
    from paper_1508_07077_gb300 import workloads as W
    hpmc = load_lib()
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    s = W.hemispheres_32768(seed=1) if kind == "hemispheres" else W.discoids_65536(seed=1)
    smp = hpmc.Sampler(s.pos, s.L, quat=s.quat, shape=s.shape, shape_params=s.shape_params,
                       q=s.q, n_r=s.n_r, d_max=0.02, a_max=s.a_max, p_translate=s.p_translate,
                       seed=1, precision=hpmc.HPMC_FP32_RECHECK, device=local)
    ctx = smp.ctx
    d = 0.02
    for _ in range(6):
        hpmc.hpmc_set_moves(ctx, d, s.a_max, s.p_translate)
        hpmc.hpmc_reset_counters(ctx)
        hpmc.hpmc_sweep(ctx, 5)
        _, c = hpmc.hpmc_get_state(ctx)
        d = min(0.1, d * min(2.0, max(0.5, (c["accept"] / max(1, c["moves"]) + 0.02) /
                                      (ACC_TARGET + 0.02))))
    hpmc.hpmc_set_moves(ctx, d, s.a_max, s.p_translate)
    nc_auto = int(s.L / (1.0 + s.q)) & ~1
    cells = (0, nc_auto - 2) if nc_auto > 4 else (0,)
    warps, ncell, tuned_ms = hpmc.hpmc_autotune(ctx, warps=(1, 2), cells=cells, n_sweeps=3)

    def step():
        hpmc.hpmc_sweep(ctx, 1, stream)

    K = min(args.steps, 10)
    for _ in range(3):
        step()
    hpmc.hpmc_reset_counters(ctx)
    ms, _ = timed_steps(step, K, stream, flush)
    _, cnt = hpmc.hpmc_get_state(ctx)
    km, kn, tc = kernel_times(hpmc, ctx, step, flush, K)
    smp.close()
    return {"workload": "%s_%d_phi%.2f_q%.2f_eta%.2f" % (kind, s.n, s.extra["phi_c"], s.q,
                                                        s.extra["eta_r"]),
            "value": cnt["moves"] / (ms * 1e-3), "unit": "moves/s", "ms_per_step": ms / K,
            "insertions_drawn_per_s": cnt["dep_drawn"] / (ms * 1e-3),
            "acceptance": cnt["accept"] / max(1, cnt["moves"]),
            "fp64_rechecks_per_move": cnt["rechecks"] / max(1, cnt["moves"]),
            "d_max": round(d, 5), "autotuned": {"warps_per_colloid": warps, "n_cell": ncell,
                                                "ms_per_sweep": tuned_ms},
            "kernel_ms_per_step": {"cells": km[0] / K, "phases": km[1] / K, "lens": km[2] / K}}


# --- Gibbs-ensemble exchange (separate workload) ------------------------------------

# Gibbs exchange kernel, per attempt of a depletant or CB-trial stream:
# Philox, the ball test, ~6 colloids within reach x 8 (point test).
OPS_PER_GIBBS_TRIAL = OPS_ATTEMPT + 6 * 8.0


def run_gibbs(args, ws, rank, local):
    """Gibbs-ensemble coexistence runs (Sec. IV.B): 152 pairs (one CTA per
    pair) of two boxes of 512 spheres at phi_c = 0.12, q = 0.8, eta_r from
    0.80 to 1.00 across the pairs, n_trial = 100.  One step = 1 sweep of
    every box + 100 exchange attempts per pair."""
    import torch
    import torch.distributed as dist
    from paper_1508_07077_gb300 import peaks, replicas as R, workloads as W

    if ws > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    hpmc = load_lib()
    pk = peaks.measure()
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
    gp = hpmc.GibbsPairs(pairs, seed=1, precision=hpmc.HPMC_FP32_RECHECK, device=local,
                         replica0=base)
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
        torch.cuda.nvtx.range_push("timed steps")
        for k in range(args.steps):
            flush.zero_()
            ev[k][0].record(stream)
            hpmc.hpmc_sweep(gp.ctx, 1, stream)
            ev[k][1].record(stream)
            hpmc.hpmc_gibbs_exchange(gp.ctx, n_ex, stream)
            ev[k][2].record(stream)
        torch.cuda.nvtx.range_pop()
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
        peak = pk["philox_rk_calls_per_s"] * OPS_PHILOX / 1e12
        trials = ATTEMPTS_PER_POINT * (gd["dep_drawn"] + blocking_all * (2 * n_trial - 1))
        achieved = OPS_PER_GIBBS_TRIAL * trials / (ex_ms * 1e-3) / 1e12
        line = {
            "metric": "Gibbs exchange attempts/s", "value": attempts_all / (ms * 1e-3),
            "unit": "attempts/s", "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
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
            "gpu_launches": args.steps * (4 + 1),
            "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "Tops/s",
                         "frac": achieved / peak, "traffic": None, "kernel": "k_gibbs_exchange",
                         "peak_basis": "measured Philox4x32-10 (round keys) calls/s x 40 "
                                       "lane-ops (of measured)"},
            "clocks": clk.summary(),
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
                "cpu": cpu_model(),
                "sample": "%d steps of pair 0 (eta_r 0.80) from the start (%d attempts, "
                          "%.1f s)" % (args.cpu_cycles_gibbs, g["attempts"], dt)}
        print(json.dumps(line))
    if ws > 1:
        dist.destroy_process_group()


SINGLE = ("spheres_16384", "hemispheres_32768", "discoids_65536")


def single_entry(args, local, name, pk):
    if name == "spheres_16384":
        return spheres_16384(args, local, pk)
    return shape_system(args, local, name.split("_")[0], pk)


def run_single(args, ws, rank, local):
    """One single-system workload on its own (rank 0 of a 1-GPU run): its
    entry of the headline line's "extra" object, printed as one JSON line."""
    import torch
    from paper_1508_07077_gb300 import peaks
    if ws > 1:
        raise SystemExit("--workload %s runs on one GPU" % args.workload)
    torch.cuda.set_device(local)
    entry = single_entry(args, local, args.workload, peaks.measure())
    print(json.dumps({"workload": args.workload, "n_gpus": 1, "steps": args.steps,
                      "warmup": args.warmup, "data": "synthetic", **entry}))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--workload", choices=("batched", "gibbs") + SINGLE, default="batched",
                    help="batched: the headline 128-replica workload, with the single-system "
                         "workloads beside it; gibbs: 152 Gibbs-ensemble pairs (exchange "
                         "attempts/s); a single-system name runs that entry alone (e.g. for "
                         "profiler captures)")
    ap.add_argument("--schedule", type=int, choices=(0, 1), default=0,
                    help="colour phases: 0 eight launches per sweep, 1 one persistent launch")
    ap.add_argument("--replicas", type=int, default=N_REPLICAS,
                    help="the first R replicas of the batch (a smaller case of the same "
                         "workload, e.g. for profiler captures); 128 is the headline")
    ap.add_argument("--no-extras", action="store_true",
                    help="the headline only (no one-at-a-time run, other schedule or "
                         "single-system workloads)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-cycles-gibbs", type=int, default=40)
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if not 1 <= args.replicas <= N_REPLICAS:
        ap.error("--replicas must be in 1..%d" % N_REPLICAS)
    ws, rank, local = _dist()
    if args.impl == "reference":
        run_reference(args, ws, rank)
        return
    if args.workload == "gibbs":
        run_gibbs(args, ws, rank, local)
        return
    if args.workload in SINGLE:
        run_single(args, ws, rank, local)
        return
    line, d = run_batched(args, ws, rank, local)
    if rank != 0:
        return
    if ws == 1 and not args.no_extras:
        pk = line["pipe_peaks_measured"]
        line["extra"] = {name: single_entry(args, local, name, pk) for name in SINGLE}
    if ws == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline_batched(d, args.warmup, rank, args.replicas)
    print(json.dumps(line))


if __name__ == "__main__":
    main()
