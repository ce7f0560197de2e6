#!/usr/bin/env python
"""Benchmark of the grey IMEX PD-ARS radiation step on the 256^3 turbulent box.

Metric: Mcell-updates/s, one cell-update = one cell advanced through both
stages of one step.  Default run: one GPU, FP64, HLL TAU mode.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--precision fp64|mixed]
                  [--hll tau|none] [--n 256] [--impl ours|reference]

* value: K steps enqueued back to back on the library stream, timed with CUDA
  events after W warm-up steps; the state (1.34 GB at 256^3 FP64) is larger
  than L2, so no flush is needed between steps.
* e2e: the same metric through the public API with host buffers: every step
  copies the full input state from pinned host memory, runs one step and
  reads the full state back (wall clock, synchronised), in one call
  (rhd_step_host) whose chunked copies overlap the stage kernels; the three
  separate calls (set, step, get) are reported beside it.
* roofline: the dominant stage kernel is bound by the FP64 pipe: its FP64
  flops per launch (ncu thread counts per cell, profiles/kernel_counts.json,
  times the cells) over its mean event-timed duration inside the timed
  region, against the FP64 multiply-add throughput measured on this GPU by
  the library's probe (rhd_fma_probe); the HBM view beside it.  Every form
  (mixed, PPM, batched, adjoint) carries the same views, mixed precision also
  the FP32 pipe's.
* cpu_baseline: the CPU oracle (serial C) on every host core at once: one
  oracle process per core, each on its own periodic sub-box of the same
  initial state with the same dt; the one-core rate beside it.
* --impl reference: the CPU oracle is the reference arm; each step is one
  oracle step on a sub-box of the workload per host core, all at once.
* Several GPUs (torchrun): every rank advances its own independent box (weak
  scaling, no data-path collective); value = all ranks' cell-updates / the
  slowest rank's time.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "Mcell-updates/s per IMEX RHD step at 256^3, FP64 vs mixed; % HBM peak; adj/fwd"
UNIT = "Mcell-updates/s"
# algorithmic HBM bytes per cell of one launch of each stage kernel:
# stage 1 reads y(n) (8 fields) + rho + kappa and writes y(n+1/2) (8 fields);
# stage 2 reads y(n), y(n+1/2), rho, kappa and writes y(n+1).
ALG_BYTES = {0: 8 * (8 + 2 + 8), 1: 8 * (8 + 8 + 2 + 8)}
KERNEL_NAMES = {0: "stage1", 1: "stage2"}
FALLBACK_HBM_GBS = 6800.0
# FP64 peak of the GB300 from its unit counts and clock: 152 SMs x 2 DFMA per
# clock x 2 flops x 2.07 GHz (the library's probe, rhd_fma_probe, reaches
# 1.24-1.25 TFLOP/s of it on the GB300)
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12
# FP64 flops per face of the hydrodynamic face kernel (PLM, ncu thread
# counts dadd + dmul + 2 dfma at 128^3)
HYDRO_FACE_FLOPS = 210


def parse(argv=None):
    ap = argparse.ArgumentParser(description=__doc__,
                                 formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="fp64", choices=["fp64", "mixed"])
    ap.add_argument("--hll", default="tau", choices=["tau", "none"])
    ap.add_argument("--reconstruction", default="plm", choices=["plm", "ppm", "ppm_cs"],
                    help="face states of the headline form (Sec. 3.3)")
    ap.add_argument("--n", type=int, default=256)
    ap.add_argument("--e2e-steps", type=int, default=0,
                    help="timed end-to-end steps (0: --steps)")
    ap.add_argument("--cpu-sample", type=int, default=96,
                    help="edge of the oracle's sub-box for the one-core cpu_baseline")
    ap.add_argument("--cpu-edge", type=int, default=64,
                    help="edge of each host core's sub-box for the all-cores cpu_baseline")
    ap.add_argument("--ref-sample", type=int, default=48,
                    help="edge of the oracle's sub-box per reference-arm step")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-batched", action="store_true",
                    help="skip the 512-problem batched workload")
    ap.add_argument("--no-adjoint", action="store_true",
                    help="skip the 512^2 differentiation workload")
    ap.add_argument("--adj-n", type=int, default=512)
    ap.add_argument("--no-split", action="store_true",
                    help="skip the hydrodynamic step and the operator-split step")
    ap.add_argument("--no-slabs", action="store_true",
                    help="skip the step of the box as two z-slabs")
    ap.add_argument("--batched-only", action="store_true",
                    help="time only the 512-problem batched workload (for profiling); "
                         "prints its own JSON line")
    ap.add_argument("--batched-steps", type=int, default=500,
                    help="steps of the batched workload (its configuration: 500)")
    ap.add_argument("--no-graph", action="store_true",
                    help="batched workload: enqueue the launches instead of replaying a "
                         "CUDA graph (for profilers that do not see graph nodes)")
    ap.add_argument("--hydro-only", action="store_true",
                    help="time only the hydrodynamic step on the --n^3 box (for "
                         "profiling); prints its own JSON line")
    ap.add_argument("--single-form", action="store_true",
                    help="time only --precision (default: FP64 and mixed)")
    return ap.parse_args(argv)


# ------------------------------------------------------------------ helpers

def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def kernel_counts_record():
    """Per-cell ncu counts (FP64/FP32 flops, DRAM bytes, pipe utilisation) of
    the stage, batch and adjoint kernels from the committed summary
    (profiles/kernel_counts.json), or None if the kernel sources have changed
    since those captures."""
    import hashlib
    path = os.path.join(ROOT, "profiles", "kernel_counts.json")
    try:
        rec = json.load(open(path))
        h = hashlib.sha256()
        for f in rec["sources"]:
            h.update(open(os.path.join(ROOT, f), "rb").read())
        return rec if h.hexdigest()[:16] == rec["sources_sha256_16"] else None
    except (OSError, ValueError, KeyError):
        return None


def measure_fma_peaks(rhd, torch):
    """FP64 and FP32 multiply-add throughput of this GPU in TFLOP/s: the
    library's probe (rhd_fma_probe, 8 independent chains per thread, 8 blocks
    of 256 threads per SM), best of 5 CUDA-event-timed launches after one
    warm-up."""
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    stream = torch.cuda.current_stream()
    out = {"method": "rhd_fma_probe: %d blocks x 256 threads x 8 independent FMA chains, "
                     "best of 5 event-timed launches" % (8 * sms), "sms": sms}
    for prec, iters in (("fp64", 2048), ("fp32", 32768)):
        best = 0.0
        for rep in range(6):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            flops = rhd.fma_probe(prec, 8 * sms, iters, stream)
            e1.record(stream)
            torch.cuda.synchronize()
            if rep:
                best = max(best, flops / (e0.elapsed_time(e1) * 1e-3) / 1e12)
        out[prec + "_tflops"] = best
    return out


def pipe_views(rec, n_cells, ms_per_launch, peaks, hbm_peak, alg_bytes):
    """Roofline views of one launch over n_cells cells lasting ms_per_launch:
    FP64 flops (and FP32 flops where the kernel has them) per cell from the
    counts record against the measured pipe peaks, algorithmic bytes against
    the copy bandwidth, and the DRAM traffic per launch."""
    sec = ms_per_launch * 1e-3
    v = {"hbm": {"achieved": alg_bytes * n_cells / sec / 1e9, "peak": hbm_peak,
                 "unit": "GB/s", "frac": alg_bytes * n_cells / sec / 1e9 / hbm_peak,
                 "alg_bytes_per_cell": alg_bytes}}
    if rec is None:
        return v
    f64 = rec["fp64_flop"] * n_cells / sec / 1e12
    v["fp64"] = {"achieved": f64, "peak": peaks["fp64_tflops"], "unit": "TFLOP/s",
                 "frac": f64 / peaks["fp64_tflops"], "flop_per_cell": rec["fp64_flop"]}
    if rec.get("fp64_warp_inst") and rec.get("fp64_thread_arith_inst"):
        # frac = (FP64 pipe busy over the launch) x (active lanes x arithmetic
        # share of the FP64-pipe instructions) x (flops per arithmetic
        # instruction / 2): the last two from the counts, the first implied
        lane_arith = rec["fp64_thread_arith_inst"] / (32.0 * rec["fp64_warp_inst"])
        fma_mix = rec["fp64_flop"] / (2.0 * rec["fp64_thread_arith_inst"])
        v["fp64"]["decomposition"] = {
            "lane_arith_share": lane_arith, "fma_mix": fma_mix,
            "fp64_pipe_busy_implied": v["fp64"]["frac"] / (lane_arith * fma_mix),
            "note": "frac = pipe busy x lane_arith_share x fma_mix; an add or multiply "
                    "fills an FMA slot with one flop, so fma_mix bounds frac even at full "
                    "lanes and a fully busy pipe"}
    if rec.get("fp32_flop", 0.0) > 1.0:
        f32 = rec["fp32_flop"] * n_cells / sec / 1e12
        v["fp32"] = {"achieved": f32, "peak": peaks["fp32_tflops"], "unit": "TFLOP/s",
                     "frac": f32 / peaks["fp32_tflops"], "flop_per_cell": rec["fp32_flop"]}
    v["traffic_per_launch"] = rec["dram_bytes"] * n_cells
    v["dram_bytes_per_cell"] = rec["dram_bytes"]
    return v


def step_record(rec):
    """Counts of one whole step from per-stage counts (stage1 + stage2)."""
    if rec is None:
        return None
    return {k: rec["stage1"][k] + rec["stage2"][k] for k in ("fp64_flop", "fp32_flop",
                                                             "dram_bytes")}


# algorithmic HBM bytes per cell of one adjoint step: the tape's y(n) and
# y(n+1/2) (16 fields) and rho, kappa read; the cotangent of the state (8
# fields) read and written; the opacity cotangent read and written
ADJ_ALG_BYTES = 8 * (16 + 2 + 16 + 2)


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            return json.load(fh), "measured"
    except (OSError, ValueError):
        return {"hbm_gbs": FALLBACK_HBM_GBS}, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.proc = None
        self.gpu = gpu_index

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.QUERY,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx),
                "reasons": sorted(reasons), "samples": len(sm)}


def reduce_max(x, dist, device):
    """Max of x over all ranks (x itself when not distributed)."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(cells_per_rank, steps, world_size, max_seconds):
    """Mcell-updates/s of all ranks together, timed by the slowest rank."""
    return world_size * cells_per_rank * steps / max_seconds / 1e6


def oracle_rate(prob, U, edge, nsteps, dt):
    """Time the CPU oracle on a periodic edge^3 sub-box of U (Mcell-updates/s)."""
    from oracle import oracle as O
    O.build()
    sub = dict(prob)
    sub["n"] = [edge, edge, edge]
    box = np.ascontiguousarray(U[:, :edge, :edge, :edge])
    t0 = time.perf_counter()
    O.step(sub, box, nsteps=nsteps, dt=dt)
    t1 = time.perf_counter()
    return edge ** 3 * nsteps / (t1 - t0) / 1e6, t1 - t0


def _oracle_ready(_):
    """Pool warm-up: import and build the oracle in the worker process."""
    from oracle import oracle as O
    O.build()
    O.lib()
    time.sleep(0.3)  # so that every worker takes one warm-up task
    return os.getpid()


def _oracle_box(payload):
    """One worker's timed oracle steps on its sub-box: (cell-updates, seconds)."""
    prob, box, nsteps, dt = payload
    from oracle import oracle as O
    t0 = time.perf_counter()
    O.step(prob, box, nsteps=nsteps, dt=dt)
    return box[0].size * nsteps, time.perf_counter() - t0


class OraclePool:
    """The serial CPU oracle on every host core at once: one process per core
    (spawned, so it is safe after CUDA initialisation), each advancing its
    own periodic edge^3 sub-box of the workload, taken at a different offset."""

    def __init__(self, cores=None):
        import multiprocessing as mp
        self.cores = cores or len(os.sched_getaffinity(0))
        self.pool = mp.get_context("spawn").Pool(self.cores)
        self.pool.map(_oracle_ready, range(self.cores), chunksize=1)

    def boxes(self, prob, U, edge):
        sub = dict(prob)
        sub["n"] = [edge, edge, edge]
        n = U.shape[1]
        out = []
        for i in range(self.cores):
            o = (i * edge) % max(n - edge + 1, 1)
            out.append((sub, np.ascontiguousarray(U[:, o:o + edge, :edge, :edge])))
        return out

    def rate(self, prob, U, edge, nsteps, dt):
        """Mcell-updates/s of all processes together over the wall time."""
        payloads = [(p, b.copy(), nsteps, dt) for p, b in self.boxes(prob, U, edge)]
        t0 = time.perf_counter()
        res = self.pool.map(_oracle_box, payloads, chunksize=1)
        t1 = time.perf_counter()
        return sum(c for c, _ in res) / (t1 - t0) / 1e6, t1 - t0

    def close(self):
        self.pool.close()
        self.pool.join()


def workload(args, rank=0):
    from paper_2404_08247_gb300 import inputs as I
    prob, U, _ = I.turbulent_box_3d(n=args.n, seed_rho=3 + 100 * rank,
                                    seed_v=4 + 100 * rank, seed_T=5 + 100 * rank,
                                    hll_mode=args.hll, reconstruction=args.reconstruction)
    return prob, U


def config_of(args, prob):
    return {
        "workload": "turbulent_box_3d %d^3 periodic: log-normal rho (k^-4 GRF, "
                    "sigma_ln=1), kappa~rho with tau_cell in [1e-3,1e3], log-uniform "
                    "T over 1 decade, rms Mach 1, chat=30 max|v|, c=10 chat"
                    % args.n,
        "cells": int(args.n ** 3),
        "precision": args.precision,
        "hll_mode": args.hll,
        "reconstruction": args.reconstruction,
        "closure": "m1",
        "vc_order": 2,
        "cfl": prob["cfl"],
        "l2_policy": "inputs larger than L2 (state %.2f GB)" % (args.n ** 3 * 80 / 1e9),
    }


# ------------------------------------------------------------- reference arm

def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    from oracle import oracle as O
    O.build()
    prob, U = workload(args)
    dt = O.dt(prob)
    edge = args.ref_sample
    pool = OraclePool()
    try:
        for _ in range(args.warmup):
            pool.rate(prob, U, edge, 1, dt)
        t = 0.0
        for _ in range(args.steps):
            _, dtime = pool.rate(prob, U, edge, 1, dt)
            t += dtime
    finally:
        pool.close()
    cells = edge ** 3 * args.steps * pool.cores
    value = cells / t / 1e6
    sample = ("each step: one oracle step on each of %d periodic %d^3 sub-boxes of the "
              "%d^3 state, one serial oracle process per host core, all at once"
              % (pool.cores, edge, args.n))
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * t / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": config_of(args, prob),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": pool.cores,
                         "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


# ------------------------------------------------------------------ our arm

def time_form(args, rhd, torch, prob, Ud, precision, barrier, stream, local):
    """Warm-up, then args.steps steps timed with CUDA events on `stream`."""
    ctx = rhd.RHDContext(prob, precision, stream=stream)
    ctx.set_state(Ud)
    ctx.step(args.warmup)
    barrier()
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    ctx.profile(True)
    l0 = ctx.launch_count()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    barrier()
    torch.cuda.synchronize()
    e0.record(stream)
    ctx.step_async(args.steps)
    e1.record(stream)
    info = ctx.sync()
    torch.cuda.synchronize()
    barrier()
    launches = ctx.launch_count() - l0
    ms = e0.elapsed_time(e1)
    klaunch, kms = ctx.profile_read()
    ctx.profile(False)
    clk = clocks.stop()
    return ctx, {"ms": ms, "launches": launches, "klaunch": klaunch, "kms": kms,
                 "clocks": clk, "info": info}


def run_batched(args, rhd, torch, rank, ws, dist, barrier, roof=None):
    """512 independent 1-D/2-D problems (mixed precision) in the persistent,
    graph-captured kernel; launch configuration from the autotuner."""
    from paper_2404_08247_gb300 import autotune
    from paper_2404_08247_gb300 import inputs as I
    problems = I.batched_problems(nprob=512, seed=11 + 100 * rank)
    tuned = autotune.tune(problems, "mixed", nsteps=4)
    stream = torch.cuda.Stream()
    probs = [p for p, _ in problems]
    with rhd.RHDBatch(probs, "mixed", stream=stream) as b:
        b.configure(tuned["tile2d"], tuned["blocks_per_sm"])
        if args.no_graph:
            b.use_graphs(False)
        for i, (_, U) in enumerate(problems):
            b.set_state(i, U)
        cells = b.cells()
        nsteps = args.batched_steps
        b.step(nsteps)  # graph capture + warm-up
        barrier()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        info = b.step(nsteps)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = reduce_max(e0.elapsed_time(e1), dist, "cuda")
    views = None
    if roof is not None:
        rec = roof["counts"]["batched"] if roof["counts"] else None
        views = pipe_views(step_record(rec), cells, ms / nsteps, roof["peaks"],
                           roof["hbm"], ALG_BYTES[0] + ALG_BYTES[1])
        views["note"] = ("one whole step (both stage launches) of the pooled cells; "
                         "flops per cell from ncu counts of the batch kernel's graph "
                         "nodes on this workload (profiles/kernel_counts.json)")
    return {"value": whole_job_rate(cells, nsteps, ws, ms * 1e-3), "unit": UNIT,
            "roofline": views,
            "ms_per_step": ms / nsteps, "steps": nsteps, "problems": len(probs),
            "cells": int(cells), "precision": "mixed",
            "n_1d": sum(1 for p in probs if p["ndim"] == 1),
            "tile2d": b.TILES[tuned["tile2d"]], "blocks_per_sm": tuned["blocks_per_sm"],
            "autotune_ms": tuned["timings_ms"],
            "mean_newton": info["sum_newton"] / max(info["n_solves"], 1),
            "workload": "512 problems, 1-D N~U{64..4096} or 2-D side~U{32..256}, "
                        "log10 tau_cell~U[-3,3], Gaussian T pulse, |v|/c~U[0,1e-3], "
                        "c=1e3, chat=100 (seed 11)"}


def run_adjoint(args, rhd, torch, rank, ws, dist, barrier, roof=None):
    """Differentiation workload: a radiation pulse through a log-normal opacity
    field on a periodic 512^2 grid, L = sum (E(200) - E_tgt)^2, gradient with
    respect to the initial temperature and log opacity by the hand-written
    adjoint with checkpoints every 20 steps (FP64)."""
    from paper_2404_08247_gb300 import adjoint as A
    from paper_2404_08247_gb300 import inputs as I
    prob, T0, lk, Et, nsteps = I.pulse_inverse_problem_2d(args.adj_n, seed_chi=7 + 100 * rank)
    every = 20
    N = T0.size
    cv = prob["kB_over_mu"] / (prob["gamma"] - 1.0)
    a = prob["a_rad"]
    stream = torch.cuda.current_stream()
    ctx = rhd.RHDContext(prob, stream=stream)
    ctx.set_state(I.rest_state(prob, T0, lk))
    Tt = torch.from_numpy(T0.reshape(-1).copy()).cuda()
    lkt = torch.from_numpy(lk.reshape(-1).copy()).cuda()
    Ett = torch.from_numpy(Et.reshape(-1).copy()).cuda()

    def events():
        return torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    # forward steps alone (the cost unit of the ratio)
    U0 = torch.from_numpy(I.rest_state(prob, T0, lk)).cuda()
    ctx.set_state(U0)
    ctx.step(3)
    ctx.set_state(U0)
    barrier()
    torch.cuda.synchronize()
    e0, e1 = events()
    e0.record(stream)
    ctx.step(nsteps)
    e1.record(stream)
    torch.cuda.synchronize()
    fwd_ms = reduce_max(e0.elapsed_time(e1), dist, "cuda") / nsteps

    def grad_pass():
        T = Tt.clone().requires_grad_(True)
        logk = lkt.clone().requires_grad_(True)
        z = torch.zeros_like(T)
        y0 = torch.stack([cv * T, z, z, z, a * T ** 4, z, z, z])
        ea, eb = events()
        y = A.trajectory(ctx, y0, torch.exp(logk), nsteps, 0.0, every)
        loss = ((y[4] - Ett) ** 2).sum()
        ea.record(stream)
        loss.backward()
        eb.record(stream)
        torch.cuda.synchronize()
        return ea.elapsed_time(eb), float(loss.detach()), T.grad, logk.grad

    grad_pass()  # warm-up (allocates the adjoint scratch)
    barrier()
    torch.cuda.synchronize()
    e0, e1 = events()
    e0.record(stream)
    bwd_ms_total, loss, gT, glk = grad_pass()
    e1.record(stream)
    torch.cuda.synchronize()
    total_ms = reduce_max(e0.elapsed_time(e1), dist, "cuda")
    bwd_ms = reduce_max(bwd_ms_total, dist, "cuda") / nsteps

    # the two parts of the backward: re-run with recording, then the adjoint
    tape = torch.empty((2 * every + 1) * 8 * N, dtype=torch.float64, device="cuda")
    ybar = torch.zeros(8 * N, dtype=torch.float64, device="cuda")
    kbar = torch.zeros(N, dtype=torch.float64, device="cuda")
    ctx.set_state(U0)
    e0, e1 = events()
    e0.record(stream)
    ctx.step_record(every, 0.0, tape)
    e1.record(stream)
    torch.cuda.synchronize()
    rec_ms = e0.elapsed_time(e1) / every
    ybar[4 * N:5 * N] = 1.0
    e0, e1 = events()
    e0.record(stream)
    ctx.adjoint(tape, every, 0.0, ybar, kbar)
    e1.record(stream)
    torch.cuda.synchronize()
    adj_ms = e0.elapsed_time(e1) / every
    launches = ctx.launch_count()
    ctx.close()
    views = None
    if roof is not None:
        rec = roof["counts"]["adjoint"]["per_step"] if roof["counts"] else None
        views = pipe_views(rec, N, adj_ms, roof["peaks"], roof["hbm"], ADJ_ALG_BYTES)
        views["note"] = ("the four adjoint kernels of one step (face_vjp_kernel and "
                         "cell_adj_kernel, both stages) against their event time; "
                         "counts from profiles/kernel_counts.json")
    return {
        "roofline": views,
        "value": whole_job_rate(N, nsteps, ws, bwd_ms * nsteps * 1e-3), "unit": UNIT,
        "what": "backward cell-updates/s (re-run with recording + adjoint)",
        "fwd_ms_per_step": fwd_ms, "bwd_ms_per_step": bwd_ms,
        "fwd_plus_bwd_ms_per_step": total_ms / nsteps,
        "record_ms_per_step": rec_ms, "adjoint_kernels_ms_per_step": adj_ms,
        "ratio_bwd_over_fwd": bwd_ms / fwd_ms,
        "ratio_adjoint_kernels_over_fwd": adj_ms / fwd_ms,
        "steps": nsteps, "checkpoint_every": every, "cells": int(N), "precision": "fp64",
        "loss": loss, "grad_T_norm": float(gT.norm()), "grad_logk_norm": float(glk.norm()),
        "launches_total": int(launches),
        "workload": "%d^2 periodic, rho=1, gas at rest, ln chi k^-4 GRF sigma=1 median "
                    "tau_cell=1 (seed 7), T=(1+9exp(-r^2/(2*0.05^2)))(1+0.2u), u iid U[-1,1] (seed 9), "
                    "c=chat=1e3, "
                    "L=sum(E_200-E_tgt)^2" % args.adj_n,
    }


# bytes per cell of one hydrodynamic step that the kernels must move (3-D):
# per stage the primitives (read 5, write 5 fields), three face kernels
# (read the primitives, write 5 face fluxes per cell each), the update (read
# the state and the three axes' fluxes, write 5 fields), stage 2 also reading
# the stage-1 state and committing (read 5, write 5): 8 B x (10 + 30 + 25)
# + 8 B x (10 + 30 + 30 + 10)
HYDRO_BYTES_PER_CELL = 8 * (10 + 30 + 25) + 8 * (10 + 30 + 30 + 10)


def run_split(args, rhd, torch, prob, Ud, rank, ws, dist, barrier):
    """The hydrodynamic step (RK2-SSP, HLLC) and one operator-split step
    (Sec. 3.1: hydrodynamics, then the subcycled radiation update) on the
    same 256^3 box, FP64."""
    stream = torch.cuda.current_stream()
    N = int(np.prod(prob["n"]))
    ctx = rhd.RHDContext(prob, "fp64", stream=stream)
    ctx.set_state(Ud)
    dt_h = ctx.hydro_dt()
    ctx.hydro_step(3, dt_h)
    ctx.set_state(Ud)
    K = 5
    barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    ctx.hydro_step(K, dt_h)
    e1.record(stream)
    torch.cuda.synchronize()
    hydro_ms = reduce_max(e0.elapsed_time(e1), dist, "cuda") / K
    ctx.set_state(Ud)
    barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    info = ctx.step_split(1, dt_h)
    torch.cuda.synchronize()
    split_ms = reduce_max((time.perf_counter() - t0) * 1e3, dist, "cuda")
    ctx.close()
    nsub = info["n_solves"] // (2 * N)
    peaks, _ = measured_peaks()
    hbm = float(peaks.get("hbm_gbs", FALLBACK_HBM_GBS))
    achieved = HYDRO_BYTES_PER_CELL * N / (hydro_ms * 1e-3) / 1e9
    nd = prob["ndim"]
    faces = sum(N // prob["n"][d] * (prob["n"][d] + 1) for d in range(nd))
    fp64_face = 2 * faces * HYDRO_FACE_FLOPS
    return {
        "hydro": {"value": whole_job_rate(N, 1, ws, hydro_ms * 1e-3), "unit": UNIT,
                  "ms_per_step": hydro_ms, "steps": K, "dt": dt_h,
                  "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm,
                               "unit": "GB/s", "frac": achieved / hbm,
                               "bytes_per_cell": HYDRO_BYTES_PER_CELL,
                               "note": "model of the multi-kernel step's traffic; the "
                                       "face kernels are bound by the FP64 pipe (84 % busy "
                                       "under ncu)",
                               "fp64_view": {
                                   "achieved": fp64_face / (hydro_ms * 1e-3) / 1e12,
                                   "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                                   "frac": fp64_face / (hydro_ms * 1e-3) / 1e12
                                           / FP64_PEAK_TFLOPS,
                                   "note": "the face kernels' flops only (2 stages x ndim "
                                           "axes x faces x HYDRO_FACE_FLOPS) over the "
                                           "whole step"}}},
        "split": {"value": whole_job_rate(N, 1, ws, split_ms * 1e-3), "unit": UNIT,
                  "ms_per_step": split_ms, "radiation_substeps": int(nsub),
                  "hydro_share": hydro_ms / split_ms,
                  "note": "host clock around rhd_step_split (two status reads per step)"},
        "reconstruction": prob.get("reconstruction", "plm"),
    }


def run_slabs(args, rhd, torch, prob, U, ws, dist, barrier, whole_ms):
    """The same box as two z-slabs on this GPU (the domain decomposition a
    multi-GPU run uses; the ghost planes exchanged by device-to-device copies
    before each stage): warm-up, then args.steps steps of rhd_step_slabs
    timed with CUDA events on the stream."""
    stream = torch.cuda.current_stream()
    nz = prob["n"][2]
    cuts = [0, nz // 2, nz]
    ctxs = [rhd.RHDContext(q, args.precision, stream=stream)
            for q in rhd.slab_problems(prob, cuts)]
    try:
        for c, z0, z1 in zip(ctxs, cuts, cuts[1:]):
            c.set_state(np.ascontiguousarray(U[:, z0:z1]))
        rhd.step_slabs(ctxs, args.warmup)
        barrier()
        torch.cuda.synchronize()
        l0 = sum(c.launch_count() for c in ctxs)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        rhd.step_slabs(ctxs, args.steps)
        e1.record(stream)
        torch.cuda.synchronize()
        launches = sum(c.launch_count() for c in ctxs) - l0
        ms = reduce_max(e0.elapsed_time(e1), dist, "cuda")
    finally:
        for c in ctxs:
            c.close()
    N = int(np.prod(prob["n"]))
    P = prob["n"][0] * prob["n"][1]
    depth = 2 if prob.get("reconstruction", "plm") == "plm" else 3
    return {"value": whole_job_rate(N, args.steps, ws, ms * 1e-3), "unit": UNIT,
            "ms_per_step": ms / args.steps, "slabs": cuts,
            "whole_over_slabs_time": whole_ms / ms,
            "exchange_bytes_per_step": 2 * 2 * 2 * 4 * depth * P * 8,
            "gpu_launches": launches,
            "note": "two z-slabs of the box, periodic in z (each slab's two faces are "
                    "HALO); per stage 16 device-to-device copies of the neighbours' "
                    "boundary planes; the TAU factors are recomputed once per call"}


def run_decomposed(args, rhd, torch, prob, U, ws, rank, dist, barrier):
    """One box decomposed in z across the ranks, one slab per rank (strong
    scaling: the total work is the box's), stepped stage by stage through
    paper_2404_08247_gb300.decomp with the ghost planes exchanged between
    ranks by NCCL point-to-point transfers before each stage (one rank: the
    whole periodic box as one slab exchanging with itself).  Every rank holds
    the same initial box and takes its z range."""
    from paper_2404_08247_gb300 import decomp
    stream = torch.cuda.current_stream()
    nz = prob["n"][2]
    cuts = [round(i * nz / ws) for i in range(ws + 1)]
    q = rhd.slab_problems(prob, cuts)[rank]
    ctx = rhd.RHDContext(q, args.precision, stream=stream)
    try:
        ctx.set_state(np.ascontiguousarray(U[:, cuts[rank]:cuts[rank + 1]]))
        slab = decomp.CtxSlab(ctx, "cuda")
        dt = rhd.rhd_default_dt(rhd.params_from_problem(prob, args.precision))
        decomp.exchange_material(slab, dist)
        decomp.step(slab, dist, args.warmup, dt)
        l0 = ctx.launch_count()
        barrier()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        res = decomp.step(slab, dist, args.steps, dt)
        e1.record(stream)
        torch.cuda.synchronize()
        barrier()
        ms = reduce_max(e0.elapsed_time(e1), dist, "cuda")
        launches = ctx.launch_count() - l0
    finally:
        ctx.close()
    N = int(np.prod(prob["n"]))
    P = prob["n"][0] * prob["n"][1]
    depth = 2 if prob.get("reconstruction", "plm") == "plm" else 3
    return {"value": N * args.steps / (ms * 1e-3) / 1e6, "unit": UNIT,
            "ms_per_step": ms / args.steps, "steps": args.steps, "ranks": ws,
            "slab_planes": cuts, "status": res["status"], "scaling": "strong",
            "exchange_bytes_per_rank_per_step": 2 * 2 * 4 * depth * P * 8,
            "gpu_launches_rank0": int(launches),
            "note": "one box in z-slabs, one per rank, ghost planes of E and F exchanged "
                    "before each stage (NCCL send/recv between ranks; one rank: its own "
                    "planes), the statuses max-reduced before each commit"}


def run_hydro_only(args):
    """2 + 3 hydrodynamic steps of the --n^3 box at its CFL step; one line."""
    import torch
    from paper_2404_08247_gb300 import build as B
    B.build()
    from paper_2404_08247_gb300 import rhd
    rhd.load()
    prob, U = workload(args)
    Ud = torch.from_numpy(U).cuda()
    ctx = rhd.RHDContext(prob, "fp64", stream=torch.cuda.current_stream())
    ctx.set_state(Ud)
    dt = ctx.hydro_dt()
    ctx.hydro_step(2, dt)
    ctx.set_state(Ud)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    ctx.hydro_step(3, dt)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / 3
    ctx.close()
    print(json.dumps({"hydro_only": True, "n": args.n, "reconstruction": args.reconstruction,
                      "ms_per_step": ms, "value": args.n ** 3 / ms / 1e3, "unit": UNIT}))
    return 0


def run_ours(args):
    import torch
    from paper_2404_08247_gb300 import rhd

    ws, rank, local = dist_env()
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    rhd.load()
    prob, U = workload(args, rank)
    # the decomposed box: every rank the same box (rank 0's seeds)
    prob0, U0 = (prob, U) if rank == 0 else workload(args, 0)
    N = U[0].size
    stream = torch.cuda.current_stream()
    Ud = torch.from_numpy(U).cuda()

    def barrier():
        if dist is not None:
            dist.barrier()

    def max_over_ranks(x):
        return reduce_max(x, dist, "cuda")

    # pipe peaks of this GPU (outside any timed region)
    fma_peaks = measure_fma_peaks(rhd, torch)

    forms = [args.precision] + [f for f in ("fp64", "mixed") if f != args.precision
                                and not args.single_form]
    if not args.single_form:
        forms.append("fp64-rk2ssp")  # the paper's comparison scheme (Sec. 4.2)
        # the paper's PPM faces (Sec. 3.3); the Colella-Sekora variant turns a
        # face state of this box's iid temperatures nonphysical in its first
        # step (it does not keep edges within the neighbours' range)
        forms += ["fp64-ppm", "mixed-ppm"]
    results = {}
    ctx = None
    for form in forms:
        fprob, fprec = prob, form
        if form == "fp64-rk2ssp":
            fprob, fprec = dict(prob, scheme="rk2ssp"), "fp64"
        elif form.endswith("-ppm"):
            fprob, fprec = dict(prob, reconstruction="ppm"), form[:-4]
        elif form.endswith("-ppm_cs"):
            fprob, fprec = dict(prob, reconstruction="ppm_cs"), form[:-7]
        c, r = time_form(args, rhd, torch, fprob, Ud, fprec, barrier, stream, local)
        r["ms"] = max_over_ranks(r["ms"])
        results[form] = r
        if form == args.precision:
            ctx = c
        else:
            c.close()
    head = results[args.precision]
    ms = head["ms"]
    value = whole_job_rate(N, args.steps, ws, ms * 1e-3)

    # dominant kernel roofline: the FP64 pipe (its bound), from the committed
    # ncu counts when they belong to these kernel sources, against the FP64
    # peak measured above; the HBM view beside it
    peaks_file, peak_src = measured_peaks()
    hbm_peak = float(peaks_file.get("hbm_gbs", FALLBACK_HBM_GBS))
    counts = kernel_counts_record()
    kms, klaunch = head["kms"], head["klaunch"]
    dom = max((0, 1), key=lambda k: kms[k])
    kname = KERNEL_NAMES[dom]
    avg_ms = kms[dom] / max(klaunch[dom], 1)
    head_form = args.precision if args.reconstruction == "plm" else \
        "%s-%s" % (args.precision, args.reconstruction)
    head_rec = None
    if counts and head_form in counts["stage_kernels"]:
        head_rec = counts["stage_kernels"][head_form][kname]
    views = pipe_views(head_rec, N, avg_ms, fma_peaks, hbm_peak, ALG_BYTES[dom])
    hbm_view = dict(views["hbm"], peak_source="%s (MEASURED_PEAKS.json hbm_gbs)" % peak_src
                    if peak_src == "measured" else "fallback")
    common = {
        "kernel": kname, "avg_launch_ms": avg_ms,
        "kernel_ms": {KERNEL_NAMES[k]: kms[k] / max(klaunch[k], 1) for k in (0, 1)},
        "traffic": views.get("traffic_per_launch"),
        "traffic_source": ("ncu dram__bytes_read+write per cell at 128^3 x cells "
                           "(profiles/kernel_counts.json)") if head_rec else None,
        "fp64_pipe_busy": ({"while_active": head_rec["fp64_pipe_active"],
                            "of_elapsed_128": head_rec["fp64_pipe_elapsed"],
                            "lanes_per_inst": head_rec["lanes"]} if head_rec else None),
    }
    if "fp64" in views and args.precision == "fp64":
        roofline = dict(
            {"bound": "alu", "achieved": views["fp64"]["achieved"],
             "peak": fma_peaks["fp64_tflops"], "unit": "TFLOP/s",
             "frac": views["fp64"]["frac"], "flop_per_cell": head_rec["fp64_flop"],
             "flop_source": "ncu thread counts dadd + dmul + 2 dfma per cell at 128^3 "
                            "(profiles/kernel_counts.json) x cells",
             "peak_source": "measured on this GPU: " + fma_peaks["method"],
             "peak_nominal": FP64_PEAK_TFLOPS,
             "hbm_view": hbm_view,
             "decomposition": views["fp64"].get("decomposition"),
             "note": "FP64-pipe bound: the fraction of the FP64 flop peak also loses "
                     "the lanes idle in the per-cell iterations and the FP64-pipe "
                     "slots of adds and multiplies (1 flop) against FMAs (2)"},
            **common)
    else:
        roofline = dict(
            {"bound": "hbm", "achieved": views["hbm"]["achieved"], "peak": hbm_peak,
             "unit": "GB/s", "frac": views["hbm"]["frac"],
             "alg_bytes_per_cell": ALG_BYTES[dom], "peak_source": hbm_view["peak_source"],
             "pipe_views": {k: views[k] for k in ("fp64", "fp32") if k in views},
             "note": "the stage kernels are bound by the FP64 pipe, not by HBM (DRAM "
                     "below 1 % busy under ncu)"},
            **common)

    # end to end through the public API with pinned host buffers: a state held
    # in host memory advanced in place, every step copying the whole state in
    # (10 fields) and the stepped state out (the 8 evolved fields; rho and
    # kappa are unchanged), over the same steps as the device-timed region (W
    # warm-up steps from the initial state, then the timed ones: a step's cost
    # follows the state's Newton iteration counts).  rhd_step_host overlaps
    # the copies with the stage kernels (chunks of z planes); the three
    # separate calls (set, step, get of all 10 fields) are timed beside it.
    e2e = None
    if not args.no_e2e:
        ne2e = args.e2e_steps if args.e2e_steps > 0 else args.steps
        hstate = torch.from_numpy(U.copy()).pin_memory()
        for _ in range(args.warmup):
            ctx.step_host(hstate, hstate, 1)
        barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(ne2e):
            ctx.step_host(hstate, hstate, 1)
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        tt = max_over_ranks(t1 - t0)
        hin = torch.from_numpy(U.copy()).pin_memory()
        hout = hin
        for _ in range(args.warmup):
            ctx.set_state(hin)
            ctx.step(1)
            ctx.get_state(hout)
        barrier()
        torch.cuda.synchronize()
        parts = [0.0, 0.0, 0.0]
        t2 = time.perf_counter()
        for _ in range(ne2e):
            ta = time.perf_counter()
            ctx.set_state(hin)
            tb = time.perf_counter()
            ctx.step(1)
            tc = time.perf_counter()
            ctx.get_state(hout)
            td = time.perf_counter()
            parts = [parts[0] + tb - ta, parts[1] + tc - tb, parts[2] + td - tc]
        torch.cuda.synchronize()
        t3 = time.perf_counter()
        ts = max_over_ranks(t3 - t2)
        e2e = {"value": whole_job_rate(N, ne2e, ws, tt), "unit": UNIT,
               "h2d_bytes_per_step": int(hstate.numel() * 8),
               "d2h_bytes_per_step": int(8 * ctx.ncell * 8),
               "steps": ne2e, "warmup": args.warmup, "precision": args.precision,
               "api": "rhd_step_host in place (copies in chunks overlapping the stage "
                      "kernels)",
               "ms_per_step": 1e3 * tt / ne2e,
               "unpipelined": {
                   "api": "rhd_state_set_all + rhd_step + rhd_state_get_all, in place",
                   "h2d_bytes_per_step": int(hin.numel() * 8),
                   "d2h_bytes_per_step": int(hout.numel() * 8),
                   "value": whole_job_rate(N, ne2e, ws, ts),
                   "ms_per_step_parts": {k: 1e3 * v / ne2e for k, v in
                                         zip(("set_state", "step", "get_state"), parts)}}}
    ctx.close()

    slabs = None
    if not args.no_slabs and prob["ndim"] == 3 and prob["n"][2] >= 6:
        slabs = run_slabs(args, rhd, torch, prob, U, ws, dist, barrier, ms)

    decomposed = None
    if not args.no_slabs and prob["ndim"] == 3 and prob["n"][2] >= 3 * ws:
        decomposed = run_decomposed(args, rhd, torch, prob0, U0, ws, rank, dist, barrier)

    roof = {"counts": counts, "peaks": fma_peaks, "hbm": hbm_peak}
    batched = None
    if not args.no_batched:
        batched = run_batched(args, rhd, torch, rank, ws, dist, barrier, roof)

    adjoint = None
    if not args.no_adjoint:
        adjoint = run_adjoint(args, rhd, torch, rank, ws, dist, barrier, roof)

    split = None
    if not args.no_split:
        split = run_split(args, rhd, torch, prob, Ud, rank, ws, dist, barrier)

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        from oracle import oracle as O
        odt = O.dt(prob)
        pool = OraclePool()
        try:
            prate, psecs = pool.rate(prob, U, args.cpu_edge, 2, odt)
        finally:
            pool.close()
        rate, secs = oracle_rate(prob, U, args.cpu_sample, 2, odt)
        cpu = {"value": prate, "unit": UNIT, "cores": pool.cores, "kind": "oracle",
               "sample": "2 oracle steps on each of %d periodic %d^3 sub-boxes of the %d^3 "
                         "initial state, same dt, one serial oracle process per host core "
                         "(%.1f s wall)" % (pool.cores, args.cpu_edge, args.n, psecs),
               "single_core": {"value": rate, "unit": UNIT, "cores": 1,
                               "sample": "2 oracle steps of a periodic %d^3 sub-box "
                                         "(%.1f s)" % (args.cpu_sample, secs)}}

    if rank == 0:
        form_lines = {}
        for form, r in results.items():
            inf = r["info"]
            fviews = {}
            for k in (0, 1):
                frec = None
                if counts and form in counts["stage_kernels"]:
                    frec = counts["stage_kernels"][form][KERNEL_NAMES[k]]
                fviews[KERNEL_NAMES[k]] = pipe_views(
                    frec, N, r["kms"][k] / max(r["klaunch"][k], 1), fma_peaks, hbm_peak,
                    ALG_BYTES[k])
            form_lines[form] = {
                "roofline": fviews,
                "value": whole_job_rate(N, args.steps, ws, r["ms"] * 1e-3),
                "ms_per_step": r["ms"] / args.steps,
                "kernel_ms": {KERNEL_NAMES[k]: r["kms"][k] / max(r["klaunch"][k], 1)
                              for k in (0, 1)},
                "hbm_frac_144B": 144 * N * args.steps / (r["ms"] * 1e-3) / 1e9 / hbm_peak,
                "mean_newton": inf["sum_newton"] / max(inf["n_solves"], 1),
                "mean_outer": inf["sum_outer"] / max(inf["n_solves"], 1),
                "max_newton": inf["max_newton"], "max_outer": inf["max_outer"],
            }
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64" if args.precision == "fp64" else "f32+f64",
            "data": "synthetic", "config": config_of(args, prob),
            "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e,
            "gpu_launches": int(head["launches"]), "clocks": head["clocks"],
            "peaks": dict(fma_peaks, hbm_gbs=hbm_peak, fp64_nominal_tflops=FP64_PEAK_TFLOPS),
            "forms": form_lines,
            "batched": batched,
            "adjoint": adjoint,
            "hydro_split": split,
            "slabs": slabs,
            "decomposed": decomposed,
        }
        print(json.dumps(line))
    if dist is not None:
        dist.destroy_process_group()
    return 0


def main(argv=None):
    args = parse(argv)
    if args.impl == "reference":
        return run_reference(args)
    if args.hydro_only:
        return run_hydro_only(args)
    if args.batched_only:
        import torch
        from paper_2404_08247_gb300 import build as B
        B.build()
        from paper_2404_08247_gb300 import rhd
        rhd.load()
        r = run_batched(args, rhd, torch, 0, 1, None, lambda: None)
        print(json.dumps(dict(r, batched_only=True)))
        return 0
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
