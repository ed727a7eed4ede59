#!/usr/bin/env python
"""Benchmark of the weighted-ensemble Gillespie-SSA path on GB300.

Workload (one "step" = one whole WE run of the batch, every row of the hot path): the Schloegl
model of Sec. III.B.1 in steady-state (MFPT) mode -- 80 bins of width 10 on X, 20 walkers per
bin, tau = 0.05, 1000 iterations, walkers recycled to X0 = 85 on reaching X >= 550 -- with
`--replicas` independent replicas per GPU (10 by default, the replicate count of Sec. III.B.3).
Each step uses fresh seeds, so every step is a new batch of synthetic trajectories.

Prints one JSON line: SSA events/s (whole job), WE iterations/s, the MFPT estimate and its
relative error against the closed form, the SSA kernel's roofline position, the CPU oracle
timed on this host, and an end-to-end figure through the one-call C ABI with host buffers.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

`--workload toggle_batch` times the batched toggle-switch sweep (64 runs with their own rate
constants in one launch per phase, general FP64 SSA kernel) and `--workload synthetic_large`
the random 354-species / 3680-reaction network (one warp per walker), each printing one JSON
line of the same form with an FP64 roofline for its SSA kernel.

`--workload toggle_learned` instead compares, on one GPU, the GPU time that plain species-count
binning and the learned progress coordinate need to reach a 10% MFPT error on a bistable
two-gene toggle switch (a_U = a_V = 40, K = 1, n = 2, d = 1; exact MFPT from the truncated
master equation), the learned arm paying for its own training data, labels and training.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import tempfile
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

ITERS = 1000
DISCARD = 300              # iterations before the flux average (steady state, Sec. III.C.3 protocol)
# Integer/FP32 lane operations one direct-method event needs on the state-indexed table path:
# Philox-4x32-10 (10 rounds x [2 multiply-high, 2 multiply-low, 4 xor, 2 key additions] = 100),
# the uniform's index and the float-float -log u1 (~68), the waiting time in clock units and
# the clock (~26), the reaction from P - 1 = 3 breakpoints (~9), the count update with its
# overflow and target checks (~7).  Peak: the issue limit, 152 SMs x 4 sub-partitions x one
# 32-lane instruction per clock x 2.07 GHz.
OPS_PER_EVENT = 210
ISSUE_PEAK_GOPS = 152 * 4 * 32 * 2.07
KERNELS_PER_ITER = 6       # SSA, bin scan, placement, split/merge, gather, finalize
# DRAM bytes (read + write) of one SSA launch on this workload, from an ncu capture of the
# kernel (dram__bytes_read.sum + dram__bytes_write.sum, mean of two 16,000-walker launches, as
# in every timed launch)
SSA_TRAFFIC_BYTES = 397440


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--replicas", type=int, default=10)
    ap.add_argument("--iters", type=int, default=ITERS)
    ap.add_argument("--cpu-seconds", type=float, default=12.0, help="CPU-oracle sample budget")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--block", type=int, default=0, help="threads per block of the SSA kernel (0: auto)")
    ap.add_argument("--workload", choices=["schlogl", "toggle_learned", "toggle_batch", "synthetic_large",
                                           "schlogl_flux"],
                    default="schlogl")
    ap.add_argument("--batch-iters", type=int, default=0,
                    help="toggle_batch / synthetic_large: WE iterations per step (0: 500 / 100)")
    ap.add_argument("--plain-iters", type=int, default=120000, help="toggle_learned: plain-binning iterations")
    ap.add_argument("--learned-iters", type=int, default=2000, help="toggle_learned: learned-binning iterations")
    return ap.parse_args()


# The SSA kernel is timed by CUDA events on every TIME_EVERY-th iteration (0, 10, 20, ... of
# each timed run); the event-record nodes cost a timed iteration a few microseconds, so timing
# a uniform sample keeps the timed run close to an untimed one.
TIME_EVERY = 10


def exact_mfpt():
    with open(os.path.join(ROOT, "tests", "golden", "exact_values.json")) as f:
        return json.load(f)["schlogl_mfpt_85_to_550_s"]


# ------------------------------------------------------------------------------------------
# CPU oracle leg (the only place besides --impl reference where bench.py runs oracle/)
# ------------------------------------------------------------------------------------------
def _oracle_sample(args):
    replica, n_iters, seed = args
    import numpy as np  # noqa: F401
    import workloads as W
    from oracle import oracle as O
    cfg = W.schlogl_mfpt_we(n_iters=n_iters, n_runs=1, seed=seed)
    cfg.run_ids = np.array([replica], dtype=np.uint32)
    t0 = time.perf_counter()
    o = O.we_run(cfg, 0)
    return int(o["events"].sum()), time.perf_counter() - t0


def _calibrate():
    ev, dt = _oracle_sample((0, 40, 123))                 # the first 40 iterations
    return ev / dt, ev / 40.0


def _oracle_pool_run(cores: int, n_iters: int, seed: int):
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    t0 = time.perf_counter()
    with ctx.Pool(cores) as pool:
        res = pool.map(_oracle_sample, [(r, n_iters, seed) for r in range(cores)])
    return sum(e for e, _ in res), time.perf_counter() - t0


def cpu_baseline(seconds: float, replicas: int):
    """The oracle as it stands, one replica per host process (spawned before any GPU work),
    each running the first n iterations of the workload; n is set so the sample takes about
    `seconds` of wall time."""
    from oracle import build as obuild
    obuild.build()
    cores = max(1, min(replicas, os.cpu_count() or 1))
    rate, per_iter = _calibrate()
    n_iters = int(max(40, min(ITERS, seconds * rate / max(per_iter * 2.5, 1.0))))
    events, wall = _oracle_pool_run(cores, n_iters, 0)
    return {"value": events / wall, "unit": "SSA events/s", "cores": cores, "kind": "oracle",
            "sample": f"{cores} replica(s) x first {n_iters} of {ITERS} iterations of the workload, "
                      f"one host process each; {events} events in {wall:.1f} s"}


# ------------------------------------------------------------------------------------------
# clocks during the timed region
# ------------------------------------------------------------------------------------------
class Clocks:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

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
        for line in open(self.path):
            p = [x.strip() for x in line.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                smax = float(p[2])
            except ValueError:
                continue
            for n, v in zip(names, p[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        os.unlink(self.path)
        sm.sort()
        med = sm[len(sm) // 2] if sm else None
        return {"sm_mhz": med, "sm_max_mhz": smax, "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------------------------------------
# reference arm: the CPU oracle on the same config
# ------------------------------------------------------------------------------------------
def run_reference(a):
    """The CPU oracle timed on this host's cores on the same workload: every step is a bounded
    sample (each replica process runs the first n iterations), sized so that the whole run
    takes about --cpu-seconds per step."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from oracle import build as obuild
    obuild.build()
    cores = max(1, min(a.replicas, os.cpu_count() or 1))
    rate, per_iter = _calibrate()
    n_iters = int(max(40, min(a.iters, a.cpu_seconds * rate / max(per_iter * 2.5, 1.0))))
    for w in range(a.warmup):
        _oracle_pool_run(cores, 20, 10_000 + w)
    tot_ev, tot_s = 0, 0.0
    for s in range(a.steps):
        ev, dt = _oracle_pool_run(cores, n_iters, s)
        tot_ev += ev
        tot_s += dt
    v = tot_ev / tot_s
    cb = {"value": v, "unit": "SSA events/s", "cores": cores, "kind": "oracle",
          "sample": f"per step {cores} replica(s) x first {n_iters} of {a.iters} iterations, one host "
                    f"process each; {tot_ev} events in {tot_s:.1f} s over {a.steps} steps"}
    line = {"impl": "reference", "metric": "SSA events/sec and WE iterations/sec on 1 GB300; MFPT rel. error per GPU-s",
            "value": v, "unit": "SSA events/s", "n_gpus": a.gpus, "steps": a.steps, "warmup": a.warmup,
            "ms_per_step": 1e3 * tot_s / a.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": workload_config(a),
            "cpu_baseline": cb,
            "e2e": {"value": v, "unit": "SSA events/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def workload_config(a):
    return {"workload": (f"Schloegl MFPT weighted ensemble (Sec. III.B): 80 bins x 20 walkers, tau=0.05, "
                         f"{a.iters} iterations, recycle X>=550 -> 85, {a.replicas} independent replicas per GPU"),
            "replicas_per_gpu": a.replicas, "iterations": a.iters, "capacity_per_replica": 1600,
            "l2": "flushed between timed steps (256 MB write)", "parallelism": f"replicas x {a.gpus} GPU(s)"}


# ------------------------------------------------------------------------------------------
# learned binning against plain binning (MFPT error per GPU-second)
# ------------------------------------------------------------------------------------------
TOGGLE_A = 40.0


def _toggle_cfg(W, np, R, n_iters, m_targ, seed):
    import math
    a = TOGGLE_A
    cfg = W.toggle_batch_we(n_runs=R, n_iters=n_iters, seed=seed, m_targ=m_targ)
    cfg.network = W.toggle_switch([a], [a])
    cfg.param_set = np.zeros(R, np.int32)
    x0 = np.tile(np.array([[int(a), 0]], np.int32), (R, 1))
    cfg.x0, cfg.recycle_state = x0, x0.copy()
    cfg.init_states = np.repeat(x0[:, None, :], m_targ, axis=1)
    cfg.init_weights = np.full((R, m_targ), 1.0 / m_targ)
    cfg.target.threshold = np.tile(np.array([[math.ceil(a / 2), math.floor(a / 4)]], np.int32), (R, 1))
    cfg.hist_len = 0
    return cfg


def _checkpointed_run(P, np, torch, ens, cfg, n_iters, n_ckpt, exact, t_fixed):
    """Advance in n_ckpt chunks; after each, the per-replica MFPT = tau/mean(flux) over the last
    80% of the iterations so far, its rms and mean relative error, and the wall time so far."""
    curve = []
    chunk = max(1, n_iters // n_ckpt)
    t = t_fixed
    done = 0
    while done < n_iters:
        k = min(chunk, n_iters - done)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ens.step(k)
        ens.sync()
        t += time.perf_counter() - t0
        done += k
        f = ens.per_iter(P.WE_OUT_FLUX)[:done]
        rate = f[done // 5:].mean(axis=0) / cfg.tau
        rel = np.where(rate > 0, 1.0 / np.maximum(rate, 1e-300) / exact - 1.0, np.inf)
        rms = float(np.sqrt(np.mean(rel ** 2))) if np.all(np.isfinite(rel)) else float("inf")
        curve.append({"iters": done, "gpu_s": round(t, 4), "rms_rel": rms,
                      "mean_rel": float(np.mean(rel)) if np.isfinite(rms) else None})
    return curve


def _time_to(curve, tol):
    """GPU time of the first checkpoint from which the rms error stays within tol."""
    for i, c in enumerate(curve):
        if all(d["rms_rel"] <= tol for d in curve[i:]):
            return c["gpu_s"]
    return None


def run_toggle_learned(a):
    import math
    import numpy as np
    import torch
    import paper_1303_5986_gb300 as P
    import workloads as W
    from oracle import exact as E
    from paper_1303_5986_gb300 import build as pbuild
    from paper_1303_5986_gb300 import learned as LN

    pbuild.build()
    R, A = 16, TOGGLE_A
    thrV, thrU = math.ceil(A / 2), math.floor(A / 4)
    exact = E.toggle_mfpt(A, A, (int(A), 0), lambda u, v: v >= thrV and u <= thrU,
                          Umax=int(2.5 * A) + 20, Vmax=int(2.5 * A) + 20)
    clocks = Clocks(int(os.environ.get("LOCAL_RANK", "0")))
    clocks.start()
    # plain arms: 30 x 30 grid of width-4 bins on (U, V), 8 walkers per bin (the batched toggle
    # configuration) and 64 walkers per bin (more of the GPU in use per iteration)
    plains = {}
    bm = None
    for m_targ, n_it in ((8, a.plain_iters), (64, a.plain_iters // 4)):
        cfg = _toggle_cfg(W, np, R, n_it, m_targ, 1)
        net = P.network_from_spec(cfg.network)
        bm = P.we_binmap_grid(cfg.bins.species, cfg.bins.edges)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        c, keep = P.run_config_from(cfg, record_iters=n_it)
        ens = P.we_ensemble_create(net, bm, c, keep)
        torch.cuda.synchronize()
        curve = _checkpointed_run(P, np, torch, ens, cfg, n_it, 40, exact, time.perf_counter() - t0)
        plains[m_targ] = {"gpu_s_to_10pct": _time_to(curve, 0.10), "final": curve[-1],
                          "walkers_end": int(ens.get(P.WE_OUT_COUNTS).sum()), "iterations": n_it,
                          "curve": curve}
        ens.close()
    # learned arm: states from a 300-iteration plain run, first-passage labels (horizon 1),
    # 2000 Adam steps, 100 bins on z, 164 walkers per bin (about 16384 walkers per replica)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    hcfg = _toggle_cfg(W, np, R, 300, 8, 2)
    hc, hkeep = P.run_config_from(hcfg, record_iters=300)
    hens = P.we_ensemble_create(net, bm, hc, hkeep)
    states = LN.harvest_states(hens, 300)
    hens.close()
    t_harvest = time.perf_counter() - t0
    tgt = ([1, 0], [P.WE_OP_GE, P.WE_OP_LE], [thrV, thrU])
    fit_t = {}
    mlp, xs, labels, losses = LN.fit_coordinate(net, states, tgt, [int(A), 0], 1.0, steps=2000,
                                                batch=4096, lr=3e-3, seed=3, timings=fit_t)
    edges = LN.coordinate_edges(mlp, xs, 100)
    lbm = P.we_binmap_learned(mlp, edges)
    M = 164
    lcfg = _toggle_cfg(W, np, R, a.learned_iters, M, 4)
    lc, lkeep = P.run_config_from(lcfg, record_iters=a.learned_iters, capacity=M * 100 + 64)
    lens = P.we_ensemble_create(net, lbm, lc, lkeep)
    torch.cuda.synchronize()
    t_fixed = time.perf_counter() - t0
    learned = _checkpointed_run(P, np, torch, lens, lcfg, a.learned_iters, 20, exact, t_fixed)
    learned_walkers = int(lens.get(P.WE_OUT_COUNTS).sum())
    clk = clocks.stop()
    tl = _time_to(learned, 0.10)
    reached = [v["gpu_s_to_10pct"] for v in plains.values() if v["gpu_s_to_10pct"] is not None]
    if tl is not None and reached:
        value, bound = min(reached) / tl, "measured against the faster plain arm"
    elif tl is not None:
        value = min(v["final"]["gpu_s"] for v in plains.values()) / tl
        bound = "lower bound: no plain arm reached 10% within its run"
    else:
        value, bound = None, "learned binning did not reach 10%"
    line = {
        "metric": "MFPT rel. error per GPU-s (learned vs plain species-count binning)",
        "value": value, "unit": "x less GPU time to 10% rms MFPT error", "value_kind": bound,
        "n_gpus": 1, "higher_is_better": True, "dtype": "f64 (SSA), fp32/bf16 (coordinate)",
        "data": "synthetic", "vs_baseline": None,
        "config": {"workload": (f"two-gene toggle a_U=a_V={A:g}, K=1, n=2, d=1; MFPT (40,0) -> "
                                f"{{V>={thrV}, U<={thrU}}}, tau=0.1, {R} replicas in one batched launch"),
                   "exact_mfpt_s": exact,
                   "plain": (f"30x30 grid (width 4) x 8 walkers, {a.plain_iters} iterations; "
                             f"x 64 walkers, {a.plain_iters // 4} iterations"),
                   "learned": (f"MLP 2->64->64->1 on log1p counts, {len(states)} harvested states, "
                               f"first-passage labels (horizon 1), 2000 Adam steps of 4096; 100 bins x {M} "
                               f"walkers, {a.learned_iters} iterations")},
        "plain_m8": plains[8], "plain_m64": plains[64],
        "learned": {"gpu_s_to_10pct": tl, "final": learned[-1], "walkers_end": learned_walkers,
                    "fixed_cost_s": t_fixed, "harvest_s": t_harvest, "labels_s": fit_t.get("labels_s"),
                    "train_s": fit_t.get("train_s"),
                    "train_loss_first_last": [float(losses[0]), float(losses[-50:].mean())],
                    "label_mean": float(labels.mean()), "curve": learned},
        "clocks": clk,
    }
    print(json.dumps(line))


# ------------------------------------------------------------------------------------------
# the batched toggle sweep and the large synthetic network (general FP64 SSA kernels)
# ------------------------------------------------------------------------------------------
FP64_PEAK_GOPS = 152 * 2 * 2.07      # 152 SMs x 2 FP64 lanes/clock x 2.07 GHz (FMA = one op)


def fp64_ops_per_event(spec, dep_degree):
    """FP64 operations one direct-method event needs on the general path: the propensities the
    dependency graph says change (mass action: one product; Hill: power, sum, quotient), their
    tree paths (log2 P additions each), the target product, the descent (log2 P), the
    reciprocal of a0 and the two clock operations.  Small networks re-evaluate every leaf."""
    import math
    import numpy as np
    P = 1 << max(0, math.ceil(math.log2(max(1, spec.n_reactions))))
    L = int(math.log2(P))
    hill = np.asarray(spec.rate_law) == 1
    per_leaf = float(np.mean(np.where(hill, 3.0, 1.0)))
    deg = float(np.mean(dep_degree)) if dep_degree is not None else float(spec.n_reactions)
    if dep_degree is None:                                # full rebuild: P leaves + P - 1 nodes
        return per_leaf * spec.n_reactions + (P - 1) + 1 + L + 1 + 2
    return deg * (per_leaf + L) + 1 + L + 1 + 2


def run_batch_workload(a):
    import numpy as np
    import torch
    import paper_1303_5986_gb300 as P
    import workloads as W
    from paper_1303_5986_gb300 import build as pbuild

    pbuild.build()
    if a.workload == "toggle_batch":
        n_iters = a.batch_iters or 500
        mk = lambda seed: W.toggle_batch_we(n_runs=64, n_iters=n_iters, seed=seed)
        desc = ("batched two-gene toggle sweep: 64 runs, a_U, a_V uniform in [20,60], K=1, n=2, d=1; "
                f"30x30 bins of width 4 x 8 walkers, tau=0.1, {n_iters} iterations, recycling into "
                "{V>=a_V/2, U<=a_U/4}, one launch per phase for all runs")
    else:
        n_iters = a.batch_iters or 100
        mk = lambda seed: W.synthetic_large_we(n_walkers=4096, n_iters=n_iters, seed=seed)
        desc = ("synthetic 354-species / 3680-reaction network (seed 7): 4096 walkers, counts "
                "uniform in [0,200], 50 bins of width 4 on species 0 x 82 walkers, tau=0.01, "
                f"{n_iters} iterations, one warp per walker")
    base = mk(0)
    net = P.network_from_spec(base.network)
    bm = P.we_binmap_grid(base.bins.species, base.bins.edges)
    deg = None if a.workload == "toggle_batch" else [net.dep_degree(j) for j in range(net.n_reactions)]
    seeds = rank_seeds(0, a.warmup + a.steps)

    def ensemble(seed):
        c, keep = P.run_config_from(mk(seed), record_iters=n_iters)
        return P.we_ensemble_create(net, bm, c, keep)

    warm = [ensemble(s) for s in seeds[:a.warmup]]
    timed = [ensemble(s) for s in seeds[a.warmup:]]
    # the large network's launches are tens of milliseconds and very uneven (the first iteration
    # runs all 4096 walkers): time every one of them
    every = 1 if a.workload == "synthetic_large" else TIME_EVERY
    for e in warm:                        # the timed path itself (graph capture, event pool)
        e.step_timed(n_iters, every=every)
        e.sync()
    for e in timed:                       # capture each timed ensemble's graphs before timing
        e.step_timed(0, every=every)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()
    clocks = Clocks(int(os.environ.get("LOCAL_RANK", "0")))
    step_ms, prop_ms = [], []
    torch.cuda.synchronize()
    clocks.start()
    for e in timed:
        flush.zero_()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        pm = e.step_timed(n_iters, every=every)
        e1.record(stream)
        e1.synchronize()
        step_ms.append(e0.elapsed_time(e1))
        prop_ms.append(pm)
    torch.cuda.synchronize()
    clk = clocks.stop()
    ev_iter = [e.per_iter(P.WE_OUT_EVENTS).sum(axis=1) for e in timed]
    events = float(sum(v.sum() for v in ev_iter))
    ev_sampled = float(sum(v[::every].sum() for v in ev_iter))
    status = [int(x) for e in timed for x in e.status()]
    total_ms = float(sum(step_ms))
    prop_total_ms = float(sum(p.sum() for p in prop_ms))
    n_launch = sum(len(p) for p in prop_ms)
    ops = fp64_ops_per_event(base.network, deg)
    achieved = ops * ev_sampled / (prop_total_ms * 1e-3) / 1e9
    ssa_ms_est = prop_total_ms / max(n_launch, 1) * n_iters * a.steps
    mapping = "warp per walker (k_propagate_warp)" if a.workload == "synthetic_large" else \
        "state chain / clock / draw warps on a two-species (U, V) table (k_propagate_pipe<8,3,2>)"
    line = {
        "metric": "SSA events/sec and WE iterations/sec on 1 GB300",
        "value": events / (total_ms * 1e-3), "unit": "SSA events/s", "n_gpus": 1, "steps": a.steps,
        "warmup": a.warmup, "ms_per_step": total_ms / a.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": desc, "iterations": n_iters, "l2": "flushed between timed steps (256 MB write)"},
        "we_iters_per_s": a.steps * n_iters / (total_ms * 1e-3),
        "status": sorted(set(status)),
        "roofline": {"bound": "alu", "achieved": achieved, "peak": FP64_PEAK_GOPS, "unit": "G FP64 ops/s",
                     "frac": achieved / FP64_PEAK_GOPS, "traffic": None, "kernel": mapping,
                     "launches": n_launch, "launches_sampled": f"every {every}th iteration",
                     "avg_launch_ms": prop_total_ms / max(n_launch, 1),
                     "share_of_step": ssa_ms_est / total_ms, "fp64_ops_per_event": ops,
                     "peak_source": "derived: 152 SMs x 2 FP64 lanes/clk x 2.07 GHz"},
        "cpu_baseline": None, "e2e": None, "gpu_launches": 6 * n_iters * a.steps, "clocks": clk,
    }
    print(json.dumps(line))


def run_schlogl_flux(a):
    """Steady-state reweighting (Sec. II.B.2, Eq. "ss") on the paper's Schloegl flux runs
    (Sec. III.B.2/3: 80 bins of width 10, 32 walkers per bin, tau = 0.1, from X = 82 with
    recycling at X >= 563, 500 iterations): the replica-mean flux into the target for
    reweighting every 100, 5 and 2 iterations and none, against the exact flux 1 / MFPT; the
    iterations (and GPU time) after which its 10-iteration moving average stays within 50 % and
    20 % of it, and the GPU cost per iteration of each schedule."""
    import numpy as np
    import torch
    import paper_1303_5986_gb300 as P
    import workloads as W
    from paper_1303_5986_gb300 import build as pbuild

    pbuild.build()
    with open(os.path.join(ROOT, "tests", "golden", "exact_values.json")) as f:
        exact = 1.0 / json.load(f)["schlogl_mfpt_82_to_563_s"]
    n_iters, R = a.batch_iters or 500, 16
    base = W.schlogl_flux_we(n_iters=n_iters, n_runs=R)
    net = P.network_from_spec(base.network)
    bm = P.we_binmap_grid(base.bins.species, base.bins.edges)
    stream = torch.cuda.current_stream()
    clocks = Clocks(int(os.environ.get("LOCAL_RANK", "0")))

    def settle(curve, tol):
        ma = np.convolve(curve, np.ones(10) / 10, mode="valid")      # ma[k]: iterations k..k+9
        ok = np.abs(ma / exact - 1.0) <= tol
        bad = np.nonzero(~ok)[0]
        if len(bad) == 0:
            return 10
        return None if bad[-1] == len(ma) - 1 else int(bad[-1] + 11)   # first iteration count after which it holds

    out = {}
    clocks.start()
    for period in (0, 100, 5, 2):
        for w in range(a.warmup + 1):                                  # warm-ups, then one timed run
            cfg = W.schlogl_flux_we(reweight_period=period, n_iters=n_iters, n_runs=R, seed=7 + w)
            c, keep = P.run_config_from(cfg, record_iters=n_iters)
            ens = P.we_ensemble_create(net, bm, c, keep)
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            ens.step(n_iters)
            e1.record(stream)
            e1.synchronize()
        ms = e0.elapsed_time(e1)
        flux = ens.per_iter(P.WE_OUT_FLUX) / cfg.tau                  # iters x replicas
        curve = flux.mean(axis=1)
        rw = ens.per_iter(P.WE_OUT_RW) if period else np.zeros((n_iters, R), dtype=np.int32)
        i50, i20 = settle(curve, 0.5), settle(curve, 0.2)
        per_it = ms / n_iters
        out[f"rw_{period}"] = {
            "iters_to_50pct": i50, "iters_to_20pct": i20,
            "gpu_s_to_50pct": None if i50 is None else i50 * per_it * 1e-3,
            "ms_per_iteration": per_it,
            "flux_over_exact_by_50_iterations": [round(float(curve[k:k + 50].mean() / exact), 3)
                                                 for k in range(0, n_iters, 50)],
            "reweightings": int((rw == 1).sum()), "skipped": int((rw == -1).sum()),
            "status": sorted(set(int(x) for x in ens.status())),
        }
    clk = clocks.stop()
    done = [k for k in ("rw_2", "rw_5", "rw_100") if out[k]["iters_to_50pct"] is not None]
    pick = min(done, key=lambda k: out[k]["iters_to_50pct"]) if done else "rw_2"
    best = out[pick]
    line = {
        "metric": "WE iterations until the Schloegl flux stays within 50% of exact (steady-state reweighting)",
        "value": best["iters_to_50pct"], "value_schedule": pick,
        "unit": "WE iterations (10-iteration moving average of 16 replicas)",
        "n_gpus": 1, "steps": 1, "warmup": a.warmup, "ms_per_step": best["ms_per_iteration"] * n_iters,
        "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"Schloegl flux runs: 80 bins of width 10 x 32 walkers, tau=0.1, {n_iters} "
                               "iterations from X=82, recycling at X>=563, 16 replicas per schedule; "
                               "reweighting every 2, 5 or 100 iterations (value: the fastest of them, "
                               "value_schedule) and never (the baseline, in schedules)",
                   "exact_flux_per_s": exact},
        "schedules": out, "clocks": clk,
    }
    print(json.dumps(line))


# ------------------------------------------------------------------------------------------
# ranks: every rank runs its own replicas (weak scaling, no data-path collective); the job's
# figures are the slowest rank's time and the sum of every rank's work
# ------------------------------------------------------------------------------------------
def rank_seeds(rank: int, n: int) -> list:
    """Seeds of a rank's ensembles: disjoint across ranks, one per warm-up/timed/e2e step."""
    return [1_000_003 * (rank + 1) + s for s in range(n)]


def combine_ranks(dist, device, total_ms: float, events: float, flux_per_replica):
    """(max time over ranks, total events, every rank's per-replica flux means in rank order).
    flux_per_replica has the same length on every rank."""
    import numpy as np
    import torch
    fl = np.asarray(flux_per_replica, dtype=np.float64)
    if dist is None:
        return total_ms, events, fl
    t = torch.tensor([total_ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    ev = torch.tensor([events], dtype=torch.float64, device=device)
    dist.all_reduce(ev, op=dist.ReduceOp.SUM)
    mine = torch.as_tensor(fl, device=device)
    parts = [torch.empty_like(mine) for _ in range(dist.get_world_size())]
    dist.all_gather(parts, mine)
    return float(t[0]), float(ev[0]), torch.cat(parts).cpu().numpy()


# ------------------------------------------------------------------------------------------
# our arm
# ------------------------------------------------------------------------------------------
def main():
    a = parse()
    if a.workload in ("toggle_batch", "synthetic_large"):
        if a.impl == "reference":
            print(json.dumps({"impl": "reference", "unavailable": "the CPU oracle arm is timed on the "
                              "default Schloegl workload only"}))
            return
        run_batch_workload(a)
        return
    if a.workload == "schlogl_flux":
        if a.impl == "reference":
            print(json.dumps({"impl": "reference", "unavailable": "the reweighting comparison has no CPU "
                              "oracle arm; its baseline is the schedule without reweighting on the same GPU"}))
            return
        run_schlogl_flux(a)
        return
    if a.workload == "toggle_learned":
        if a.impl == "reference":
            print(json.dumps({"impl": "reference", "unavailable": "the learned-binning comparison has no CPU "
                              "oracle arm; its baseline is the plain-binning arm on the same GPU"}))
            return
        run_toggle_learned(a)
        return
    if a.impl == "reference":
        run_reference(a)
        return
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    cb = None
    if rank == 0 and world == 1 and not a.no_cpu_baseline:
        cb = cpu_baseline(a.cpu_seconds, a.replicas)       # before the first GPU call

    import numpy as np
    import torch
    import paper_1303_5986_gb300 as P
    import workloads as W
    from paper_1303_5986_gb300 import build as pbuild

    pbuild.build()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if dist is not None:
            dist.barrier()

    stream = torch.cuda.current_stream()
    mk = lambda seed: W.schlogl_mfpt_we(n_iters=a.iters, n_runs=a.replicas, seed=seed)
    base = mk(0)
    net = P.network_from_spec(base.network)
    bm = P.we_binmap_grid(base.bins.species, base.bins.edges)

    def ensemble(seed):
        cfg = mk(seed)
        c, keep = P.run_config_from(cfg, record_iters=a.iters, block_threads=a.block)
        return P.we_ensemble_create(net, bm, c, keep)

    seeds = rank_seeds(rank, a.warmup + a.steps + 1)
    # every ensemble of the timed region is uploaded before timing starts (inputs resident)
    warm = [ensemble(s) for s in seeds[:a.warmup]]
    timed = [ensemble(s) for s in seeds[a.warmup:a.warmup + a.steps]]
    for e in warm:                        # the timed path itself (graph capture, event pool)
        e.step_timed(a.iters, every=TIME_EVERY)
        e.sync()
    for e in timed:                       # capture each timed ensemble's graphs before timing
        e.step_timed(0, every=TIME_EVERY)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    clocks = Clocks(local)
    step_ms, prop_ms = [], []
    barrier()
    torch.cuda.synchronize()
    clocks.start()
    for e in timed:
        flush.zero_()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        pm = e.step_timed(a.iters, every=TIME_EVERY)
        e1.record(stream)
        e1.synchronize()
        step_ms.append(e0.elapsed_time(e1))
        prop_ms.append(pm)
    torch.cuda.synchronize()
    barrier()
    clk = clocks.stop()
    for e in timed:
        e.sync()

    ev_iter = [e.per_iter(P.WE_OUT_EVENTS).sum(axis=1) for e in timed]   # events per iteration
    events = [int(v.sum()) for v in ev_iter]
    ev_sampled = float(sum(v[::TIME_EVERY].sum() for v in ev_iter))     # of the timed launches
    fluxes = [e.per_iter(P.WE_OUT_FLUX) for e in timed]              # iters x replicas
    prop_total_ms = float(sum(p.sum() for p in prop_ms))
    n_launch = sum(len(p) for p in prop_ms)
    # MFPT = 1/flux over the replicas of all timed steps of all ranks (Eq. "mfpt")
    fl_rank = np.concatenate([f[DISCARD:].mean(axis=0) for f in fluxes]) / base.tau
    total_ms, ev_total, fl = combine_ranks(dist, "cuda", float(sum(step_ms)), float(sum(events)), fl_rank)
    value = ev_total / (total_ms * 1e-3)
    we_iters_per_s = a.steps * a.iters / (total_ms * 1e-3)
    mfpt = 1.0 / fl.mean()
    exact = exact_mfpt()
    rel_err = abs(mfpt - exact) / exact
    se = fl.std(ddof=1) / np.sqrt(len(fl)) / fl.mean() if len(fl) > 1 else None

    # roofline of the dominant kernel (the SSA kernel), from the events around the timed launches
    prop_s = prop_total_ms * 1e-3
    achieved = OPS_PER_EVENT * ev_sampled / prop_s / 1e9
    ssa_ms_est = prop_total_ms / max(n_launch, 1) * a.iters * a.steps
    roofline = {"bound": "alu", "achieved": achieved, "peak": ISSUE_PEAK_GOPS, "unit": "G lane-ops/s",
                "frac": achieved / ISSUE_PEAK_GOPS, "traffic": SSA_TRAFFIC_BYTES,
                "kernel": "k_propagate_pipe<4,2,1> (state chain / clock / draw warps, state-indexed table)",
                "launches": n_launch, "launches_sampled": f"every {TIME_EVERY}th iteration",
                "avg_launch_ms": prop_total_ms / max(n_launch, 1),
                "share_of_step": ssa_ms_est / total_ms if dist is None else None,
                "peak_source": "derived: 152 SMs x 4 SMSPs x 32 lanes x 2.07 GHz (issue limit)",
                "ops_per_event": OPS_PER_EVENT, "events_per_launch": ev_sampled / max(n_launch, 1)}

    # end to end: one we_run() call per step from host buffers, observables back to the host
    e2e = None
    if rank == 0:
        cfg = mk(seeds[-1])
        c, keep = P.run_config_from(cfg, record_iters=a.iters)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ens = P.we_run(net, bm, c, keep)
        fh = ens.get(P.WE_OUT_FLUX)
        evh = ens.get(P.WE_OUT_EVENTS)
        t1 = time.perf_counter()
        S, R, cap = cfg.network.n_species, cfg.n_runs, cfg.capacity
        h2d = 4 * S * R * cap + 8 * R * cap + 4 * R * cap + 16 * R
        d2h = fh.nbytes + evh.nbytes
        e2e = {"value": float(evh.sum()) / (t1 - t0), "unit": "SSA events/s", "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": d2h, "wall_s": t1 - t0, "path": "we_run() + we_ensemble_get(host)"}
        ens.close()

    if rank == 0:
        line = {
            "metric": "SSA events/sec and WE iterations/sec on 1 GB300; MFPT rel. error per GPU-s",
            "value": value, "unit": "SSA events/s", "n_gpus": world, "steps": a.steps,
            "warmup": a.warmup, "ms_per_step": total_ms / a.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(a), "we_iters_per_s": we_iters_per_s,
            "replica_iters_per_s": we_iters_per_s * a.replicas * world,
            "mfpt_s": mfpt, "mfpt_exact_s": exact, "mfpt_rel_error": rel_err, "mfpt_rel_se": se,
            "mfpt_rel_error_per_gpu_s": rel_err / (total_ms * 1e-3 / a.steps),
            "roofline": roofline, "cpu_baseline": cb, "e2e": e2e,
            "gpu_launches": KERNELS_PER_ITER * a.iters * a.steps, "clocks": clk,
        }
        print(json.dumps(line))
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
