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
# Algorithmic FP64 operations of one direct-method event of the Schloegl model (four reactions):
# four propensity products, three tree additions, the target u2 * a0, two descent subtractions,
# the division dt = -log(u1) / a0 and the clock addition -- 12, plus one logarithm.
FP64_OPS_PER_EVENT_SCHLOGL = 12
# DRAM bytes (read + write) of one SSA launch on this workload, from an ncu capture of the
# kernel (dram__bytes_read.sum + dram__bytes_write.sum of the launch of iteration 600, 10,540
# live walkers in 16,000 slots, as in the timed launches of that stage of the run)
SSA_TRAFFIC_BYTES = 393472


def with_resample_kernel(ens, a):
    """Apply --resample-kernel / --resample-blocks (the library's automatic choice by default)."""
    import paper_1303_5986_gb300 as P
    kinds = {"auto": P.WE_RESAMPLE_AUTO, "chain": P.WE_RESAMPLE_CHAIN, "one_launch": P.WE_RESAMPLE_ONE_LAUNCH}
    if a.resample_kernel != "auto" or a.resample_blocks:
        ens.set_resample_kernel(kinds[a.resample_kernel], a.resample_blocks)
    return ens


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
                                           "schlogl_flux", "schlogl_e50", "birth_death"],
                    default="schlogl")
    ap.add_argument("--resample-kernel", choices=["auto", "chain", "one_launch"], default="auto",
                    help="kernels of the grouping and split/merge step (same results)")
    ap.add_argument("--resample-blocks", type=int, default=0,
                    help="one_launch: blocks per run (0: the library's choice)")
    ap.add_argument("--report-iter", type=int, default=-1,
                    help="also report the SSA events of this iteration of the first timed step (for ncu; "
                         "default and batch workloads)")
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
def host_cpu() -> dict:
    """This host's logical core count and CPU model (lscpu's model name, else /proc/cpuinfo)."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().lower().startswith("model name"):
                model = line.split(":", 1)[1].strip()
                break
    except (OSError, subprocess.SubprocessError):
        pass
    if model is None:
        try:
            for line in open("/proc/cpuinfo"):
                if line.lower().startswith(("model name", "cpu model")):
                    model = line.split(":", 1)[1].strip()
                    break
        except OSError:
            pass
    return {"host_cores": os.cpu_count(), "cpu_model": model}


def _oracle_sample(args):
    replica, n_iters, seed = args[:3]
    depgraph = len(args) > 3 and args[3]
    import numpy as np  # noqa: F401
    import workloads as W
    from oracle import oracle as O
    cfg = W.schlogl_mfpt_we(n_iters=n_iters, n_runs=1, seed=seed)
    cfg.run_ids = np.array([replica], dtype=np.uint32)
    t0 = time.perf_counter()
    o = O.we_run(cfg, 0, depgraph=depgraph)
    return int(o["events"].sum()), time.perf_counter() - t0


def _calibrate():
    ev, dt = _oracle_sample((0, 40, 123))                 # the first 40 iterations
    return ev / dt, ev / 40.0


def _oracle_pool_run(cores: int, n_iters: int, seed: int, depgraph: bool = False):
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    t0 = time.perf_counter()
    with ctx.Pool(cores) as pool:
        res = pool.map(_oracle_sample, [(r, n_iters, seed, depgraph) for r in range(cores)])
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
    ev_dg, wall_dg = _oracle_pool_run(cores, n_iters, 0, depgraph=True)
    return {"value": events / wall, "unit": "SSA events/s", "cores": cores, "kind": "oracle",
            "sample": f"{cores} replica(s) x first {n_iters} of {ITERS} iterations of the workload, "
                      f"one host process each; {events} events in {wall:.1f} s", **host_cpu(),
            "depgraph": {"value": ev_dg / wall_dg, "unit": "SSA events/s", "cores": cores,
                         "kind": "dependency-graph CPU SSA (same results as the oracle)",
                         "sample": f"the same sample; {ev_dg} events in {wall_dg:.1f} s"}}


def _batch_cpu_task(args):
    """One CPU sample task of the batched or large-network workloads: (kind, item, n_iters,
    depgraph) -> (events, seconds).  toggle: the first n_iters iterations of run `item` of the
    64-run sweep; synthetic: `n_iters` intervals of plain propagation of walker `item` of the
    4096 from its initial state (iteration i, slot item)."""
    kind, item, n_iters, depgraph = args
    import workloads as W
    from oracle import oracle as O
    t0 = time.perf_counter()
    if kind == "toggle":
        cfg = W.toggle_batch_we(n_runs=64, n_iters=n_iters, seed=0)
        ev = int(O.we_run(cfg, item, n_iters=n_iters, depgraph=depgraph)["events"].sum())
    else:
        cfg = W.synthetic_large_we(n_walkers=4096, n_iters=n_iters)
        net = O.Network(cfg.network)
        x = cfg.init_states[0, item]
        ev = 0
        for it in range(n_iters):
            x, e, _, _ = O.propagate_one(cfg, x, it, item, net=net, depgraph=depgraph)
            ev += e
    return ev, time.perf_counter() - t0


def batch_cpu_baseline(kind: str):
    """CPU figures (SSA events/s on this host's cores) for the toggle sweep and the large network:
    the oracle and the dependency-graph CPU SSA on a bounded sample of the same workload, one
    spawned process per core, before any GPU work."""
    import multiprocessing as mp
    from oracle import build as obuild
    obuild.build()
    cores = os.cpu_count() or 1
    if kind == "toggle":
        items, n_iters = list(range(min(64, cores))), 300
        what = f"{len(items)} of the 64 toggle runs x their first {n_iters} iterations (WE, resampling included)"
    else:
        items, n_iters = list(range(64)), 2
        what = f"64 of the 4096 walkers x {n_iters} intervals of tau=0.01 from their initial states (SSA only)"
    out = {}
    ctx = mp.get_context("spawn")
    for dg in (False, True):
        t0 = time.perf_counter()
        with ctx.Pool(min(cores, len(items))) as pool:
            res = pool.map(_batch_cpu_task, [(kind, i, n_iters, dg) for i in items])
        wall = time.perf_counter() - t0
        ev = sum(e for e, _ in res)
        out["depgraph" if dg else "oracle"] = {"value": ev / wall, "events": ev, "wall_s": wall,
                                               "per_event_core_us": 1e6 * sum(t for _, t in res) / max(ev, 1)}
    o = out["oracle"]
    return {"value": o["value"], "unit": "SSA events/s", "cores": min(cores, len(items)), "kind": "oracle",
            "sample": what + f"; {o['events']} events in {o['wall_s']:.1f} s", **host_cpu(),
            "per_event_core_us": o["per_event_core_us"],
            "depgraph": {"value": out["depgraph"]["value"], "unit": "SSA events/s",
                         "kind": "dependency-graph CPU SSA (same results as the oracle)",
                         "per_event_core_us": out["depgraph"]["per_event_core_us"],
                         "sample": f"the same sample; {out['depgraph']['events']} events in "
                                   f"{out['depgraph']['wall_s']:.1f} s"}}


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
                    f"process each; {tot_ev} events in {tot_s:.1f} s over {a.steps} steps", **host_cpu()}
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
    cb = None if a.no_cpu_baseline else batch_cpu_baseline("toggle" if a.workload == "toggle_batch" else "synthetic")
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
        return with_resample_kernel(P.we_ensemble_create(net, bm, c, keep), a)

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
    fp64_peak = P.measure_alu_peaks()["fp64_fma_per_s"] / 1e9     # builder-measured (we_peaks.cu)
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
                     "measured_fp64_peak": fp64_peak, "frac_of_measured_fp64_peak": achieved / fp64_peak,
                     "launches": n_launch, "launches_sampled": f"every {every}th iteration",
                     "avg_launch_ms": prop_total_ms / max(n_launch, 1),
                     "share_of_step": ssa_ms_est / total_ms, "fp64_ops_per_event": ops,
                     "peak_source": "derived: 152 SMs x 2 FP64 lanes/clk x 2.07 GHz; measured beside it by "
                                    "we_measure_alu_peaks (FP64 FMA lanes/s, this GPU)"},
        "cpu_baseline": cb, "e2e": None, "gpu_launches": timed[0].iteration_kernels() * n_iters * a.steps,
        "report_iter": ({"iteration": a.report_iter,
                         "ssa_events": int(timed[0].per_iter(P.WE_OUT_EVENTS)[a.report_iter].sum()),
                         "walkers_propagated": int(timed[0].per_iter(P.WE_OUT_NWALKERS)[a.report_iter - 1].sum())
                         if a.report_iter > 0 else None}
                        if 0 <= a.report_iter < n_iters else None),
        "clocks": clk,
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
# E50%: brute-force SSA against WE on the Schloegl MFPT (Sec. II.C, Sec. III.B.3)
# ------------------------------------------------------------------------------------------
def _settled(err, tol=0.5):
    """First index from which every later entry of err is <= tol (None if the last is not)."""
    bad = [k for k, v in enumerate(err) if not (v <= tol)]
    if not bad:
        return 0
    return None if bad[-1] == len(err) - 1 else bad[-1] + 1


def run_schlogl_e50(a):
    """E50% of Sec. II.C measured on GB300: the dynamics time (simulated seconds of all segments
    or runs) brute-force SSA and WE need before their MFPT estimates stay within 50 % of the
    exact value, for the Schloegl transition 82 -> X >= 563 (50,308 s).
      brute force: 128 campaigns of 16 SSA runs from X = 82, absorbed at X >= 563, up to
        1e5 s each; for run lengths T' on a grid the library's Eq. "mld" MLE per campaign
        (we_ensemble_fpt_mle with T'), whose dynamics time is sum_i min(t_i, T') = n mu;
      WE: the paper's flux runs (80 bins of width 10 x 32 walkers, tau = 0.1, recycling
        82 <- X >= 563) with reweighting every 2, 5 and 100 iterations and without, 32
        replicas each; the running MFPT of a replica after iteration i is tau / mean flux over
        iterations i/2 .. i, its dynamics time tau x the walkers propagated so far.
    A method has settled when the median over campaigns / replicas of |estimate / exact - 1|
    stays <= 0.5 from then on; its dynamics time is the median at that point.  value = brute
    force / WE (the paper's E50%, ~500 with reweighting); GPU seconds per campaign / replica
    from CUDA events around every iteration of the batched launches are reported beside it."""
    import numpy as np
    import torch
    import paper_1303_5986_gb300 as P
    import workloads as W
    from paper_1303_5986_gb300 import build as pbuild

    pbuild.build()
    with open(os.path.join(ROOT, "tests", "golden", "exact_values.json")) as f:
        exact = json.load(f)["schlogl_mfpt_82_to_563_s"]
    clocks = Clocks(int(os.environ.get("LOCAL_RANK", "0")))
    clocks.start()
    # brute force
    n_camp, n_per, tau_bf, it_bf = 128, 16, 50.0, 2000
    bcfg = W.schlogl_bruteforce(n_walkers=n_per, tau=tau_bf, n_iters=it_bf, n_runs=n_camp, seed=11,
                                x0=82, threshold=563)
    net = P.network_from_spec(bcfg.network)
    one = P.we_binmap_grid(bcfg.bins.species, bcfg.bins.edges)
    c, keep = P.run_config_from(bcfg, record_iters=it_bf, resample=False)
    ens = P.we_ensemble_create(net, one, c, keep)
    ms_bf = ens.step_timed(it_bf, every=1)                 # SSA kernel time per interval
    ens.sync()
    grid = np.unique(np.concatenate([np.geomspace(100.0, tau_bf * it_bf, 120), [tau_bf * it_bf]]))
    err_bf, dyn_bf = [], []
    for Tp in grid:
        m = ens.fpt_mle(float(Tp))                         # (N, n, sum t, mu, sigma) per campaign
        err_bf.append(float(np.median(np.abs(m[:, 3] / exact - 1.0))))
        dyn_bf.append(float(np.median(m[:, 2] + (m[:, 0] - m[:, 1]) * Tp)))
    kb = _settled(err_bf)
    bf_events = float(ens.per_iter(P.WE_OUT_EVENTS).sum())
    ens.close()
    ssa_bf_ms = np.cumsum(ms_bf)
    bf = {"campaigns": n_camp, "runs_per_campaign": n_per, "max_run_s": tau_bf * it_bf,
          "settled_run_length_s": None if kb is None else float(grid[kb]),
          "dynamics_s_to_50pct": None if kb is None else dyn_bf[kb],
          "gpu_s_per_campaign_to_50pct": None if kb is None else
          float(ssa_bf_ms[min(it_bf, int(np.ceil(grid[kb] / tau_bf))) - 1]) * 1e-3 / n_camp,
          "ssa_events": bf_events, "ssa_gpu_s": float(ssa_bf_ms[-1]) * 1e-3,
          "median_rel_err_at_max_length": err_bf[-1]}
    # weighted ensemble, per reweighting schedule
    R, n_it = 32, 500
    we = {}
    for period in (0, 100, 5, 2):
        cfg = W.schlogl_flux_we(reweight_period=period, n_iters=n_it, n_runs=R, seed=13)
        bm = P.we_binmap_grid(cfg.bins.species, cfg.bins.edges)
        c, keep = P.run_config_from(cfg, record_iters=n_it)
        e = P.we_ensemble_create(net, bm, c, keep)
        ms = e.step_timed(n_it, every=1)
        e.sync()
        flux = e.per_iter(P.WE_OUT_FLUX)                   # iters x replicas
        nw = e.per_iter(P.WE_OUT_NWALKERS)
        prop = np.vstack([np.full((1, R), cfg.m_targ), nw[:-1]])      # walkers propagated per iteration
        dyn = np.cumsum(prop, axis=0) * cfg.tau
        err = []
        for i in range(n_it):
            f = flux[i // 2:i + 1].mean(axis=0)
            est = np.where(f > 0, cfg.tau / np.maximum(f, 1e-300), np.inf)
            err.append(float(np.median(np.abs(est / exact - 1.0))))
        k = _settled(err)
        we[f"rw_{period}"] = {
            "iterations_to_50pct": None if k is None else k + 1,
            "dynamics_s_to_50pct": None if k is None else float(np.median(dyn[k])),
            "segments_to_50pct": None if k is None else float(np.median(np.cumsum(prop, axis=0)[k])),
            "gpu_s_per_replica_to_50pct": None if k is None else float(np.sum(ms[:k + 1])) * 1e-3 / R,
            "median_rel_err_end": err[-1]}
        e.close()
    clk = clocks.stop()
    ok = {k: v for k, v in we.items() if v["dynamics_s_to_50pct"] is not None}
    best = min(ok, key=lambda k: ok[k]["dynamics_s_to_50pct"]) if ok else None
    value = None
    if best is not None and bf["dynamics_s_to_50pct"] is not None:
        value = bf["dynamics_s_to_50pct"] / we[best]["dynamics_s_to_50pct"]
    gpu_ratio = None
    if best is not None and bf["gpu_s_per_campaign_to_50pct"] is not None:
        gpu_ratio = bf["gpu_s_per_campaign_to_50pct"] / we[best]["gpu_s_per_replica_to_50pct"]
    line = {
        "metric": "E50%: brute-force / WE dynamics time to a Schloegl MFPT within 50% of exact",
        "value": value, "unit": "x (dynamics-time ratio, Sec. II.C)", "value_schedule": best,
        "gpu_time_ratio": gpu_ratio, "n_gpus": 1, "higher_is_better": True, "dtype": "f64",
        "data": "synthetic", "vs_baseline": None,
        "config": {"workload": "Schloegl 82 -> X >= 563 (exact MFPT %.1f s); brute force: 128 campaigns x 16 "
                               "absorbed SSA runs up to 1e5 s, Eq. \"mld\" MLE on the device; WE: 80 bins of "
                               "width 10 x 32 walkers, tau=0.1, 500 iterations, 32 replicas, reweighting every "
                               "2/5/100 iterations or never" % exact},
        "bruteforce": bf, "we": we, "clocks": clk,
    }
    print(json.dumps(line))


# ------------------------------------------------------------------------------------------
# the 1-D birth-death configuration: WE iterations/s against the launch floor
# ------------------------------------------------------------------------------------------
def run_birth_death(a):
    """The 1-D birth-death configuration (kb = 10, kd = 0.1, X0 = 100; 60 bins of width 5 plus
    overflow, 10 walkers per bin, tau = 0.1, 200 iterations), 10 replicas (run ids 0-9) in one
    batch per step.  About 2 events per walker per interval: the iteration is launch-latency
    bound, so its roofline is the measured floor of a CUDA graph of the same number of empty
    launches (one block per SM each)."""
    import numpy as np
    import torch
    import paper_1303_5986_gb300 as P
    import workloads as W
    from paper_1303_5986_gb300 import build as pbuild

    pbuild.build()
    n_iters, R = a.batch_iters or 200, 10
    base = W.birth_death_we(n_iters=n_iters, n_runs=R)
    net = P.network_from_spec(base.network)
    bm = P.we_binmap_grid(base.bins.species, base.bins.edges)
    seeds = rank_seeds(0, a.warmup + a.steps)

    # the library's autotuner picks the SSA mapping and block shape for this configuration (with
    # ~2 events per walker per interval the plain thread-per-walker table kernel can beat the
    # pipelined one, whose rounds of 16 draws pay off only for long event chains)
    c0, keep0 = P.run_config_from(base, record_iters=n_iters)
    mapping, block = P.we_autotune(net, bm, c0)

    def ensemble(seed):
        c, keep = P.run_config_from(W.birth_death_we(n_iters=n_iters, n_runs=R, seed=seed), record_iters=n_iters,
                                    mapping=mapping, block_threads=block)
        return with_resample_kernel(P.we_ensemble_create(net, bm, c, keep), a)

    warm = [ensemble(s) for s in seeds[:a.warmup]]
    timed = [ensemble(s) for s in seeds[a.warmup:]]
    for e in warm:
        e.step_timed(n_iters, every=n_iters)
        e.sync()
    for e in timed:                       # capture each timed ensemble's graphs before timing
        e.step_timed(0, every=n_iters)
    k_iter = timed[0].iteration_kernels()
    floor_ms = P.measure_graph_floor(k_iter, 2000)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()
    clocks = Clocks(int(os.environ.get("LOCAL_RANK", "0")))
    step_ms = []
    torch.cuda.synchronize()
    clocks.start()
    for e in timed:
        flush.zero_()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        e.step_timed(n_iters, every=n_iters)      # the first iteration's SSA launch timed too
        e1.record(stream)
        e1.synchronize()
        step_ms.append(e0.elapsed_time(e1))
    torch.cuda.synchronize()
    clk = clocks.stop()
    total_ms = float(sum(step_ms))
    events = float(sum(e.per_iter(P.WE_OUT_EVENTS).sum() for e in timed))
    status = sorted(set(int(x) for e in timed for x in e.status()))
    it_per_s = a.steps * n_iters / (total_ms * 1e-3)
    per_iter_ms = total_ms / (a.steps * n_iters)
    line = {
        "metric": "SSA events/sec and WE iterations/sec on 1 GB300",
        "value": it_per_s, "unit": "WE iterations/s (10 replicas per iteration)", "n_gpus": 1,
        "steps": a.steps, "warmup": a.warmup, "ms_per_step": total_ms / a.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "1-D birth-death kb=10, kd=0.1, X0=100: 60 bins of width 5 + overflow x 10 "
                               f"walkers, tau=0.1, {n_iters} iterations, 10 replicas per step",
                   "iterations": n_iters, "l2": "flushed between timed steps (256 MB write)",
                   "ssa_mapping": {1: "thread", 2: "warp", 3: "thread, state-indexed table"}.get(mapping, mapping),
                   "ssa_block_threads": block},
        "ssa_events_per_s": events / (total_ms * 1e-3), "status": status,
        "roofline": {"bound": "latency", "achieved": 1.0 / per_iter_ms * 1e3, "peak": 1.0 / floor_ms * 1e3,
                     "unit": "WE iterations/s", "frac": floor_ms / per_iter_ms, "traffic": None,
                     "kernel": f"whole iteration graph ({k_iter} kernels: SSA, grouping by bin and split/merge, "
                               "finalize)",
                     "ms_per_iteration": per_iter_ms, "floor_ms_per_iteration": floor_ms,
                     "peak_source": f"measured: CUDA graph of {k_iter} empty launches of one "
                                    "block per SM, replayed 2000 times (we_measure_graph_floor)"},
        "cpu_baseline": None, "e2e": None, "gpu_launches": k_iter * n_iters * a.steps, "clocks": clk,
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
    if a.workload in ("schlogl_e50", "birth_death"):
        if a.impl == "reference":
            print(json.dumps({"impl": "reference", "unavailable": "the CPU oracle arm is timed on the "
                              "default Schloegl workload only"}))
            return
        (run_schlogl_e50 if a.workload == "schlogl_e50" else run_birth_death)(a)
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
        return with_resample_kernel(P.we_ensemble_create(net, bm, c, keep), a)

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
    report_iter = None
    if 0 <= a.report_iter < a.iters:
        report_iter = {"iteration": a.report_iter, "ssa_events": int(ev_iter[0][a.report_iter]),
                       "walkers": int(timed[0].per_iter(P.WE_OUT_NWALKERS)[a.report_iter - 1].sum())
                       if a.report_iter > 0 else None}
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
    peaks = P.measure_alu_peaks()                     # builder-measured denominators (we_peaks.cu)
    ev_rate = ev_sampled / prop_s                     # events/s inside the SSA kernel
    fp64_achieved = FP64_OPS_PER_EVENT_SCHLOGL * ev_rate / 1e9
    # the roofline of the method's algorithmic work (FP64 operations per event) against the FP64
    # peak derived from the unit counts and clock; beside it the same against the FP64 FMA rate
    # the library measures, and the implementation's issue form (its own lane-operation model)
    roofline = {"bound": "alu", "achieved": fp64_achieved, "peak": FP64_PEAK_GOPS, "unit": "G FP64 ops/s",
                "frac": fp64_achieved / FP64_PEAK_GOPS, "traffic": SSA_TRAFFIC_BYTES,
                "kernel": "k_propagate_pipe<4,2,1> (state chain / clock / draw warps, state-indexed table)",
                "fp64_ops_per_event": FP64_OPS_PER_EVENT_SCHLOGL, "plus_per_event": "one logarithm",
                "peak_source": "derived: 152 SMs x 2 FP64 lanes/clk x 2.07 GHz",
                "measured_fp64_peak": peaks["fp64_fma_per_s"] / 1e9,
                "frac_of_measured_fp64_peak": FP64_OPS_PER_EVENT_SCHLOGL * ev_rate / peaks["fp64_fma_per_s"],
                "measured_peak_source": "we_measure_alu_peaks (FP64 FMA lanes/s on this GPU)",
                "issue_form": {"achieved": achieved, "peak": ISSUE_PEAK_GOPS, "unit": "G lane-ops/s",
                               "frac": achieved / ISSUE_PEAK_GOPS, "ops_per_event": OPS_PER_EVENT,
                               "peak_source": "derived: 152 SMs x 4 SMSPs x 32 lanes x 2.07 GHz (issue limit)",
                               "measured_int32_alu_peak": peaks["ialu_per_s"] / 1e9,
                               "measured_int32_imad_peak": peaks["imad_per_s"] / 1e9},
                "launches": n_launch, "launches_sampled": f"every {TIME_EVERY}th iteration",
                "avg_launch_ms": prop_total_ms / max(n_launch, 1),
                "share_of_step": ssa_ms_est / total_ms if dist is None else None,
                "events_per_launch": ev_sampled / max(n_launch, 1)}

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
            "roofline": roofline, "cpu_baseline": cb, "e2e": e2e, "report_iter": report_iter,
            "gpu_launches": timed[0].iteration_kernels() * a.iters * a.steps, "clocks": clk,
        }
        print(json.dumps(line))
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
