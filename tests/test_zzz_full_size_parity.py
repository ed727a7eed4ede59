"""GPU path against the CPU oracle at the benchmarks' full sizes, in the launch configurations
the benchmarks time (collected late: these are the longest GPU tests): the Schloegl MFPT
workload, the 64-run toggle sweep in full, the 354 x 3680 network (sampled walkers of its first
interval, and whole iterations through resampling), the paper-scale Schloegl PDF run and the
1-D birth-death configuration.

The Schloegl MFPT workload with 10 replicas of 1,600 walker slots each (80 bins x 20 walkers,
tau = 0.05, recycling at X >= 550 back to X = 85; default mapping and block shape) runs 600
iterations on the GPU, into the regime the benchmark spends its time in: walkers spread up to
the high state and recycle every interval (~1,060 walkers and ~1.8e5 SSA events per run and
iteration).  Three more iterations then run on the GPU and, from the GPU's own populations at
iteration 600 (first iteration 600, so the same counter-based random numbers), on the oracle:
every run's walkers, weights, parents, event counts, fluxes and histograms must agree (bit for
bit; observables summed by device atomics within 1e-12 relative)."""
import numpy as np
import pytest

import workloads as W

from gpu_helpers import assert_run_parity, gpu_outputs, gpu_run, oracle_run

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1303_5986_gb300 import build
    build.build()


def test_schlogl_benchmark_configuration_at_full_size():
    k, m, R = 600, 3, 10
    cfg = W.schlogl_mfpt_we(n_iters=k + m, n_runs=R)
    ens = gpu_run(cfg, k, record_iters=k + m)
    ens.sync()
    states = [ens.states(r) for r in range(R)]
    weights = [ens.weights(r) for r in range(R)]
    ens.step(m)
    ens.sync()
    recycled, events = 0.0, 0
    for r in range(R):
        g = gpu_outputs(ens, r)
        for key in ("flux_weight", "total_weight", "n_walkers", "events", "hist", "near_tau"):
            g[key] = g[key][k:]
        o = oracle_run(cfg, r, n_iters=m, init_states=states, init_weights=weights, first_iter=k)
        assert_run_parity(g, o, label=f"benchmark configuration, run {r}")
        recycled += float(g["flux_weight"].sum())
        events += int(g["events"].sum())
    assert recycled > 0.0
    assert events > R * m * 100_000


def test_synthetic_354x3680_first_interval_at_full_size_sampled():
    """The 354-species / 3680-reaction network at the benchmark's full size (4,096 walkers with
    counts uniform in [0, 200], one warp per walker as the benchmark launches it): the first
    interval (~3.9e4 events per walker) on the GPU, then eight sampled walkers (both ends of
    the population and six between) replayed one by one on the oracle from the same initial
    counts and random-number counters: their counts after the interval agree bit for bit."""
    from oracle import oracle as O
    cfg = W.synthetic_large_we(n_walkers=4096, n_iters=1)
    ens = gpu_run(cfg, 0, record_iters=1)
    ens.propagate()
    ens.sync()
    after = ens.states(0)
    assert after.shape == (4096, 354)
    x0 = np.asarray(cfg.init_states)[0]
    net = O.Network(cfg.network, 0)
    for s in (0, 1, 1000, 2047, 2048, 3000, 4094, 4095):
        x, ev, rec, rc = O.propagate_one(cfg, x0[s], 0, s, run=0, net=net)
        assert rc == 0 and ev > 10_000, (s, rc, ev)
        assert np.array_equal(after[s], x), s


def test_toggle_sweep_at_full_size():
    """The batched toggle sweep as the benchmark runs it: 64 runs, each with its own production
    rates, 500 iterations, every phase one launch for all runs; every run's walkers, weights,
    parents, event counts, fluxes and histograms against the oracle's."""
    cfg = W.toggle_batch_we()
    assert (cfg.n_runs, cfg.n_iters) == (64, 500)
    ens = gpu_run(cfg, cfg.n_iters)
    ens.sync()
    for r in range(cfg.n_runs):
        assert_run_parity(gpu_outputs(ens, r), oracle_run(cfg, r, n_iters=cfg.n_iters),
                          label=f"toggle sweep, run {r}")


@pytest.mark.parametrize("target", [None, 250])
def test_birth_death_at_full_size(target):
    """The 1-D birth-death configuration in full: 60 bins of width 5 plus an overflow bin,
    10 walkers per bin, tau = 0.1, 200 iterations, with and without recycling at X >= 250."""
    cfg = W.birth_death_we(target=target)
    assert cfg.n_iters == 200
    ens = gpu_run(cfg, cfg.n_iters)
    ens.sync()
    assert_run_parity(gpu_outputs(ens, 0), oracle_run(cfg, 0, n_iters=cfg.n_iters),
                      label=f"birth-death, target {target}")


def test_synthetic_354x3680_through_resampling_at_full_size():
    """The 354 x 3680 network at the benchmark's full size through resampling: 4,096 walkers
    run 4 iterations on the GPU (the first interval of all 4,096 walkers, then the population
    the benchmark spends its later iterations in, ~160-250 walkers in the 2-3 occupied bins of
    82 walkers), then 2 more on the GPU and, from the GPU's own population at iteration 4, on
    the oracle (its full propensity recomputation per event): walkers, weights, parents, event
    counts and observables agree."""
    k, m = 4, 2
    cfg = W.synthetic_large_we(n_walkers=4096, n_iters=k + m)
    ens = gpu_run(cfg, k, record_iters=k + m)
    ens.sync()
    states = [ens.states(0)]
    weights = [ens.weights(0)]
    assert 80 <= len(states[0]) <= 600
    ens.step(m)
    ens.sync()
    g = gpu_outputs(ens, 0)
    for key in ("flux_weight", "total_weight", "n_walkers", "events", "hist", "near_tau"):
        g[key] = g[key][k:]
    o = oracle_run(cfg, 0, n_iters=m, init_states=states, init_weights=weights, first_iter=k)
    assert_run_parity(g, o, label="354 x 3680 through resampling")
    assert int(g["events"].sum()) > 500_000


def test_schlogl_pdf_paper_scale_at_full_size():
    """The paper's Schloegl PDF run at its scale (802 unit bins x 100 walkers, tau = 0.05, from
    X = 82; Sec. III.B.2), two replicas: 99 iterations on the GPU (tens of thousands of walkers
    per replica spread over hundreds of bins), then the last two iterations (to t = 5) on the GPU
    and, from the GPU's own populations, on the oracle: the split/merge of every bin at this
    width, and every walker, weight, parent and histogram entry, agree."""
    k, m, R = 99, 2, 2
    cfg = W.schlogl_pdf_we(n_iters=k + m, n_runs=R)
    ens = gpu_run(cfg, k, record_iters=k + m)
    ens.sync()
    states = [ens.states(r) for r in range(R)]
    weights = [ens.weights(r) for r in range(R)]
    assert min(len(s) for s in states) > 20_000
    ens.step(m)
    ens.sync()
    for r in range(R):
        g = gpu_outputs(ens, r)
        for key in ("flux_weight", "total_weight", "n_walkers", "events", "hist", "near_tau"):
            g[key] = g[key][k:]
        o = oracle_run(cfg, r, n_iters=m, init_states=states, init_weights=weights, first_iter=k)
        assert_run_parity(g, o, label=f"Schloegl PDF at paper scale, run {r}")
