"""GPU path (through the C ABI) against the CPU oracle on identical seeded inputs.

Bar: bit-exact species counts, walker order, parents and weights after every resampling, exact
event counts; event times within 1e-12 relative; observables that device atomics sum in
arbitrary order within 1e-12 relative."""
import numpy as np
import pytest

import paper_1303_5986_gb300 as P
import workloads as W
from oracle import oracle as O

from gpu_helpers import assert_run_parity, gpu_outputs, gpu_run, oracle_run

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1303_5986_gb300 import build
    build.build()


def _parity(cfg, n_iters, runs=None, **kw):
    ens = gpu_run(cfg, n_iters, **kw)
    ens.sync()
    runs = range(cfg.n_runs) if runs is None else runs
    for r in runs:
        g = gpu_outputs(ens, r)
        o = oracle_run(cfg, r, n_iters=n_iters, resample=kw.get("resample", True),
                       max_steps=kw.get("max_steps"))
        assert_run_parity(g, o, label=f"{cfg.name} run {r}")
    return ens


MAPPINGS = [P.WE_MAP_AUTO, P.WE_MAP_THREAD]        # auto picks the state-indexed tables here


@pytest.mark.parametrize("mapping", MAPPINGS)
def test_birth_death_we(mapping):
    _parity(W.birth_death_we(n_iters=60), 60, mapping=mapping)


@pytest.mark.parametrize("mapping", MAPPINGS)
def test_birth_death_we_with_recycling(mapping):
    _parity(W.birth_death_we(n_iters=60, target=130), 60, mapping=mapping)


@pytest.mark.parametrize("edges", [
    W.uniform_edges(93, 4, 9),                        # integer inner edges 97..125 with an offset
    np.array([0.0, 103.0, np.inf]),                   # two bins
    W.uniform_edges(90.5, 3, 8, overflow=True),       # uniform but not integers: searched
    np.array([0.0, 95, 99, 100, 104, 120, np.inf]),   # integers, not uniform: searched
], ids=["uniform_offset", "two_bins", "non_integer", "non_uniform"])
@pytest.mark.parametrize("mapping", [P.WE_MAP_AUTO, P.WE_MAP_THREAD, P.WE_MAP_WARP])
def test_grid_bin_forms(edges, mapping):
    """A count's bin by division (integer inner edges in arithmetic progression) or by searching
    the edges (any other grid) equals the oracle's search, counts below the first inner edge and
    above the last included (birth-death around X = 100)."""
    cfg = W.birth_death_we(n_iters=30)
    cfg.bins = W.GridBins([0], [np.asarray(edges, dtype=np.float64)])
    _parity(cfg, 30, mapping=mapping)


@pytest.mark.parametrize("mapping", MAPPINGS)
@pytest.mark.parametrize("block", [0, 32])
def test_schlogl_mfpt_batched_replicas(mapping, block):
    _parity(W.schlogl_mfpt_we(n_iters=40, n_runs=3), 40, mapping=mapping, block_threads=block)


def test_schlogl_table_beyond_its_range():
    """Walkers above the table's last count take the directly evaluated row."""
    cfg = W.schlogl_pdf_we(n_iters=6, m_targ=4, n_unit_bins=80)
    cfg.bins = W.GridBins([0], [W.uniform_edges(0, 100, 80)])
    cfg.x0[:, 0] = 5000
    cfg.init_states[:, :, 0] = 5000
    cfg.recycle_state[:, 0] = 5000
    cfg.capacity = 4 * 80
    _parity(cfg, 6, mapping=P.WE_MAP_THREAD_TABLE)


@pytest.mark.parametrize("mapping,block", [(P.WE_MAP_THREAD_TABLE, 0), (P.WE_MAP_THREAD_TABLE, 64),
                                           (P.WE_MAP_THREAD, 0)])
def test_event_just_before_the_end_of_the_interval(mapping, block):
    """An interval whose only event of one walker falls 1.6e-8 tau before tau (toggle a = 40 at
    (U, V) = (10, 2), iteration 50392, run id 11, walker slot 65): the waiting time's leading
    float product rounds up to the end of the interval, so the fire test must use the full
    product.  Plain SSA for one interval, against the oracle."""
    cfg = W.toggle_batch_we(n_runs=1, n_iters=1)
    cfg.network = W.toggle_switch([40.0], [40.0])
    cfg.param_set = np.zeros(1, np.int32)
    cfg.run_ids = np.array([11], dtype=np.uint32)
    cfg.seed = 1
    cfg.x0 = np.array([[40, 0]], dtype=np.int32)
    cfg.recycle_state = cfg.x0.copy()
    cfg.target.threshold = np.array([[20, 10]], dtype=np.int32)
    n = 240
    cfg.init_states = np.tile(np.array([10, 2], dtype=np.int32), (1, n, 1))
    cfg.init_weights = np.full((1, n), 1.0 / n)
    cfg.capacity = n
    cfg.first_iter = 50392
    ens = gpu_run(cfg, 1, resample=False, mapping=mapping, block_threads=block, first_iter=50392)
    ens.sync()
    g = gpu_outputs(ens, 0, hist=False)
    o = oracle_run(cfg, 0, n_iters=1, resample=False, first_iter=50392)
    assert np.array_equal(g["states"][65], [10, 1])        # the event at t = 0.0999999984 fires
    assert_run_parity(g, o, label=f"end-of-interval {mapping} {block}")
    t = ens.get(P.WE_OUT_TLAST, 0)
    assert abs(t[65] - 0.09999999837240271) < 1e-15


@pytest.mark.parametrize("mapping,block", [(P.WE_MAP_AUTO, 0), (P.WE_MAP_AUTO, 32), (P.WE_MAP_THREAD, 0),
                                           (P.WE_MAP_THREAD, 32), (P.WE_MAP_WARP, 0)])
def test_near_tau_stop_decisions_are_counted(mapping, block):
    """An interval chosen to end exactly at a walker's first event: the host computes that
    event's time t1 = -log(u1) / a0 from the same counter-based draw (slot 0, iteration 0) and
    sets tau = t1.  Whatever the kernel decides for that event, the walker's stop decision is
    within 2^-40 tau of tau and WE_OUT_NEAR_TAU counts it; the other walkers of the run start
    elsewhere and are not counted unless they too end that close."""
    import math
    cfg = W.birth_death_we(n_iters=1)
    key = [int(cfg.seed) & 0xffffffff, ((int(cfg.seed) >> 32) + int(cfg.run_ids[0])) & 0xffffffff]
    r = O.philox([0, 0, 0, 0], key)
    u1 = O.u01(r[0], r[1])
    a0 = O.tree_total(O.Network(cfg.network).propensities([100]))
    cfg.tau = -math.log(u1) / a0
    ens = gpu_run(cfg, 1, resample=False, mapping=mapping, block_threads=block)
    ens.sync()
    near = ens.per_iter(P.WE_OUT_NEAR_TAU, 0)
    assert near[0] >= 1, (mapping, block, near)
    assert near[0] <= 3
    ens2 = gpu_run(W.birth_death_we(n_iters=1), 1, resample=False, mapping=mapping, block_threads=block)
    ens2.sync()
    assert ens2.per_iter(P.WE_OUT_NEAR_TAU, 0)[0] == 0


@pytest.mark.parametrize("block", [0, 64])
def test_two_species_table_beyond_its_range(block):
    """A toggle whose counts run past the two-species table (256 x 256 for one parameter set):
    walkers above it take the directly evaluated row, in the pipelined kernel (block 128) and
    the thread kernel (block 64)."""
    cfg = W.toggle_batch_we(n_runs=2, n_iters=8)
    a = np.array([400.0, 300.0])
    cfg.network = W.toggle_switch(a, a[::-1].copy())
    cfg.x0 = np.array([[400, 0], [300, 2]], dtype=np.int32)
    cfg.init_states = np.repeat(cfg.x0[:, None, :], cfg.m_targ, axis=1)
    cfg.recycle_state = cfg.x0.copy()
    cfg.target.threshold = np.array([[150, 100], [200, 75]], dtype=np.int32)
    cfg.bins = W.GridBins(species=[0, 1], edges=[W.uniform_edges(0, 40, 12, overflow=True)] * 2)
    cfg.capacity = cfg.m_targ * cfg.bins.n_bins
    _parity(cfg, 8, mapping=P.WE_MAP_THREAD_TABLE, block_threads=block)


@pytest.mark.parametrize("block", [0, 64])
def test_toggle_batch_uneven_runs(block):
    cfg = W.toggle_batch_we(n_runs=8, n_iters=30)
    ens = _parity(cfg, 30, block_threads=block)
    counts = ens.get(P.WE_OUT_COUNTS)
    assert len(set(counts.tolist())) > 1          # uneven live-walker counts across runs


def test_epigenetic_switch_paper_bins():
    """The paper's switch (n=3, m=1) with its non-uniform 15 x 31 bins (Sec. III.C.2)."""
    spec = W.epigenetic_switch()
    e1 = np.concatenate([np.arange(0, 11, dtype=float), [20.0, 30.0, 40.0, 50.0, np.inf]])
    e2 = np.concatenate([np.arange(0, 31, dtype=float), [np.inf]])
    cfg = W.WEConfig(network=spec, bins=W.GridBins([0, 1], [e1, e2]), tau=0.1, m_targ=16,
                     n_iters=25, x0=[150, 0], hist_species=1, hist_len=64, name="epigenetic")
    _parity(cfg, 25)


def test_futile_cycle():
    spec = W.futile_cycle()
    cfg = W.WEConfig(network=spec, bins=W.GridBins([0], [W.uniform_edges(0, 1, 101)]), tau=1.0,
                     m_targ=10, n_iters=15, x0=[50, 50, 1, 1, 0, 0], hist_species=0, hist_len=102,
                     name="futile")
    _parity(cfg, 15)


@pytest.mark.parametrize("mapping", MAPPINGS)
@pytest.mark.parametrize("block", [32, 96, 128])
def test_plain_ssa_counts_and_times(block, mapping):
    """No resampling: 3000 Schloegl walkers for three intervals; counts bit-exact, last event
    times within 1e-12 relative (device log vs host log may differ in the last bit)."""
    cfg = W.schlogl_mfpt_we(n_iters=3)
    cfg.target = None
    n = 3000
    rng = np.random.default_rng(4)
    init = np.zeros((1, n, 3), dtype=np.int32)
    init[0, :, 0] = rng.integers(0, 700, size=n)
    init[0, :, 1], init[0, :, 2] = 100000, 200000
    w = np.full((1, n), 1.0 / n)
    cfg.capacity = n
    ens = gpu_run(cfg, 3, resample=False, init_states=init, init_weights=w, block_threads=block,
                  mapping=mapping)
    ens.sync()
    o = oracle_run(cfg, 0, n_iters=3, resample=False, init_states=init, init_weights=w)
    g = gpu_outputs(ens, 0)
    assert_run_parity(g, o, "plain ssa")
    tl = ens.get(P.WE_OUT_TLAST, 0)
    np.testing.assert_allclose(tl, o["t_last"][:n], rtol=1e-12, atol=0)
    rel = np.abs(tl - o["t_last"][:n]) / np.maximum(o["t_last"][:n], 1e-300)
    assert rel.max() < 1e-13                          # the float-float logarithm: ~1e-14
    assert np.all(tl <= cfg.tau) and np.count_nonzero(tl) > n // 2


def test_zero_propensity_walkers_idle():
    dead = W.NetworkSpec(species=["X", "Y"], reactants=[[(0, 1)], [(1, 2)]], products=[[(1, 1)], []],
                         rate=[[1.0, 2.0]])
    cfg = W.WEConfig(network=dead, bins=W.GridBins([0], [W.uniform_edges(0, 1, 4)]), tau=1.0,
                     m_targ=3, n_iters=4, x0=[0, 1], hist_species=1, hist_len=4, name="dead")
    _parity(cfg, 4)


def test_many_merges_in_one_bin():
    """600 walkers of random weight in one bin merged down to M=3 (the serial merge path)."""
    spec = W.birth_death(kb=1e-9, kd=1e-9)
    n = 600
    rng = np.random.default_rng(8)
    init = np.full((1, n, 1), 7, dtype=np.int32)
    w = rng.exponential(size=(1, n)) * 10.0 ** rng.uniform(-30, 0, size=(1, n))
    w /= w.sum()
    cfg = W.WEConfig(network=spec, bins=W.GridBins([0], [W.uniform_edges(0, 5, 4)]), tau=0.1,
                     m_targ=3, n_iters=2, x0=[7], init_states=init, init_weights=w, capacity=n,
                     hist_species=0, hist_len=16, name="merges")
    _parity(cfg, 2)


def test_single_walker_m1_and_split_to_many():
    cfg = W.birth_death_we(n_iters=10)
    cfg.m_targ = 1
    cfg.init_states = cfg.init_states[:, :1]
    cfg.init_weights = np.ones((1, 1))
    cfg.capacity = 61
    _parity(cfg, 10)
    cfg2 = W.birth_death_we(n_iters=6)
    cfg2.m_targ = 37
    cfg2.init_states = cfg2.init_states[:, :1]
    cfg2.init_weights = np.ones((1, 1))
    cfg2.capacity = 37 * 61
    _parity(cfg2, 6)


def test_recycle_on_first_event():
    cfg = W.birth_death_we(n_iters=8, target=101)
    _parity(cfg, 8)


def test_step_cap_status():
    cfg = W.schlogl_mfpt_we(n_iters=3)
    ens = gpu_run(cfg, 3, max_steps=5)
    with pytest.raises(P.WEError) as ei:
        ens.sync()
    assert ei.value.status == P.WE_ESTEPCAP
    o = oracle_run(cfg, 0, n_iters=3, max_steps=5)
    assert o["status"] == P.WE_ESTEPCAP and int(ens.status()[0]) == P.WE_ESTEPCAP


def test_count_overflow_status():
    grow = W.NetworkSpec(species=["X"], reactants=[[]], products=[[(0, 1)]], rate=[[1e9]])
    cfg = W.WEConfig(network=grow, bins=W.GridBins([0], [W.uniform_edges(0, 1e6, 4)]), tau=1.0,
                     m_targ=2, n_iters=1, x0=[P.WE_MAX_COUNT - 3], name="overflow")
    ens = gpu_run(cfg, 1)
    with pytest.raises(P.WEError) as ei:
        ens.sync()
    assert ei.value.status == P.WE_EOVERFLOW
    o = oracle_run(cfg, 0, n_iters=1)
    assert o["status"] == P.WE_EOVERFLOW
    s = ens.states(0)
    assert np.all(s[:, 0] == P.WE_MAX_COUNT)


def test_checkpoint_resume_is_bit_identical():
    cfg = W.schlogl_mfpt_we(n_iters=24, n_runs=2)
    full = gpu_run(cfg, 24)
    full.sync()
    first = gpu_run(cfg, 12)
    first.sync()
    R = cfg.n_runs
    states = [first.states(r) for r in range(R)]
    weights = [first.weights(r) for r in range(R)]
    n = min(len(w) for w in weights)
    # resume each run separately from its checkpoint (walker counts may differ per run)
    for r in range(R):
        c1 = W.schlogl_mfpt_we(n_iters=12, n_runs=1)
        c1.run_ids = np.array([r], dtype=np.uint32)
        c1.first_iter = 12
        ens = gpu_run(c1, 12, init_states=states[r][None], init_weights=weights[r][None], first_iter=12)
        ens.sync()
        assert np.array_equal(ens.states(0), full.states(r))
        assert np.array_equal(ens.weights(0).view(np.int64), full.weights(r).view(np.int64))
        assert np.array_equal(ens.per_iter(P.WE_OUT_EVENTS, 0), full.per_iter(P.WE_OUT_EVENTS, r)[12:])
    assert n > 0


@pytest.mark.parametrize("case", ["schlogl", "toggle", "reweighted"])
def test_checkpoint_and_resume_a_batch(case):
    """we_ensemble_checkpoint after 12 iterations, we_ensemble_resume, 12 more: every run of the
    batch (uneven walker counts) ends bit-identical to 24 uninterrupted iterations, including
    the steady-state reweighting state (transfers and the last split/merge's bin layout)."""
    if case == "schlogl":
        mk = lambda n: W.schlogl_mfpt_we(n_iters=n, n_runs=3)
    elif case == "toggle":
        mk = lambda n: W.toggle_batch_we(n_runs=4, n_iters=n)
    else:
        mk = lambda n: W.schlogl_flux_we(reweight_period=3, n_iters=n, n_runs=2, m_targ=6)
    cfg = mk(24)
    full = gpu_run(cfg, 24)
    full.sync()
    first = gpu_run(cfg, 12, record_iters=24)
    first.sync()
    blob = first.checkpoint()
    c2 = mk(12)
    net = P.network_from_spec(c2.network)
    bm = P.we_binmap_grid(c2.bins.species, c2.bins.edges)
    conf, keep = P.run_config_from(c2, record_iters=12)
    ens = P.we_ensemble_resume(net, bm, conf, blob, keep)
    ens.step(12)
    ens.sync()
    assert int(ens.get(P.WE_OUT_ITER)[0]) == 24
    for r in range(cfg.n_runs):
        assert np.array_equal(ens.states(r), full.states(r)), r
        assert np.array_equal(ens.weights(r).view(np.int64), full.weights(r).view(np.int64)), r
        assert np.array_equal(ens.per_iter(P.WE_OUT_EVENTS, r), full.per_iter(P.WE_OUT_EVENTS, r)[12:]), r
    if case == "reweighted":
        assert np.array_equal(ens.per_iter(P.WE_OUT_RW), full.per_iter(P.WE_OUT_RW)[12:])


def test_failed_device_allocations_are_reported_and_undone():
    """Host-side fault injection: the k-th device allocation of an MLP (4 of them) or of a
    library-owned ensemble workspace fails; the call returns WE_ENOMEM, frees what it had
    allocated, and the same call succeeds once disarmed."""
    import torch
    L = P._lib.lib()
    p = W.mlp_init_params(2, 64, seed=3)
    cfg = W.schlogl_mfpt_we(n_iters=2, n_runs=1)
    net = P.network_from_spec(cfg.network)
    bm = P.we_binmap_grid(cfg.bins.species, cfg.bins.edges)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    try:
        for k in (1, 2, 3, 4):
            assert L.we_debug_fail_allocation(k) == 0
            with pytest.raises(P.WEError) as ei:
                P.we_mlp_create(2, 64, p)
            assert ei.value.status == -2, ei.value
        assert L.we_debug_fail_allocation(1) == 0
        with pytest.raises(P.WEError) as ei:
            P.we_run(net, bm, P.run_config_from(cfg)[0])
        assert ei.value.status == -2
    finally:
        L.we_debug_fail_allocation(0)
    torch.cuda.synchronize()
    assert abs(torch.cuda.mem_get_info()[0] - free0) < (8 << 20)
    mlp = P.we_mlp_create(2, 64, p)
    assert mlp.params().shape[0] == len(p)
    ens = P.we_run(net, bm, P.run_config_from(cfg)[0])
    ens.sync()


def test_autotuner_choice_and_cache(tmp_path):
    """The autotuner picks a valid (mapping, block) for a one-species, a two-species Hill and
    a large network; the trajectories do not depend on the pick; its cache survives a save,
    clear and load (the second call returns the same pick from the cache)."""
    cases = [W.schlogl_mfpt_we(n_iters=6, n_runs=2), W.toggle_batch_we(n_runs=2, n_iters=6),
             _small_synthetic(n_walkers=24, n_iters=2)]
    P.autotune_cache_clear()
    picks = []
    for cfg in cases:
        net = P.network_from_spec(cfg.network)
        bm = P.we_binmap_grid(cfg.bins.species, cfg.bins.edges)
        c, keep = P.run_config_from(cfg)
        mapping, block = P.we_autotune(net, bm, c)
        assert mapping in (P.WE_MAP_THREAD, P.WE_MAP_WARP, P.WE_MAP_THREAD_TABLE) and block in (32, 64, 96, 128)
        picks.append((mapping, block))
        a = gpu_run(cfg, cfg.n_iters)
        b = gpu_run(cfg, cfg.n_iters, mapping=mapping, block_threads=block)
        for r in range(cfg.n_runs):
            assert np.array_equal(a.states(r), b.states(r))
            assert np.array_equal(a.weights(r).view(np.int64), b.weights(r).view(np.int64))
    path = tmp_path / "tune.txt"
    P.autotune_cache_save(path)
    assert len(path.read_text().splitlines()) == len(cases)
    P.autotune_cache_clear()
    P.autotune_cache_load(path)
    for cfg, pick in zip(cases, picks):
        net = P.network_from_spec(cfg.network)
        bm = P.we_binmap_grid(cfg.bins.species, cfg.bins.edges)
        c, keep = P.run_config_from(cfg)
        assert P.we_autotune(net, bm, c) == pick


def test_repeat_runs_are_identical():
    cfg = W.toggle_batch_we(n_runs=4, n_iters=20)
    a = gpu_run(cfg, 20)
    b = gpu_run(cfg, 20)
    for r in range(4):
        assert np.array_equal(a.states(r), b.states(r))
        assert np.array_equal(a.weights(r).view(np.int64), b.weights(r).view(np.int64))


def test_phase_api_matches_step():
    """propagate()/resample() issued one by one equal the graph-replayed step()."""
    cfg = W.schlogl_mfpt_we(n_iters=6, n_runs=2)
    a = gpu_run(cfg, 6)
    b = gpu_run(cfg, 0, record_iters=6)
    for _ in range(6):
        b.propagate()
        b.resample()
    b.sync()
    for r in range(2):
        assert np.array_equal(a.states(r), b.states(r))
        assert np.array_equal(a.per_iter(P.WE_OUT_NWALKERS, r), b.per_iter(P.WE_OUT_NWALKERS, r))


def test_we_run_one_call_host_outputs():
    cfg = W.birth_death_we(n_iters=20)
    net = P.network_from_spec(cfg.network)
    bm = P.we_binmap_grid(cfg.bins.species, cfg.bins.edges)
    c, keep = P.run_config_from(cfg, record_iters=20)
    ens = P.we_run(net, bm, c, keep)
    assert ens.run_status == 0
    o = oracle_run(cfg, 0, n_iters=20)
    assert_run_parity(gpu_outputs(ens, 0), o, "we_run")


def test_library_owned_workspace():
    cfg = W.birth_death_we(n_iters=5)
    ens = gpu_run(cfg, 5, workspace=None)
    ens.sync()
    assert_run_parity(gpu_outputs(ens, 0), oracle_run(cfg, 0, n_iters=5), "own workspace")


def test_timed_step_matches_step_and_reports_kernel_times():
    cfg = W.schlogl_mfpt_we(n_iters=12, n_runs=2)
    a = gpu_run(cfg, 12)
    b = gpu_run(cfg, 0, record_iters=12)
    ms = b.step_timed(12)
    b.sync()
    assert ms.shape == (12,) and np.all(ms > 0)
    for r in range(2):
        assert np.array_equal(a.states(r), b.states(r))
        assert np.array_equal(a.per_iter(P.WE_OUT_EVENTS, r), b.per_iter(P.WE_OUT_EVENTS, r))


def test_sampled_timed_step_matches_step():
    """Every 5th iteration timed (0, 5, 10), the others from the plain graph, across two calls
    (the second after a capture-only call): the same trajectories as untimed steps."""
    cfg = W.schlogl_mfpt_we(n_iters=24, n_runs=2)
    a = gpu_run(cfg, 24)
    b = gpu_run(cfg, 0, record_iters=24)
    assert b.step_timed(0, every=5).shape == (0,)
    ms1 = b.step_timed(12, every=5)
    ms2 = b.step_timed(12, every=5)
    b.sync()
    assert ms1.shape == (3,) and ms2.shape == (3,) and np.all(ms1 > 0) and np.all(ms2 > 0)
    for r in range(2):
        assert np.array_equal(a.states(r), b.states(r))
        assert np.array_equal(a.weights(r).view(np.int64), b.weights(r).view(np.int64))
        assert np.array_equal(a.per_iter(P.WE_OUT_EVENTS, r), b.per_iter(P.WE_OUT_EVENTS, r))


# ------------------------------------------------------------------ steady-state reweighting --
@pytest.mark.parametrize("period", [1, 2, 5])
def test_reweighting_parity_schlogl(period):
    """Steady-state reweighting (Sec. II.B.2, Eq. "ss") on the Schloegl flux run, three runs in
    one batch: the accumulated transfers, the GTH elimination and the rescaling give the
    oracle's weights bit for bit, and the same iterations are reweighted or skipped."""
    cfg = W.schlogl_flux_we(reweight_period=period, n_iters=24, n_runs=3, m_targ=6)
    ens = _parity(cfg, 24)
    rw = ens.per_iter(P.WE_OUT_RW)
    for r in range(3):
        o = oracle_run(cfg, r, n_iters=24)
        assert np.array_equal(rw[:, r], o["reweighted"]), (period, r, rw[:, r], o["reweighted"])
    assert (rw == 1).sum() >= 3 * (24 // period) // 2


@pytest.mark.parametrize("mapping", [P.WE_MAP_WARP, P.WE_MAP_THREAD])
def test_reweighting_parity_other_mappings(mapping):
    """The transfer accumulation reads the end bins that every SSA kernel writes: the same
    reweighted weights with the warp-per-walker and the general thread kernels."""
    cfg = W.schlogl_flux_we(reweight_period=3, n_iters=15, n_runs=2, m_targ=5)
    ens = _parity(cfg, 15, mapping=mapping)
    assert (ens.per_iter(P.WE_OUT_RW)[[5, 8, 11, 14]] == 1).all()


def test_epigenetic_switch_parity():
    """The epigenetic switch with the paper's non-uniform 2-D bins (15 x 31), Hill exponents 3
    and 1, recycling into the last g1 bin and reweighting every 5 iterations: bit-exact."""
    cfg = W.epigenetic_mfpt_we(n_iters=20, n_runs=2, reweight_period=5)
    ens = _parity(cfg, 20)
    rw = ens.per_iter(P.WE_OUT_RW)
    for r in range(2):
        assert np.array_equal(rw[:, r], oracle_run(cfg, r, n_iters=20)["reweighted"])


def test_reweighting_parity_toggle_2d():
    """Reweighting over a 30 x 30 grid (900 bins) with Hill kinetics and one parameter set per
    run."""
    cfg = W.toggle_batch_we(n_runs=3, n_iters=12)
    cfg.reweight_period = 3
    ens = _parity(cfg, 12)
    rw = ens.per_iter(P.WE_OUT_RW)
    for r in range(3):
        assert np.array_equal(rw[:, r], oracle_run(cfg, r, n_iters=12)["reweighted"])
    assert (rw[[5, 8, 11]] == 1).all()


# ------------------------------------------------------------------ warp per walker ----------
@pytest.mark.parametrize("factory", ["schlogl", "toggle", "futile"])
def test_warp_mapping_small_networks(factory):
    """The warp-per-walker kernel on networks the thread kernels also handle."""
    if factory == "schlogl":
        cfg = W.schlogl_mfpt_we(n_iters=12, n_runs=2)
    elif factory == "toggle":
        cfg = W.toggle_batch_we(n_runs=4, n_iters=12)
    else:
        cfg = W.WEConfig(network=W.futile_cycle(), bins=W.GridBins([0], [W.uniform_edges(0, 1, 101)]),
                         tau=1.0, m_targ=6, n_iters=8, x0=[50, 50, 1, 1, 0, 0], hist_species=0,
                         hist_len=102, name="futile")
    _parity(cfg, cfg.n_iters, mapping=P.WE_MAP_WARP)


def _small_synthetic(n_walkers=24, m_targ=2, tau=2e-5, n_iters=3):
    cfg = W.synthetic_large_we(n_walkers=n_walkers, n_iters=n_iters, m_targ=m_targ)
    cfg.tau = tau
    cfg.capacity = max(n_walkers, m_targ * cfg.bins.n_bins)
    return cfg


def test_warp_mapping_synthetic_354x3680():
    """FceRI-sized random network (354 species, 3680 reactions): dependency-graph updates of the
    shared-memory tree against the oracle's full recomputation, through resampling."""
    cfg = _small_synthetic()
    ens = _parity(cfg, cfg.n_iters, mapping=P.WE_MAP_WARP)
    ev = ens.per_iter(P.WE_OUT_EVENTS, 0)
    assert ev.min() > 1000                      # hundreds of events per walker per interval


def _hub_network(n_x=40):
    """A hub species H read by 102 reactions (H -> H + X_k for 100 rate constants, H -> 0 and
    H -> X_0 + ... + X_39), so the reactions that change H have more dependents than an event
    record holds (96), and H -> X_0 + ... + X_39 has 41 net changes (a record holds 32)."""
    H = n_x
    reactants, products, rate = [], [], []
    for k in range(100):
        reactants.append([(H, 1)]); products.append([(H, 1), (k % n_x, 1)]); rate.append(0.05 + 0.001 * k)
    for k in range(n_x):
        reactants.append([(k, 1)]); products.append([]); rate.append(1.0)
    reactants.append([]); products.append([(H, 1)]); rate.append(5.0)
    reactants.append([(H, 1)]); products.append([]); rate.append(1.0)
    reactants.append([(H, 1)]); products.append([(k, 1) for k in range(n_x)]); rate.append(0.2)
    return W.NetworkSpec(species=[f"X{k}" for k in range(n_x)] + ["H"], reactants=reactants,
                         products=products, rate=[rate], name="hub")


def test_warp_mapping_past_the_event_record():
    """Dependents and net changes beyond what the warp kernel's per-reaction record holds are
    read from the CSR arrays; trajectories stay bit-exact."""
    net = _hub_network()
    x0 = [0] * 40 + [5]
    cfg = W.WEConfig(network=net, bins=W.GridBins([40], [W.uniform_edges(0, 1, 21)]), tau=2.0,
                     m_targ=4, n_iters=6, x0=x0, hist_species=40, hist_len=22, name="hub")
    ens = _parity(cfg, cfg.n_iters, mapping=P.WE_MAP_WARP)
    assert ens.per_iter(P.WE_OUT_EVENTS, 0).min() > 100


def test_warp_mapping_synthetic_plain_ssa_times():
    cfg = _small_synthetic(n_walkers=40, n_iters=2)
    ens = gpu_run(cfg, 2, resample=False, mapping=P.WE_MAP_WARP)
    ens.sync()
    o = oracle_run(cfg, 0, n_iters=2, resample=False)
    assert_run_parity(gpu_outputs(ens, 0), o, "synthetic plain")
    tl = ens.get(P.WE_OUT_TLAST, 0)
    np.testing.assert_allclose(tl, o["t_last"][:40], rtol=1e-12, atol=0)
