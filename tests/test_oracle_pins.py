"""Pins of the CPU oracle to things other than itself (closed forms, a library generator, the
paper's printed numbers, brute force, invariants).  CPU only."""
import ctypes
import math
import os

import numpy as np
import pytest
from scipy import stats

import workloads as W
from oracle import exact as E
from oracle import oracle as O


# ---------------------------------------------------------------- Philox-4x32-10 ---------------
def _curand():
    for p in ["/usr/local/cuda/lib64/libcurand.so", "libcurand.so", "libcurand.so.10"]:
        try:
            return ctypes.CDLL(p)
        except OSError:
            continue
    return None


@pytest.mark.parametrize("seed", [0, 1, 0x123456789ABCDEF0, 2**64 - 1])
def test_philox_matches_curand_host_generator(seed):
    """CURAND's host Philox4_32_10 generator (run, not read) emits block k of its stream as
    Philox(counter=(0,0,k,0), key=(seed_lo, seed_hi)); the oracle must reproduce it."""
    cur = _curand()
    if cur is None:
        pytest.skip("libcurand not available")
    gen = ctypes.c_void_p()
    if cur.curandCreateGeneratorHost(ctypes.byref(gen), 161) != 0:   # CURAND_RNG_PSEUDO_PHILOX4_32_10
        pytest.skip("curand host generator unavailable")
    try:
        assert cur.curandSetPseudoRandomGeneratorSeed(gen, ctypes.c_ulonglong(seed)) == 0
        n = 4 * 2048
        buf = (ctypes.c_uint32 * n)()
        assert cur.curandGenerate(gen, buf, ctypes.c_size_t(n)) == 0
        ref = np.frombuffer(buf, dtype=np.uint32).reshape(-1, 4)
        key = (seed & 0xFFFFFFFF, seed >> 32)
        for k in list(range(0, 64)) + list(range(1900, 2048)):
            assert np.array_equal(O.philox((0, 0, k, 0), key), ref[k]), k
    finally:
        cur.curandDestroyGenerator(gen)


def test_philox_uniformity_and_counter_sensitivity():
    """Every counter word and key word changes the output; words are uniform (chi-square)."""
    base = O.philox((1, 2, 3, 4), (5, 6))
    for i in range(4):
        c = [1, 2, 3, 4]
        c[i] ^= 1
        assert not np.array_equal(O.philox(c, (5, 6)), base)
    for i in range(2):
        k = [5, 6]
        k[i] ^= 1
        assert not np.array_equal(O.philox((1, 2, 3, 4), k), base)
    words = np.concatenate([O.philox((s, 7, 0, 1), (11, 13)) for s in range(4000)])
    counts = np.bincount((words >> 28).astype(np.int64), minlength=16)
    assert stats.chisquare(counts).pvalue > 1e-4


def test_u01_exact_values():
    assert O.u01(0, 0) == 2.0 ** -53
    assert O.u01(0xFFFFFFFF, 0xFFFFFFFF) == 1.0 - 2.0 ** -53
    assert O.u01(0, 1 << 12) == 3.0 * 2.0 ** -53
    assert O.u01(1, 0) == (2.0 ** 21 + 1) * 2.0 ** -53
    assert O.u01(0x80000000, 0) == 0.5 + 2.0 ** -53
    # low 12 bits of the second word are dropped
    assert O.u01(123, 0xFFF) == O.u01(123, 0)


# ---------------------------------------------------------------- propensities -----------------
def test_schlogl_modes_pin_combinatorial_convention():
    """With combinatorial mass action, the stationary law of the oracle's own Schloegl
    propensities peaks at X=82 and X=563 with the barrier at X=256 (Sec. III.B.3)."""
    net = O.Network(W.schlogl())
    N = 1500
    a = np.array([net.propensities([x, 100000, 200000]) for x in range(N + 1)])
    birth = a[:, 0] + a[:, 2]
    death = a[:, 1] + a[:, 3]
    lp = np.concatenate([[0.0], np.cumsum(np.log(birth[:-1]) - np.log(death[1:]))])
    maxima = [x for x in range(1, N) if lp[x] >= lp[x - 1] and lp[x] >= lp[x + 1]]
    minima = [x for x in range(1, N) if lp[x] <= lp[x - 1] and lp[x] <= lp[x + 1]]
    assert maxima == [82, 563]
    assert minima == [256]


def test_propensity_hand_values():
    net = O.Network(W.schlogl())
    # folded constants: c1*A and c3*B
    assert net.keff(0) == 3e-7 * 100000.0 and net.keff(2) == 1e-3 * 200000.0
    a = net.propensities([5, 100000, 200000])
    # C(5,2)=10, C(5,3)=10
    assert a[0] == net.keff(0) * 10.0 and a[1] == 1e-4 * 10.0 and a[2] == 200.0 and a[3] == 3.5 * 5.0
    for x in (0, 1, 2):
        a = net.propensities([x, 100000, 200000])
        assert a[1] == 0.0 and (x >= 2 or a[0] == 0.0)
    fut = O.Network(W.futile_cycle())
    a = fut.propensities([50, 50, 1, 1, 0, 0])
    assert list(a) == [50.0, 0.0, 0.0, 50.0, 0.0, 0.0]
    tog = O.Network(W.toggle_switch(40.0, 30.0))
    a = tog.propensities([7, 3])
    assert a[0] == 40.0 / 10.0 and a[1] == 30.0 / 50.0 and a[2] == 7.0 and a[3] == 3.0
    epi = O.Network(W.epigenetic_switch())
    a = epi.propensities([4, 2])
    assert a[0] == 156.0 / 9.0 and a[2] == 30.0 / 5.0


def test_network_validation():
    bad = W.NetworkSpec(species=["X"], reactants=[[(0, 4)]], products=[[]], rate=[[1.0]])
    with pytest.raises(ValueError):
        O.Network(bad)
    bad = W.NetworkSpec(species=["X"], reactants=[[(1, 1)]], products=[[]], rate=[[1.0]])
    with pytest.raises(ValueError):
        O.Network(bad)
    bad = W.NetworkSpec(species=["X"], reactants=[[]], products=[[(0, 1)]], rate=[[-1.0]])
    with pytest.raises(ValueError):
        O.Network(bad)


# ---------------------------------------------------------------- canonical tree ---------------
def test_tree_total_is_a_correct_sum():
    rng = np.random.default_rng(1)
    for n in [1, 2, 3, 4, 5, 7, 8, 9, 100, 3680]:
        a = rng.exponential(size=n) * (rng.random(n) < 0.8)
        t = O.tree_total(a)
        exact = math.fsum(a)
        depth = max(1, math.ceil(math.log2(n)))
        assert abs(t - exact) <= depth * 2.0 ** -52 * exact + 1e-300
    assert O.tree_total([3.0]) == 3.0
    assert O.tree_total([0.0, 0.0, 0.0]) == 0.0
    # pairwise shape: ((a+b)+(c+d)) differs from the left fold for these values
    v = [1.0, 0.0, 2.0 ** -53, 2.0 ** -53]
    assert O.tree_total(v) == 1.0 + 2.0 ** -52       # a left-to-right fold would give 1.0


def test_tree_select_boundaries_and_zeros():
    a = [1.0, 2.0, 3.0, 4.0]
    cases = {0.0: 0, 0.999: 0, 1.0: 1, 2.999: 1, 3.0: 2, 5.999: 2, 6.0: 3, 9.999: 3}
    for tgt, j in cases.items():
        assert O.tree_select(a, tgt) == j
    z = [0.0, 1.0, 0.0, 0.0, 2.0, 0.0, 0.0]
    for tgt in np.linspace(0.0, 3.0, 61):
        assert z[O.tree_select(z, tgt)] > 0.0
    assert O.tree_select(z, 1e300) == 4      # a target rounded past the total stays on a live leaf


def test_tree_select_frequencies():
    rng = np.random.default_rng(2)
    a = np.array([0.5, 0.0, 3.0, 1.5, 0.0, 2.0])
    tot = O.tree_total(a)
    n = 30000
    picks = np.bincount([O.tree_select(a, u * tot) for u in rng.random(n)], minlength=len(a))
    assert picks[1] == 0 and picks[4] == 0
    expected = a / a.sum() * n
    live = a > 0
    assert stats.chisquare(picks[live], expected[live]).pvalue > 1e-4


# ---------------------------------------------------------------- SSA dynamics -----------------
def _brute_force(cfg, n_walkers, n_iters, seed=5):
    S = cfg.network.n_species
    init = np.repeat(cfg.x0[:1], n_walkers, axis=0)
    cfg.seed = seed
    return O.we_run(cfg, 0, n_iters=n_iters, resample=False, init_states=init,
                    init_weights=np.full(n_walkers, 1.0 / n_walkers))


def test_ssa_immigration_death_matches_closed_form():
    """Brute-force SSA (no resampling) of 0->X, X->0 against Binomial * Poisson at t=2."""
    cfg = W.birth_death_we()
    out = _brute_force(cfg, 20000, 20)
    x = out["states"][:, 0]
    p = E.immigration_death_pmf(100, 10.0, 0.1, 2.0, 400)
    obs = np.bincount(x, minlength=401)[:401]
    exp = p * len(x)
    keep = exp > 20
    chi = ((obs[keep] - exp[keep]) ** 2 / exp[keep]).sum()
    dof = keep.sum() - 1
    assert stats.chi2.sf(chi, dof) > 1e-4
    assert abs(x.mean() - (p * np.arange(401)).sum()) < 5 * x.std() / np.sqrt(len(x))


def test_ssa_schlogl_matches_cme():
    """Brute-force SSA of the Schloegl model from X=82 against the truncated CME at t=0.5."""
    cfg = W.schlogl_mfpt_we()
    cfg.target = None
    cfg.x0[:, 0] = 82
    cfg.recycle_state[:, 0] = 82
    out = _brute_force(cfg, 8000, 10)
    x = out["states"][:, 0]
    b, d = E.schlogl_rates()
    p = E.bd_transient(b, d, 82, 0.5, 1500)
    obs = np.bincount(x, minlength=1501)[:1501]
    exp = p * len(x)
    # pool into blocks of 4 states for power
    ob = obs[:1500].reshape(-1, 4).sum(1)
    ex = exp[:1500].reshape(-1, 4).sum(1)
    keep = ex > 20
    chi = ((ob[keep] - ex[keep]) ** 2 / ex[keep]).sum()
    assert stats.chi2.sf(chi, keep.sum() - 1) > 1e-4


def test_recycling_rate_is_inverse_mfpt():
    """With recycling and no resampling, each walker is a renewal process whose rate of hits is
    1/MFPT(A -> B) (Eq. "mfpt"); MFPT(100 -> 115) of the birth-death chain is a closed form."""
    cfg = W.birth_death_we(target=115)
    n_w, n_it = 2000, 1500
    out = _brute_force(cfg, n_w, n_it, seed=9)
    hits = out["flux_weight"] * n_w            # every walker carries weight 1/n_w
    bb, dd = E.birth_death_rates()
    mfpt = E.bd_mfpt(100, 115, bb, dd)
    rate = hits[200:].sum() / (n_w * (n_it - 200) * cfg.tau)
    se = np.sqrt(hits[200:].sum()) / (n_w * (n_it - 200) * cfg.tau)
    assert abs(rate - 1.0 / mfpt) < 3 * se, (rate, 1.0 / mfpt, se)


def test_step_cap_and_overflow_statuses():
    cfg = W.birth_death_we()
    x, ev, rec, rc = O.propagate_one(cfg, [100], 0, 0, max_steps=1)
    assert rc == -5 and ev == 1
    grow = W.NetworkSpec(species=["X"], reactants=[[]], products=[[(0, 1)]], rate=[[1e9]])
    cfg2 = W.WEConfig(network=grow, bins=W.GridBins([0], [W.uniform_edges(0, 1, 1)]), tau=1.0,
                      m_targ=1, n_iters=1, x0=[O.MAX_COUNT - 2])
    x, ev, rec, rc = O.propagate_one(cfg2, [O.MAX_COUNT - 2], 0, 0)
    assert rc == -4 and x[0] == O.MAX_COUNT and ev == 2


def test_zero_propensity_walker_idles():
    dead = W.NetworkSpec(species=["X"], reactants=[[(0, 1)]], products=[[]], rate=[[1.0]])
    cfg = W.WEConfig(network=dead, bins=W.GridBins([0], [W.uniform_edges(0, 1, 1)]), tau=1.0,
                     m_targ=1, n_iters=1, x0=[0])
    x, ev, rec, rc = O.propagate_one(cfg, [0], 0, 0)
    assert rc == 0 and ev == 0 and x[0] == 0


# ---------------------------------------------------------------- split / merge -----------------
def test_resample_invariants_random():
    rng = np.random.default_rng(3)
    for trial in range(40):
        n = int(rng.integers(1, 300))
        nb = int(rng.integers(1, 12))
        M = int(rng.integers(1, 15))
        st = rng.integers(0, 1000, size=(n, 2)).astype(np.int32)
        w = rng.exponential(size=n) * 10.0 ** rng.uniform(-40, 0, size=n)
        b = rng.integers(0, nb, size=n).astype(np.int32)
        s2, w2, p2 = O.resample(st, w, b, nb, M, trial, 77)
        occ = np.unique(b)
        assert len(w2) == M * len(occ)
        assert abs(w2.sum() - math.fsum(w)) <= 1e-14 * math.fsum(w)
        for bin_ in occ:
            assert abs(math.fsum(w2[b[p2] == bin_]) - math.fsum(w[b == bin_])) <= 1e-14 * math.fsum(w[b == bin_])
        assert np.array_equal(s2, st[p2])
        assert np.all(np.diff(b[p2]) >= 0)          # concatenation over ascending bins


def test_lone_walker_split_gives_paper_weights():
    s2, w2, p2 = O.resample([[5]], [0.3], [0], 1, 10, 0, 1)
    assert len(w2) == 10 and np.all(w2 == 0.3 / 10) and np.all(p2 == 0)


def test_split_allocation_greedy():
    # weights 0.6, 0.2 with M=4: copies go to the largest per-copy weight: 0.6 -> 0.3 -> 0.2 tie
    s2, w2, p2 = O.resample([[1], [2]], [0.6, 0.2], [0, 0], 1, 4, 0, 1)
    assert list(p2) == [0, 0, 0, 1] and list(w2) == [0.6 / 3, 0.6 / 3, 0.6 / 3, 0.2]


def test_merge_survivor_probability_and_unbiasedness():
    """Merging keeps the expected weight of every walker (Sec. II.B; Huber & Kim): over many
    draws the earlier of the two lightest walkers survives with probability w_p/(w_p+w_q)."""
    w = np.array([0.1, 0.3, 0.2, 0.4])
    b = np.zeros(4, dtype=np.int32)
    st = np.arange(4, dtype=np.int32)[:, None]
    n = 20000
    acc = np.zeros(4)
    first_merge_p = 0
    for it in range(n):
        s2, w2, p2 = O.resample(st, w, b, 1, 3, it, 1234)
        for slot, ww in zip(p2, w2):
            acc[slot] += ww
        first_merge_p += int(0 in p2)
    mean = acc / n
    # walker 0 (0.1) merges with walker 2 (0.2): survives with prob 1/3
    p = 1.0 / 3.0
    assert abs(first_merge_p / n - p) < 4 * np.sqrt(p * (1 - p) / n)
    sd = np.array([0.3 * np.sqrt(p * (1 - p)), 0, 0.3 * np.sqrt(p * (1 - p)), 0]) / np.sqrt(n)
    assert np.all(np.abs(mean - w) <= 4 * sd + 1e-12)


def test_merge_ties_take_earliest():
    w = np.array([0.25, 0.25, 0.25, 0.25])
    s2, w2, p2 = O.resample(np.arange(4)[:, None], w, np.zeros(4, dtype=np.int32), 1, 3, 0, 5)
    # the pair is (slot 0, slot 1); exactly one of them survives with weight 0.5
    assert sorted(w2.tolist()) == [0.25, 0.25, 0.5]
    assert set(p2.tolist()) in ({0, 2, 3}, {1, 2, 3})


# ---------------------------------------------------------------- epigenetic switch -----------
def test_epigenetic_switch_mfpt_matches_paper():
    """The exact MFPT of the epigenetic switch (Sec. III.C) from the g2-high state (0, 30) into
    the last g1 bin (g1 >= 50), by a sparse solve of the truncated master equation, is the
    1.3e6 s the paper prints (its WE and brute-force estimates); the truncation is converged,
    and the opposite transition is four orders of magnitude faster."""
    T = E.epigenetic_mfpt((0, 30), lambda u, v: u >= 50)
    assert round(T, -5) == 1.3e6
    assert abs(E.epigenetic_mfpt((0, 30), lambda u, v: u >= 50, G1=300, G2=90) - T) < 1e-6 * T
    assert E.epigenetic_mfpt((156, 0), lambda u, v: v >= 30) < 1e4


# ---------------------------------------------- brute-force transition-time estimator ----------
def test_mle_transition_time_maximises_the_censored_likelihood():
    """Eq. "mld" is the maximum-likelihood mean of exponential waiting times, the runs without a
    transition censored at T: the estimate sits where a bounded numerical search finds the
    likelihood's maximum (densities of the observed times, survival T of the other runs); with
    every run transitioning it is the sample mean; sigma is mu / sqrt(n)."""
    from scipy.optimize import minimize_scalar
    rng = np.random.default_rng(5)
    T, N = 1.0, 500
    t = rng.exponential(1.3, N)
    seen = t[t <= T]
    n = len(seen)

    def minus_log_likelihood(mu):
        return sum(math.log(mu) + ti / mu for ti in seen) + (N - n) * T / mu

    best = minimize_scalar(minus_log_likelihood, bounds=(0.01, 100.0), method="bounded",
                           options={"xatol": 1e-10})
    mu, sig = E.mle_transition_time(T, N, seen)
    assert mu == pytest.approx(best.x, rel=1e-6)
    assert sig == pytest.approx(mu / math.sqrt(n), rel=1e-14)
    every = rng.exponential(2.0, 50)
    assert E.mle_transition_time(every.max(), 50, every)[0] == pytest.approx(every.mean(), rel=1e-14)
    with pytest.raises(ValueError):
        E.mle_transition_time(1.0, 10, [])


def test_mle_transition_time_is_consistent_and_gives_the_paper_figures():
    """Censored exponential samples of mean 1.3 (200,000 runs of length 1) give 1.3 back within 4
    standard errors.  The expected data of the paper's brute-force campaign (Sec. III.C: 753 runs
    of 1e6 s of a switch whose mean transition time is 1.3e6 s, so 404 transitions at a mean
    observed time of 4.37e5 s) give the 1.3e6 s and 6.5e4 s it prints; the factor (1 - n/N) of
    the printed equation would give 9.0e5 s."""
    rng = np.random.default_rng(11)
    t = rng.exponential(1.3, 200_000)
    seen = t[t <= 1.0]
    mu, sig = E.mle_transition_time(1.0, len(t), seen)
    assert abs(mu - 1.3) < 4 * sig
    m, T, N = 1.3e6, 1e6, 753
    p = -math.expm1(-T / m)                          # P(transition within one run)
    n = round(N * p)
    mean_seen = m - T * math.exp(-T / m) / p         # mean of an exponential conditioned on t <= T
    mu, sig = E.mle_transition_time(T, N, np.full(n, mean_seen))
    assert n == 404
    assert round(mu, -5) == 1.3e6
    assert round(sig, -3) == 6.5e4


# ----------------------------- the dependency-graph CPU baseline equals the oracle --------------
@pytest.mark.parametrize("case", ["schlogl", "toggle", "futile", "absorbing"])
def test_dependency_graph_cpu_baseline_equals_oracle(case):
    """The CPU baseline with a dependency graph (incremental tree updates) gives the oracle's
    runs bit for bit: it only skips recomputing propensities that cannot have changed."""
    if case == "schlogl":
        cfg = W.schlogl_mfpt_we(n_iters=30)
    elif case == "toggle":
        cfg = W.toggle_batch_we(n_runs=2, n_iters=20)
    elif case == "futile":
        cfg = W.futile_pdf_we(n_iters=8, m_targ=10)
    else:
        cfg = W.birth_death_bruteforce(n_walkers=64, tau=1.0, n_iters=30, threshold=112)
    resample = case != "absorbing"
    for r in range(cfg.n_runs):
        a = O.we_run(cfg, r, resample=resample)
        b = O.we_run(cfg, r, resample=resample, depgraph=True)
        for k in ("states", "weights", "parent", "events", "flux_weight", "hist", "first_passage", "n_walkers"):
            assert np.array_equal(a[k], b[k]), (case, r, k)


def test_dependency_graph_cpu_baseline_on_the_large_network():
    """The 354 x 3680 network: one interval of eight walkers, propagated by the oracle (all 3680
    propensities and the whole tree after every event) and by the dependency-graph baseline."""
    cfg = W.synthetic_large_we(n_walkers=8, n_iters=1)
    cfg.tau = 1e-4
    net = O.Network(cfg.network)
    for i in range(8):
        a = O.propagate_one(cfg, cfg.init_states[0, i], 0, i, net=net)
        b = O.propagate_one(cfg, cfg.init_states[0, i], 0, i, net=net, depgraph=True)
        assert np.array_equal(a[0], b[0]) and a[1:] == b[1:] and a[1] > 100


# --------------------------------------- brute-force runs with an absorbing target --------------
def test_absorbing_runs_give_erlang_first_passage_times():
    """Pure birth at rate 2 (the birth-death network with kd = 0) from 100, absorbed at X >= 130:
    the first-passage time is the sum of 30 exponential waits, Erlang(30, 2) (mean 15, variance
    7.5).  Intervals of 0.25 put each passage ~60 intervals in, so a time recorded without its
    interval's start fl(i tau), or one interval off, or the time of the event before the
    entrance, fails; so does a walker that keeps firing after its entrance."""
    net = W.networks.NetworkSpec(species=["X"], reactants=[[], [(0, 1)]], products=[[(0, 1)], []],
                                 rate=[[2.0, 0.0]], name="pure_birth")
    tgt = W.Target(species=[0], op=[W.configs.OP_GE], threshold=np.full((1, 1), 130, dtype=np.int32))
    cfg = W.bruteforce_fpt(net, [100], tgt, n_walkers=1500, tau=0.25, n_iters=160)
    o = O.we_run(cfg, 0, resample=False)
    fp = o["first_passage"]
    assert o["status"] == 0 and np.all(fp > 0) and np.all(o["states"][:, 0] == 130)
    assert np.all(fp <= 160 * 0.25)
    assert int(o["events"].sum()) == 30 * 1500                       # nothing fires after absorption
    se = fp.std(ddof=1) / np.sqrt(len(fp))
    assert abs(fp.mean() - 15.0) < 3 * se, (fp.mean(), se)
    assert stats.kstest(fp, stats.gamma(30, scale=0.5).cdf).pvalue > 0.01
    n = len(fp)                                   # sd of s^2 / sigma^2: 2/(n-1) + excess kurtosis 6/30 over n
    assert abs(fp.var(ddof=1) / 7.5 - 1.0) < 3 * np.sqrt(2.0 / (n - 1) + 0.2 / n)


def test_absorbing_runs_mean_first_passage_matches_closed_form():
    """Birth-death (kb = 10, kd = 0.1) from 100, absorbed at X >= 110, runs of 400 s in intervals
    of 1 s (every run passes): the mean first-passage time equals the closed form
    sum_k (sum_{j<=k} pi_j) / (lambda_k pi_k) = 20.91 within 3 standard errors, and the
    censored-exponential MLE of Eq. "mld" with no censored run is the sample mean."""
    b, d = E.birth_death_rates()
    exact = E.bd_mfpt(100, 110, b, d)
    cfg = W.birth_death_bruteforce(n_walkers=1200, tau=1.0, n_iters=400, threshold=110)
    o = O.we_run(cfg, 0, resample=False)
    fp = o["first_passage"]
    assert o["status"] == 0 and np.all(fp > 0)
    se = fp.std(ddof=1) / np.sqrt(len(fp))
    assert abs(fp.mean() - exact) < 3 * se, (fp.mean(), exact, se)
    mu, sig = E.mle_transition_time(400.0, len(fp), fp)
    assert mu == pytest.approx(fp.mean(), rel=1e-12)


def test_absorbing_walker_starting_inside_fires_nothing():
    """A walker that starts inside the absorbing set fires no event and its first passage is the
    start of the run; walkers outside are unaffected by it (their draws are keyed by slot)."""
    cfg = W.birth_death_bruteforce(n_walkers=4, tau=1.0, n_iters=30, threshold=105)
    cfg.init_states[0, 1, 0] = 107
    o = O.we_run(cfg, 0, resample=False)
    assert o["first_passage"][1] == 0.0 and o["states"][1, 0] == 107
    cfg2 = W.birth_death_bruteforce(n_walkers=4, tau=1.0, n_iters=30, threshold=105)
    o2 = O.we_run(cfg2, 0, resample=False)
    keep = [0, 2, 3]
    assert np.array_equal(o["first_passage"][keep], o2["first_passage"][keep])
    assert np.array_equal(o["states"][keep], o2["states"][keep])


# ---------------------------------------------------------------- futile-cycle CME -------------
def test_futile_cme_matches_paper_and_invariants():
    """The futile cycle's exact law (uniformized CME over its 400 states): P(S1 > 90, t = 100)
    from S1 = S2 = 50 equals the 2.72e-18 printed in Sec. III.A; S1 and S2 have the same law
    (the two half-cycles have the same rates), the law sums to 1, and it agrees with a dense
    matrix exponential where that is accurate (the bulk)."""
    law = E.futile_s1_law(100.0)
    assert round(law[91:].sum(), 20) == pytest.approx(2.72e-18, abs=0.005e-18)
    assert abs(law.sum() - 1.0) < 1e-10
    from scipy.linalg import expm
    st, idx, tr = E.futile_generator()
    n = len(st)
    assert n == 400
    p0 = np.zeros(n)
    p0[idx[(0, 0, 50)]] = 1.0
    pt = E.uniformized_transient(n, tr, p0, 100.0)
    s1_law, s2_law = np.zeros(101), np.zeros(101)
    for k, (b1, b2, s1) in enumerate(st):
        s1_law[s1] += pt[k]
        s2_law[100 - s1 - b1 - b2] += pt[k]
    np.testing.assert_allclose(s1_law, law, rtol=1e-12)
    np.testing.assert_allclose(s1_law, s2_law, rtol=1e-9, atol=0)     # S1 <-> S2 symmetry
    Q = np.zeros((n, n))
    for a_, b_, r in tr:
        Q[a_, b_] += r
        Q[a_, a_] -= r
    p = p0 @ expm(Q * 20.0)
    dense = np.zeros(101)
    for k, (b1, b2, s1) in enumerate(st):
        dense[s1] += p[k]
    short = E.futile_s1_law(20.0)
    bulk = dense > 1e-6
    np.testing.assert_allclose(short[bulk], dense[bulk], rtol=1e-9)


def test_futile_cme_generator_against_the_oracle_network():
    """Every CME transition out of a state equals the oracle's propensity of the reaction that
    makes it (S1, S2, E1, E2, B1, B2 order), and the CME's total exit rate equals a0."""
    net = O.Network(W.futile_cycle())
    st, idx, tr = E.futile_generator()
    out = {}
    for a_, b_, r in tr:
        out[a_] = out.get(a_, 0.0) + r
    for k, (b1, b2, s1) in enumerate(st[::37]):
        kk = idx[(b1, b2, s1)]
        s2 = 100 - s1 - b1 - b2
        a = net.propensities([s1, s2, 1 - b1, 1 - b2, b1, b2])
        assert math.isclose(sum(a), out.get(kk, 0.0), rel_tol=1e-15)


# ---------------------------------------------------------------- whole WE runs ------------------
def _replicas(cfg, R, **kw):
    outs = []
    for r in range(R):
        cfg.run_ids = np.array([r], dtype=np.uint32)
        outs.append(O.we_run(cfg, 0, **kw))
    return outs


def test_we_schlogl_tail_matches_cme():
    """WE estimate of P(X >= x, t = 1) for the Schloegl model from X=82 (unit-width bins as in
    Sec. III.B.2, 10 walkers per bin) against the truncated CME, within 3 standard errors over
    48 independent replicas (the protocol of Sec. III.B.3).  Transient WE tail estimates are
    unbiased but right-skewed; the checks stay where the replicas' log-spread is below 1.5, so
    that their standard error is a fair measure."""
    cfg = W.schlogl_pdf_we(n_iters=20, m_targ=10, n_unit_bins=400)
    outs = _replicas(cfg, 48)
    b, d = E.schlogl_rates()
    p = E.bd_transient(b, d, 82, 1.0, 1500)
    for thr in (120, 150):
        est = np.array([o["hist"][-1, thr:].sum() for o in outs])
        exact = p[thr:].sum()
        se = est.std(ddof=1) / np.sqrt(len(est))
        assert np.log(est).std(ddof=1) < 1.5, thr
        assert abs(est.mean() - exact) < 3 * se, (thr, est.mean(), exact, se)
    for o in outs:
        assert np.all(np.abs(o["total_weight"] - 1.0) < 1e-12)


def test_we_birth_death_stationary_tails_match_poisson():
    """Stationary WE of the birth-death process (kb=10, kd=0.1; 61 bins, 10 walkers per bin):
    the time-averaged weighted histogram reproduces the Poisson(100) law in both tails
    (P(X >= 150) ~ 1.9e-6, P(X <= 50) ~ 2.4e-8), within 3 standard errors over 32 replicas."""
    cfg = W.birth_death_we(n_iters=1500)
    outs = _replicas(cfg, 32)
    x = np.arange(401)
    pois = np.exp(E.log_poisson_pmf(x, 100.0))
    H = np.array([o["hist"][375:].mean(0) for o in outs])
    for sel in (slice(150, None), slice(None, 51)):
        est = H[:, sel].sum(1)
        exact = pois[sel].sum()
        se = est.std(ddof=1) / np.sqrt(len(est))
        assert abs(est.mean() - exact) < 3 * se, (sel, est.mean(), exact, se)


def test_we_mfpt_matches_closed_form():
    """Steady-state WE with recycling: MFPT = 1/flux (Eq. "mfpt") for the rare passage
    100 -> 140 of the birth-death chain (closed form ~9.8e3), 3 standard errors over 32
    replicas."""
    cfg = W.birth_death_we(n_iters=400, target=140)
    outs = _replicas(cfg, 32)
    bb, dd = E.birth_death_rates()
    exact = 1.0 / E.bd_mfpt(100, 140, bb, dd)
    est = np.array([1.0 / O.mfpt_from_flux(o["flux_weight"], cfg.tau, discard=150) for o in outs])
    se = est.std(ddof=1) / np.sqrt(len(est))
    assert abs(est.mean() - exact) < 3 * se, (est.mean(), exact, se)
    for o in outs:
        assert np.all(np.abs(o["total_weight"] - 1.0) < 1e-12)


def test_toggle_recycling_rate_matches_master_equation():
    """Hill-repression dynamics (Sec. III.C.1 form, n=2): the renewal rate of first passages of
    a toggle switch with a_U = a_V = 8 into {V >= 4, U <= 2} equals 1/MFPT from an exact sparse
    solve of the 2-D master equation (~39.6)."""
    a = 8.0
    net = W.toggle_switch([a], [a])
    tgt = W.Target(species=[1, 0], op=[W.configs.OP_GE, W.configs.OP_LE],
                   threshold=np.array([[4, 2]], dtype=np.int32))
    e = W.uniform_edges(0, 4, 29, overflow=True)
    cfg = W.WEConfig(network=net, bins=W.GridBins([0, 1], [e, e]), tau=0.1, m_targ=8,
                     n_iters=1, x0=[8, 0], target=tgt)
    n_w, n_it = 2000, 1200
    out = _brute_force(cfg, n_w, n_it, seed=21)
    hits = out["flux_weight"] * n_w
    mfpt = E.toggle_mfpt(a, a, (8, 0), lambda u, v: v >= 4 and u <= 2, Umax=60, Vmax=60)
    span = n_w * (n_it - 300) * cfg.tau
    rate = hits[300:].sum() / span
    se = np.sqrt(hits[300:].sum()) / span
    assert abs(rate - 1.0 / mfpt) < 3 * se, (rate, 1.0 / mfpt, se)


def test_synthetic_network_homodimer_and_conservation():
    spec = W.synthetic_large()
    assert spec.n_species == 354 and spec.n_reactions == 3680
    net = O.Network(spec)
    x = np.arange(354, dtype=np.int32) % 200
    a = net.propensities(x)
    seen_dimer = seen_bi = False
    for j, (reac, prod) in enumerate(zip(spec.reactants, spec.products)):
        assert sum(m for _, m in reac) == sum(m for _, m in prod)     # molecules conserved
        if len(reac) == 1 and reac[0][1] == 2:
            v = int(x[reac[0][0]])
            assert a[j] == spec.rate[0, j] * float(v * (v - 1) // 2)
            seen_dimer = True
        if len(reac) == 2:
            assert a[j] == spec.rate[0, j] * float(int(x[reac[0][0]]) * int(x[reac[1][0]]))
            seen_bi = True
    assert seen_dimer and seen_bi


# ---------------------------------------------------------------- steady-state reweighting -----
def _transfers(K, W):
    """F[e, b] = P_eb W_b: the transfers over one interval of a chain whose moves b -> e (e != b)
    have probabilities K[e, b]; the rest of the weight stays (P_bb = 1 - sum_e K[e, b]), so that
    W_b = sum_e F[e, b] as in a WE run."""
    P = K.copy()
    np.fill_diagonal(P, 0.0)
    np.fill_diagonal(P, 1.0 - P.sum(axis=0))
    assert (P >= 0).all()
    return P * W[None, :]


def test_rw_solve_birth_death_chain_detailed_balance():
    """Tridiagonal moves: the steady state is fixed by detailed balance,
    pi_{i+1} / pi_i = up_i / down_{i+1}, with no linear solve.  The factors must give every bin
    that holds walkers the weight pi_i scaled to the bins' current total -- to 1e-10 relative
    even where pi is 1e-60 of its largest entry (the solve keeps relative accuracy)."""
    rng = np.random.default_rng(3)
    n = 40
    up = rng.uniform(0.02, 0.4, n)
    down = rng.uniform(0.02, 0.4, n)
    up[:20] *= 1e-3                                               # a steep left tail
    K = np.zeros((n, n))
    for i in range(n - 1):
        K[i + 1, i] = up[i]
        K[i, i + 1] = down[i + 1]
    W = rng.uniform(0.5, 3.0, n)
    pi = np.ones(n)
    for i in range(n - 1):
        pi[i + 1] = pi[i] * up[i] / down[i + 1]
    cb = rng.uniform(0.01, 1.0, n)
    st, fac = O.rw_solve(_transfers(K, W), cb)
    assert st == 1
    new = fac * cb
    np.testing.assert_allclose(new / new.sum(), pi / pi.sum(), rtol=1e-10)
    assert abs(new.sum() - cb.sum()) < 1e-14 * cb.sum() * n


def test_rw_solve_cycle_and_partial_occupancy():
    """A one-way cycle 0 -> 1 -> 2 -> 0 with move probabilities a, b, c per interval has pi
    proportional to (1/a, 1/b, 1/c) (inflow of each state = outflow).  A bin that holds no walkers keeps factor 0 and the others
    share the current total in the solved proportions."""
    a, b, c = 0.07, 0.25, 0.13
    K = np.zeros((4, 4))
    K[1, 0], K[2, 1], K[0, 2] = a, b, c
    W = np.array([1.0, 2.0, 0.5, 0.0])                 # bin 3 never started an interval: inactive
    cb = np.array([0.2, 0.0, 0.5, 0.3])                # bin 1 holds no walkers now
    st, fac = O.rw_solve(_transfers(K, W), cb)
    assert st == 1
    pi = np.array([1 / a, 1 / b, 1 / c])
    assert fac[1] == 0.0 and fac[3] == 0.0
    held = fac[[0, 2]] * cb[[0, 2]]
    np.testing.assert_allclose(held / held.sum(), pi[[0, 2]] / pi[[0, 2]].sum(), rtol=1e-12)
    assert abs(held.sum() - (cb[0] + cb[2])) < 1e-15


def test_rw_solve_matches_a_null_space_on_dense_chains():
    """Random dense chains (every move possible): the solved bin weights are the null vector of
    the rate matrix (singular value decomposition), to 1e-10 relative."""
    rng = np.random.default_rng(11)
    for n in (3, 7, 20, 45):
        K = rng.uniform(0.0, 0.5 / n, (n, n))
        W = rng.uniform(0.2, 2.0, n)
        F = _transfers(K, W)
        cb = rng.uniform(0.1, 1.0, n)
        st, fac = O.rw_solve(F, cb)
        assert st == 1
        P_ = F / F.sum(axis=0)[None, :]                  # column-stochastic move matrix
        G = P_ - np.eye(n)
        _, _, vt = np.linalg.svd(G)
        pi = np.abs(vt[-1])
        new = fac * cb
        np.testing.assert_allclose(new / new.sum(), pi / pi.sum(), rtol=1e-10)


def test_rw_solve_takes_the_largest_strongly_connected_set():
    """One active bin leaves everything as is.  Of two closed pairs {0, 1} and {2, 3} (equal
    size) the one with the lower bin is reweighted (pi_0 / pi_1 = 0.2 / 0.1) and the other keeps
    its weights.  A bin that was only ever seen staying (absorbing in the estimate) and a bin
    that only feeds the chain are left out of a 4-bin cycle, which is solved alone."""
    F = np.zeros((3, 3))
    F[0, 0] = 1.0
    st, fac = O.rw_solve(F, np.array([1.0, 0.0, 0.0]))
    assert st == -1 and not fac.any()
    K = np.zeros((4, 4))
    K[1, 0], K[0, 1], K[3, 2], K[2, 3] = 0.1, 0.2, 0.1, 0.3
    cb = np.array([0.1, 0.3, 0.25, 0.35])
    st, fac = O.rw_solve(_transfers(K, np.ones(4)), cb)
    assert st == 1 and fac[2] == 0.0 and fac[3] == 0.0
    new = fac[:2] * cb[:2]
    assert new[0] / new[1] == pytest.approx(2.0, rel=1e-14)
    assert new.sum() == pytest.approx(0.4, rel=1e-15)
    K = np.zeros((6, 6))
    K[1, 0], K[2, 1], K[3, 2], K[0, 3] = 0.1, 0.2, 0.3, 0.4     # cycle 0 -> 1 -> 2 -> 3 -> 0
    K[4, 3] = 0.05                                              # 3 -> 4; 4 only stays
    K[0, 5] = 0.2                                               # 5 -> 0 only
    cb = np.full(6, 1.0 / 6)
    st, fac = O.rw_solve(_transfers(K, np.ones(6)), cb)
    assert st == 1 and fac[4] == 0.0 and fac[5] == 0.0
    pi = 1.0 / np.array([0.1, 0.2, 0.3, 0.4])                   # moves within the set only
    new = fac[:4] * cb[:4]
    np.testing.assert_allclose(new / new.sum(), pi / pi.sum(), rtol=1e-12)


def test_we_with_reweighting_keeps_total_weight_and_schedule():
    """Schloegl flux run with reweighting every 3 iterations: the schedule, the total weight
    (1 to 1e-12 at every iteration) and the first reweighting only after transfers exist."""
    cfg = W.schlogl_flux_we(reweight_period=3, n_iters=12, m_targ=4)
    o = O.we_run(cfg, 0)
    assert o["status"] == 0
    rw = o["reweighted"]
    assert list(np.nonzero(rw)[0]) == [2, 5, 8, 11]
    assert (rw[[5, 8, 11]] == 1).all()
    assert np.all(np.abs(o["total_weight"] - 1.0) < 1e-12)
    assert abs(o["weights"].sum() - 1.0) < 1e-12


def test_we_reweighting_is_unbiased_with_state_resolved_bins():
    """With one state per bin the bin-to-bin chain that reweighting estimates is the exact lumped
    chain, so the steady-state flux it produces matches 1 / MFPT (birth-death 100 -> 140 with
    recycling, unit bins, reweighting every 5 iterations; 16 replicas, iterations 100-300), within
    3 standard errors."""
    b, d = E.birth_death_rates()
    exact = 1.0 / E.bd_mfpt(100, 140, b, d)
    cfg = W.birth_death_we(n_iters=300, target=140)
    cfg.bins = W.GridBins(species=[0], edges=[W.uniform_edges(0, 1, 150)])
    cfg.capacity = cfg.m_targ * cfg.bins.n_bins
    cfg.reweight_period = 5
    m = []
    for r in range(16):
        cfg.run_ids = np.array([r], dtype=np.uint32)
        o = O.we_run(cfg, 0)
        assert o["status"] == 0 and (o["reweighted"][4::5] == 1).all()
        m.append(o["flux_weight"][100:].mean() / cfg.tau / exact)
    m = np.array(m)
    se = m.std(ddof=1) / np.sqrt(len(m))
    assert abs(m.mean() - 1.0) < 3 * se, (m.mean(), se)


# ---------------------------------------------------------------- grid bins ----------------------
def test_grid_bins_match_a_library_search():
    """Grid bin assignment (Sec. II.B: non-overlapping bins on a 1-D or 2-D grid): per dimension
    the bin whose half-open interval [e_k, e_k+1) holds the count, clamped into the first and last
    bins, the flat index row-major with the last dimension fastest.  WE stays unbiased under any
    binning, so whole-run statistics cannot see a wrong bin map; here every count of the paper's
    grids (Schloegl, toggle with an overflow edge at infinity, the epigenetic switch's non-uniform
    2-D grid) and of random uneven 3-D grids goes against numpy's searchsorted and
    ravel_multi_index."""
    def by_library(cfg, x):
        idx = []
        for sp, e in zip(cfg.bins.species, cfg.bins.edges):
            e = np.asarray(e, dtype=np.float64)
            k = int(np.searchsorted(e, float(x[sp]), side="right")) - 1
            idx.append(min(max(k, 0), len(e) - 2))
        dims = [len(e) - 1 for e in cfg.bins.edges]
        return int(np.ravel_multi_index(tuple(idx), tuple(dims)))

    rng = np.random.default_rng(3)
    cfgs = [W.schlogl_mfpt_we(n_iters=1), W.toggle_batch_we(n_runs=1, n_iters=1), W.epigenetic_mfpt_we(n_iters=1)]
    for cfg in cfgs:
        S = len(cfg.network.fixed_count)
        hi = [int(np.max(np.where(np.isfinite(e), e, 0))) + 20 for e in cfg.bins.edges]
        for _ in range(400):
            x = np.zeros(S, np.int32)
            for sp, h in zip(cfg.bins.species, hi):
                x[sp] = rng.integers(0, h + 1)
            assert O.bin_of(cfg, x) == by_library(cfg, x), (cfg.name, x)
        # every edge and its neighbours along each dimension
        for d, (sp, e) in enumerate(zip(cfg.bins.species, cfg.bins.edges)):
            for v in np.asarray(e)[np.isfinite(e)]:
                for dv in (-1, 0, 1):
                    x = np.zeros(S, np.int32)
                    x[sp] = max(int(v) + dv, 0)
                    assert O.bin_of(cfg, x) == by_library(cfg, x), (cfg.name, d, x)
    cfg = W.futile_pdf_we(n_iters=1)                  # six species: room for 3-D grids
    S = len(cfg.network.fixed_count)
    assert S >= 3
    for trial in range(20):
        ndim = 3
        sp = list(rng.choice(S, size=ndim, replace=False))
        edges = [np.concatenate([[0.0], np.cumsum(rng.integers(1, 9, size=rng.integers(1, 7))).astype(np.float64)])
                 for _ in range(ndim)]
        if trial % 2:
            edges[-1] = np.append(edges[-1], np.inf)
        cfg.bins = W.GridBins(species=[int(s) for s in sp], edges=edges)
        for _ in range(200):
            x = rng.integers(0, 60, size=S).astype(np.int32)
            assert O.bin_of(cfg, x) == by_library(cfg, x), (trial, x)


# ------------------------------------------------------- exact birth-death tools -------------------
def test_birth_death_exact_tools_agree_with_independent_forms():
    """The exact tools that other tests take as expected values, each against an independent
    computation: the truncated-CME transient (matrix exponential) of immigration-death against
    its Binomial-Poisson closed form, the stationary law against Poisson(kb/kd), and the
    first-passage-time sum against a sparse solve of the first-passage equations Q_sub T = -1 on
    the states below the target (Schloegl and birth-death)."""
    from scipy.sparse.linalg import spsolve
    kb, kd = 10.0, 0.1
    b, d = E.birth_death_rates(kb, kd)
    for t in (0.5, 2.0, 20.0):
        p = E.bd_transient(b, d, 100, t, 400)
        q = E.immigration_death_pmf(100, kb, kd, t, 400)
        assert np.max(np.abs(p - q)) < 1e-10, t
    pi = E.bd_stationary(b, d, 400)
    assert np.max(np.abs(pi - np.exp(E.log_poisson_pmf(np.arange(401), kb / kd)))) < 1e-12
    for (rates, a, target) in ((E.birth_death_rates(), 100, 140), (E.schlogl_rates(), 85, 550),
                               (E.schlogl_rates(), 0, 300)):
        Q = E.bd_generator(*rates, target).tocsc()[:target, :target]     # exit to the target removed
        T = spsolve(Q, -np.ones(target))
        assert E.bd_mfpt(a, target, *rates) == pytest.approx(T[a], rel=1e-9), (a, target)


def test_two_species_mfpt_solvers_reduce_to_known_cases():
    """The 2-D master-equation solvers behind the toggle and epigenetic-switch expected values:
    with the repression switched off (K far above any count) the species entering the target
    is an immigration-death process of its own, so the MFPT is the 1-D first-passage sum; with
    equal Hill exponents and unit constants the two models are the same chain, so the two
    solvers (each written from its own model's equations) agree; and the toggle's MFPT is
    unchanged when the two genes swap roles."""
    ind = lambda a: (lambda x: np.full(np.shape(x), a, dtype=np.float64))
    lin = lambda x: 1.0 * np.asarray(x, dtype=np.float64)
    t = E.toggle_mfpt(30.0, 12.0, (30, 0), lambda u, v: v >= 20, K=1e30, Umax=70, Vmax=40)
    assert t == pytest.approx(E.bd_mfpt(0, 20, ind(12.0), lin), rel=1e-9)
    g = E.epigenetic_mfpt((0, 30), lambda u, v: u >= 50, K1=1e30, K2=1e30, G1=90, G2=70)
    assert g == pytest.approx(E.bd_mfpt(0, 50, ind(156.0), lin), rel=1e-9)
    target = lambda u, v: v >= 10 and u <= 5
    a = E.toggle_mfpt(20.0, 20.0, (20, 0), target, n=2, Umax=60, Vmax=60)
    b = E.epigenetic_mfpt((20, 0), target, a1=20.0, a2=20.0, n=2, m=2, G1=60, G2=60)
    assert a == pytest.approx(b, rel=1e-10)
    swapped = E.toggle_mfpt(20.0, 20.0, (0, 20), lambda u, v: target(v, u), n=2, Umax=60, Vmax=60)
    assert a == pytest.approx(swapped, rel=1e-10)
    assert 10.0 < a < 1e6


def test_stored_golden_values_are_the_oracles():
    """tests/golden/exact_values.json holds exactly what tests/golden/make_golden.py computes from
    oracle/ today (a stale file, or one written by anything else, fails here), and its entries
    agree with the values the paper prints: P(X >= 700, t = 5 | X0 = 82) = 1.148e-9 and an MFPT
    of about 5e4 s between the Schloegl modes (Sec. III.B.3), P(S1 > 90, t = 100) = 2.72e-18
    (Sec. III.A), the epigenetic switch's 1.3e6 s (Sec. III.C)."""
    import importlib.util
    import json
    here = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
    spec = importlib.util.spec_from_file_location("make_golden", os.path.join(here, "make_golden.py"))
    mg = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mg)
    fresh = mg.compute()
    stored = json.load(open(os.path.join(here, "exact_values.json")))
    assert set(fresh) == set(stored)
    for k, v in fresh.items():
        if isinstance(v, float):
            assert stored[k] == pytest.approx(v, rel=1e-9), k
        else:
            assert stored[k] == v, k
    assert round(stored["schlogl_p_ge_700_t5_from_82"], 12) == 1.148e-9
    assert round(stored["schlogl_mfpt_82_to_563_s"], -4) == 5e4
    assert round(stored["futile_p_s1_gt_90_t100"], 20) == 2.72e-18
    assert round(stored["epigenetic_mfpt_0_30_to_g1_ge_50_s"], -5) == 1.3e6


def test_end_of_interval_target_check_renewal_flux():
    """Target checked at the end of each interval only (B checked at a prescribed time step,
    Sec. IV), against the renewal closed form: a pure-birth process X -> X + 1 at rate k from 0,
    recycled to 0, reaches X >= n at the Erlang(n, k) time T and stays there, so a cycle lasts
    N = ceil(T / tau) intervals and the long-run flux per interval is 1 / E[N], with
    E[N] = sum_{m >= 0} P(T > m tau) = sum_m P(Poisson(k m tau) <= n - 1).  Checked at the
    event instead, the flux is tau k / n; the two differ by about 5 % here, many standard errors."""
    k, n, tau = 1.0, 5, 0.5
    R, N, iters, burn = 8, 250, 300, 40
    en = 0.0
    for m in range(0, 10000):
        term = stats.poisson.cdf(n - 1, k * m * tau)
        en += term
        if term < 1e-16:
            break
    net = W.NetworkSpec(species=["X"], reactants=[[]], products=[[(0, 1)]], rate=[[k]])
    tgt = W.Target(species=[0], op=[W.configs.OP_GE], threshold=np.full((R, 1), n, dtype=np.int32))
    expect = {True: 1.0 / en, False: tau * k / n}
    ses = []
    for endpoint in (True, False):
        cfg = W.bruteforce_fpt(net, [0], tgt, N, tau, iters, n_runs=R, name="pure_birth")
        cfg.absorb = False
        cfg.endpoint = endpoint
        per_run = [O.we_run(cfg, r, resample=False)["flux_weight"][burn:].mean() for r in range(R)]
        mean, se = float(np.mean(per_run)), float(np.std(per_run, ddof=1) / math.sqrt(R))
        assert abs(mean - expect[endpoint]) < 3 * se, (endpoint, mean, expect[endpoint], se)
        ses.append(se)
    assert abs(expect[True] - expect[False]) > 10 * max(ses)
