"""Run settings (bins, tau, walkers per bin, iterations, targets, initial states) for the WE runs.

The factories below give the benchmark workloads: the 1-D birth-death process, the Schloegl
model in steady-state (MFPT) and PDF modes (Sec. III.B.2), a batched sweep of two-gene toggle
switches shaped like the epigenetic switch (Sec. III.C), and a random network shaped like the
FceRI model (Sec. III.D).  Every random draw here is seeded; none of it is the method's own
randomness, which comes from the counter-based generator inside each implementation.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from .networks import (NetworkSpec, birth_death, epigenetic_switch, futile_cycle, schlogl, synthetic_large,
                       toggle_switch)

OP_GE = 0
OP_LE = 1


def uniform_edges(lo: float, width: float, n: int, overflow: bool = False) -> np.ndarray:
    """n bins of equal width starting at lo; with overflow, one more bin up to +infinity."""
    e = lo + width * np.arange(n + 1, dtype=np.float64)
    if overflow:
        e = np.append(e, np.inf)
    return e


@dataclass
class GridBins:
    species: list
    edges: list

    @property
    def ndim(self) -> int:
        return len(self.species)

    @property
    def n_bins_per_dim(self) -> list:
        return [len(e) - 1 for e in self.edges]

    @property
    def n_bins(self) -> int:
        return int(np.prod(self.n_bins_per_dim))

    def flat_edges(self) -> np.ndarray:
        return np.concatenate([np.asarray(e, dtype=np.float64) for e in self.edges])


@dataclass
class Target:
    """Target set B = AND_c (x[species_c] op_c threshold[run, c])."""

    species: list
    op: list
    threshold: np.ndarray   # (n_runs, n_clauses) int32


@dataclass
class WEConfig:
    network: NetworkSpec
    bins: GridBins
    tau: float
    m_targ: int
    n_iters: int
    x0: np.ndarray                       # (n_runs, S) int32
    n_runs: int = 1
    seed: int = 0
    run_ids: np.ndarray = None           # (n_runs,) uint32
    param_set: np.ndarray = None         # (n_runs,) which rate row each run uses
    init_states: np.ndarray = None       # (n_runs, n_init, S) int32
    init_weights: np.ndarray = None      # (n_runs, n_init) float64
    target: Target = None
    recycle_state: np.ndarray = None     # (n_runs, S) int32
    hist_species: int = 0
    hist_len: int = 0
    capacity: int = 0
    max_steps: int = 0
    first_iter: int = 0
    reweight_period: int = 0             # >0: steady-state reweighting every this many iterations
    absorb: bool = False                 # with a target: walkers stop at their first entrance
    endpoint: bool = False               # with a target: checked at each interval's end only
                                         # (brute-force first-passage runs, no resampling)
    name: str = ""
    notes: dict = field(default_factory=dict)

    def __post_init__(self):
        S = self.network.n_species
        self.x0 = np.asarray(self.x0, dtype=np.int32).reshape(-1, S)
        if self.x0.shape[0] == 1 and self.n_runs > 1:
            self.x0 = np.repeat(self.x0, self.n_runs, axis=0)
        assert self.x0.shape[0] == self.n_runs
        if self.run_ids is None:
            self.run_ids = np.arange(self.n_runs, dtype=np.uint32)
        self.run_ids = np.asarray(self.run_ids, dtype=np.uint32)
        if self.param_set is None:
            self.param_set = np.arange(self.n_runs, dtype=np.int32) % self.network.n_param_sets
        self.param_set = np.asarray(self.param_set, dtype=np.int32)
        if self.init_states is None:
            n = self.m_targ
            self.init_states = np.repeat(self.x0[:, None, :], n, axis=1)
        self.init_states = np.asarray(self.init_states, dtype=np.int32)
        if self.init_weights is None:
            n = self.init_states.shape[1]
            self.init_weights = np.full((self.n_runs, n), 1.0 / n)
        self.init_weights = np.asarray(self.init_weights, dtype=np.float64)
        if self.recycle_state is None:
            self.recycle_state = self.x0.copy()
        self.recycle_state = np.asarray(self.recycle_state, dtype=np.int32).reshape(self.n_runs, S)
        if self.capacity <= 0:
            self.capacity = max(self.m_targ * self.bins.n_bins, self.init_states.shape[1])

    @property
    def n_init(self) -> int:
        return self.init_states.shape[1]

    @property
    def feedback(self) -> bool:
        return self.target is not None


def birth_death_we(n_iters: int = 200, n_runs: int = 1, target: int | None = None,
                   seed: int = 0) -> WEConfig:
    """1-D birth-death: kb=10, kd=0.1, X0=100; 60 bins of width 5 on [0,300) plus [300,inf);
    10 walkers per bin; tau=0.1.  With ``target`` the run recycles at X >= target."""
    net = birth_death()
    bins = GridBins(species=[0], edges=[uniform_edges(0, 5, 60, overflow=True)])
    tgt = None
    if target is not None:
        tgt = Target(species=[0], op=[OP_GE], threshold=np.full((n_runs, 1), target, dtype=np.int32))
    return WEConfig(network=net, bins=bins, tau=0.1, m_targ=10, n_iters=n_iters, x0=[100],
                    n_runs=n_runs, seed=seed, target=tgt, hist_species=0, hist_len=401,
                    name="birth_death")


def schlogl_mfpt_we(n_iters: int = 1000, n_runs: int = 1, seed: int = 0, x0: int = 85,
                    threshold: int = 550, m_targ: int = 20) -> WEConfig:
    """Schloegl steady state (Sec. III.B.2 flux runs, with the settings of the benchmark):
    80 bins of width 10 on [0,800) (X >= 800 falls in the last bin), 20 walkers per bin,
    tau=0.05, recycling at X >= 550 back to X0=85."""
    net = schlogl()
    A, B = int(net.fixed_count[1]), int(net.fixed_count[2])
    bins = GridBins(species=[0], edges=[uniform_edges(0, 10, 80)])
    tgt = Target(species=[0], op=[OP_GE], threshold=np.full((n_runs, 1), threshold, dtype=np.int32))
    return WEConfig(network=net, bins=bins, tau=0.05, m_targ=m_targ, n_iters=n_iters,
                    x0=[x0, A, B], n_runs=n_runs, seed=seed, target=tgt, hist_species=0,
                    hist_len=1001, name="schlogl_mfpt")


def schlogl_flux_we(reweight_period: int = 0, n_iters: int = 500, n_runs: int = 1, seed: int = 0,
                    m_targ: int = 32) -> WEConfig:
    """Schloegl flux run of Sec. III.B.2/3: 80 bins of width 10 on [0,800), 32 walkers per bin,
    tau=0.1, 500 iterations from X0=82, recycling at X >= 563 back to 82; steady-state
    reweighting every ``reweight_period`` iterations (the paper's RW-100, RW-5, RW-2)."""
    cfg = schlogl_mfpt_we(n_iters=n_iters, n_runs=n_runs, seed=seed, x0=82, threshold=563,
                          m_targ=m_targ)
    cfg.tau = 0.1
    cfg.reweight_period = reweight_period
    cfg.name = "schlogl_flux"
    return cfg


def schlogl_pdf_we(n_iters: int = 101, n_runs: int = 1, seed: int = 0, m_targ: int = 100,
                   n_unit_bins: int = 802, x0: int = 82) -> WEConfig:
    """Schloegl probability distribution (Sec. III.B.2): 802 unit-width bins, 100 walkers per
    bin, tau=0.05, 101 iterations, from X0=82 (the last bin holds X >= 801)."""
    net = schlogl()
    A, B = int(net.fixed_count[1]), int(net.fixed_count[2])
    bins = GridBins(species=[0], edges=[uniform_edges(0, 1, n_unit_bins)])
    return WEConfig(network=net, bins=bins, tau=0.05, m_targ=m_targ, n_iters=n_iters,
                    x0=[x0, A, B], n_runs=n_runs, seed=seed, hist_species=0, hist_len=1201,
                    name="schlogl_pdf")


def futile_pdf_we(n_iters: int = 100, n_runs: int = 1, seed: int = 0, m_targ: int = 100) -> WEConfig:
    """Enzymatic futile cycle distribution (Sec. III.A): 101 unit-width bins on S1, 100 walkers
    per bin, tau=1, 100 iterations, from S1 = S2 = 50 with both enzymes free."""
    bins = GridBins(species=[0], edges=[uniform_edges(0, 1, 101)])
    return WEConfig(network=futile_cycle(), bins=bins, tau=1.0, m_targ=m_targ, n_iters=n_iters,
                    x0=[50, 50, 1, 1, 0, 0], n_runs=n_runs, seed=seed, hist_species=0,
                    hist_len=102, name="futile_pdf")


def epigenetic_mfpt_we(n_iters: int = 500, n_runs: int = 6, seed: int = 0, m_targ: int = 16,
                       reweight_period: int = 100) -> WEConfig:
    """Epigenetic switch MFPT runs (Sec. III.C): 15 x 31 bins -- g1 unit-width on [0,10], width
    10 on [10,50], one bin [50,inf); g2 unit-width on [0,30], one bin [30,inf) -- 16 walkers per
    bin, tau = 0.1, 500 iterations, reweighting every 100; from the g2-high state (g1, g2) =
    (0, 30), recycling on reaching g1 >= 50 (the last g1 bin)."""
    net = epigenetic_switch()
    e1 = np.concatenate([np.arange(0, 10, dtype=np.float64), np.arange(10, 51, 10, dtype=np.float64), [np.inf]])
    e2 = uniform_edges(0, 1, 30, overflow=True)
    bins = GridBins(species=[0, 1], edges=[e1, e2])
    tgt = Target(species=[0], op=[OP_GE], threshold=np.full((n_runs, 1), 50, dtype=np.int32))
    return WEConfig(network=net, bins=bins, tau=0.1, m_targ=m_targ, n_iters=n_iters, x0=[0, 30],
                    n_runs=n_runs, seed=seed, target=tgt, hist_species=0, hist_len=101,
                    reweight_period=reweight_period, name="epigenetic_mfpt")


def bruteforce_fpt(network: NetworkSpec, x0, target: Target, n_walkers: int, tau: float, n_iters: int,
                   n_runs: int = 1, seed: int = 0, name: str = "bruteforce") -> WEConfig:
    """Brute-force transition-time campaign (Sec. II.C): n_walkers unweighted SSA runs per run id
    from x0, each stopped at its first entrance into the target set; tau is only the length of
    the intervals the runs are advanced by (n_iters of them: runs of length T = n_iters tau).
    Run without resampling; one bin."""
    S = network.n_species
    x0 = np.asarray(x0, dtype=np.int32).reshape(-1, S)
    if x0.shape[0] == 1:
        x0 = np.repeat(x0, n_runs, axis=0)
    init = np.repeat(x0[:, None, :], n_walkers, axis=1)
    bins = GridBins(species=[0], edges=[np.array([0.0, np.inf])])
    return WEConfig(network=network, bins=bins, tau=tau, m_targ=1, n_iters=n_iters, x0=x0,
                    n_runs=n_runs, seed=seed, init_states=init,
                    init_weights=np.full((n_runs, n_walkers), 1.0 / n_walkers), target=target,
                    capacity=n_walkers, absorb=True, name=name)


def schlogl_bruteforce(n_walkers: int = 1024, tau: float = 10.0, n_iters: int = 100, n_runs: int = 1,
                       seed: int = 0, x0: int = 85, threshold: int = 550) -> WEConfig:
    """Brute-force Schloegl transition runs (Sec. III.B.3's E50% comparison): walkers from X0 = 85
    absorbed at X >= 550, runs of length n_iters * tau."""
    net = schlogl()
    A, B = int(net.fixed_count[1]), int(net.fixed_count[2])
    tgt = Target(species=[0], op=[OP_GE], threshold=np.full((n_runs, 1), threshold, dtype=np.int32))
    return bruteforce_fpt(net, [x0, A, B], tgt, n_walkers, tau, n_iters, n_runs, seed, "schlogl_bruteforce")


def birth_death_bruteforce(n_walkers: int = 256, tau: float = 1.0, n_iters: int = 100, n_runs: int = 1,
                           seed: int = 0, x0: int = 100, threshold: int = 130) -> WEConfig:
    """Brute-force birth-death first passages 100 -> X >= threshold (kb = 10, kd = 0.1)."""
    tgt = Target(species=[0], op=[OP_GE], threshold=np.full((n_runs, 1), threshold, dtype=np.int32))
    return bruteforce_fpt(birth_death(), [x0], tgt, n_walkers, tau, n_iters, n_runs, seed,
                          "birth_death_bruteforce")


def toggle_params(n_runs: int = 64, seed: int = 0, lo: float = 20.0, hi: float = 60.0):
    rng = np.random.default_rng(seed)
    a_u = rng.uniform(lo, hi, size=n_runs)
    a_v = rng.uniform(lo, hi, size=n_runs)
    return a_u, a_v


def toggle_batch_we(n_runs: int = 64, n_iters: int = 500, seed: int = 0, m_targ: int = 8,
                    param_seed: int = 0) -> WEConfig:
    """Batched sweep of toggle switches (K=1, n=2, d=1, no basal production): production rates
    a_U, a_V uniform in [20,60], one WE run per parameter set; 2-D bins of width 4 on [0,116)
    plus [116,inf) on each of U and V (30 x 30); 8 walkers per bin; tau=0.1.  Each run starts
    at (round(a_U), 0) and recycles on reaching {V >= a_V/2 and U <= a_U/4}."""
    a_u, a_v = toggle_params(n_runs, param_seed)
    net = toggle_switch(a_u, a_v)
    e = uniform_edges(0, 4, 29, overflow=True)
    bins = GridBins(species=[0, 1], edges=[e, e])
    x0 = np.stack([np.rint(a_u), np.zeros(n_runs)], axis=1).astype(np.int32)
    thr = np.stack([np.ceil(a_v / 2.0), np.floor(a_u / 4.0)], axis=1).astype(np.int32)
    tgt = Target(species=[1, 0], op=[OP_GE, OP_LE], threshold=thr)
    return WEConfig(network=net, bins=bins, tau=0.1, m_targ=m_targ, n_iters=n_iters, x0=x0,
                    n_runs=n_runs, seed=seed, target=tgt, hist_species=1, hist_len=129,
                    name="toggle_batch", notes=dict(a_u=a_u, a_v=a_v))


def synthetic_large_we(n_walkers: int = 4096, n_iters: int = 100, seed: int = 0,
                       net_seed: int = 7, state_seed: int = 11, m_targ: int = 82) -> WEConfig:
    """Random 354 x 3680 network (FceRI's shape): 4096 walkers with counts uniform in [0,200],
    weights 1/4096, 50 bins of width 4 on species 0 over [0,200) (higher counts fall in the last
    bin), 82 walkers per bin, tau=0.01."""
    net = synthetic_large(seed=net_seed)
    S = net.n_species
    rng = np.random.default_rng(state_seed)
    init = rng.integers(0, 201, size=(1, n_walkers, S)).astype(np.int32)
    bins = GridBins(species=[0], edges=[uniform_edges(0, 4, 50)])
    return WEConfig(network=net, bins=bins, tau=0.01, m_targ=m_targ, n_iters=n_iters,
                    x0=init[0, 0], n_runs=1, seed=seed, init_states=init,
                    init_weights=np.full((1, n_walkers), 1.0 / n_walkers), hist_species=0,
                    hist_len=401, capacity=max(n_walkers, m_targ * 50), name="synthetic_large")
