"""The two kernels of the grouping-by-bin and split/merge step (Sec. II.B) give the same
ensembles: the three-launch chain (per-run scan, grid-wide grouping, one warp per occupied bin)
and the one-launch form (each of G blocks per run groups the run's walkers in shared memory and
splits/merges its share of the bins, merging through two key-ordered lists).  Both are held to the oracle bit for bit: counts, weights,
order, parents and event counts exact, accumulated observables within 1e-12 relative."""
import functools

import numpy as np
import pytest

import paper_1303_5986_gb300 as P
import workloads as W

from gpu_helpers import assert_run_parity, gpu_outputs, gpu_run, oracle_run

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1303_5986_gb300 import build
    build.build()


def _many_merges():
    """600 walkers of random weight in one bin merged down to M = 3 (more than 128 walkers: the
    serial floating-point merge path, on shared-memory lists in the one-launch form)."""
    spec = W.birth_death(kb=1e-9, kd=1e-9)
    n = 600
    rng = np.random.default_rng(8)
    init = np.full((1, n, 1), 7, dtype=np.int32)
    w = rng.exponential(size=(1, n)) * 10.0 ** rng.uniform(-30, 0, size=(1, n))
    w /= w.sum()
    return W.WEConfig(network=spec, bins=W.GridBins([0], [W.uniform_edges(0, 5, 4)]), tau=0.1,
                      m_targ=3, n_iters=2, x0=[7], init_states=init, init_weights=w, capacity=n,
                      hist_species=0, hist_len=16, name="merges")


def _one_bin(w, m_targ, name):
    """Walkers of the given weights in one bin of a network that does not move (every interval
    is a pure split/merge)."""
    spec = W.birth_death(kb=1e-9, kd=1e-9)
    n = w.shape[1]
    init = np.full((1, n, 1), 7, dtype=np.int32)
    return W.WEConfig(network=spec, bins=W.GridBins([0], [W.uniform_edges(0, 5, 4)]), tau=0.1,
                      m_targ=m_targ, n_iters=3, x0=[7], init_states=init, init_weights=w,
                      capacity=max(n, 4 * m_targ), hist_species=0, hist_len=16, name=name)


def _equal_weights():
    """100 walkers of one weight merged to 7: every pair ties on weight, and so do the merged
    sums (order by slot)."""
    return _one_bin(np.full((1, 100), 0.01), 7, "equal_weights")


def _few_distinct_weights():
    """90 walkers with weights from {1, 2, 3} / norm merged to 5: merged sums tie with one another
    and with unmerged walkers."""
    rng = np.random.default_rng(3)
    w = rng.integers(1, 4, size=(1, 90)).astype(np.float64)
    return _one_bin(w / w.sum(), 5, "few_weights")


def _tiny_weights():
    """110 walkers below 2^-999 merged to 4: the survivor decision takes the FP64 quotient."""
    rng = np.random.default_rng(4)
    return _one_bin(rng.exponential(size=(1, 110)) * 1e-305, 4, "tiny_weights")


def _equal_split():
    """5 walkers of one weight split to 23 copies: every per-copy weight ties (order by slot)."""
    return _one_bin(np.full((1, 5), 0.2), 23, "equal_split")


def _split_32():
    """32 walkers of random weight (the most the sorted split form takes) split to 61."""
    rng = np.random.default_rng(5)
    w = rng.exponential(size=(1, 32))
    return _one_bin(w / w.sum(), 61, "split_32")


def _tiny_split():
    """3 walkers below 2^-999 split to 20: the per-copy weights by FP64 division."""
    return _one_bin(np.array([[3e-306, 1e-305, 7e-306]]), 20, "tiny_split")


def _toggle_small_grid():
    """Two-species toggle runs on a 12 x 12 grid (144 bins), four parameter sets."""
    cfg = W.toggle_batch_we(n_runs=4, n_iters=25, m_targ=6)
    e = W.uniform_edges(0, 8, 11, overflow=True)
    cfg.bins = W.GridBins([0, 1], [e, e])
    cfg.capacity = 6 * 144
    return cfg


CASES = {
    "schlogl_mfpt": lambda: W.schlogl_mfpt_we(n_iters=30, n_runs=3),
    "birth_death_recycling": lambda: W.birth_death_we(n_iters=40, target=130),
    "reweighted": lambda: W.schlogl_flux_we(reweight_period=3, n_iters=15, n_runs=2, m_targ=5),
    "toggle_2d": _toggle_small_grid,
    "many_merges": _many_merges,
    "equal_weights": _equal_weights,
    "few_distinct_weights": _few_distinct_weights,
    "tiny_weights": _tiny_weights,
    "equal_split": _equal_split,
    "split_32": _split_32,
    "tiny_split": _tiny_split,
}


@functools.lru_cache(maxsize=None)
def _oracle(case, r):
    cfg = CASES[case]()
    return oracle_run(cfg, r, n_iters=cfg.n_iters)


def _check(ens, cfg, case, label):
    ens.sync()
    for r in range(cfg.n_runs):
        assert_run_parity(gpu_outputs(ens, r), _oracle(case, r), label=f"{case} run {r} {label}")


@pytest.mark.parametrize("case", list(CASES))
@pytest.mark.parametrize("kind,blocks", [(P.WE_RESAMPLE_CHAIN, 0), (P.WE_RESAMPLE_ONE_LAUNCH, 0),
                                         (P.WE_RESAMPLE_ONE_LAUNCH, 1), (P.WE_RESAMPLE_ONE_LAUNCH, 3),
                                         (P.WE_RESAMPLE_ONE_LAUNCH, 32)])
def test_resample_kernels_match_the_oracle(case, kind, blocks):
    cfg = CASES[case]()
    ens = gpu_run(cfg, 0, record_iters=cfg.n_iters)
    ens.set_resample_kernel(kind, blocks)
    ens.step(cfg.n_iters)
    _check(ens, cfg, case, f"kind {kind} blocks {blocks}")
    if case == "reweighted":
        rw = ens.per_iter(P.WE_OUT_RW)
        for r in range(cfg.n_runs):
            assert np.array_equal(rw[:, r], _oracle(case, r)["reweighted"])


def test_switching_kernels_between_iterations():
    """Chain for 12 iterations, one launch for 10, chain again for 8: the bin counts each form
    leaves behind are what the other expects, and the captured graphs are replaced."""
    case = "schlogl_mfpt"
    cfg = CASES[case]()
    ens = gpu_run(cfg, 0, record_iters=cfg.n_iters)
    ens.set_resample_kernel(P.WE_RESAMPLE_CHAIN, 0)
    ens.step(12)
    ens.set_resample_kernel(P.WE_RESAMPLE_ONE_LAUNCH, 2)
    ens.step(10)
    ens.set_resample_kernel(P.WE_RESAMPLE_CHAIN, 0)
    ens.step(8)
    _check(ens, cfg, case, "switched")


def test_phase_calls_with_the_one_launch_kernel():
    """propagate() + resample() per iteration, the one-launch kernel chosen explicitly."""
    case = "birth_death_recycling"
    cfg = CASES[case]()
    ens = gpu_run(cfg, 0, record_iters=cfg.n_iters)
    ens.set_resample_kernel(P.WE_RESAMPLE_ONE_LAUNCH, 2)
    for _ in range(cfg.n_iters):
        ens.propagate()
        ens.resample()
    _check(ens, cfg, case, "phase calls")


def test_iteration_kernel_counts():
    """Kernel nodes of the iteration graph: SSA + split/merge + bookkeeping in one launch each,
    SSA + scan + grouping + split/merge + bookkeeping with the chain."""
    cfg = CASES["schlogl_mfpt"]()
    ens = gpu_run(cfg, 0, record_iters=cfg.n_iters)
    assert ens.iteration_kernels() == 3
    ens.set_resample_kernel(P.WE_RESAMPLE_CHAIN, 0)
    assert ens.iteration_kernels() == 5


def test_capacity_overflow_is_flagged_by_both_kernels():
    """A capacity below M_targ x occupied bins: both kernels report WE_EOVERFLOW, as the oracle."""
    cfg = W.birth_death_we(n_iters=3)
    cfg.capacity = 15                                   # 10 walkers spread over 2 or more bins
    o = oracle_run(cfg, 0, n_iters=3)
    assert o["status"] == P.WE_EOVERFLOW
    for kind in (P.WE_RESAMPLE_CHAIN, P.WE_RESAMPLE_ONE_LAUNCH):
        ens = gpu_run(cfg, 0, record_iters=3)
        ens.set_resample_kernel(kind, 0)
        ens.step(3)
        with pytest.raises(P.WEError) as ei:
            ens.sync()
        assert ei.value.status == P.WE_EOVERFLOW
        assert int(ens.status()[0]) == P.WE_EOVERFLOW


def test_resample_kernel_errors():
    ens = gpu_run(W.birth_death_we(n_iters=2), 0, record_iters=2)
    for kind, blocks in ((3, 0), (-1, 0), (P.WE_RESAMPLE_ONE_LAUNCH, 33), (P.WE_RESAMPLE_CHAIN, -1)):
        with pytest.raises(P.WEError) as ei:
            ens.set_resample_kernel(kind, blocks)
        assert ei.value.status == P.WE_EINVAL
    ens.propagate()
    with pytest.raises(P.WEError) as ei:
        ens.set_resample_kernel(P.WE_RESAMPLE_CHAIN, 0)            # a resample is pending
    assert ei.value.status == P.WE_EINVAL
    ens.resample()
    ens.sync()
    # 354 species: the split/merge does not gather them, so the one-launch form does not apply
    big = gpu_run(W.synthetic_large_we(n_walkers=24, n_iters=1), 0, mapping=P.WE_MAP_WARP)
    with pytest.raises(P.WEError) as ei:
        big.set_resample_kernel(P.WE_RESAMPLE_ONE_LAUNCH, 0)
    assert ei.value.status == P.WE_EINVAL
    big.set_resample_kernel(P.WE_RESAMPLE_CHAIN, 0)
