"""Brute-force transition runs (Sec. II.C) on the GPU: plain SSA walkers stopped at their first
entrance into an absorbing target set, with each walker's first-passage time, and the
censored-exponential maximum-likelihood transition time of Eq. "mld" computed by the library.

Bar: counts, event counts and absorption flags bit-exact against the CPU oracle; first-passage
times within 1e-12 relative (device and host logarithms may differ in the last bits); the MLE
within 1e-12 of the oracle's estimator applied to the same times."""
import numpy as np
import pytest

import paper_1303_5986_gb300 as P
import workloads as W
from oracle import exact as E
from oracle import oracle as O

from gpu_helpers import gpu_outputs, gpu_run

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1303_5986_gb300 import build
    build.build()


def _bf_parity(cfg, **kw):
    ens = gpu_run(cfg, cfg.n_iters, resample=False, **kw)
    ens.sync()
    for r in range(cfg.n_runs):
        g = gpu_outputs(ens, r, hist=False)
        o = O.we_run(cfg, r, resample=False)
        lab = f"{cfg.name} run {r} {kw}"
        assert g["status"] == o["status"] == 0, lab
        assert np.array_equal(g["events"], o["events"]), lab
        assert np.array_equal(g["states"], o["states"]), lab
        gf, of = ens.first_passage(r), o["first_passage"]
        assert np.array_equal(gf < 0, of < 0), lab
        np.testing.assert_allclose(gf, of, rtol=1e-12, atol=0, err_msg=lab)
        np.testing.assert_allclose(g["flux_weight"], o["flux_weight"], rtol=1e-12, atol=1e-300, err_msg=lab)
    return ens


@pytest.mark.parametrize("mapping,block", [(P.WE_MAP_AUTO, 0), (P.WE_MAP_AUTO, 32),
                                           (P.WE_MAP_THREAD, 0), (P.WE_MAP_THREAD, 32),
                                           (P.WE_MAP_WARP, 0)])
def test_birth_death_bruteforce_parity(mapping, block):
    """Birth-death 100 -> X >= 115 in 60 intervals of 1 s, 300 walkers in 2 runs, on every kernel
    (state-indexed table pipelined and plain, general FP64 warp-specialised and plain, warp per
    walker): about half the walkers pass."""
    cfg = W.birth_death_bruteforce(n_walkers=300, tau=1.0, n_iters=60, n_runs=2, threshold=115)
    ens = _bf_parity(cfg, mapping=mapping, block_threads=block)
    f = ens.first_passage(0)
    assert 0.2 < (f >= 0).mean() < 0.9


@pytest.mark.parametrize("block", [0, 32])
def test_schlogl_bruteforce_parity(block):
    """Schloegl from X = 85 absorbed at X >= 125, 256 walkers, 12 intervals of 2 s."""
    cfg = W.schlogl_bruteforce(n_walkers=256, tau=2.0, n_iters=12, threshold=125)
    ens = _bf_parity(cfg, block_threads=block)
    assert (ens.first_passage(0) >= 0).sum() > 10


def test_toggle_bruteforce_parity():
    """Two-species Hill dynamics (the two-species table kernel): a toggle with a_U = a_V = 8 from
    (8, 0) into {V >= 4, U <= 2}."""
    net = W.toggle_switch([8.0], [8.0])
    tgt = W.Target(species=[1, 0], op=[W.configs.OP_GE, W.configs.OP_LE],
                   threshold=np.array([[4, 2]], dtype=np.int32))
    cfg = W.bruteforce_fpt(net, [8, 0], tgt, n_walkers=256, tau=1.0, n_iters=40, name="toggle_bf")
    for mapping in (P.WE_MAP_AUTO, P.WE_MAP_THREAD):
        ens = _bf_parity(cfg, mapping=mapping)
    assert (ens.first_passage(0) >= 0).sum() > 20


def test_synthetic_network_bruteforce_parity():
    """Warp per walker on the 354 x 3680 network: species 0 absorbed at >= 150 within 3
    intervals of 1e-5."""
    base = W.synthetic_large_we(n_walkers=24, n_iters=3)
    tgt = W.Target(species=[0], op=[W.configs.OP_GE], threshold=np.full((1, 1), 150, dtype=np.int32))
    cfg = W.bruteforce_fpt(base.network, base.init_states[0, 0], tgt, n_walkers=24, tau=1e-5, n_iters=3,
                           name="synthetic_bf")
    cfg.init_states = base.init_states.copy()
    _bf_parity(cfg, mapping=P.WE_MAP_WARP)


def test_walker_starting_inside_the_target_fires_nothing():
    cfg = W.birth_death_bruteforce(n_walkers=4, tau=1.0, n_iters=30, threshold=105)
    cfg.init_states[0, 1, 0] = 107
    for mapping in (P.WE_MAP_AUTO, P.WE_MAP_THREAD, P.WE_MAP_WARP):
        ens = _bf_parity(cfg, mapping=mapping)
        f = ens.first_passage(0)
        assert f[1] == 0.0 and ens.states(0)[1, 0] == 107


def test_mle_matches_the_estimator_on_the_same_times():
    """we_ensemble_fpt_mle (sums on the device) against Eq. "mld" evaluated on the host from the
    GPU's own first-passage times: for the whole run (T = time simulated) and censored at an
    earlier T, per run."""
    cfg = W.birth_death_bruteforce(n_walkers=700, tau=1.0, n_iters=50, n_runs=3, threshold=118)
    ens = gpu_run(cfg, cfg.n_iters, resample=False)
    ens.sync()
    for T in (0.0, 50.0, 20.0):
        res = ens.fpt_mle(T)
        Te = 50.0 if T <= 0 else T
        for r in range(cfg.n_runs):
            f = ens.first_passage(r)
            seen = f[(f >= 0) & (f <= Te)]
            mu, sig = E.mle_transition_time(Te, len(f), seen)
            assert res[r, 0] == len(f) and res[r, 1] == len(seen)
            assert res[r, 2] == pytest.approx(seen.sum(), rel=1e-12)
            assert res[r, 3] == pytest.approx(mu, rel=1e-12)
            assert res[r, 4] == pytest.approx(sig, rel=1e-12)


def test_bruteforce_configuration_errors():
    cfg = W.birth_death_bruteforce(n_walkers=8, tau=1.0, n_iters=2, threshold=110)
    with pytest.raises(P.WEError) as ei:
        gpu_run(cfg, 0, resample=True)                  # absorbing needs plain propagation
    assert ei.value.status == P.WE_EINVAL
    ens = gpu_run(W.birth_death_we(n_iters=2), 2)
    with pytest.raises(P.WEError) as ei:
        ens.fpt_mle()                                    # not an absorbing ensemble
    assert ei.value.status == P.WE_EINVAL
    bf = gpu_run(cfg, 1, resample=False)
    with pytest.raises(P.WEError) as ei:
        bf.checkpoint()
    assert ei.value.status == P.WE_ENOTSUPPORTED
    with pytest.raises(P.WEError) as ei:
        bf.fpt_mle(5.0)                                  # past the 1.0 simulated so far
    assert ei.value.status == P.WE_EINVAL


def test_mle_without_transitions_and_with_every_walker_absorbed():
    """Degenerate campaigns: runs too short for any passage give n = 0 and an infinite estimate
    (Eq. "mld" has no maximum); walkers that all start inside the target give n = N, times 0,
    and fire nothing."""
    cfg = W.birth_death_bruteforce(n_walkers=64, tau=0.01, n_iters=2, threshold=200)
    ens = gpu_run(cfg, cfg.n_iters, resample=False)
    ens.sync()
    N, n, st, mu, sig = ens.fpt_mle()[0]
    assert N == 64 and n == 0 and st == 0.0 and np.isinf(mu) and np.isinf(sig)
    assert np.all(ens.first_passage(0) == -1.0)
    cfg2 = W.birth_death_bruteforce(n_walkers=32, tau=1.0, n_iters=3, threshold=50)
    ens2 = gpu_run(cfg2, cfg2.n_iters, resample=False)
    ens2.sync()
    N, n, st, mu, sig = ens2.fpt_mle()[0]
    assert N == 32 and n == 32 and st == 0.0 and mu == 0.0
    assert np.all(ens2.first_passage(0) == 0.0)
    assert int(ens2.per_iter(P.WE_OUT_EVENTS, 0).sum()) == 0
