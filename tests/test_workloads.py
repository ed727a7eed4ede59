"""The synthetic workloads have the stated shapes: bins, walkers per bin, tau, start states,
targets and rate constants of the benchmark configurations (1-D birth-death, Schloegl MFPT,
the batched toggle sweep, the 354 x 3680 synthetic network) and of the paper's runs they stand
for.  Host logic only; no GPU."""
import numpy as np
import pytest

import workloads as W
from workloads.configs import OP_GE


def _order(side):
    return sum(m for _, m in side)


def test_birth_death_and_schloegl_runs():
    c = W.birth_death_we()
    e = np.asarray(c.bins.edges[0])
    assert len(e) - 1 == 61 and e[0] == 0 and e[60] == 300 and np.isinf(e[-1])
    assert np.all(np.diff(e[:61]) == 5)
    assert (c.m_targ, c.tau, int(np.asarray(c.x0).ravel()[0]), c.n_iters) == (10, 0.1, 100, 200)
    assert np.allclose(c.network.rate[0], [10.0, 0.1])

    c = W.schlogl_mfpt_we()
    e = np.asarray(c.bins.edges[0])
    assert len(e) - 1 == 80 and e[0] == 0 and e[-1] == 800 and np.all(np.diff(e) == 10)
    assert (c.m_targ, c.tau, c.n_iters) == (20, 0.05, 1000)
    assert int(np.asarray(c.x0).ravel()[0]) == 85
    assert list(c.target.op) == [OP_GE] and int(np.asarray(c.target.threshold).ravel()[0]) == 550
    net = c.network
    assert [_order(r) for r in net.reactants] == [3, 3, 1, 1]   # A+2X, 3X, B, X
    fixed = np.asarray(net.fixed_count)
    assert sorted(fixed[fixed >= 0].tolist()) == [100000, 200000]


def test_toggle_sweep():
    c = W.toggle_batch_we()
    assert c.n_runs == 64 and c.m_targ == 8 and c.n_iters == 500
    for e in c.bins.edges:
        e = np.asarray(e)
        assert len(e) - 1 == 30 and np.isinf(e[-1]) and np.all(np.diff(e[:-1]) == 4)
    a_u, a_v = c.notes["a_u"], c.notes["a_v"]
    for a in (a_u, a_v):
        assert a.shape == (64,) and np.all((a >= 20) & (a <= 60)) and len(np.unique(a)) == 64
    x0 = np.asarray(c.x0)
    assert np.array_equal(x0[:, 0], np.rint(a_u).astype(np.int32)) and np.all(x0[:, 1] == 0)
    thr = np.asarray(c.target.threshold)
    assert np.array_equal(thr[:, 0], np.ceil(a_v / 2).astype(np.int32))
    assert np.array_equal(thr[:, 1], np.floor(a_u / 4).astype(np.int32))
    assert len(c.network.reactants) == 6 and c.network.rate.shape[0] == 64


def test_synthetic_network_shape():
    c = W.synthetic_large_we()
    net = c.network
    assert len(net.species) == 354 and len(net.reactants) == 3680
    orders = np.array([_order(r) for r in net.reactants])
    assert (orders == 1).sum() == 2208 and (orders == 2).sum() == 1472
    assert all(_order(r) == _order(p) for r, p in zip(net.reactants, net.products))   # conserving
    k = net.rate[0]
    assert np.all((k >= 1e-4) & (k <= 1e1))
    lk = np.log10(k)                                   # log-uniform: flat histogram over 5 decades
    hist, _ = np.histogram(lk, bins=5, range=(-4, 1))
    assert hist.min() > 0.8 * len(k) / 5
    init = np.asarray(c.init_states)
    assert init.shape == (1, 4096, 354) and init.min() >= 0 and init.max() <= 200
    assert np.allclose(np.asarray(c.init_weights).sum(), 1.0)
    e = np.asarray(c.bins.edges[0])
    assert c.bins.species == [0] and len(e) - 1 == 50 and e[-1] == 200 and c.tau == 0.01
    # deterministic for its seed
    again = W.synthetic_large_we().network
    assert np.array_equal(again.rate, net.rate) and again.reactants == net.reactants
