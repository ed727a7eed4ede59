"""Shared helpers of the GPU tests: run a configuration through the C ABI and through the CPU
oracle, and compare."""
import numpy as np

import paper_1303_5986_gb300 as P
from oracle import oracle as O


def gpu_run(cfg, n_iters=None, resample=True, mapping=P.WE_MAP_AUTO, block_threads=0,
            max_steps=None, init_states=None, init_weights=None, first_iter=None, workspace="torch",
            record_iters=None, bins=None, capacity=None):
    n_iters = cfg.n_iters if n_iters is None else n_iters
    net = P.network_from_spec(cfg.network)
    bm = P.we_binmap_grid(cfg.bins.species, cfg.bins.edges) if bins is None else bins
    rec = max(n_iters, 1) if record_iters is None else record_iters
    c, keep = P.run_config_from(cfg, record_iters=rec, resample=resample, mapping=mapping,
                                block_threads=block_threads, max_steps=max_steps,
                                init_states=init_states, init_weights=init_weights,
                                first_iter=first_iter, capacity=capacity)
    ens = P.we_ensemble_create(net, bm, c, keep, workspace=workspace)
    ens._net, ens._bm = net, bm
    if n_iters:
        ens.step(n_iters)
    return ens


def gpu_outputs(ens, run, hist=True):
    o = {
        "states": ens.states(run), "weights": ens.weights(run), "parent": ens.parents(run),
        "flux_weight": ens.per_iter(P.WE_OUT_FLUX, run), "total_weight": ens.per_iter(P.WE_OUT_TOTAL_W, run),
        "n_walkers": ens.per_iter(P.WE_OUT_NWALKERS, run), "events": ens.per_iter(P.WE_OUT_EVENTS, run),
        "status": int(ens.status()[run]),
        "near_tau": ens.per_iter(P.WE_OUT_NEAR_TAU, run),
    }
    if hist:
        o["hist"] = ens.per_iter(P.WE_OUT_HIST, run)
    return o


def assert_run_parity(g, o, label="", check_parent=True):
    """Bit-exact trajectories (counts, weights, order, parents, event counts); observables
    accumulated by device atomics within 1e-12 relative."""
    assert g["status"] == o["status"], (label, g["status"], o["status"])
    # no interval ended within 2^-40 tau of an event, where a stop decision could flip
    assert int(np.sum(g.get("near_tau", 0))) == 0, (label, "near-tau stop decisions")
    assert np.array_equal(g["n_walkers"], o["n_walkers"]), label
    assert np.array_equal(g["events"], o["events"]), label
    assert g["states"].shape == o["states"].shape, (label, g["states"].shape, o["states"].shape)
    assert np.array_equal(g["states"], o["states"]), label
    assert np.array_equal(g["weights"].view(np.int64), o["weights"].view(np.int64)), label
    if check_parent:
        assert np.array_equal(g["parent"], o["parent"]), label
    np.testing.assert_allclose(g["flux_weight"], o["flux_weight"], rtol=1e-12, atol=1e-300, err_msg=label)
    np.testing.assert_allclose(g["total_weight"], o["total_weight"], rtol=1e-12, atol=0, err_msg=label)
    if "hist" in g and "hist" in o:
        np.testing.assert_allclose(g["hist"], o["hist"][:, :g["hist"].shape[1]], rtol=1e-12, atol=1e-300,
                                   err_msg=label)


def oracle_run(cfg, run, n_iters=None, resample=True, max_steps=None, init_states=None,
               init_weights=None, first_iter=None):
    return O.we_run(cfg, run, n_iters=n_iters, resample=resample, max_steps=max_steps,
                    init_states=None if init_states is None else init_states[run],
                    init_weights=None if init_weights is None else init_weights[run],
                    first_iter=first_iter)
