"""Learned bins for WE: harvest walker states from a plain WE run, label them by first passage
with the SSA kernel, fit the progress coordinate with the training kernels, and place bin
edges on it.  WE stays unbiased under any binning (Sec. II.B); choosing bins automatically is
the open problem of Sec. IV.B.  Every step runs in the library's kernels; this module only
moves arrays between the calls.
"""
import numpy as np

from .api import MLP, first_passage_labels, we_mlp_coordinate_edges, we_mlp_create_init


def harvest_states(ens, n_iters: int, every: int = 1, runs=None) -> np.ndarray:
    """Advance `ens` by n_iters WE iterations and collect the walkers' states (after each
    resampling, every `every` iterations, over the given runs).  Returns (n, S) int32."""
    out = []
    for it in range(n_iters):
        ens.step(1)
        if (it + 1) % every == 0:
            if runs is None:
                out.append(ens.states(-1))
            else:
                out.extend(ens.states(r) for r in runs)
    return np.concatenate(out, axis=0) if out else np.zeros((0, ens.n_species), np.int32)


def fit_coordinate(net, states, target, recycle_state, horizon: float, hidden: int = 64,
                   steps: int = 2000, batch: int = 4096, lr: float = 3e-3, seed: int = 0,
                   param_set: int = 0, max_states: int = 2_000_000, stream=None, timings=None):
    """Label `states` by first passage into `target` within `horizon` (one SSA shot each) and
    train a fresh MLP on them.  Returns (mlp, device states, device labels, losses).  With a dict
    `timings`, the wall time of the labelling and of the training (device synchronised) go in
    'labels_s' and 'train_s'."""
    import time
    import torch
    st = np.ascontiguousarray(states, dtype=np.int32)
    rng = np.random.default_rng(seed)
    if len(st) > max_states:
        st = st[rng.choice(len(st), size=max_states, replace=False)]
    st = st[rng.permutation(len(st))]
    t0 = time.perf_counter()
    labels = first_passage_labels(net, st, horizon, target, recycle_state, seed=seed,
                                  param_set=param_set, stream=stream)
    xs = torch.as_tensor(st, device=labels.device)
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    mlp = we_mlp_create_init(st.shape[1], hidden, seed)
    losses = mlp.train(xs, labels, steps, batch, lr, stream=stream)
    torch.cuda.synchronize()
    if timings is not None:
        timings["labels_s"] = t1 - t0
        timings["train_s"] = time.perf_counter() - t1
    return mlp, xs, labels, losses


def coordinate_edges(mlp: MLP, states_dev, n_bins: int, lo_q: float = 0.001, stream=None) -> np.ndarray:
    """n_bins equal intervals of z (with the BF16 weights that the bin map will use) from a low
    order statistic of z over the given states to its maximum, computed by the library."""
    return we_mlp_coordinate_edges(mlp, states_dev, n_bins, lo_q, stream=stream)


__all__ = ["harvest_states", "fit_coordinate", "coordinate_edges"]
