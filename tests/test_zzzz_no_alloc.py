"""The allocation-free split/merge entry point (we_resample_static), for callers that may not
allocate device memory, must give exactly what the ensemble's own resampling gives.

Kept in a file of its own that pytest collects last."""
import numpy as np
import pytest

import paper_1303_5986_gb300 as P
import workloads as W

from gpu_helpers import gpu_run

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1303_5986_gb300 import build
    build.build()


def _grid_bins(states, cfg):
    e = np.asarray(cfg.bins.edges[0], dtype=np.float64)
    v = states[:, cfg.bins.species[0]].astype(np.float64)
    return np.clip(np.searchsorted(e, v, side="right") - 1, 0, len(e) - 2).astype(np.int32)


def test_static_resample_matches_ensemble_resample_on_consecutive_calls():
    import torch
    cfg = W.schlogl_mfpt_we(n_iters=40, n_runs=1)
    ens = gpu_run(cfg, 0, record_iters=40)
    ens.step(12)
    dev = torch.device("cuda", torch.cuda.current_device())
    cap = cfg.capacity
    for call in range(2):
        it = ens.iteration()
        ens.propagate()
        states = ens.states(0)
        w = ens.weights(0)
        bins = _grid_bins(states, cfg)
        ens.resample()
        ref_w = ens.weights(0)
        ref_p = ens.parents(0)
        tb = torch.as_tensor(bins, device=dev)
        tw = torch.as_tensor(w, device=dev)
        ow = torch.zeros(cap, dtype=torch.float64, device=dev)
        op = torch.full((cap,), -1, dtype=torch.int32, device=dev)
        oc = torch.zeros(1, dtype=torch.int32, device=dev)
        P.we_resample_static(tb, tw, cfg.bins.n_bins, cfg.m_targ, it, cfg.seed, int(cfg.run_ids[0]),
                             ow, op, oc)
        torch.cuda.synchronize()
        n = int(oc.item())
        assert n == len(ref_w), (call, n, len(ref_w))
        assert np.array_equal(ow[:n].cpu().numpy().view(np.int64), ref_w.view(np.int64)), call
        assert np.array_equal(op[:n].cpu().numpy(), ref_p), call
        ens.step(4)


def test_static_resample_rejects_sizes_beyond_its_array():
    import torch
    dev = torch.device("cuda", torch.cuda.current_device())
    n = 65537
    tb = torch.zeros(n, dtype=torch.int32, device=dev)
    tw = torch.full((n,), 1.0 / n, dtype=torch.float64, device=dev)
    ow = torch.zeros(n, dtype=torch.float64, device=dev)
    op = torch.zeros(n, dtype=torch.int32, device=dev)
    oc = torch.zeros(1, dtype=torch.int32, device=dev)
    with pytest.raises(P.WEError) as ei:
        P.we_resample_static(tb, tw, 4, 10, 0, 0, 0, ow, op, oc)
    assert ei.value.status == P.WE_EINVAL
