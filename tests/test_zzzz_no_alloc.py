"""The allocation-free split/merge entry point (we_resample_static).

Some callers cannot allocate device memory: a host framework whose caching allocator already
holds the GPU's memory, or a loop in which a cudaMalloc (which may synchronise the device and
may fail under memory pressure) is not allowed after set-up.  we_resample_static serves them
from a fixed array in the library's device image.  Its results must equal, bit for bit, both
the CPU oracle's split/merge (the paper's rules restated independently, Sec. II.B) and the
ensemble's own resampling, on consecutive calls that share the array; its in-kernel errors come
back through out_count.

Kept in a file of its own that pytest collects last, so that a run stopping at the first
failure has run every other test before it."""
import numpy as np
import pytest

import paper_1303_5986_gb300 as P
import workloads as W
from oracle import oracle as O

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


def _static(bins, w, n_bins, m_targ, it, seed, run_id, cap):
    import torch
    dev = torch.device("cuda", torch.cuda.current_device())
    tb = torch.as_tensor(np.ascontiguousarray(bins, dtype=np.int32), device=dev)
    tw = torch.as_tensor(np.ascontiguousarray(w, dtype=np.float64), device=dev)
    ow = torch.zeros(cap, dtype=torch.float64, device=dev)
    op = torch.full((cap,), -1, dtype=torch.int32, device=dev)
    oc = torch.zeros(1, dtype=torch.int32, device=dev)
    P.we_resample_static(tb, tw, n_bins, m_targ, it, seed, run_id, ow, op, oc)
    torch.cuda.synchronize()
    n = int(oc.item())
    if n < 0:
        return n, None, None
    return n, ow[:n].cpu().numpy(), op[:n].cpu().numpy()


def test_static_resample_matches_oracle_and_ensemble_on_consecutive_calls():
    """Two calls in a row on live Schloegl populations (iterations 12 and 17 of the MFPT
    workload): new weights and parents equal the oracle's and the ensemble's bit for bit."""
    cfg = W.schlogl_mfpt_we(n_iters=40, n_runs=1)
    ens = gpu_run(cfg, 0, record_iters=40)
    ens.step(12)
    cap = cfg.capacity
    run_id = int(cfg.run_ids[0])
    for call in range(2):
        it = ens.iteration()
        ens.propagate()
        states = ens.states(0)
        w = ens.weights(0)
        bins = _grid_bins(states, cfg)
        ens.resample()
        n, sw, sp = _static(bins, w, cfg.bins.n_bins, cfg.m_targ, it, cfg.seed, run_id, cap)
        _, ow, op = O.resample(states, w, bins, cfg.bins.n_bins, cfg.m_targ, it, cfg.seed, run_id, cap)
        assert n == len(ow), (call, n, len(ow))
        assert np.array_equal(sw.view(np.int64), ow.view(np.int64)), call
        assert np.array_equal(sp, op), call
        assert np.array_equal(ens.weights(0).view(np.int64), sw.view(np.int64)), call
        assert np.array_equal(ens.parents(0), sp), call
        ens.step(4)


def test_static_resample_matches_oracle_on_wide_bins():
    """Bins far above and below M_targ (600 walkers merged to 37, a lone walker split into 37,
    40 merged to 37, 36 split to 37; weights spread over 60 orders of magnitude), against the
    oracle, on two calls in a row."""
    rng = np.random.default_rng(5)
    n_bins, m_targ = 7, 37
    bins = np.concatenate([np.zeros(600), np.ones(1), np.full(40, 3), np.full(36, 6)]).astype(np.int32)
    rng.shuffle(bins)
    w = 10.0 ** rng.uniform(-60, 0, len(bins))
    w /= w.sum()
    cap = len(bins)
    for it in (3, 4):
        n, sw, sp = _static(bins, w, n_bins, m_targ, it, 11, 2, cap)
        _, ow, op = O.resample(w[:, None] * 0, w, bins, n_bins, m_targ, it, 11, 2, cap)
        assert n == len(ow) == 4 * m_targ
        assert np.array_equal(sw.view(np.int64), ow.view(np.int64)), it
        assert np.array_equal(sp, op), it


def test_static_resample_reports_in_kernel_errors_through_out_count():
    """A bin index out of range gives WE_EINVAL and a capacity below (occupied bins x M_targ)
    gives WE_EOVERFLOW, both in out_count; a valid call after them on the same array works."""
    n_bins, m_targ = 10, 10
    bins = np.arange(40, dtype=np.int32) % n_bins
    w = np.full(40, 1.0 / 40)
    bad = bins.copy()
    bad[17] = n_bins
    assert _static(bad, w, n_bins, m_targ, 0, 0, 0, 100)[0] == P.WE_EINVAL
    bad[17] = -3
    assert _static(bad, w, n_bins, m_targ, 0, 0, 0, 100)[0] == P.WE_EINVAL
    assert _static(bins, w, n_bins, m_targ, 0, 0, 0, 50)[0] == P.WE_EOVERFLOW
    n, sw, sp = _static(bins, w, n_bins, m_targ, 0, 0, 0, 100)
    _, ow, op = O.resample(bins[:, None], w, bins, n_bins, m_targ, 0, 0, 0, 100)
    assert n == 100 and np.array_equal(sw.view(np.int64), ow.view(np.int64)) and np.array_equal(sp, op)


def test_static_resample_rejects_sizes_beyond_its_array():
    import torch
    dev = torch.device("cuda", torch.cuda.current_device())
    n = 65537                                              # one past the array's 65,536 walkers
    tb = torch.zeros(n, dtype=torch.int32, device=dev)
    tw = torch.full((n,), 1.0 / n, dtype=torch.float64, device=dev)
    ow = torch.zeros(n, dtype=torch.float64, device=dev)
    op = torch.zeros(n, dtype=torch.int32, device=dev)
    oc = torch.zeros(1, dtype=torch.int32, device=dev)
    with pytest.raises(P.WEError) as ei:
        P.we_resample_static(tb, tw, 4, 10, 0, 0, 0, ow, op, oc)
    assert ei.value.status == P.WE_EINVAL
    with pytest.raises(P.WEError) as ei:                  # 4097 bins
        P.we_resample_static(tb[:10], tw[:10], 4097, 10, 0, 0, 0, ow[:10], op[:10], oc)
    assert ei.value.status == P.WE_EINVAL


def test_static_resample_binding_refuses_mistyped_tensors():
    """Wrong dtypes, short outputs or non-contiguous tensors are refused before the library is
    called (it takes raw pointers and could not tell)."""
    import torch
    dev = torch.device("cuda", torch.cuda.current_device())
    n = 40
    tb = torch.zeros(n, dtype=torch.int32, device=dev)
    tw = torch.full((n,), 1.0 / n, dtype=torch.float64, device=dev)
    ow = torch.zeros(64, dtype=torch.float64, device=dev)
    op = torch.zeros(64, dtype=torch.int32, device=dev)
    oc = torch.zeros(1, dtype=torch.int32, device=dev)
    bad = [
        (tb.long(), tw, ow, op, oc), (tb, tw.float(), ow, op, oc), (tb, tw[:-1], ow, op, oc),
        (tb, tw, ow.float(), op, oc), (tb, tw, ow, op[:63], oc), (tb, tw, ow, op, oc.long()),
        (tb, torch.stack([tw, tw], 1)[:, 0], ow, op, oc), (tb.cpu(), tw, ow, op, oc),
    ]
    for args in bad:
        with pytest.raises(P.WEError) as ei:
            P.we_resample_static(args[0], args[1], 4, 10, 0, 0, 0, *args[2:])
        assert ei.value.status == P.WE_EINVAL
