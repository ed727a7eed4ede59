"""The target set checked at the end of each interval only (WE_FEEDBACK_ENDPOINT: B checked at a
prescribed time step, Sec. IV) on the GPU, bit for bit against the oracle's same mode: walkers
found in B when the interval ends are put in the recycle state, counted as flux and binned
there; crossings into B and back within an interval are not counted."""
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


def _parity(cfg, n_iters, resample=True, **kw):
    ens = gpu_run(cfg, n_iters, resample=resample, **kw)
    ens.sync()
    for r in range(cfg.n_runs):
        assert_run_parity(gpu_outputs(ens, r), oracle_run(cfg, r, n_iters=n_iters, resample=resample),
                          label=f"{cfg.name} run {r} {kw}")
    return ens


@pytest.mark.parametrize("mapping,block", [(P.WE_MAP_AUTO, 0), (P.WE_MAP_AUTO, 32),
                                           (P.WE_MAP_THREAD, 0), (P.WE_MAP_WARP, 0)])
def test_birth_death_we_end_of_interval_check(mapping, block):
    cfg = W.birth_death_we(n_iters=50, target=130)
    cfg.endpoint = True
    ens = _parity(cfg, 50, mapping=mapping, block_threads=block)
    assert ens.per_iter(P.WE_OUT_FLUX).sum() > 0


@pytest.mark.parametrize("block", [0, 32])
def test_schlogl_mfpt_end_of_interval_check(block):
    cfg = W.schlogl_mfpt_we(n_iters=40, n_runs=3)
    cfg.endpoint = True
    _parity(cfg, 40, block_threads=block)


@pytest.mark.parametrize("mapping", [P.WE_MAP_AUTO, P.WE_MAP_THREAD, P.WE_MAP_WARP])
def test_pure_birth_plain_end_of_interval_check(mapping):
    """Plain SSA walkers of a pure-birth process, recycled to 0 when X >= 5 at an interval's end:
    the flux counts each walker once per interval at most, and every walker ends below 5."""
    R, n = 2, 5
    net = W.NetworkSpec(species=["X"], reactants=[[]], products=[[(0, 1)]], rate=[[1.0]])
    tgt = W.Target(species=[0], op=[W.configs.OP_GE], threshold=np.full((R, 1), n, dtype=np.int32))
    cfg = W.bruteforce_fpt(net, [0], tgt, 200, 0.5, 60, n_runs=R, name="pure_birth")
    cfg.absorb = False
    cfg.endpoint = True
    ens = _parity(cfg, 60, resample=False, mapping=mapping)
    for r in range(R):
        assert np.all(ens.states(r)[:, 0] < n)
        nrec = ens.get(P.WE_OUT_NREC, r)
        assert set(np.unique(nrec)) <= {0, 1}


def test_recycle_state_inside_the_target_is_refused():
    cfg = W.birth_death_we(n_iters=2, target=101)
    cfg.endpoint = True
    cfg.recycle_state = np.full((1, 1), 105, dtype=np.int32)
    with pytest.raises(P.WEError) as ei:
        gpu_run(cfg, 1)
    assert ei.value.status == P.WE_EINVAL
