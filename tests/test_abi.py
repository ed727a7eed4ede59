"""The C-ABI library loads, exports every entry point include/we_ssa.h declares, and its host-only
entry points (network compilation, bin maps, validation) behave -- no GPU needed."""
import ctypes
import os
import re

import numpy as np
import pytest

import paper_1303_5986_gb300 as P
import workloads as W
from oracle import oracle as O

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "we_ssa.h")


def _declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(we_[a-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1303_5986_gb300 import build
    build.build()


def test_every_declared_symbol_is_exported_and_bound():
    lib = ctypes.CDLL(P._lib.LIB_PATH)
    declared = _declared_functions()
    assert len(declared) >= 20
    for name in declared:
        assert hasattr(lib, name), name
    bound = {n for n, _, _ in P.SIGNATURES}
    assert set(declared) == bound


def test_run_config_struct_layout_matches_header():
    # offsets follow the C declaration order with natural alignment
    c = P._lib.we_run_config
    assert c.tau.offset == 0 and c.seed.offset == 16 and c.init_states.offset == 48
    assert c.tgt_threshold.offset == 120 and c.max_steps.offset == 136
    assert c.block_threads.offset == 160 and c.reweight_period.offset == 164
    assert c.n_init_per_run.offset == 168
    assert ctypes.sizeof(c) == 176


def test_status_strings_and_last_error():
    lib = P.lib()
    assert lib.we_status_string(0) == b"WE_OK"
    assert lib.we_status_string(-5) == b"WE_ESTEPCAP"
    assert lib.we_version() >= 100
    with pytest.raises(P.WEError) as ei:
        P.we_binmap_grid([0], [[0.0, 5.0, 5.0]])
    assert ei.value.status == P.WE_EINVAL
    assert b"ascend" in lib.we_last_error()


@pytest.mark.parametrize("factory", [W.birth_death, W.schlogl, W.futile_cycle, W.epigenetic_switch,
                                     lambda: W.toggle_switch([20.0, 33.3, 59.9], [41.0, 22.2, 30.1]),
                                     W.synthetic_large])
def test_folded_rate_constants_match_oracle_bits(factory):
    spec = factory()
    net = P.network_from_spec(spec)
    for p in range(spec.n_param_sets):
        onet = O.Network(spec, p)
        for j in range(spec.n_reactions):
            assert net.keff(p, j) == onet.keff(j)


def test_dependency_graph_degrees():
    net = P.network_from_spec(W.schlogl())
    assert [net.dep_degree(j) for j in range(4)] == [3, 3, 3, 3]
    tog = P.network_from_spec(W.toggle_switch([30.0], [30.0]))
    # U production changes U: U decay and V's Hill production read U
    assert tog.dep_degree(0) == 2 and tog.dep_degree(2) == 2
    syn = W.synthetic_large()
    net = P.network_from_spec(syn)
    degs = np.array([net.dep_degree(j) for j in range(syn.n_reactions)])
    assert 30 < degs.mean() < 55 and degs.max() <= 120


def test_network_validation_errors():
    bad = W.NetworkSpec(species=["X"], reactants=[[(0, 2), (0, 2)]], products=[[]], rate=[[1.0]])
    with pytest.raises(P.WEError):
        P.network_from_spec(bad)
    bad = W.NetworkSpec(species=["X"], reactants=[[]], products=[[(0, 1)]], rate=[[np.inf]])
    with pytest.raises(P.WEError):
        P.network_from_spec(bad)
    hill_with_reactant = W.NetworkSpec(species=["X"], reactants=[[(0, 1)]], products=[[]], rate=[[1.0]],
                                       rate_law=[1], hill_species=[0], hill_K=[[1.0]], hill_n=[2])
    with pytest.raises(P.WEError):
        P.network_from_spec(hill_with_reactant)


def test_config_validation_without_gpu():
    cfg = W.schlogl_mfpt_we(n_iters=4)
    net = P.network_from_spec(cfg.network)
    bm = P.we_binmap_grid(cfg.bins.species, cfg.bins.edges)
    c, keep = P.run_config_from(cfg)
    assert P.we_ensemble_workspace_bytes(net, bm, c) > 0
    c.tau = -1.0
    with pytest.raises(P.WEError):
        P.we_ensemble_workspace_bytes(net, bm, c)
    c.tau = 0.05
    c.m_targ = 0
    with pytest.raises(P.WEError):
        P.we_ensemble_workspace_bytes(net, bm, c)


def test_reweighting_config_validation_without_gpu():
    """Steady-state reweighting: a negative period, plain propagation, or more than 1024 bins
    are refused before any device work; a valid period adds the per-run transfer matrix and
    solve scratch (16 n_bins^2 bytes and more) to the workspace."""
    cfg = W.schlogl_flux_we(reweight_period=0, n_iters=4, n_runs=3)
    net = P.network_from_spec(cfg.network)
    bm = P.we_binmap_grid(cfg.bins.species, cfg.bins.edges)
    c, keep = P.run_config_from(cfg)
    base = P.we_ensemble_workspace_bytes(net, bm, c)
    c.reweight_period = 5
    grown = P.we_ensemble_workspace_bytes(net, bm, c)
    assert grown - base >= 16 * 80 * 80 * 3
    c.reweight_period = -1
    with pytest.raises(P.WEError):
        P.we_ensemble_workspace_bytes(net, bm, c)
    c.reweight_period = 2
    c.resample = 0
    with pytest.raises(P.WEError):
        P.we_ensemble_workspace_bytes(net, bm, c)
    big = P.we_binmap_grid([0], [W.uniform_edges(0, 1, 1100)])
    c.resample = 1
    with pytest.raises(P.WEError):
        P.we_ensemble_workspace_bytes(net, big, c)


def test_resume_refuses_malformed_checkpoints_without_gpu():
    """The checkpoint is validated on the host before any device work: wrong magic, wrong run or
    species count, truncation, and reweighting data the configuration does not use."""
    cfg = W.schlogl_mfpt_we(n_iters=4, n_runs=2)
    net = P.network_from_spec(cfg.network)
    bm = P.we_binmap_grid(cfg.bins.species, cfg.bins.edges)
    c, keep = P.run_config_from(cfg)
    S = cfg.network.n_species

    def blob(magic=0x31434557, runs=2, species=S, nb=0, counts=(3, 2), cut=0):
        hdr = np.array([magic, 1, runs, species, 7, nb, cfg.m_targ, 0], dtype=np.int32).tobytes()
        body = np.array(counts, dtype=np.int32).tobytes()
        for k in counts:
            body += np.zeros(k * species, dtype=np.int32).tobytes() + np.full(k, 0.1).tobytes()
        b = hdr + body
        return np.frombuffer(b[:len(b) - cut], dtype=np.uint8)

    L = P._lib.lib()
    for bad in (blob(magic=1), blob(runs=3, counts=(1, 1, 1)), blob(species=S + 1), blob(cut=4),
                blob(nb=80), blob(counts=(0, 2))):
        h = ctypes.c_void_p()
        st = L.we_ensemble_resume(net.h, bm.h, ctypes.byref(c), ctypes.c_void_p(bad.ctypes.data), bad.nbytes,
                                  None, ctypes.byref(h))
        assert st == -1 and h.value is None, st


def test_autotune_cache_file_round_trip_without_gpu(tmp_path):
    """The autotuner's cache as a text file: entries load, save back unchanged (sorted), and a
    malformed line is refused."""
    src = tmp_path / "tune.txt"
    src.write_text("NVIDIA_GB300 1 4 16000 20 3 128\nNVIDIA_GB300 2 6 57600 8 1 64\n")
    P.autotune_cache_clear()
    P.autotune_cache_load(src)
    out = tmp_path / "out.txt"
    P.autotune_cache_save(out)
    assert sorted(out.read_text().splitlines()) == sorted(src.read_text().splitlines())
    bad = tmp_path / "bad.txt"
    bad.write_text("NVIDIA_GB300 1 4 16000 20 9 128\n")
    with pytest.raises(P.WEError):
        P.autotune_cache_load(bad)
    with pytest.raises(P.WEError):
        P.autotune_cache_load(tmp_path / "missing.txt")
    P.autotune_cache_clear()
    P.autotune_cache_save(out)
    assert out.read_text() == ""


def test_run_config_marshalling_reads_back():
    """run_config_from writes a run description into the C struct field by field: scalars,
    the per-run arrays behind its pointers (initial walkers and weights, target thresholds,
    parameter sets), the target clauses, and the reweighting period, which plain propagation
    (resample off) forces to 0."""
    cfg = W.toggle_batch_we(n_runs=4, n_iters=7, seed=123)
    cfg.reweight_period = 3
    c, keep = P.run_config_from(cfg)
    assert (c.tau, c.m_targ, c.n_runs, c.seed, c.record_iters) == (0.1, 8, 4, 123, 7)
    assert (c.hist_species, c.hist_len, c.reweight_period) == (cfg.hist_species, cfg.hist_len, 3)
    ist, iw = np.asarray(cfg.init_states), np.asarray(cfg.init_weights)
    assert c.n_init == ist.shape[1]
    n_st = ist.size
    assert np.array_equal(np.ctypeslib.as_array(c.init_states, shape=(n_st,)), ist.ravel())
    assert np.array_equal(np.ctypeslib.as_array(c.init_weights, shape=(iw.size,)), iw.ravel())
    assert c.feedback == 1 and c.n_clauses == 2
    assert [c.tgt_species[k] for k in range(2)] == list(cfg.target.species)
    assert [c.tgt_op[k] for k in range(2)] == list(cfg.target.op)
    thr = np.asarray(cfg.target.threshold)
    assert np.array_equal(np.ctypeslib.as_array(c.tgt_threshold, shape=(thr.size,)), thr.ravel())
    if cfg.param_set is not None:
        ps = np.asarray(cfg.param_set)
        assert np.array_equal(np.ctypeslib.as_array(c.param_set, shape=(ps.size,)), ps)
    plain, keep2 = P.run_config_from(cfg, resample=False)
    assert plain.reweight_period == 0 and plain.resample == 0


def test_every_run_description_check_is_made_on_the_host():
    """Each malformed field of a run description is refused with WE_EINVAL before any device
    work (through the host-only workspace-size call, so no GPU is needed): an empty initial
    population, capacity below it, record slots, negative first iteration, target clauses
    (count, species, operator), histogram species, per-run initial counts, parameter sets,
    initial counts and weights out of range."""
    import ctypes as C
    cfg = W.toggle_batch_we(n_runs=2, n_iters=4)
    net = P.network_from_spec(cfg.network)
    bm = P.we_binmap_grid(cfg.bins.species, cfg.bins.edges)

    def fresh():                       # the config's arrays may be the description's own
        import copy
        cc = copy.deepcopy(cfg)
        c, keep = P.run_config_from(cc)
        keep["cfg"] = cc
        return c, keep

    c, keep = fresh()
    assert P.we_ensemble_workspace_bytes(net, bm, c) > 0
    assert c.n_init == 8                # eight initial walkers per run
    S = len(cfg.network.fixed_count)
    cases = {
        "n_init 0": lambda c, k: setattr(c, "n_init", 0),
        "capacity below n_init": lambda c, k: setattr(c, "capacity", c.n_init - 1),
        "record_iters 0": lambda c, k: setattr(c, "record_iters", 0),
        "first_iter < 0": lambda c, k: setattr(c, "first_iter", -1),
        "no clauses": lambda c, k: setattr(c, "n_clauses", 0),
        "too many clauses": lambda c, k: setattr(c, "n_clauses", 5),
        "clause species": lambda c, k: c.tgt_species.__setitem__(0, S),
        "clause operator": lambda c, k: c.tgt_op.__setitem__(0, 7),
        "histogram species": lambda c, k: setattr(c, "hist_species", S),
        "param set": lambda c, k: k["ps"].__setitem__(0, 99),
        "negative count": lambda c, k: k["ist"].__setitem__((0, 0, 0), -1),
        "count too large": lambda c, k: k["ist"].__setitem__((0, 0, 0), 1 << 30),
        "negative weight": lambda c, k: k["iw"].__setitem__((0, 0), -1.0),
        "NaN weight": lambda c, k: k["iw"].__setitem__((0, 0), float("nan")),
        "infinite weight": lambda c, k: k["iw"].__setitem__((0, 0), float("inf")),
    }
    for name, mutate in cases.items():
        c, keep = fresh()
        mutate(c, keep)
        with pytest.raises(P.WEError) as e:
            P.we_ensemble_workspace_bytes(net, bm, c)
        assert e.value.status == -1, name
    # per-run initial counts, given through the raw field
    c, keep = fresh()
    bad = np.array([0, 1], dtype=np.int32)
    c.n_init_per_run = bad.ctypes.data_as(C.POINTER(C.c_int32))
    with pytest.raises(P.WEError):
        P.we_ensemble_workspace_bytes(net, bm, c)
    ok = np.array([1, c.n_init], dtype=np.int32)
    c.n_init_per_run = ok.ctypes.data_as(C.POINTER(C.c_int32))
    assert P.we_ensemble_workspace_bytes(net, bm, c) > 0
