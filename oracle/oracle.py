"""ctypes wrapper of the plain C oracle (we_oracle.c).  TEST INFRASTRUCTURE ONLY.

Every function forwards to the C code, which cites the passage of arXiv:1303.5986 it follows;
this module only marshals numpy arrays.  Batched configurations run one run at a time.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

_I32P = C.POINTER(C.c_int32)
_F64P = C.POINTER(C.c_double)
_I64P = C.POINTER(C.c_int64)

STATUS = {0: "OK", -1: "EINVAL", -2: "ENOMEM", -4: "EOVERFLOW", -5: "ESTEPCAP"}
MAX_COUNT = 2097151


class NetworkIn(C.Structure):
    _fields_ = [("n_species", C.c_int32), ("n_reactions", C.c_int32),
                ("reac_ptr", _I32P), ("reac_species", _I32P), ("reac_mult", _I32P),
                ("prod_ptr", _I32P), ("prod_species", _I32P), ("prod_mult", _I32P),
                ("rate", _F64P), ("rate_law", _I32P), ("hill_species", _I32P),
                ("hill_K", _F64P), ("hill_n", _I32P), ("fixed_count", _I32P)]


class WEConfigC(C.Structure):
    _fields_ = [("tau", C.c_double), ("m_targ", C.c_int32), ("n_iters", C.c_int32),
                ("first_iter", C.c_int32), ("seed", C.c_uint64), ("run_id", C.c_uint32),
                ("n_init", C.c_int32), ("init_states", _I32P), ("init_weights", _F64P),
                ("bin_ndim", C.c_int32), ("bin_species", C.c_int32 * 4),
                ("bin_nbins", C.c_int32 * 4), ("bin_edges", _F64P), ("feedback", C.c_int32),
                ("n_clauses", C.c_int32), ("tgt_species", C.c_int32 * 4),
                ("tgt_op", C.c_int32 * 4), ("tgt_threshold", C.c_int32 * 4),
                ("recycle_state", _I32P), ("max_steps", C.c_int64), ("capacity", C.c_int32),
                ("hist_species", C.c_int32), ("hist_len", C.c_int32), ("resample", C.c_int32),
                ("reweight_period", C.c_int32)]


class WEOut(C.Structure):
    _fields_ = [("flux_weight", _F64P), ("total_weight", _F64P), ("n_walkers", _I32P),
                ("events", _I64P), ("hist", _F64P), ("states", _I32P), ("weights", _F64P),
                ("parent", _I32P), ("t_last", _F64P), ("n_final", C.c_int32), ("status", C.c_int32),
                ("first_passage", _F64P), ("reweighted", _I32P)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = C.CDLL(path)
        L.orc_philox4x32_10.argtypes = [C.POINTER(C.c_uint32), C.POINTER(C.c_uint32), C.POINTER(C.c_uint32)]
        L.orc_philox4x32_10.restype = None
        L.orc_u01.argtypes = [C.c_uint32, C.c_uint32]
        L.orc_u01.restype = C.c_double
        L.orc_net_create.argtypes = [C.POINTER(NetworkIn), C.POINTER(C.c_void_p)]
        L.orc_net_create.restype = C.c_int
        L.orc_net_destroy.argtypes = [C.c_void_p]
        L.orc_net_keff.argtypes = [C.c_void_p, C.c_int32]
        L.orc_net_keff.restype = C.c_double
        L.orc_propensities.argtypes = [C.c_void_p, _I32P, _F64P]
        L.orc_tree_total.argtypes = [C.c_int32, _F64P]
        L.orc_tree_total.restype = C.c_double
        L.orc_tree_select.argtypes = [C.c_int32, _F64P, C.c_double]
        L.orc_tree_select.restype = C.c_int32
        L.orc_propagate.argtypes = [C.c_void_p, C.POINTER(WEConfigC), C.c_int32, C.c_int32, _I32P,
                                    _I64P, _I32P, _F64P]
        L.orc_propagate.restype = C.c_int
        L.orc_bin_of.argtypes = [C.POINTER(WEConfigC), _I32P]
        L.orc_bin_of.restype = C.c_int32
        L.orc_resample.argtypes = [C.c_int32, C.c_int32, _I32P, _F64P, _I32P, C.c_int32, C.c_int32,
                                   C.c_int32, C.c_uint64, C.c_uint32, C.c_int32, _I32P, _F64P, _I32P]
        L.orc_resample.restype = C.c_int32
        L.orc_we_run.argtypes = [C.c_void_p, C.POINTER(WEConfigC), C.POINTER(WEOut)]
        L.orc_rw_solve.argtypes = [C.c_int32, _F64P, _F64P, _F64P]
        L.orc_dg_create.argtypes = [C.c_void_p, C.POINTER(C.c_void_p)]
        L.orc_dg_create.restype = C.c_int
        L.orc_dg_destroy.argtypes = [C.c_void_p]
        L.orc_propagate_dg.argtypes = [C.c_void_p, C.POINTER(WEConfigC), C.c_int32, C.c_int32, _I32P,
                                       _I64P, _I32P, _F64P]
        L.orc_propagate_dg.restype = C.c_int
        L.orc_we_run_dg.argtypes = [C.c_void_p, C.POINTER(WEConfigC), C.POINTER(WEOut)]
        L.orc_we_run_dg.restype = C.c_int
        L.orc_rw_solve.restype = C.c_int32
        L.orc_we_run.restype = C.c_int
        _lib = L
    return _lib


def _p(a, t):
    return a.ctypes.data_as(t)


def philox(ctr, key) -> np.ndarray:
    c = (C.c_uint32 * 4)(*[int(v) & 0xffffffff for v in ctr])
    k = (C.c_uint32 * 2)(*[int(v) & 0xffffffff for v in key])
    o = (C.c_uint32 * 4)()
    lib().orc_philox4x32_10(c, k, o)
    return np.array(list(o), dtype=np.uint32)


def u01(hi: int, lo: int) -> float:
    return lib().orc_u01(int(hi) & 0xffffffff, int(lo) & 0xffffffff)


class Network:
    """The oracle's compiled form of a NetworkSpec for one parameter set."""

    def __init__(self, spec, param_set: int = 0):
        self.spec = spec
        csr = spec.csr()
        self._keep = dict(csr)
        self._keep["rate"] = np.ascontiguousarray(spec.rate[param_set % spec.n_param_sets])
        self._keep["rate_law"] = np.ascontiguousarray(spec.rate_law)
        self._keep["hill_species"] = np.ascontiguousarray(spec.hill_species)
        self._keep["hill_K"] = np.ascontiguousarray(spec.hill_K_row(param_set))
        self._keep["hill_n"] = np.ascontiguousarray(spec.hill_n)
        self._keep["fixed_count"] = np.ascontiguousarray(spec.fixed_count)
        k = self._keep
        self._in = NetworkIn(
            spec.n_species, spec.n_reactions,
            _p(k["reac_ptr"], _I32P), _p(k["reac_species"], _I32P), _p(k["reac_mult"], _I32P),
            _p(k["prod_ptr"], _I32P), _p(k["prod_species"], _I32P), _p(k["prod_mult"], _I32P),
            _p(k["rate"], _F64P), _p(k["rate_law"], _I32P), _p(k["hill_species"], _I32P),
            _p(k["hill_K"], _F64P), _p(k["hill_n"], _I32P), _p(k["fixed_count"], _I32P))
        h = C.c_void_p()
        rc = lib().orc_net_create(C.byref(self._in), C.byref(h))
        if rc != 0:
            raise ValueError(f"oracle network rejected: {STATUS.get(rc, rc)}")
        self.h = h
        self.S, self.M = spec.n_species, spec.n_reactions

    def __del__(self):
        if getattr(self, "_dg", None) is not None and _lib is not None:
            _lib.orc_dg_destroy(self._dg)
            self._dg = None
        if getattr(self, "h", None) and _lib is not None:
            _lib.orc_net_destroy(self.h)
            self.h = None

    def depgraph(self):
        """The dependency-graph CPU baseline's handle for this network (created once)."""
        if getattr(self, "_dg", None) is None:
            h = C.c_void_p()
            rc = lib().orc_dg_create(self.h, C.byref(h))
            if rc != 0:
                raise ValueError(f"dependency graph: {STATUS.get(rc, rc)}")
            self._dg = h
        return self._dg

    def keff(self, j: int) -> float:
        return lib().orc_net_keff(self.h, j)

    def propensities(self, x) -> np.ndarray:
        x = np.ascontiguousarray(x, dtype=np.int32)
        a = np.zeros(self.M)
        lib().orc_propensities(self.h, _p(x, _I32P), _p(a, _F64P))
        return a


def tree_total(a) -> float:
    a = np.ascontiguousarray(a, dtype=np.float64)
    return lib().orc_tree_total(len(a), _p(a, _F64P))


def tree_select(a, target: float) -> int:
    a = np.ascontiguousarray(a, dtype=np.float64)
    return lib().orc_tree_select(len(a), _p(a, _F64P), float(target))


def make_config(cfg, run: int = 0, n_iters: int | None = None, first_iter: int | None = None,
                resample: bool = True, init_states=None, init_weights=None, max_steps=None):
    """Fill the C config for run ``run`` of a workloads.WEConfig.  Returns (struct, keepalive)."""
    S = cfg.network.n_species
    keep = {}
    ist = cfg.init_states[run] if init_states is None else init_states
    iw = cfg.init_weights[run] if init_weights is None else init_weights
    keep["init_states"] = np.ascontiguousarray(ist, dtype=np.int32).reshape(-1, S)
    keep["init_weights"] = np.ascontiguousarray(iw, dtype=np.float64)
    keep["edges"] = np.ascontiguousarray(cfg.bins.flat_edges())
    keep["recycle"] = np.ascontiguousarray(cfg.recycle_state[run], dtype=np.int32)
    c = WEConfigC()
    c.tau = cfg.tau
    c.m_targ = cfg.m_targ
    c.n_iters = cfg.n_iters if n_iters is None else n_iters
    c.first_iter = cfg.first_iter if first_iter is None else first_iter
    c.seed = int(cfg.seed)
    c.run_id = int(cfg.run_ids[run])
    c.n_init = keep["init_states"].shape[0]
    c.init_states = _p(keep["init_states"], _I32P)
    c.init_weights = _p(keep["init_weights"], _F64P)
    c.bin_ndim = cfg.bins.ndim
    for d in range(cfg.bins.ndim):
        c.bin_species[d] = cfg.bins.species[d]
        c.bin_nbins[d] = cfg.bins.n_bins_per_dim[d]
    c.bin_edges = _p(keep["edges"], _F64P)
    if cfg.target is not None:
        c.feedback = 2 if getattr(cfg, "absorb", False) else (3 if getattr(cfg, "endpoint", False) else 1)
        c.n_clauses = len(cfg.target.species)
        for i in range(c.n_clauses):
            c.tgt_species[i] = cfg.target.species[i]
            c.tgt_op[i] = cfg.target.op[i]
            c.tgt_threshold[i] = int(cfg.target.threshold[run, i])
    c.recycle_state = _p(keep["recycle"], _I32P)
    c.max_steps = cfg.max_steps if max_steps is None else max_steps
    c.capacity = max(cfg.capacity, c.n_init)
    c.hist_species = cfg.hist_species
    c.hist_len = cfg.hist_len
    c.resample = 1 if resample else 0
    c.reweight_period = int(getattr(cfg, "reweight_period", 0) or 0)
    return c, keep


def we_run(cfg, run: int = 0, n_iters: int | None = None, first_iter: int | None = None,
           resample: bool = True, init_states=None, init_weights=None, max_steps=None,
           net: Network | None = None, depgraph: bool = False) -> dict:
    """One WE run of the paper's algorithm (Sec. II.B) for run ``run`` of the config.  With
    depgraph=True the propagation runs the dependency-graph CPU baseline instead of the
    oracle's full recomputation (same results, less work)."""
    if net is None:
        net = Network(cfg.network, int(cfg.param_set[run]))
    c, keep = make_config(cfg, run, n_iters, first_iter, resample, init_states, init_weights, max_steps)
    n = c.n_iters
    S = cfg.network.n_species
    cap = c.capacity
    o = {
        "flux_weight": np.zeros(n), "total_weight": np.zeros(n),
        "n_walkers": np.zeros(n, dtype=np.int32), "events": np.zeros(n, dtype=np.int64),
        "hist": np.zeros((n, max(cfg.hist_len, 1))), "states": np.zeros((cap, S), dtype=np.int32),
        "weights": np.zeros(cap), "parent": np.zeros(cap, dtype=np.int32), "t_last": np.zeros(cap),
        "reweighted": np.zeros(n, dtype=np.int32), "first_passage": np.zeros(cap),
    }
    out = WEOut(_p(o["flux_weight"], _F64P), _p(o["total_weight"], _F64P),
                _p(o["n_walkers"], _I32P), _p(o["events"], _I64P),
                _p(o["hist"], _F64P) if cfg.hist_len > 0 else None,
                _p(o["states"], _I32P), _p(o["weights"], _F64P), _p(o["parent"], _I32P),
                _p(o["t_last"], _F64P), 0, 0, _p(o["first_passage"], _F64P), _p(o["reweighted"], _I32P))
    if depgraph:
        lib().orc_we_run_dg(net.depgraph(), C.byref(c), C.byref(out))
    else:
        lib().orc_we_run(net.h, C.byref(c), C.byref(out))
    nf = out.n_final
    o["t_last_prev"] = o["t_last"]
    o["states"] = o["states"][:nf]
    o["weights"] = o["weights"][:nf]
    o["parent"] = o["parent"][:nf]
    o["first_passage"] = o["first_passage"][:nf]
    o["n_final"] = nf
    o["status"] = out.status
    return o


def propagate_one(cfg, x, iteration: int, slot: int, run: int = 0, net: Network | None = None,
                  max_steps=None, depgraph: bool = False):
    """SSA for one interval of one walker; returns (new_state, events, recycles, status).
    depgraph=True: the dependency-graph CPU baseline (same result)."""
    if net is None:
        net = Network(cfg.network, int(cfg.param_set[run]))
    c, keep = make_config(cfg, run, max_steps=max_steps)
    xs = np.ascontiguousarray(x, dtype=np.int32).copy()
    ev = C.c_int64(0)
    rec = C.c_int32(0)
    tl = C.c_double(0.0)
    fn = lib().orc_propagate_dg if depgraph else lib().orc_propagate
    rc = fn(net.depgraph() if depgraph else net.h, C.byref(c), iteration, slot, _p(xs, _I32P), C.byref(ev),
            C.byref(rec), C.byref(tl))
    return xs, ev.value, rec.value, rc


def bin_of(cfg, x) -> int:
    c, keep = make_config(cfg, 0)
    xs = np.ascontiguousarray(x, dtype=np.int32)
    return lib().orc_bin_of(C.byref(c), _p(xs, _I32P))


def resample(states, weights, bins, n_bins: int, m_targ: int, iteration: int, seed: int,
             run_id: int = 0, capacity: int | None = None):
    """Split/merge of one ensemble given every walker's bin; returns (states, weights, parent)."""
    states = np.ascontiguousarray(states, dtype=np.int32)
    if states.ndim == 1:
        states = states[:, None]
    n, S = states.shape
    weights = np.ascontiguousarray(weights, dtype=np.float64)
    bins = np.ascontiguousarray(bins, dtype=np.int32)
    cap = capacity if capacity is not None else max(n, m_targ * n_bins)
    os_ = np.zeros((cap, S), dtype=np.int32)
    ow = np.zeros(cap)
    op = np.zeros(cap, dtype=np.int32)
    m = lib().orc_resample(n, S, _p(states, _I32P), _p(weights, _F64P), _p(bins, _I32P), n_bins,
                           m_targ, iteration, int(seed), int(run_id), cap, _p(os_, _I32P),
                           _p(ow, _F64P), _p(op, _I32P))
    if m < 0:
        raise RuntimeError(f"oracle resample failed: {STATUS.get(m, m)}")
    return os_[:m], ow[:m], op[:m]


def rw_solve(F, cb):
    """Steady-state reweighting factors per bin from accumulated transfers F[end, start] and the
    current bin weights (Sec. II.B.2, Eq. "ss"); returns (status, factors)."""
    F = np.ascontiguousarray(F, dtype=np.float64)
    nb = F.shape[0]
    cb = np.ascontiguousarray(cb, dtype=np.float64)
    fac = np.zeros(nb)
    st = lib().orc_rw_solve(nb, _p(F, _F64P), _p(cb, _F64P), _p(fac, _F64P))
    return st, fac


def we_run_all(cfg, **kw) -> list:
    """Every run of a (batched) config, one after another."""
    return [we_run(cfg, r, **kw) for r in range(cfg.n_runs)]


def mfpt_from_flux(flux_weight, tau: float, discard: int = 0) -> float:
    """MFPT = 1 / steady-state flux (Eq. "mfpt"), the flux being recycled weight per unit time
    averaged over the iterations after ``discard``."""
    f = np.asarray(flux_weight, dtype=np.float64)[discard:]
    mean_flux = f.mean() / tau
    return np.inf if mean_flux == 0 else 1.0 / mean_flux


if __name__ == "__main__":  # pragma: no cover
    print(os.path.abspath(_build.build()))
