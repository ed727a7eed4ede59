"""Thin Python binding of the C ABI (include/we_ssa.h): argument marshalling only.

Every computation happens in libwe_ssa.so (CUDA kernels for sm_103a).  PyTorch is used for
device memory (the ensemble workspace) and for the CUDA stream; numpy for host arrays.
Function names follow the C entry points; the small classes only own the handles.
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import _lib as L
from ._lib import check, lib, we_run_config

_I32P = C.POINTER(C.c_int32)
_U32P = C.POINTER(C.c_uint32)
_F64P = C.POINTER(C.c_double)


def _i32(a):
    return None if a is None else np.ascontiguousarray(a, dtype=np.int32)


def _f64(a):
    return None if a is None else np.ascontiguousarray(a, dtype=np.float64)


def _ptr(a, t):
    return None if a is None else a.ctypes.data_as(t)


def _stream_handle(stream=None):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return C.c_void_p(stream.cuda_stream)


class Network:
    def __init__(self, handle, n_species, n_reactions, n_param_sets):
        self.h = handle
        self.n_species, self.n_reactions, self.n_param_sets = n_species, n_reactions, n_param_sets

    def __del__(self):
        if getattr(self, "h", None) and L._lib is not None:
            L._lib.we_network_destroy(self.h)
            self.h = None

    def keff(self, p: int, j: int) -> float:
        v = C.c_double()
        check(lib().we_network_keff(self.h, p, j, C.byref(v)))
        return v.value

    def dep_degree(self, j: int) -> int:
        v = C.c_int32()
        check(lib().we_network_dep_degree(self.h, j, C.byref(v)))
        return v.value


def we_network_create(n_species, n_reactions, reac_ptr, reac_species, reac_mult, prod_ptr,
                      prod_species, prod_mult, rate, rate_law=None, hill_species=None,
                      hill_K=None, hill_n=None, fixed_count=None) -> Network:
    rate = np.atleast_2d(_f64(rate))
    nps = rate.shape[0]
    arrs = [_i32(reac_ptr), _i32(reac_species), _i32(reac_mult), _i32(prod_ptr), _i32(prod_species),
            _i32(prod_mult)]
    hk = None if hill_K is None else np.atleast_2d(_f64(hill_K))
    h = C.c_void_p()
    check(lib().we_network_create(
        n_species, n_reactions, *[_ptr(a, _I32P) for a in arrs], nps, _ptr(rate, _F64P),
        _ptr(_i32(rate_law), _I32P), _ptr(_i32(hill_species), _I32P),
        0 if hk is None else hk.shape[0], _ptr(hk, _F64P), _ptr(_i32(hill_n), _I32P),
        _ptr(_i32(fixed_count), _I32P), C.byref(h)))
    return Network(h, n_species, n_reactions, nps)


def network_from_spec(spec) -> Network:
    """Marshal a network description (reaction lists, rates, laws) into we_network_create."""
    csr = spec.csr()
    return we_network_create(spec.n_species, spec.n_reactions, csr["reac_ptr"], csr["reac_species"],
                             csr["reac_mult"], csr["prod_ptr"], csr["prod_species"], csr["prod_mult"],
                             spec.rate, spec.rate_law, spec.hill_species, spec.hill_K, spec.hill_n,
                             spec.fixed_count)


class BinMap:
    def __init__(self, handle):
        self.h = handle

    def __del__(self):
        if getattr(self, "h", None) and L._lib is not None:
            L._lib.we_binmap_destroy(self.h)
            self.h = None

    @property
    def n_bins(self) -> int:
        return lib().we_binmap_n_bins(self.h)


def we_binmap_grid(species, edges) -> BinMap:
    """species: list of species ids; edges: list of ascending edge arrays, one per dimension."""
    sp = _i32(species)
    nb = _i32([len(e) - 1 for e in edges])
    ed = _f64(np.concatenate([np.asarray(e, dtype=np.float64) for e in edges]))
    h = C.c_void_p()
    check(lib().we_binmap_grid(len(sp), _ptr(sp, _I32P), _ptr(nb, _I32P), _ptr(ed, _F64P), C.byref(h)))
    return BinMap(h)


def make_run_config(tau, m_targ, init_states, init_weights, *, n_runs=None, seed=0, run_ids=None,
                    param_set=None, first_iter=0, capacity=0, record_iters=1, target=None,
                    recycle_state=None, max_steps=0, hist_species=0, hist_len=0, resample=True,
                    mapping=L.WE_MAP_AUTO, block_threads=0, reweight_period=0, absorb=False,
                    endpoint=False):
    """Build a we_run_config.  init_states: (runs, n_init, S); init_weights: (runs, n_init);
    target: None or (species list, op list, thresholds (runs, clauses)); absorb: the target set
    is absorbing (brute-force first-passage runs, needs resample=False) instead of recycling;
    endpoint: the target set is checked at each interval's end only.  Returns
    (config, keepalive) -- keep the second object alive while the config is used."""
    ist = _i32(init_states)
    iw = _f64(init_weights)
    R = ist.shape[0] if n_runs is None else n_runs
    keep = {"ist": ist, "iw": iw}
    c = we_run_config()
    c.tau = float(tau)
    c.m_targ = int(m_targ)
    c.n_runs = int(R)
    c.seed = int(seed)
    if run_ids is not None:
        keep["rid"] = np.ascontiguousarray(run_ids, dtype=np.uint32)
        c.run_ids = _ptr(keep["rid"], _U32P)
    if param_set is not None:
        keep["ps"] = _i32(param_set)
        c.param_set = _ptr(keep["ps"], _I32P)
    c.n_init = int(ist.shape[1])
    c.init_states = _ptr(ist, _I32P)
    c.init_weights = _ptr(iw, _F64P)
    c.first_iter = int(first_iter)
    c.capacity = int(capacity)
    c.record_iters = int(record_iters)
    if target is not None:
        sp, ops, thr = target
        keep["thr"] = _i32(thr).reshape(R, len(sp))
        c.feedback = (L.WE_FEEDBACK_ABSORB if absorb else
                      L.WE_FEEDBACK_ENDPOINT if endpoint else L.WE_FEEDBACK_RECYCLE)
        c.n_clauses = len(sp)
        for k in range(len(sp)):
            c.tgt_species[k] = int(sp[k])
            c.tgt_op[k] = int(ops[k])
        c.tgt_threshold = _ptr(keep["thr"], _I32P)
    if recycle_state is not None:
        keep["rec"] = _i32(recycle_state)
        c.recycle_state = _ptr(keep["rec"], _I32P)
    c.max_steps = int(max_steps)
    c.hist_species = int(hist_species)
    c.hist_len = int(hist_len)
    c.resample = 1 if resample else 0
    c.mapping = int(mapping)
    c.block_threads = int(block_threads)
    c.reweight_period = int(reweight_period)
    return c, keep


def run_config_from(cfg, record_iters=None, resample=True, first_iter=None, init_states=None,
                    init_weights=None, mapping=L.WE_MAP_AUTO, block_threads=0, max_steps=None,
                    capacity=None):
    """Marshal a run description (attributes tau, m_targ, init_states, target, ...) into a
    we_run_config."""
    tgt = None
    if cfg.target is not None:
        tgt = (cfg.target.species, cfg.target.op, cfg.target.threshold)
    return make_run_config(
        cfg.tau, cfg.m_targ, cfg.init_states if init_states is None else init_states,
        cfg.init_weights if init_weights is None else init_weights, n_runs=cfg.n_runs,
        seed=cfg.seed, run_ids=cfg.run_ids, param_set=cfg.param_set,
        first_iter=cfg.first_iter if first_iter is None else first_iter,
        capacity=cfg.capacity if capacity is None else capacity,
        record_iters=cfg.n_iters if record_iters is None else record_iters, target=tgt,
        recycle_state=cfg.recycle_state, max_steps=cfg.max_steps if max_steps is None else max_steps,
        hist_species=cfg.hist_species, hist_len=cfg.hist_len, resample=resample, mapping=mapping,
        block_threads=block_threads, reweight_period=getattr(cfg, "reweight_period", 0) if resample else 0,
        absorb=bool(getattr(cfg, "absorb", False)), endpoint=bool(getattr(cfg, "endpoint", False)))


_OUT_DTYPES = {
    L.WE_OUT_COUNTS: np.int32, L.WE_OUT_STATES: np.int32, L.WE_OUT_WEIGHTS: np.float64,
    L.WE_OUT_PARENT: np.int32, L.WE_OUT_FLUX: np.float64, L.WE_OUT_TOTAL_W: np.float64,
    L.WE_OUT_NWALKERS: np.int32, L.WE_OUT_EVENTS: np.int64, L.WE_OUT_HIST: np.float64,
    L.WE_OUT_STATUS: np.int32, L.WE_OUT_ITER: np.int32, L.WE_OUT_RECORDED: np.int32,
    L.WE_OUT_TLAST: np.float64, L.WE_OUT_Z: np.float32, L.WE_OUT_NREC: np.int32,
    L.WE_OUT_RW: np.int32, L.WE_OUT_FPT: np.float64, L.WE_OUT_NEAR_TAU: np.int32,
}


class Ensemble:
    """A we_ensemble handle.  By default its workspace is a PyTorch CUDA tensor."""

    def __init__(self, handle, workspace=None, keep=None, n_runs=1, n_species=1, hist_len=0):
        self.h = handle
        self.workspace = workspace
        self._keep = keep
        self.n_runs, self.n_species, self.hist_len = n_runs, n_species, hist_len

    def close(self):
        if getattr(self, "h", None) and L._lib is not None:
            L._lib.we_ensemble_destroy(self.h)
            self.h = None
        self.workspace = None

    def __del__(self):
        self.close()

    def propagate(self, stream=None):
        check(lib().we_ensemble_propagate(self.h, _stream_handle(stream)))

    def resample(self, stream=None):
        check(lib().we_ensemble_resample(self.h, _stream_handle(stream)))

    def set_resample_kernel(self, kind: int, blocks_per_run: int = 0):
        """WE_RESAMPLE_AUTO / WE_RESAMPLE_CHAIN / WE_RESAMPLE_ONE_LAUNCH (same results)."""
        check(lib().we_ensemble_set_resample_kernel(self.h, int(kind), int(blocks_per_run)))

    def iteration_kernels(self) -> int:
        """Kernel launches of one WE iteration (kernel nodes of the captured iteration graph)."""
        n = C.c_int32(0)
        check(lib().we_ensemble_iteration_kernels(self.h, C.byref(n)))
        return int(n.value)

    def step(self, n_iters: int, stream=None):
        check(lib().we_ensemble_step(self.h, int(n_iters), _stream_handle(stream)))

    def step_timed(self, n_iters: int, stream=None, every: int = 1) -> np.ndarray:
        """step() with the SSA kernel of every `every`-th iteration (0, every, ...) timed by CUDA
        events (ms, one entry per timed iteration)."""
        n_t = (int(n_iters) + every - 1) // every
        ms = np.zeros(max(n_t, 1), dtype=np.float32)
        check(lib().we_ensemble_step_timed_every(self.h, int(n_iters), int(every), _stream_handle(stream),
                                                 ms.ctypes.data_as(C.POINTER(C.c_float))))
        return ms[:n_t]

    def sync(self, stream=None):
        check(lib().we_ensemble_sync(self.h, _stream_handle(stream)))

    def checkpoint(self, stream=None) -> np.ndarray:
        """The ensemble's state between iterations as bytes (see we_ensemble_checkpoint)."""
        n = C.c_size_t()
        check(lib().we_ensemble_checkpoint(self.h, None, 0, C.byref(n), _stream_handle(stream)))
        buf = np.zeros(n.value, dtype=np.uint8)
        check(lib().we_ensemble_checkpoint(self.h, C.c_void_p(buf.ctypes.data), buf.nbytes, C.byref(n),
                                           _stream_handle(stream)))
        return buf

    def nbytes(self, what: int, run: int = -1, stream=None) -> int:
        n = C.c_size_t()
        check(lib().we_ensemble_get(self.h, what, run, None, 0, C.byref(n), _stream_handle(stream)))
        return n.value

    def get(self, what: int, run: int = -1, out=None, stream=None):
        """Copy an output array into `out` (numpy or torch, host or device) or a new numpy array."""
        dt = _OUT_DTYPES[what]
        nb = self.nbytes(what, run, stream)
        if out is None:
            out = np.zeros(nb // np.dtype(dt).itemsize, dtype=dt)
        if hasattr(out, "data_ptr"):
            ptr, size = out.data_ptr(), out.numel() * out.element_size()
        else:
            ptr, size = out.ctypes.data, out.nbytes
        n = C.c_size_t()
        check(lib().we_ensemble_get(self.h, what, run, C.c_void_p(ptr), size, C.byref(n),
                                    _stream_handle(stream)))
        return out

    # convenience views of get()
    def states(self, run: int = 0):
        return self.get(L.WE_OUT_STATES, run).reshape(-1, self.n_species)

    def weights(self, run: int = 0):
        return self.get(L.WE_OUT_WEIGHTS, run)

    def parents(self, run: int = 0):
        return self.get(L.WE_OUT_PARENT, run)

    def per_iter(self, what: int, run: int = -1):
        a = self.get(what, run)
        if what == L.WE_OUT_HIST:
            return a.reshape(-1, self.hist_len) if run >= 0 else a.reshape(-1, self.n_runs, self.hist_len)
        return a if run >= 0 else a.reshape(-1, self.n_runs)

    def status(self):
        return self.get(L.WE_OUT_STATUS, -1)

    def iteration(self) -> int:
        return int(self.get(L.WE_OUT_ITER)[0])

    def first_passage(self, run: int = 0):
        """Absorbing ensembles: each walker's first-passage time from the run's start (-1: none)."""
        return self.get(L.WE_OUT_FPT, run)

    def fpt_mle(self, T: float = 0.0, stream=None) -> np.ndarray:
        """Brute-force transition time of every run (Sec. II.C, Eq. "mld") from the first-passage
        times in [0, T] (T <= 0: the time simulated so far): rows (N, n, sum t_i, mu, sigma)."""
        out = np.zeros((self.n_runs, 5))
        check(lib().we_ensemble_fpt_mle(self.h, float(T), C.c_void_p(out.ctypes.data), out.nbytes,
                                        _stream_handle(stream)))
        return out


def we_ensemble_workspace_bytes(net: Network, bins: BinMap, cfg) -> int:
    n = C.c_size_t()
    check(lib().we_ensemble_workspace_bytes(net.h, bins.h, C.byref(cfg), C.byref(n)))
    return n.value


def we_ensemble_create(net: Network, bins: BinMap, cfg, keep=None, workspace="torch",
                       stream=None, device=None) -> Ensemble:
    """workspace='torch': a CUDA uint8 tensor from PyTorch; None: the library allocates; or a
    tensor supplied by the caller."""
    ws = None
    ptr, size = None, 0
    if isinstance(workspace, str) and workspace == "torch":
        import torch
        nb = we_ensemble_workspace_bytes(net, bins, cfg)
        ws = torch.empty(nb, dtype=torch.uint8, device=device or torch.device("cuda", torch.cuda.current_device()))
        ptr, size = C.c_void_p(ws.data_ptr()), nb
    elif workspace is not None:
        ws = workspace
        ptr, size = C.c_void_p(ws.data_ptr()), ws.numel() * ws.element_size()
    h = C.c_void_p()
    check(lib().we_ensemble_create(net.h, bins.h, C.byref(cfg), ptr, size, _stream_handle(stream),
                                   C.byref(h)))
    hl = cfg.hist_len if cfg.hist_len > 0 else 1
    return Ensemble(h, ws, keep, cfg.n_runs, net.n_species, hl)


def we_ensemble_resume(net: Network, bins: BinMap, cfg, checkpoint, keep=None, stream=None) -> Ensemble:
    """A new ensemble continuing from Ensemble.checkpoint() bytes; cfg supplies everything else
    (its initial walkers and first iteration are replaced by the checkpoint's)."""
    blob = np.ascontiguousarray(checkpoint, dtype=np.uint8)
    h = C.c_void_p()
    check(lib().we_ensemble_resume(net.h, bins.h, C.byref(cfg), C.c_void_p(blob.ctypes.data), blob.nbytes,
                                   _stream_handle(stream), C.byref(h)))
    hl = cfg.hist_len if cfg.hist_len > 0 else 1
    return Ensemble(h, None, keep, cfg.n_runs, net.n_species, hl)


def we_run(net: Network, bins: BinMap, cfg, keep=None, stream=None) -> Ensemble:
    """Whole WE procedure in one call (host inputs, library-owned device memory)."""
    h = C.c_void_p()
    st = lib().we_run(net.h, bins.h, C.byref(cfg), _stream_handle(stream), C.byref(h))
    if h.value is None:
        check(st)
    hl = cfg.hist_len if cfg.hist_len > 0 else 1
    ens = Ensemble(h, None, keep, cfg.n_runs, net.n_species, hl)
    ens.run_status = st
    return ens


def we_autotune(net: Network, bins: BinMap, cfg, stream=None):
    m = C.c_int32()
    b = C.c_int32()
    check(lib().we_autotune(net.h, bins.h, C.byref(cfg), _stream_handle(stream), C.byref(m), C.byref(b)))
    return m.value, b.value


def measure_alu_peaks(stream=None) -> dict:
    """Measured whole-GPU lane operations per second of FP64 FMA, INT32 multiply-add and INT32
    ALU (xor/add) -- the denominators of the SSA kernels' rooflines."""
    f, m, a = C.c_double(), C.c_double(), C.c_double()
    check(lib().we_measure_alu_peaks(_stream_handle(stream), C.byref(f), C.byref(m), C.byref(a)))
    return {"fp64_fma_per_s": f.value, "imad_per_s": m.value, "ialu_per_s": a.value}


def measure_graph_floor(kernels: int, n_replays: int = 2000, stream=None) -> float:
    """Milliseconds per replay of a CUDA graph of `kernels` empty launches (the launch floor of a
    WE iteration with that many kernels)."""
    ms = C.c_double()
    check(lib().we_measure_graph_floor(int(kernels), int(n_replays), _stream_handle(stream), C.byref(ms)))
    return ms.value


def autotune_cache_save(path: str):
    """Write the autotuner's cached choices to a text file."""
    check(lib().we_autotune_cache_save(str(path).encode()))


def autotune_cache_load(path: str):
    """Merge cached choices from a file written by autotune_cache_save."""
    check(lib().we_autotune_cache_load(str(path).encode()))


def autotune_cache_clear():
    lib().we_autotune_cache_clear()


def _require_cuda_tensor(t, dtype, min_numel: int, name: str, device=None):
    """Raise WEError(WE_EINVAL) unless t is a contiguous CUDA tensor of `dtype` with at least
    `min_numel` elements (on `device` when given).  The C entry points take raw device pointers
    and cannot check any of this themselves."""
    import torch
    ok = (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == dtype and t.is_contiguous()
          and t.numel() >= min_numel and (device is None or t.device == device))
    if not ok:
        desc = (f"{getattr(t, 'dtype', type(t).__name__)} on {getattr(t, 'device', '?')}, "
                f"{getattr(t, 'numel', lambda: '?')()} elements")
        raise L.WEError(L.WE_EINVAL, f"{name} must be a contiguous CUDA {dtype} tensor with at "
                                     f"least {min_numel} elements on {device or 'a CUDA device'} ({desc})")


def we_resample_static(bins, weights, n_bins: int, m_targ: int, iteration: int, seed: int,
                       run_id: int, out_weights, out_parent, out_count, stream=None):
    """Split/merge of one run held in device tensors, with no allocation by the library
    (for callers that may not allocate device memory).  Arguments are contiguous CUDA tensors on
    the current device: bins int32 and weights float64 of n entries; out_weights float64 and
    out_parent int32 with the same capacity (out_weights.numel()); out_count int32[>= 1], which
    receives the new count or a negative status.  Anything else raises WEError(WE_EINVAL) before
    the library is called."""
    import torch
    _require_cuda_tensor(bins, torch.int32, 1, "bins")
    dev = bins.device
    if dev.index != torch.cuda.current_device():
        raise L.WEError(L.WE_EINVAL, f"bins is on {dev}, not on the current device "
                                     f"cuda:{torch.cuda.current_device()}")
    n = int(bins.numel())
    _require_cuda_tensor(weights, torch.float64, n, "weights", dev)
    if weights.numel() != n:
        raise L.WEError(L.WE_EINVAL, f"weights has {weights.numel()} entries for {n} bins")
    _require_cuda_tensor(out_weights, torch.float64, 1, "out_weights", dev)
    cap = int(out_weights.numel())
    _require_cuda_tensor(out_parent, torch.int32, cap, "out_parent", dev)
    _require_cuda_tensor(out_count, torch.int32, 1, "out_count", dev)
    check(lib().we_resample_static(n, C.c_void_p(bins.data_ptr()), C.c_void_p(weights.data_ptr()),
                                   int(n_bins), int(m_targ), int(iteration), int(seed), int(run_id),
                                   cap, C.c_void_p(out_weights.data_ptr()),
                                   C.c_void_p(out_parent.data_ptr()), C.c_void_p(out_count.data_ptr()),
                                   _stream_handle(stream)))


# ------------------------------------------------------------------------------ learned bins
_F32P = C.POINTER(C.c_float)


class MLP:
    """A we_mlp handle (device-resident FP32 master weights and Adam moments)."""

    def __init__(self, handle, n_in, hidden):
        self.h = handle
        self.n_in, self.hidden = n_in, hidden
        self.n_params = lib().we_mlp_n_params(handle)

    def close(self):
        if getattr(self, "h", None) and L._lib is not None:
            L._lib.we_mlp_destroy(self.h)
            self.h = None

    def __del__(self):
        self.close()

    def params(self) -> np.ndarray:
        out = np.zeros(self.n_params, dtype=np.float32)
        check(lib().we_mlp_get_params(self.h, out.ctypes.data_as(_F32P), out.size))
        return out

    def train(self, states, labels, steps: int, batch: int, lr: float, stream=None) -> np.ndarray:
        """Adam steps on device tensors states (n x n_in int32) and labels (n float32)."""
        losses = np.zeros(max(int(steps), 1), dtype=np.float32)
        check(lib().we_mlp_train(self.h, C.c_void_p(states.data_ptr()), C.c_void_p(labels.data_ptr()),
                                 int(labels.numel()), int(steps), int(batch), float(lr),
                                 losses.ctypes.data_as(_F32P), _stream_handle(stream)))
        return losses[:int(steps)]

    def forward(self, states, bf16: bool = False, stream=None):
        """z of device states (n x n_in int32) as a device float32 tensor."""
        import torch
        n = int(states.shape[0])
        z = torch.empty(n, dtype=torch.float32, device=states.device)
        check(lib().we_mlp_forward(self.h, C.c_void_p(states.data_ptr()), n, 1 if bf16 else 0,
                                   C.c_void_p(z.data_ptr()), _stream_handle(stream)))
        return z

    def gradient(self, states, labels, stream=None):
        import torch
        g = torch.empty(self.n_params, dtype=torch.float32, device=labels.device)
        loss = np.zeros(1, dtype=np.float32)
        check(lib().we_mlp_gradient(self.h, C.c_void_p(states.data_ptr()), C.c_void_p(labels.data_ptr()),
                                    int(labels.numel()), C.c_void_p(g.data_ptr()),
                                    loss.ctypes.data_as(_F32P), _stream_handle(stream)))
        return g.cpu().numpy(), float(loss[0])


def we_mlp_create(n_in: int, hidden: int, params) -> MLP:
    p = np.ascontiguousarray(params, dtype=np.float32)
    h = C.c_void_p()
    check(lib().we_mlp_create(int(n_in), int(hidden), p.ctypes.data_as(_F32P), C.byref(h)))
    return MLP(h, n_in, hidden)


def we_mlp_create_init(n_in: int, hidden: int, seed: int = 0) -> MLP:
    """A new MLP with the library's own seeded initial weights (uniform +-1/sqrt(fan_in))."""
    h = C.c_void_p()
    check(lib().we_mlp_create_init(int(n_in), int(hidden), int(seed), C.byref(h)))
    return MLP(h, n_in, hidden)


def we_mlp_coordinate_edges(mlp: MLP, states, n_bins: int, lo_q: float = 0.001, stream=None) -> np.ndarray:
    """Bin edges on the learned coordinate, computed by the library: n_bins equal intervals from
    the floor(lo_q (n-1))-th smallest z of the device states (n x n_in int32) to the largest."""
    edges = np.zeros(int(n_bins) + 1, dtype=np.float32)
    check(lib().we_mlp_coordinate_edges(mlp.h, C.c_void_p(states.data_ptr()), int(states.shape[0]), int(n_bins),
                                        float(lo_q), C.c_void_p(edges.ctypes.data), _stream_handle(stream)))
    return edges


def we_binmap_learned(mlp: MLP, edges) -> BinMap:
    e = np.ascontiguousarray(edges, dtype=np.float32)
    h = C.c_void_p()
    check(lib().we_binmap_learned(mlp.h, len(e) - 1, e.ctypes.data_as(_F32P), C.byref(h)))
    return BinMap(h)


def first_passage_labels(net: Network, states, horizon: float, target, recycle_state=None, seed: int = 0,
                         param_set: int = 0, stream=None):
    """Shooting labels for training a progress coordinate: label 1 where a plain SSA trajectory
    (Sec. II.A) started at a state enters the target set within `horizon` (or starts inside it),
    else 0.  states: (n, S) int; target: (species, ops, thresholds (clauses,)).  Runs one
    unresampled interval of length `horizon` through the SSA kernel with the target as an
    absorbing set and reads each walker's first-passage time (-1: none; 0: started inside).
    `recycle_state` is not needed and ignored.  Returns float32 labels on the device."""
    import torch
    st = np.ascontiguousarray(states, dtype=np.int32)
    n, S = st.shape
    sp, ops, thr = target
    thr = np.asarray(thr, dtype=np.int32).reshape(1, -1)
    c, keep = make_run_config(horizon, 1, st.reshape(1, n, S), np.full((1, n), 1.0 / n), n_runs=1,
                              seed=seed, param_set=[param_set], capacity=n, record_iters=1,
                              target=(sp, ops, thr), resample=False, absorb=True)
    bm = we_binmap_grid([0], [np.array([0.0, 2.0 ** 31])])
    ens = we_ensemble_create(net, bm, c, keep, stream=stream)
    ens.propagate(stream)
    dev = ens.workspace.device
    fpt = torch.empty(n, dtype=torch.float64, device=dev)
    ens.get(L.WE_OUT_FPT, 0, out=fpt, stream=stream)             # device copy of the passage times
    ens.close()
    return (fpt >= 0).to(torch.float32)
