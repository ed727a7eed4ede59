"""ctypes declarations of the C ABI in include/we_ssa.h (libwe_ssa.so, built in-tree).

There is no fallback: if the CUDA library is missing or fails to load, every call raises.
"""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libwe_ssa.so")

WE_OK = 0
WE_EINVAL = -1
WE_ENOMEM = -2
WE_ECUDA = -3
WE_EOVERFLOW = -4
WE_ESTEPCAP = -5
WE_ETIMEOUT = -6
WE_ENOTSUPPORTED = -7
WE_MAX_COUNT = 2097151
WE_MASS_ACTION = 0
WE_HILL_REPRESSION = 1
WE_OP_GE = 0
WE_OP_LE = 1
WE_MAP_AUTO = 0
WE_MAP_THREAD = 1
WE_MAP_WARP = 2
WE_MAP_THREAD_TABLE = 3
WE_RESAMPLE_AUTO = 0
WE_RESAMPLE_CHAIN = 1
WE_RESAMPLE_ONE_LAUNCH = 2
WE_OUT_COUNTS = 1
WE_OUT_STATES = 2
WE_OUT_WEIGHTS = 3
WE_OUT_PARENT = 4
WE_OUT_FLUX = 5
WE_OUT_TOTAL_W = 6
WE_OUT_NWALKERS = 7
WE_OUT_EVENTS = 8
WE_OUT_HIST = 9
WE_OUT_STATUS = 10
WE_OUT_ITER = 11
WE_OUT_RECORDED = 12
WE_OUT_TLAST = 13
WE_OUT_Z = 14
WE_OUT_NREC = 15
WE_OUT_RW = 16
WE_OUT_FPT = 17
WE_OUT_NEAR_TAU = 18
WE_FEEDBACK_RECYCLE = 1
WE_FEEDBACK_ABSORB = 2
WE_FEEDBACK_ENDPOINT = 3

_I32P = C.POINTER(C.c_int32)
_U32P = C.POINTER(C.c_uint32)
_F64P = C.POINTER(C.c_double)
_F32P = C.POINTER(C.c_float)
_VP = C.c_void_p


class we_run_config(C.Structure):
    _fields_ = [
        ("tau", C.c_double), ("m_targ", C.c_int32), ("n_runs", C.c_int32), ("seed", C.c_uint64),
        ("run_ids", _U32P), ("param_set", _I32P), ("n_init", C.c_int32), ("init_states", _I32P),
        ("init_weights", _F64P), ("first_iter", C.c_int32), ("capacity", C.c_int32),
        ("record_iters", C.c_int32), ("feedback", C.c_int32), ("n_clauses", C.c_int32),
        ("tgt_species", C.c_int32 * 4), ("tgt_op", C.c_int32 * 4), ("tgt_threshold", _I32P),
        ("recycle_state", _I32P), ("max_steps", C.c_int64), ("hist_species", C.c_int32),
        ("hist_len", C.c_int32), ("resample", C.c_int32), ("mapping", C.c_int32),
        ("block_threads", C.c_int32), ("reweight_period", C.c_int32), ("n_init_per_run", _I32P),
    ]


# (name, restype, argtypes) for every exported entry point of we_ssa.h
SIGNATURES = [
    ("we_status_string", C.c_char_p, [C.c_int32]),
    ("we_last_error", C.c_char_p, []),
    ("we_debug_fail_allocation", C.c_int32, [C.c_int32]),
    ("we_version", C.c_int32, []),
    ("we_network_create", C.c_int32, [C.c_int32, C.c_int32, _I32P, _I32P, _I32P, _I32P, _I32P, _I32P,
                                      C.c_int32, _F64P, _I32P, _I32P, C.c_int32, _F64P, _I32P, _I32P,
                                      C.POINTER(_VP)]),
    ("we_network_destroy", None, [_VP]),
    ("we_network_keff", C.c_int32, [_VP, C.c_int32, C.c_int32, _F64P]),
    ("we_network_dep_degree", C.c_int32, [_VP, C.c_int32, _I32P]),
    ("we_binmap_grid", C.c_int32, [C.c_int32, _I32P, _I32P, _F64P, C.POINTER(_VP)]),
    ("we_binmap_destroy", None, [_VP]),
    ("we_binmap_n_bins", C.c_int32, [_VP]),
    ("we_ensemble_workspace_bytes", C.c_int32, [_VP, _VP, C.POINTER(we_run_config), C.POINTER(C.c_size_t)]),
    ("we_ensemble_create", C.c_int32, [_VP, _VP, C.POINTER(we_run_config), _VP, C.c_size_t, _VP,
                                       C.POINTER(_VP)]),
    ("we_ensemble_destroy", C.c_int32, [_VP]),
    ("we_ensemble_propagate", C.c_int32, [_VP, _VP]),
    ("we_ensemble_resample", C.c_int32, [_VP, _VP]),
    ("we_ensemble_set_resample_kernel", C.c_int32, [_VP, C.c_int32, C.c_int32]),
    ("we_ensemble_iteration_kernels", C.c_int32, [_VP, C.POINTER(C.c_int32)]),
    ("we_ensemble_step", C.c_int32, [_VP, C.c_int32, _VP]),
    ("we_ensemble_step_timed", C.c_int32, [_VP, C.c_int32, _VP, C.POINTER(C.c_float)]),
    ("we_ensemble_step_timed_every", C.c_int32, [_VP, C.c_int32, C.c_int32, _VP, C.POINTER(C.c_float)]),
    ("we_ensemble_checkpoint", C.c_int32, [_VP, _VP, C.c_size_t, C.POINTER(C.c_size_t), _VP]),
    ("we_ensemble_resume", C.c_int32, [_VP, _VP, C.POINTER(we_run_config), _VP, C.c_size_t, _VP,
                                       C.POINTER(_VP)]),
    ("we_ensemble_sync", C.c_int32, [_VP, _VP]),
    ("we_ensemble_get", C.c_int32, [_VP, C.c_int32, C.c_int32, _VP, C.c_size_t,
                                    C.POINTER(C.c_size_t), _VP]),
    ("we_ensemble_fpt_mle", C.c_int32, [_VP, C.c_double, _VP, C.c_size_t, _VP]),
    ("we_run", C.c_int32, [_VP, _VP, C.POINTER(we_run_config), _VP, C.POINTER(_VP)]),
    ("we_measure_alu_peaks", C.c_int32, [_VP, _F64P, _F64P, _F64P]),
    ("we_measure_graph_floor", C.c_int32, [C.c_int32, C.c_int32, _VP, _F64P]),
    ("we_autotune", C.c_int32, [_VP, _VP, C.POINTER(we_run_config), _VP, _I32P, _I32P]),
    ("we_autotune_cache_save", C.c_int32, [C.c_char_p]),
    ("we_autotune_cache_load", C.c_int32, [C.c_char_p]),
    ("we_autotune_cache_clear", None, []),
    ("we_mlp_create", C.c_int32, [C.c_int32, C.c_int32, _F32P, C.POINTER(_VP)]),
    ("we_mlp_destroy", None, [_VP]),
    ("we_mlp_n_params", C.c_int32, [_VP]),
    ("we_mlp_get_params", C.c_int32, [_VP, _F32P, C.c_size_t]),
    ("we_mlp_train", C.c_int32, [_VP, _VP, _VP, C.c_int32, C.c_int32, C.c_int32, C.c_float, _F32P, _VP]),
    ("we_mlp_gradient", C.c_int32, [_VP, _VP, _VP, C.c_int32, _VP, _F32P, _VP]),
    ("we_mlp_forward", C.c_int32, [_VP, _VP, C.c_int32, C.c_int32, _VP, _VP]),
    ("we_binmap_learned", C.c_int32, [_VP, C.c_int32, _F32P, C.POINTER(_VP)]),
    ("we_mlp_create_init", C.c_int32, [C.c_int32, C.c_int32, C.c_uint64, C.POINTER(_VP)]),
    ("we_mlp_coordinate_edges", C.c_int32, [_VP, _VP, C.c_int32, C.c_int32, C.c_double, _VP, _VP]),
    ("we_resample_static", C.c_int32, [C.c_int32, _VP, _VP, C.c_int32, C.c_int32, C.c_int32,
                                       C.c_uint64, C.c_uint32, C.c_int32, _VP, _VP, _VP, _VP]),
]

_lib = None


class WEError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{status_name(status)}: {message}")
        self.status = status


_NAMES = {0: "WE_OK", -1: "WE_EINVAL", -2: "WE_ENOMEM", -3: "WE_ECUDA", -4: "WE_EOVERFLOW",
          -5: "WE_ESTEPCAP", -6: "WE_ETIMEOUT", -7: "WE_ENOTSUPPORTED"}


def status_name(s: int) -> str:
    return _NAMES.get(s, f"status {s}")


def lib() -> C.CDLL:
    """The loaded CUDA library; raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with paper_1303_5986_gb300.build.build()")
        L = C.CDLL(LIB_PATH)
        for name, res, args in SIGNATURES:
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def check(status: int) -> int:
    if status != WE_OK:
        raise WEError(status, lib().we_last_error().decode(errors="replace"))
    return status
