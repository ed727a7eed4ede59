"""GB300-native weighted-ensemble Gillespie-SSA (arXiv:1303.5986 hot path).

The compute lives in libwe_ssa.so (hand-written CUDA for sm_103a) behind the C ABI of
include/we_ssa.h; this package is its Python binding.  Build with ``build.build()``.
"""
from ._lib import (WEError, WE_OK, WE_EINVAL, WE_ENOMEM, WE_ECUDA, WE_EOVERFLOW, WE_ESTEPCAP,
                   WE_ETIMEOUT, WE_ENOTSUPPORTED, WE_MAX_COUNT, WE_MAP_AUTO, WE_MAP_THREAD,
                   WE_MAP_WARP, WE_MAP_THREAD_TABLE, WE_RESAMPLE_AUTO, WE_RESAMPLE_CHAIN, WE_RESAMPLE_ONE_LAUNCH, WE_OP_GE, WE_OP_LE, WE_OUT_COUNTS, WE_OUT_STATES, WE_OUT_WEIGHTS,
                   WE_OUT_PARENT, WE_OUT_FLUX, WE_OUT_TOTAL_W, WE_OUT_NWALKERS, WE_OUT_EVENTS,
                   WE_OUT_HIST, WE_OUT_STATUS, WE_OUT_ITER, WE_OUT_RECORDED, WE_OUT_TLAST,
                   WE_OUT_Z, WE_OUT_NREC, WE_OUT_RW, WE_OUT_FPT, WE_OUT_NEAR_TAU, WE_FEEDBACK_RECYCLE, WE_FEEDBACK_ABSORB, WE_FEEDBACK_ENDPOINT,
                   SIGNATURES, lib, status_name)
from .api import (Network, BinMap, Ensemble, we_network_create, network_from_spec, we_binmap_grid,
                  make_run_config, run_config_from, we_ensemble_workspace_bytes,
                  we_ensemble_create, we_ensemble_resume, we_run, we_autotune, autotune_cache_save, autotune_cache_load, autotune_cache_clear, we_resample_static, MLP, we_mlp_create,
                  we_binmap_learned, first_passage_labels, measure_alu_peaks, measure_graph_floor,
                  we_mlp_create_init, we_mlp_coordinate_edges)

__all__ = [n for n in dir() if not n.startswith("_")]
