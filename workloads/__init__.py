"""Seeded synthetic inputs for the weighted-ensemble SSA path (networks and run settings).

This package holds input data only -- reaction lists, rate constants, bin edges, initial states --
and none of the method's arithmetic (no propensities, no SSA, no resampling).  Both the CUDA path
(through its C-ABI binding) and the CPU oracle read their inputs from here, so that the two are
fed identical bytes.
"""
from .networks import (NetworkSpec, birth_death, schlogl, toggle_switch, epigenetic_switch,
                       futile_cycle, synthetic_large)
from .mlp_init import mlp_init_params, mlp_n_params, logit_edges
from .configs import (WEConfig, GridBins, Target, birth_death_we, schlogl_mfpt_we, schlogl_flux_we, schlogl_pdf_we, futile_pdf_we, epigenetic_mfpt_we,
                      toggle_batch_we, synthetic_large_we, uniform_edges, bruteforce_fpt, schlogl_bruteforce,
                      birth_death_bruteforce)

__all__ = [
    "NetworkSpec", "birth_death", "schlogl", "toggle_switch", "epigenetic_switch", "futile_cycle",
    "synthetic_large", "WEConfig", "GridBins", "Target", "birth_death_we", "schlogl_mfpt_we",
    "schlogl_flux_we", "schlogl_pdf_we", "futile_pdf_we", "epigenetic_mfpt_we", "toggle_batch_we", "synthetic_large_we", "uniform_edges", "mlp_init_params",
    "mlp_n_params", "logit_edges", "bruteforce_fpt", "schlogl_bruteforce", "birth_death_bruteforce",
]
