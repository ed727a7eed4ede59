"""Seeded initial weights and bin edges for the learned progress coordinate (inputs only).

Layout of the flat parameter vector: W1[H][n_in], b1[H], W2[H][H], b2[H], w3[H], b3.
"""
import numpy as np


def mlp_n_params(n_in: int, hidden: int = 64) -> int:
    return hidden * n_in + 3 * hidden + hidden * hidden + 1


def mlp_init_params(n_in: int, hidden: int = 64, seed: int = 0) -> np.ndarray:
    """Uniform(-1/sqrt(fan_in), 1/sqrt(fan_in)) weights, zero biases, float32."""
    rng = np.random.default_rng(seed)
    parts = [rng.uniform(-1, 1, size=hidden * n_in) / np.sqrt(n_in), np.zeros(hidden),
             rng.uniform(-1, 1, size=hidden * hidden) / np.sqrt(hidden), np.zeros(hidden),
             rng.uniform(-1, 1, size=hidden) / np.sqrt(hidden), np.zeros(1)]
    return np.concatenate(parts).astype(np.float32)


def logit_edges(n_bins: int = 100, lo: float = -12.0, hi: float = 12.0) -> np.ndarray:
    """n_bins equal intervals of the logit z on [lo, hi] (z outside falls in the end bins)."""
    return np.linspace(lo, hi, n_bins + 1).astype(np.float32)
