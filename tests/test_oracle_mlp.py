"""Pins of the FP64 reference of the learned progress coordinate (CPU only).

The coordinate is not in the paper (adaptive binning is the open problem of Sec. IV.B; WE is
unbiased under any binning, Sec. II.B), so its reference is pinned by mathematics: central
differences of the loss, closed forms of the logistic loss and of Adam's first step, exact BF16
rounding cases, and a brute-force bin search."""
import numpy as np

import workloads as W
from oracle import mlp as M


def _data(n_in=2, n=40, seed=0, hi=80):
    rng = np.random.default_rng(seed)
    return rng.integers(0, hi, size=(n, n_in)), rng.random(n)


def test_gradient_matches_central_differences():
    """Every parameter's gradient (all six blocks, hidden width 8, two inputs) against a
    central difference of the FP64 loss: a dropped term or a transposed weight block fails."""
    n_in, H = 2, 8
    p = W.mlp_init_params(n_in, H, seed=3).astype(np.float64)
    p[W.mlp_n_params(n_in, H) - 1] = 0.3                 # non-zero b3
    X, y = _data(n_in)
    _, g = M.loss_and_grad(p, X, y, n_in, H)
    h = 1e-6
    fd = np.empty_like(p)
    for k in range(len(p)):
        e = np.zeros_like(p)
        e[k] = h
        fd[k] = (M.loss_and_grad(p + e, X, y, n_in, H)[0] - M.loss_and_grad(p - e, X, y, n_in, H)[0]) / (2 * h)
    assert np.max(np.abs(fd - g)) < 1e-8 * max(1.0, np.max(np.abs(g)))


def test_gradient_three_inputs_wide_hidden():
    n_in, H = 3, 64
    p = W.mlp_init_params(n_in, H, seed=5).astype(np.float64)
    X, y = _data(n_in, n=12, seed=1)
    _, g = M.loss_and_grad(p, X, y, n_in, H)
    rng = np.random.default_rng(2)
    for k in rng.choice(len(p), size=40, replace=False):
        e = np.zeros_like(p)
        e[k] = 1e-6
        fd = (M.loss_and_grad(p + e, X, y, n_in, H)[0] - M.loss_and_grad(p - e, X, y, n_in, H)[0]) / 2e-6
        assert abs(fd - g[k]) < 1e-8, k


def test_zero_network_gives_log2_loss():
    """All weights zero: z = b3 = 0, so BCE = log 2 for any label, and dL/db3 = mean(1/2 - y)."""
    n_in, H = 2, 4
    p = np.zeros(W.mlp_n_params(n_in, H))
    X, y = _data(n_in, n=10)
    loss, g = M.loss_and_grad(p, X, y, n_in, H)
    assert abs(loss - np.log(2.0)) < 1e-15
    assert abs(g[-1] - np.mean(0.5 - y)) < 1e-15
    assert np.all(g[:-1] == 0.0)


def test_forward_by_hand():
    """One input, one hidden unit: z = w3 silu(w2 silu(w1 log1p(x) + b1) + b2) + b3."""
    p = np.array([0.7, -0.2, 1.3, 0.1, -0.9, 0.25])      # W1, b1, W2, b2, w3, b3
    x = 5
    silu = lambda a: a / (1 + np.exp(-a))
    z = -0.9 * silu(1.3 * silu(0.7 * np.log(6.0) - 0.2) + 0.1) + 0.25
    assert abs(M.forward(p, [[x]], 1, 1)[0] - z) < 1e-15


def test_adam_first_step_is_signed_lr():
    """With zero moments the bias-corrected first Adam step is lr g / (|g| + eps)."""
    g = np.array([0.5, -2.0, 1e-3])
    p1, m, v = M.adam_step(np.zeros(3), g, np.zeros(3), np.zeros(3), 1, 0.01)
    np.testing.assert_allclose(p1, -0.01 * g / (np.abs(g) + 1e-8), rtol=1e-12)
    np.testing.assert_allclose(m, 0.1 * g, rtol=1e-12)
    np.testing.assert_allclose(v, 0.001 * g * g, rtol=1e-12)


def test_bf16_round_to_nearest_even():
    f = lambda u: np.array([u], dtype=np.uint32).view(np.float32)
    b = lambda x: int(M.bf16_round(x).view(np.uint32)[0])
    assert b(f(0x3F808000)) == 0x3F800000                # tie, even stays
    assert b(f(0x3F818000)) == 0x3F820000                # tie, odd rounds up
    assert b(f(0x3F808001)) == 0x3F810000                # above half
    assert b(f(0x3F807FFF)) == 0x3F800000                # below half
    assert b(f(0xBF818000)) == 0xBF820000                # sign kept


def test_bins_of_matches_brute_force():
    edges = W.logit_edges(10, -5.0, 5.0)
    z = np.concatenate([np.linspace(-7, 7, 301), edges.astype(np.float64)])
    got = M.bins_of(z, edges)
    for zi, b in zip(z, got):
        want = 0
        for k in range(10):
            if edges[k] <= zi:
                want = k
        assert b == want, (zi, b, want)


def test_inference_params_round_only_weights():
    n_in, H = 2, 4
    p = W.mlp_init_params(n_in, H, seed=1)
    p[H * n_in:H * n_in + H] = 0.123456789                # b1 unchanged by rounding
    q = M.inference_params(p, n_in, H)
    assert np.all(q[H * n_in:H * n_in + H] == p[H * n_in:H * n_in + H])
    assert np.all(q[:H * n_in].view(np.uint32) & 0xFFFF == 0)
    assert np.max(np.abs(q[:H * n_in] - p[:H * n_in])) <= np.max(np.abs(p[:H * n_in])) * 2 ** -8
