"""The learned progress coordinate on the GPU against its FP64 reference (oracle/mlp.py):
gradients, Adam steps and training losses of the hand-written training kernels; the BF16-weight
inference fused into bin assignment; shooting labels; and unbiasedness of WE under learned bins
(Sec. II.B: any binning leaves the estimator unbiased)."""
import numpy as np
import pytest

import paper_1303_5986_gb300 as P
import workloads as W
from oracle import exact as E
from oracle import mlp as M

from gpu_helpers import gpu_run

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1303_5986_gb300 import build
    build.build()


def _dev(a, dtype):
    import torch
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")


def _params(n_in, H, seed):
    p = W.mlp_init_params(n_in, H, seed=seed)
    rng = np.random.default_rng(seed + 100)
    nb = W.mlp_n_params(n_in, H)
    o1, o2 = H * n_in, H * n_in + H + H * H
    p[o1:o1 + H] = rng.uniform(-0.5, 0.5, H)
    p[o2:o2 + H] = rng.uniform(-0.5, 0.5, H)
    p[nb - 1] = 0.2
    return p


@pytest.mark.parametrize("n_in,H,n", [(2, 64, 257), (354, 64, 96), (1, 16, 1), (3, 7, 130)])
def test_gradient_matches_oracle(n_in, H, n):
    """FP32 batch gradient of the mean BCE loss against the FP64 reference, all parameters."""
    p = _params(n_in, H, 4)
    rng = np.random.default_rng(n)
    X = rng.integers(0, 200, size=(n, n_in)).astype(np.int32)
    y = rng.random(n).astype(np.float32)
    mlp = P.we_mlp_create(n_in, H, p)
    assert np.array_equal(mlp.params(), p)
    g, loss = mlp.gradient(_dev(X, _i32()), _dev(y, _f32()))
    lo, go = M.loss_and_grad(p.astype(np.float64), X, y.astype(np.float64), n_in, H)
    assert abs(loss - lo) <= 2e-6 * max(1.0, lo), (loss, lo)
    scale = np.abs(go).max()
    err = np.abs(g - go)
    assert err.max() <= 1e-5 * scale + 1e-9, (err.max(), scale, int(err.argmax()))


def _i32():
    import torch
    return torch.int32


def _f32():
    import torch
    return torch.float32


def test_adam_step_matches_oracle():
    """One full-batch Adam step: params with a clear gradient move by lr g/(|g|+eps) as in the
    reference; no parameter moves by more than lr."""
    n_in, H, n, lr = 2, 32, 128, 1e-3
    p = _params(n_in, H, 7)
    rng = np.random.default_rng(1)
    X = rng.integers(0, 80, size=(n, n_in)).astype(np.int32)
    y = (rng.random(n) < 0.3).astype(np.float32)
    mlp = P.we_mlp_create(n_in, H, p)
    losses = mlp.train(_dev(X, _i32()), _dev(y, _f32()), 1, n, lr)
    q = mlp.params().astype(np.float64)
    lo, go = M.loss_and_grad(p.astype(np.float64), X, y.astype(np.float64), n_in, H)
    qo, _, _ = M.adam_step(p.astype(np.float64), go, 0.0 * go, 0.0 * go, 1, lr)
    assert abs(losses[0] - lo) <= 2e-6 * max(1.0, lo)
    clear = np.abs(go) > 1e-3 * np.abs(go).max()
    assert clear.sum() > 0.5 * len(go)
    assert np.max(np.abs(q - qo)[clear]) <= 1e-3 * lr
    assert np.max(np.abs(q - p)) <= lr * (1 + 1e-5)


def test_training_losses_follow_oracle():
    """Five Adam steps on consecutive batches (wrapping around the data): each reported batch
    loss against the reference loss of the same batch at the reference's parameters."""
    n_in, H, n, B, lr = 2, 64, 300, 128, 3e-3
    p = _params(n_in, H, 9)
    rng = np.random.default_rng(3)
    X = rng.integers(0, 100, size=(n, n_in)).astype(np.int32)
    y = (X[:, 1] > X[:, 0]).astype(np.float32)
    mlp = P.we_mlp_create(n_in, H, p)
    losses = mlp.train(_dev(X, _i32()), _dev(y, _f32()), 5, B, lr)
    po, m, v = p.astype(np.float64), 0.0, 0.0
    for t in range(5):
        idx = (t * B + np.arange(B)) % n
        lo, go = M.loss_and_grad(po, X[idx], y[idx].astype(np.float64), n_in, H)
        assert abs(losses[t] - lo) <= 1e-4 * max(1.0, lo), (t, losses[t], lo)
        po, m, v = M.adam_step(po, go, m, v, t + 1, lr)


def test_training_separates_toggle_basins():
    """Trained on labels V > U, the coordinate classifies held-out states (its sign, computed by
    the reference from the GPU's weights) and the batch loss falls well below log 2."""
    n_in, H = 2, 64
    rng = np.random.default_rng(5)
    X = rng.integers(0, 100, size=(8192, 2)).astype(np.int32)
    y = (X[:, 1] > X[:, 0]).astype(np.float32)
    mlp = P.we_mlp_create(n_in, H, W.mlp_init_params(n_in, H, seed=2))
    losses = mlp.train(_dev(X, _i32()), _dev(y, _f32()), 600, 1024, 3e-3)
    assert losses[-20:].mean() < 0.2, losses[-20:].mean()
    T = rng.integers(0, 100, size=(2000, 2))
    z = M.forward(mlp.params(), T, n_in, H)
    keep = T[:, 0] != T[:, 1]
    acc = np.mean((z[keep] > 0) == (T[keep, 1] > T[keep, 0]))
    assert acc > 0.95, acc


def _learned_toggle_ensemble(p, n_in, H, edges, n_runs=3, n_init=200, seed=0):
    a = 14.0
    cfg = W.toggle_batch_we(n_runs=n_runs, n_iters=1, seed=seed)
    rng = np.random.default_rng(seed + 1)
    cfg.network = W.toggle_switch(np.full(n_runs, a), np.full(n_runs, a))
    cfg.init_states = rng.integers(0, 40, size=(n_runs, n_init, 2)).astype(np.int32)
    cfg.init_weights = np.full((n_runs, n_init), 1.0 / n_init)
    cfg.x0 = np.tile(np.array([[14, 0]], dtype=np.int32), (n_runs, 1))
    cfg.recycle_state = cfg.x0.copy()
    cfg.target.threshold = np.tile(np.array([[7, 3]], dtype=np.int32), (n_runs, 1))
    cfg.m_targ = 5
    mlp = P.we_mlp_create(n_in, H, p)
    bm = P.we_binmap_learned(mlp, edges)
    assert bm.n_bins == len(edges) - 1
    ens = gpu_run(cfg, 0, bins=bm, capacity=n_init + 5 * (len(edges) - 1))
    ens._mlp = mlp
    return ens, cfg


def test_learned_bins_match_oracle():
    """z of every walker after one interval (BF16 weights, FP32 arithmetic) against the FP64
    reference with the same BF16 weights; then split/merge on the learned bins gives each
    occupied bin exactly M walkers and keeps the total weight."""
    n_in, H = 2, 64
    p = _params(n_in, H, 11)
    grid = np.stack(np.meshgrid(np.arange(60), np.arange(60)), -1).reshape(-1, 2)
    zg = M.forward(M.inference_params(p, n_in, H), grid, n_in, H)
    edges = np.linspace(zg.min(), zg.max(), 41).astype(np.float32)
    ens, cfg = _learned_toggle_ensemble(p, n_in, H, edges)
    ens.propagate()
    pi = M.inference_params(p, n_in, H)
    zs = []
    for r in range(cfg.n_runs):
        X = ens.states(r)
        z = ens.get(P.WE_OUT_Z, r)
        assert len(z) == len(X) == 200
        zo = M.forward(pi, X, n_in, H)
        np.testing.assert_allclose(z, zo, rtol=1e-5, atol=2e-5)
        far = np.min(np.abs(zo[:, None] - edges[None, :].astype(np.float64)), axis=1) > 1e-4
        assert np.array_equal(M.bins_of(z, edges)[far], M.bins_of(zo, edges)[far])
        # the standalone forward pass: BF16 form equals the binning kernel's z bit for bit;
        # FP32 form against the reference with unrounded weights
        Xd = _dev(X, _i32())
        assert np.array_equal(ens._mlp.forward(Xd, bf16=True).cpu().numpy().view(np.uint32), z.view(np.uint32))
        np.testing.assert_allclose(ens._mlp.forward(Xd).cpu().numpy(), M.forward(p, X, n_in, H),
                                   rtol=1e-5, atol=2e-5)
        zs.append(z)
    ens.resample()
    counts = ens.get(P.WE_OUT_COUNTS)
    for r in range(cfg.n_runs):
        assert counts[r] == cfg.m_targ * len(np.unique(M.bins_of(zs[r], edges))), r
        assert abs(ens.weights(r).sum() - 1.0) < 1e-12
    tot = ens.per_iter(P.WE_OUT_TOTAL_W)
    assert np.all(np.abs(tot - 1.0) < 1e-12)


def test_first_passage_labels():
    """Shooting labels from the SSA kernel: states inside the target are 1; over many shots from
    one state the label mean is the probability of entering the target within the horizon, checked
    on the birth-death chain against the exact absorbing-chain solution."""
    net_spec = W.birth_death(kb=10.0, kd=0.1)
    net = P.network_from_spec(net_spec)
    n = 20000
    X = np.concatenate([np.full((n, 1), 120), np.full((10, 1), 140)]).astype(np.int32)
    lab = P.first_passage_labels(net, X, 2.0, ([0], [P.WE_OP_GE], [130]), [100], seed=3)
    lab = lab.cpu().numpy()
    assert np.all(lab[n:] == 1.0)
    # exact P(hit 130 by t = 2 from 120): absorbing chain on 0..130, matrix exponential
    b, d = E.birth_death_rates(10.0, 0.1)
    Q = np.zeros((131, 131))
    for x in range(130):
        Q[x, x + 1] = b(x)
        if x > 0:
            Q[x, x - 1] = d(x)
        Q[x, x] = -Q[x].sum()
    p0 = np.zeros(131)
    p0[120] = 1.0
    exact = E.small_generator_expm(Q, p0, 2.0)[130]
    est = lab[:n].mean()
    se = np.sqrt(exact * (1 - exact) / n)
    assert abs(est - exact) < 3 * se, (est, exact, se)
    assert lab.dtype == np.float32


def test_we_with_learned_bins_is_unbiased():
    """Immigration-death chain (kb = 10, kd = 0.1, X0 = 100), tau = 0.1, 200 intervals, 10 walkers
    per bin on 100 bins of a coordinate trained on soft labels sigmoid((x - 130)/8): the weighted
    tail P(X >= k, t = 20) against the exact transient distribution within 3 standard errors over
    64 replicas -- and the same for the plain species-count grid (60 bins of width 5 plus
    overflow) as the control."""
    n_in, H = 1, 64
    xs = np.arange(0, 301, dtype=np.int32).reshape(-1, 1)
    ys = (1.0 / (1.0 + np.exp(-(xs[:, 0] - 130.0) / 8.0))).astype(np.float32)
    mlp = P.we_mlp_create(n_in, H, W.mlp_init_params(n_in, H, seed=1))
    losses = mlp.train(_dev(xs, _i32()), _dev(ys, _f32()), 2000, 301, 1e-2)
    assert losses[-1] < losses[0]
    z = M.forward(mlp.params(), np.arange(60, 220).reshape(-1, 1), n_in, H)
    assert np.all(np.diff(z) > 0), "coordinate not monotone on [60, 220)"
    edges = W.logit_edges(100, -10.0, 12.0)
    exact = E.immigration_death_pmf(100, 10.0, 0.1, 20.0, 400)
    for learned in (True, False):
        cfg = W.birth_death_we(n_iters=200, n_runs=64, seed=5)
        bm = P.we_binmap_learned(mlp, edges) if learned else None
        ens = gpu_run(cfg, 200, bins=bm, capacity=10 * 100 + 64)
        ens.sync()
        Hh = ens.per_iter(P.WE_OUT_HIST)           # iters x runs x len; iteration 199 ends at t = 20
        for k in (120, 130, 140):
            est = Hh[199, :, k:].sum(axis=1)
            ex = exact[k:].sum()
            se = est.std(ddof=1) / np.sqrt(len(est))
            assert abs(est.mean() - ex) < 3 * se, (learned, k, est.mean(), ex, se)
        tot = ens.per_iter(P.WE_OUT_TOTAL_W)
        assert np.all(np.abs(tot - 1.0) < 1e-12)


def test_harvest_states_all_runs():
    """States of all runs in one call (run = -1) equal the per-run arrays concatenated, and the
    harvest collects them after every iteration."""
    from paper_1303_5986_gb300 import learned as LN
    cfg = W.toggle_batch_we(n_runs=5, n_iters=3, seed=2)
    ens = gpu_run(cfg, 2, record_iters=4)
    allx = ens.states(-1)
    per = np.concatenate([ens.states(r) for r in range(cfg.n_runs)])
    assert np.array_equal(allx, per)
    assert len(allx) == ens.get(P.WE_OUT_COUNTS).sum()
    h = LN.harvest_states(ens, 2)
    assert h.shape[1] == 2 and len(h) > len(allx)


def test_learned_bins_on_the_large_network():
    """A learned bin map on the 354-species synthetic network (warp-per-walker SSA kernel, an MLP
    with 354 inputs): z against the FP64 reference, each occupied bin resampled to M walkers, and
    the total weight kept."""
    cfg = W.synthetic_large_we(n_walkers=256, n_iters=1, m_targ=6)
    S = cfg.network.n_species
    H = 16
    p = _params(S, H, 21)
    states0 = cfg.init_states[0]
    zg = M.forward(M.inference_params(p, S, H), states0, S, H)
    edges = np.linspace(zg.min() - 1.0, zg.max() + 1.0, 21).astype(np.float32)
    mlp = P.we_mlp_create(S, H, p)
    bm = P.we_binmap_learned(mlp, edges)
    cfg.capacity = 256 + 6 * 20
    cfg.tau = 2e-4
    ens = gpu_run(cfg, 0, bins=bm, capacity=cfg.capacity)
    ens.propagate()
    X = ens.states(0)
    z = ens.get(P.WE_OUT_Z, 0)
    zo = M.forward(M.inference_params(p, S, H), X, S, H)
    np.testing.assert_allclose(z, zo, rtol=1e-5, atol=5e-5)
    ens.resample()
    n_occ = len(np.unique(M.bins_of(z, edges)))
    assert ens.get(P.WE_OUT_COUNTS)[0] == 6 * n_occ
    assert abs(ens.weights(0).sum() - 1.0) < 1e-12


def test_coordinate_edges_are_order_statistics_of_z():
    """Bin placement on the learned coordinate runs in the library: the low edge is the
    floor(lo_q (n-1))-th smallest z of the states (inference form), the top edge the largest,
    found by radix selection on the device; the edges equal fl32(lo + (hi - lo) i / n_bins)."""
    import torch
    rng = np.random.default_rng(8)
    S, H, n = 3, 64, 50_001
    mlp = P.we_mlp_create_init(S, H, seed=4)
    X = rng.integers(0, 400, size=(n, S)).astype(np.int32)
    X[:10] = X[10]                                        # ties
    xd = torch.as_tensor(X, device="cuda")
    z = mlp.forward(xd, bf16=True).cpu().numpy()
    zs = np.sort(z)
    for lo_q, nb in ((0.001, 100), (0.0, 7), (0.5, 1)):
        e = P.we_mlp_coordinate_edges(mlp, xd, nb, lo_q)
        lo = float(zs[int(np.floor(lo_q * (n - 1)))])
        hi = float(zs[-1])
        want = (lo + (hi - lo) * np.arange(nb + 1, dtype=np.float64) / nb).astype(np.float32)
        assert np.array_equal(e, want), (lo_q, nb)


def test_library_initial_weights():
    """we_mlp_create_init: deterministic for a seed, different across seeds, weights within
    +-1/sqrt(fan_in) and spread over that range, zero biases."""
    S, H = 5, 64
    a = P.we_mlp_create_init(S, H, seed=1).params()
    b = P.we_mlp_create_init(S, H, seed=1).params()
    c = P.we_mlp_create_init(S, H, seed=2).params()
    assert np.array_equal(a, b) and not np.array_equal(a, c)
    w1 = a[:H * S]
    b1 = a[H * S:H * S + H]
    w2 = a[H * S + H:H * S + H + H * H]
    assert np.all(b1 == 0) and a[-1] == 0
    assert np.abs(w1).max() <= 1 / np.sqrt(S) and np.abs(w1).max() > 0.9 / np.sqrt(S)
    assert np.abs(w2).max() <= 1 / np.sqrt(H) and abs(w2.mean()) < 0.05 / np.sqrt(H)
