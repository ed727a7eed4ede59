"""FP64 reference of the learned progress coordinate.  TEST INFRASTRUCTURE ONLY.

z(x) = w3 . silu(W2 silu(W1 phi + b1) + b2) + b3, phi = log1p(x); loss = mean BCE with logits
against labels in [0,1]; gradients by hand-written backpropagation (checked against central
differences in the tests); Adam as in Kingma & Ba (2015).  Weights can be rounded to BF16 with
round-to-nearest-even to mirror the inference path.
"""
import numpy as np


def unpack(p, n_in, H):
    p = np.asarray(p, dtype=np.float64)
    o = 0
    W1 = p[o:o + H * n_in].reshape(H, n_in); o += H * n_in
    b1 = p[o:o + H]; o += H
    W2 = p[o:o + H * H].reshape(H, H); o += H * H
    b2 = p[o:o + H]; o += H
    w3 = p[o:o + H]; o += H
    b3 = p[o]
    return W1, b1, W2, b2, w3, b3


def _sig(a):
    return 1.0 / (1.0 + np.exp(-a))


def forward(p, states, n_in, H):
    W1, b1, W2, b2, w3, b3 = unpack(p, n_in, H)
    phi = np.log1p(np.asarray(states, dtype=np.float64))
    a1 = phi @ W1.T + b1
    h1 = a1 * _sig(a1)
    a2 = h1 @ W2.T + b2
    h2 = a2 * _sig(a2)
    return h2 @ w3 + b3


def loss_and_grad(p, states, labels, n_in, H):
    W1, b1, W2, b2, w3, b3 = unpack(p, n_in, H)
    y = np.asarray(labels, dtype=np.float64)
    B = len(y)
    phi = np.log1p(np.asarray(states, dtype=np.float64))
    a1 = phi @ W1.T + b1
    s1 = _sig(a1)
    h1 = a1 * s1
    a2 = h1 @ W2.T + b2
    s2 = _sig(a2)
    h2 = a2 * s2
    z = h2 @ w3 + b3
    loss = np.mean(np.maximum(z, 0) - z * y + np.log1p(np.exp(-np.abs(z))))
    dz = (_sig(z) - y) / B
    dw3 = h2.T @ dz
    db3 = dz.sum()
    da2 = np.outer(dz, w3) * (s2 * (1 + a2 * (1 - s2)))
    dW2 = da2.T @ h1
    db2 = da2.sum(0)
    da1 = (da2 @ W2) * (s1 * (1 + a1 * (1 - s1)))
    dW1 = da1.T @ phi
    db1 = da1.sum(0)
    g = np.concatenate([dW1.ravel(), db1, dW2.ravel(), db2, dw3, [db3]])
    return loss, g


def adam_step(p, g, m, v, t, lr, b1=0.9, b2=0.999, eps=1e-8):
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    mh = m / (1 - b1 ** t)
    vh = v / (1 - b2 ** t)
    return p - lr * mh / (np.sqrt(vh) + eps), m, v


def bf16_round(x):
    """Round float32 values to BF16 (round to nearest, ties to even), returned as float32."""
    u = np.asarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) >> 16 << 16
    return u.astype(np.uint32).view(np.float32)


def inference_params(p, n_in, H):
    """The inference path's parameters: weights rounded to BF16, biases kept in FP32."""
    p = np.asarray(p, dtype=np.float32).copy()
    o = 0
    p[o:o + H * n_in] = bf16_round(p[o:o + H * n_in]); o += H * n_in + H
    p[o:o + H * H] = bf16_round(p[o:o + H * H]); o += H * H + H
    p[o:o + H] = bf16_round(p[o:o + H])
    return p


def bins_of(z, edges):
    """Bin k holds [edges[k], edges[k+1]); values beyond the ends fall in the end bins."""
    e = np.asarray(edges, dtype=np.float64)
    return np.clip(np.searchsorted(e, np.asarray(z, dtype=np.float64), side="right") - 1, 0, len(e) - 2)
