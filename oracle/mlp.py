"""Float64 reference of the learned beam-width predictor. TEST INFRASTRUCTURE ONLY.

The paper has no learned component; this network is the search-budget
predictor of the GPU library, restated plainly so that its GPU forward pass,
gradients and Adam steps can be checked:

    x_hat = (x - mu) / sigma                        (per-feature standardisation)
    h1 = relu(W1^T x_hat + b1)                      W1: [F, 64]
    h2 = relu(W2^T h1 + b2)                         W2: [64, 64]
    y  = W3^T h2 + b3                               W3: [64, 2]
    loss = mean over rows and outputs of rho_q(t - y),
    rho_q(u) = max(q u, (q - 1) u)                  (pinball loss, quantile q)

Flat parameter layout (shared convention): W1 row-major [F * 64], b1 [64],
W2 [64 * 64], b2 [64], W3 [64 * 2], b3 [2].
"""
from __future__ import annotations

import numpy as np

HIDDEN = 64
OUT = 2


def n_params(F: int) -> int:
    return F * HIDDEN + HIDDEN + HIDDEN * HIDDEN + HIDDEN + HIDDEN * OUT + OUT


def unpack(p: np.ndarray, F: int):
    p = np.asarray(p, dtype=np.float64)
    o = 0
    W1 = p[o:o + F * HIDDEN].reshape(F, HIDDEN); o += F * HIDDEN
    b1 = p[o:o + HIDDEN]; o += HIDDEN
    W2 = p[o:o + HIDDEN * HIDDEN].reshape(HIDDEN, HIDDEN); o += HIDDEN * HIDDEN
    b2 = p[o:o + HIDDEN]; o += HIDDEN
    W3 = p[o:o + HIDDEN * OUT].reshape(HIDDEN, OUT); o += HIDDEN * OUT
    b3 = p[o:o + OUT]; o += OUT
    return W1, b1, W2, b2, W3, b3


def forward(p, X, mu, sigma):
    """Outputs y [B, 2] and the intermediates (x_hat, z1, h1, z2, h2)."""
    X = np.asarray(X, dtype=np.float64)
    F = X.shape[1]
    W1, b1, W2, b2, W3, b3 = unpack(p, F)
    xh = (X - np.asarray(mu, np.float64)) / np.asarray(sigma, np.float64)
    z1 = xh @ W1 + b1
    h1 = np.maximum(z1, 0.0)
    z2 = h1 @ W2 + b2
    h2 = np.maximum(z2, 0.0)
    y = h2 @ W3 + b3
    return y, (xh, z1, h1, z2, h2)


def pinball(y, T, q):
    u = np.asarray(T, np.float64) - y
    return float(np.mean(np.maximum(q * u, (q - 1.0) * u)))


def loss_and_grad(p, X, T, mu, sigma, q):
    """Pinball loss and its gradient with respect to the flat parameters
    (backpropagation written out layer by layer; at u = 0 the subgradient
    of the (1 - q) side is used)."""
    X = np.asarray(X, dtype=np.float64)
    B, F = X.shape
    W1, b1, W2, b2, W3, b3 = unpack(p, F)
    y, (xh, z1, h1, z2, h2) = forward(p, X, mu, sigma)
    u = np.asarray(T, np.float64) - y
    loss = float(np.mean(np.maximum(q * u, (q - 1.0) * u)))
    # d rho / d y = -q when t > y, (1 - q) otherwise; mean over B * OUT terms
    dy = np.where(u > 0, -q, 1.0 - q) / (B * OUT)
    dW3 = h2.T @ dy
    db3 = dy.sum(0)
    dh2 = dy @ W3.T
    dz2 = dh2 * (z2 > 0)
    dW2 = h1.T @ dz2
    db2 = dz2.sum(0)
    dh1 = dz2 @ W2.T
    dz1 = dh1 * (z1 > 0)
    dW1 = xh.T @ dz1
    db1 = dz1.sum(0)
    g = np.concatenate([dW1.ravel(), db1, dW2.ravel(), db2, dW3.ravel(), db3])
    return loss, g


def adam_step(p, g, m, v, t, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (Kingma & Ba) at step t >= 1; returns (p, m, v)."""
    m = beta1 * m + (1 - beta1) * g
    v = beta2 * v + (1 - beta2) * g * g
    mh = m / (1 - beta1 ** t)
    vh = v / (1 - beta2 ** t)
    return p - lr * mh / (np.sqrt(vh) + eps), m, v
