"""Plain FP64 reference of the warm-start network (test infrastructure only).

The learned warm start predicts, for every RWG edge i, the correction of the
cubic time extrapolation of its current from local features (the edge's and
its four neighbours' past currents and Jacobi-scaled right-hand sides, all
divided by their RMS).  The network is an odd three-layer perceptron without
biases,

    z1 = W1 x,  h1 = tanh(z1),  z2 = W2 h1,  h2 = tanh(z2),  y = w3 . h2,

so that flipping every input flips the output (the march is linear in the
incident field).  Loss of a batch: mean of w (y - t)^2, with sample weights w
(1 when none are given).

This module is the CPU check of the GPU forward and backward kernels: plain
numpy in float64, one formula per line, no batching tricks beyond matrix
products.  Parameters are flattened as [W1 (H x F, row-major), W2 (H x H),
w3 (H)].  Only tests may import it.
"""
from __future__ import annotations

import numpy as np


def unpack(theta: np.ndarray, F: int, H: int):
    theta = np.asarray(theta, dtype=np.float64)
    W1 = theta[: H * F].reshape(H, F)
    W2 = theta[H * F: H * F + H * H].reshape(H, H)
    w3 = theta[H * F + H * H: H * F + H * H + H]
    return W1, W2, w3


def forward(theta: np.ndarray, X: np.ndarray, F: int, H: int) -> np.ndarray:
    """y for every row of X (n x F)."""
    W1, W2, w3 = unpack(theta, F, H)
    h1 = np.tanh(X @ W1.T)
    h2 = np.tanh(h1 @ W2.T)
    return h2 @ w3


def loss_and_grad(theta: np.ndarray, X: np.ndarray, T: np.ndarray, F: int, H: int, W=None):
    """Weighted mean squared error over the batch and its gradient (chain
    rule, one layer at a time)."""
    X = np.asarray(X, dtype=np.float64)
    T = np.asarray(T, dtype=np.float64)
    w = np.ones(len(T)) if W is None else np.asarray(W, dtype=np.float64)
    W1, W2, w3 = unpack(theta, F, H)
    n = X.shape[0]
    h1 = np.tanh(X @ W1.T)          # n x H
    h2 = np.tanh(h1 @ W2.T)         # n x H
    y = h2 @ w3                     # n
    loss = float(np.mean(w * (y - T) ** 2))
    dy = 2.0 * w * (y - T) / n      # n
    g3 = h2.T @ dy                  # H
    dz2 = np.outer(dy, w3) * (1.0 - h2 ** 2)   # n x H
    g2 = dz2.T @ h1                 # H x H
    dz1 = (dz2 @ W2) * (1.0 - h1 ** 2)         # n x H
    g1 = dz1.T @ X                  # H x F
    return loss, np.concatenate([g1.ravel(), g2.ravel(), g3])


def adam(theta, m, v, g, t: int, lr: float, b1: float = 0.9, b2: float = 0.999, eps: float = 1e-8):
    """One Adam update (Kingma and Ba, 2015) with bias correction; returns
    the new (theta, m, v)."""
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    mh = m / (1 - b1 ** t)
    vh = v / (1 - b2 ** t)
    return theta - lr * mh / (np.sqrt(vh) + eps), m, v
