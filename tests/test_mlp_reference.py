"""Pins of the FP64 reference network (oracle/mlp.py) that checks the GPU
training kernels: its gradient against central finite differences of its own
loss, and the symmetries the warm start relies on (odd in the input, so the
prediction flips with the data)."""
import numpy as np

from oracle import mlp

F, H = 25, 64


def _theta(rng, scale=1.0):
    W1 = rng.standard_normal((H, F)) * scale / np.sqrt(F)
    W2 = rng.standard_normal((H, H)) * scale / np.sqrt(H)
    w3 = rng.standard_normal(H) * scale / np.sqrt(H)
    return np.concatenate([W1.ravel(), W2.ravel(), w3])


def test_gradient_matches_finite_differences():
    rng = np.random.default_rng(0)
    th = _theta(rng)
    X = rng.standard_normal((37, F))
    T = rng.standard_normal(37)
    Wt = rng.uniform(0.1, 3.0, 37)
    _, g = mlp.loss_and_grad(th, X, T, F, H, Wt)
    # every w3 entry, and a seeded sample of W1 and W2 entries
    idx = np.concatenate([np.arange(H * F + H * H, H * F + H * H + H),
                          rng.choice(H * F, 40, replace=False),
                          H * F + rng.choice(H * H, 40, replace=False)])
    h = 1e-6
    for k in idx:
        e = np.zeros_like(th)
        e[k] = h
        fd = (mlp.loss_and_grad(th + e, X, T, F, H, Wt)[0] - mlp.loss_and_grad(th - e, X, T, F, H, Wt)[0]) / (2 * h)
        assert abs(fd - g[k]) <= 1e-7 * max(1.0, abs(g[k])) + 1e-9, (k, fd, g[k])


def test_network_is_odd_and_zero_at_zero():
    rng = np.random.default_rng(1)
    th = _theta(rng, 3.0)
    X = rng.standard_normal((50, F))
    assert np.allclose(mlp.forward(th, -X, F, H), -mlp.forward(th, X, F, H), atol=1e-14)
    assert np.all(mlp.forward(th, np.zeros((3, F)), F, H) == 0.0)


def test_loss_of_exact_targets_is_zero():
    rng = np.random.default_rng(2)
    th = _theta(rng)
    X = rng.standard_normal((20, F))
    loss, g = mlp.loss_and_grad(th, X, mlp.forward(th, X, F, H), F, H)
    assert loss < 1e-28 and np.abs(g).max() < 1e-13


def test_adam_first_step_moves_each_parameter_by_lr():
    # with bias correction the first Adam step is lr * sign(g) (|g| >> eps)
    th = np.zeros(5)
    g = np.array([1.0, -2.0, 0.5, 3.0, -0.1])
    th1, m, v = mlp.adam(th, np.zeros(5), np.zeros(5), g, 1, 0.01)
    assert np.allclose(th1, -0.01 * np.sign(g), rtol=1e-6)
