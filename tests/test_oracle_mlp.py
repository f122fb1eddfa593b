"""Pins of the oracle's MLP: finite differences of its loss, and a network
whose output is known in closed form."""
import numpy as np

from oracle import mlp


def test_gradient_matches_finite_differences():
    rng = np.random.default_rng(0)
    p = rng.normal(0, 0.5, mlp.NPARAM)
    X = rng.normal(0, 1, (40, 4))
    T = rng.normal(0, 1, 40)
    _, g = mlp.loss_and_grad(p, X, T)
    h = 1e-6
    for i in rng.choice(mlp.NPARAM, 120, replace=False):
        q = p.copy(); q[i] += h
        lp, _ = mlp.loss_and_grad(q, X, T)
        q[i] -= 2 * h
        lm, _ = mlp.loss_and_grad(q, X, T)
        assert abs((lp - lm) / (2 * h) - g[i]) < 1e-6 * max(1.0, abs(g[i]))


def test_closed_form_network():
    # W1 = [I4; 0], W2 = I (on the first 4 units), W3 = ones on them: for
    # nonnegative inputs y = b3 + sum(x)
    d = {"W1": np.vstack([np.eye(4), np.zeros((28, 4))]), "b1": np.zeros(32),
         "W2": np.eye(32), "b2": np.zeros(32), "W3": np.r_[np.ones(4), np.zeros(28)],
         "b3": np.array([0.5])}
    X = np.abs(np.random.default_rng(1).normal(0, 1, (10, 4)))
    y, _ = mlp.forward(mlp.pack(d), X)
    assert np.allclose(y, X.sum(1) + 0.5)
    assert mlp.NPARAM == 1249
