"""Pins of the planner-network oracle: its gradient against central finite differences
of its own loss (a different computation: no chain rule), a closed form for the output
bias, and the Adam step's first-iteration property (the step is lr * sign(g))."""
import numpy as np

from oracle import mlp


def _data(seed, n=37):
    rng = np.random.default_rng(seed)
    return rng.normal(size=(n, 8)), rng.normal(size=(n, 2))


def test_gradient_matches_central_differences():
    p = mlp.init_params(3)
    X, T = _data(4)
    _, g = mlp.loss_grad(p, X, T)
    rng = np.random.default_rng(5)
    idx = rng.choice(mlp.NPARAMS, size=200, replace=False)
    h = 1e-6
    for i in idx:
        e = np.zeros_like(p)
        e[i] = h
        fd = (mlp.loss(p + e, X, T) - mlp.loss(p - e, X, T)) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(fd)), i


def test_output_bias_gradient_closed_form():
    """With all weights zero the output is b3, so dL/db3 = mean(b3 - t)."""
    p = np.zeros(mlp.NPARAMS)
    p[-2:] = [0.3, -1.2]
    X, T = _data(6)
    L, g = mlp.loss_grad(p, X, T)
    assert np.allclose(g[-2:], (p[-2:] - T).mean(axis=0), rtol=0, atol=1e-15)
    assert np.all(g[:-2] == 0)
    assert abs(L - np.sum((p[-2:] - T) ** 2) / (2 * len(T))) <= 1e-14


def test_adam_first_step_is_signed_lr():
    g = np.array([0.5, -2.0, 1e-3])
    p1, _, _ = mlp.adam_step(np.zeros(3), g, np.zeros(3), np.zeros(3), 1, lr=0.01)
    assert np.allclose(p1, -0.01 * np.sign(g), rtol=1e-5)
