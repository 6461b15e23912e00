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


def test_forward_closed_form_abs_and_hinge():
    """Hand-set weights make the network compute y0 = |x0| + 1/4 and
    y1 = 2 max(x1 - 1, 0) - 1/2 (|x| = relu(x) + relu(-x)); this pins the wiring of
    every layer (which weight index feeds which unit, the biases, where the ReLUs sit)."""
    w = {name: np.zeros(shape) for name, shape in mlp.SHAPES}
    w["W1"][0, 0], w["W1"][1, 0] = 1.0, -1.0          # z1_0 = x0, z1_1 = -x0
    w["W1"][2, 1], w["b1"][2] = 1.0, -1.0             # z1_2 = x1 - 1
    w["b1"][3] = 5.0                                  # a live unit that no later weight reads
    w["W2"][0, 0], w["W2"][0, 1] = 1.0, 1.0           # z2_0 = |x0|
    w["W2"][1, 2], w["b2"][1] = 2.0, 0.5              # z2_1 = 2 max(x1 - 1, 0) + 1/2
    w["b2"][4] = -3.0                                 # a dead unit (ReLU of a negative)
    w["W3"][0, 0], w["b3"][0] = 1.0, 0.25
    w["W3"][1, 1], w["b3"][1] = 1.0, -1.0
    w["W3"][:, 4] = 7.0
    X = np.random.default_rng(8).uniform(-3, 3, size=(50, 8))
    y, _ = mlp.forward(mlp.pack(w), X)
    assert np.allclose(y[:, 0], np.abs(X[:, 0]) + 0.25, rtol=0, atol=1e-15)
    assert np.allclose(y[:, 1], 2 * np.maximum(X[:, 1] - 1, 0) - 0.5, rtol=0, atol=1e-15)


def test_adam_constant_gradient_steps():
    """Under a constant gradient the bias-corrected moments equal g and g^2 at every
    step, so each step moves by lr g / (|g| + eps): after t steps p = -t lr g / (|g| + eps).
    (At t = 1 a correction by (1 - beta) instead of (1 - beta^t) looks the same; this
    covers t up to 25.)"""
    g = np.array([0.5, -2.0, 1e-3, 3.0])
    p, m, v = np.zeros(4), np.zeros(4), np.zeros(4)
    lr, eps = 0.01, 1e-8
    for t in range(1, 26):
        p, m, v = mlp.adam_step(p, g, m, v, t, lr=lr, eps=eps)
        expect = -t * lr * g / (np.abs(g) + eps)
        assert np.allclose(p, expect, rtol=1e-12, atol=0), t
