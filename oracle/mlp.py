"""Oracle of the tile-planner network: FP64 numpy forward, backward and Adam step.

TEST INFRASTRUCTURE (see the package docstring). The network is 8 -> 64 -> 64 -> 2 with
ReLU hidden layers; the parameter vector is W1[64][8], b1[64], W2[64][64], b2[64],
W3[2][64], b3[2]; the loss over n samples is L = sum (y - t)^2 / (2n). The backward pass
is the chain rule written out layer by layer.
"""
from __future__ import annotations

import numpy as np

IN, H, OUT = 8, 64, 2
SHAPES = [("W1", (H, IN)), ("b1", (H,)), ("W2", (H, H)), ("b2", (H,)), ("W3", (OUT, H)), ("b3", (OUT,))]
NPARAMS = sum(int(np.prod(s)) for _, s in SHAPES)


def unpack(p: np.ndarray) -> dict:
    out, o = {}, 0
    for name, shape in SHAPES:
        k = int(np.prod(shape))
        out[name] = np.asarray(p[o:o + k], dtype=np.float64).reshape(shape)
        o += k
    return out


def pack(d: dict) -> np.ndarray:
    return np.concatenate([np.asarray(d[name], dtype=np.float64).ravel() for name, _ in SHAPES])


def forward(p: np.ndarray, X: np.ndarray):
    w = unpack(p)
    X = np.asarray(X, dtype=np.float64)
    z1 = X @ w["W1"].T + w["b1"]
    a1 = np.maximum(z1, 0.0)
    z2 = a1 @ w["W2"].T + w["b2"]
    a2 = np.maximum(z2, 0.0)
    y = a2 @ w["W3"].T + w["b3"]
    return y, (X, z1, a1, z2, a2)


def loss(p, X, T) -> float:
    y, _ = forward(p, X)
    return float(np.sum((y - np.asarray(T, dtype=np.float64)) ** 2) / (2 * len(X)))


def loss_grad(p, X, T):
    """(loss, gradient) by the chain rule."""
    w = unpack(p)
    y, (X, z1, a1, z2, a2) = forward(p, X)
    n = len(X)
    dy = (y - np.asarray(T, dtype=np.float64)) / n          # dL/dy
    g = {"W3": dy.T @ a2, "b3": dy.sum(axis=0)}
    dz2 = (dy @ w["W3"]) * (z2 > 0)
    g["W2"], g["b2"] = dz2.T @ a1, dz2.sum(axis=0)
    dz1 = (dz2 @ w["W2"]) * (z1 > 0)
    g["W1"], g["b1"] = dz1.T @ X, dz1.sum(axis=0)
    return float(np.sum((y - T) ** 2) / (2 * n)), pack(g)


def adam_step(p, g, m, v, t, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam step (Kingma & Ba): returns new (p, m, v); t counts from 1."""
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    mh = m / (1 - b1 ** t)
    vh = v / (1 - b2 ** t)
    return p - lr * mh / (np.sqrt(vh) + eps), m, v


def init_params(seed: int) -> np.ndarray:
    """He-uniform weights, zero biases (the initialisation the planner trainer uses)."""
    rng = np.random.default_rng(seed)
    d = {}
    for name, shape in SHAPES:
        if name.startswith("W"):
            lim = np.sqrt(6.0 / shape[1])
            d[name] = rng.uniform(-lim, lim, size=shape)
        else:
            d[name] = np.zeros(shape)
    return pack(d)
