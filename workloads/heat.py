"""2-D heat chain: explicit 5-point diffusion with a zero Dirichlet boundary.

Per time step (one chain holds `steps` steps):
  loop A  u_new = 0.6*u + 0.1*(u_E + u_W + u_N + u_S)   (u + 0.1 * 5-point Laplacian)
  loop B  u = u_new
  loop R  max |u| over the interior (one reduction handle per step)
Interior n x n, halo 1 (held at zero). Initial data: U(0,1) from a seed, or the
discrete eigenmode sin(pi*(x+1)/(n+1)) * sin(pi*(y+1)/(n+1)).
"""
from __future__ import annotations

import numpy as np

from .spec import READ, REDUCE, WRITE, Arg, DatSpec, Loop, RedSpec

SEED = 1709 + 1
STENCIL5 = [(0, 0), (1, 0), (-1, 0), (0, 1), (0, -1)]


def initial(n: int = 256, kind: str = "random", seed: int = SEED) -> np.ndarray:
    u = np.zeros((n + 2, n + 2))
    if kind == "random":
        u[1:-1, 1:-1] = np.random.default_rng(seed).uniform(0.0, 1.0, size=(n, n))
    elif kind == "eigen":
        s = np.sin(np.pi * np.arange(1, n + 1) / (n + 1))
        u[1:-1, 1:-1] = np.outer(s, s)
    else:
        raise ValueError(kind)
    return u


def build(n: int = 256, steps: int = 10, kind: str = "random", seed: int = SEED,
          dtype: str = "f64"):
    """Return (datasets, reductions, loops) of one chain of `steps` heat steps."""
    dats = [DatSpec("u", (n, n), (1, 1), (1, 1), dtype, init=initial(n, kind, seed)),
            DatSpec("u_new", (n, n), (1, 1), (1, 1), dtype, init=np.zeros((n + 2, n + 2)))]
    reds = [RedSpec(f"max{s}", "max") for s in range(steps)]
    loops = []
    for s in range(steps):
        loops.append(Loop("lincomb", (0, 0), (n, n),
                          [Arg("u_new", WRITE), Arg("u", READ, STENCIL5)],
                          [0.0, 0.6, 0.1, 0.1, 0.1, 0.1]))
        loops.append(Loop("copy", (0, 0), (n, n), [Arg("u", WRITE), Arg("u_new", READ)]))
        loops.append(Loop("reduce", (0, 0), (n, n),
                          [Arg("u", READ), Arg(f"max{s}", REDUCE)], [1.0]))
    return dats, reds, loops
