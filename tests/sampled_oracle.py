"""Oracle values at single points of grids too large for the oracle to step whole.

An explicit step reaches a fixed distance: one Euler MacCormack step with fourth-order
dissipation reads U up to 2 cells away, one Navier-Stokes RK3 step up to 12 (4 per
stage). After k steps the value at a point therefore depends only on the state within
k times that reach. These helpers cut a periodic window of the initial state around the
point, wide enough that the wrap at the window's edge cannot reach its centre within k
steps, step the window with the oracle's full step functions, and return the centre.
The oracle evaluates every point of the window with the same operations, in the same
order, on the same inputs as on the full grid, so the centre is bit-identical to the
full-grid oracle's value there (checked on grids the oracle can step whole).
"""
from __future__ import annotations

import numpy as np

EULER_REACH = 2
NS_REACH = 12


def _window(U, centre, R):
    """U[:, c - R .. c + R] (periodic) for every spatial axis; centre in array-axis order."""
    idx = [np.arange(c - R, c + R + 1) % n for c, n in zip(centre, U.shape[1:])]
    return np.ascontiguousarray(U[np.ix_(range(U.shape[0]), *idx)])


def euler_points(physics, U0, points, dt, dx, dy, steps, gamma, eps4):
    """Conserved state after `steps` steps of fixed dt at each (y, x) of `points`."""
    R = EULER_REACH * steps + 1
    out = []
    for y, x in points:
        W = _window(U0, (y, x), R)
        for _ in range(steps):
            physics.euler_step(W, dt, dx, dy, gamma, eps4)
        out.append(W[:, R, R].copy())
    return np.array(out)


def ns_points(physics, U0, points, dt, prm, steps):
    """Conserved state after `steps` RK3 steps at each (z, y, x) of `points`."""
    R = NS_REACH * steps + 1
    out = []
    for z, y, x in points:
        W = _window(U0, (z, y, x), R)
        for _ in range(steps):
            physics.ns_step(W, dt, prm)
        out.append(W[:, R, R, R].copy())
    return np.array(out)
