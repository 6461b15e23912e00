"""The windowed oracle (tests/sampled_oracle.py) equals the full-grid oracle bit for bit
at sampled points, including points whose window wraps around the periodic edges."""
import numpy as np
import pytest

from workloads import euler, tgv

import sampled_oracle


@pytest.fixture(scope="module")
def phys(oracle_lib):
    from oracle import physics
    return physics


@pytest.mark.parametrize("steps", [1, 3])
def test_euler_window_equals_full_grid(phys, steps):
    n = 64
    U0 = euler.initial(n)
    dt = euler.CFL * phys.euler_dt_min(U0, 1.0 / n, 1.0 / n, euler.GAMMA)
    U = U0.copy()
    for _ in range(steps):
        phys.euler_step(U, dt, 1.0 / n, 1.0 / n, euler.GAMMA, euler.EPS4)
    rng = np.random.default_rng(7)
    pts = [(0, 0), (n - 1, 3), (31, 24), (40, n - 2)] + [tuple(rng.integers(0, n, 2)) for _ in range(12)]
    got = sampled_oracle.euler_points(phys, U0, pts, dt, 1.0 / n, 1.0 / n, steps, euler.GAMMA, euler.EPS4)
    want = np.array([U[:, y, x] for y, x in pts])
    assert np.array_equal(got, want)


def test_euler_window_too_narrow_differs(phys):
    """The reach is real: a window one cell too narrow changes the centre (near the
    square's edge, where the state varies)."""
    n = 64
    U0 = euler.initial(n)
    dt = euler.CFL * phys.euler_dt_min(U0, 1.0 / n, 1.0 / n, euler.GAMMA)
    U = U0.copy()
    phys.euler_step(U, dt, 1.0 / n, 1.0 / n, euler.GAMMA, euler.EPS4)
    y, x = 24, 24
    R = sampled_oracle.EULER_REACH - 1
    W = sampled_oracle._window(U0, (y, x), R)
    phys.euler_step(W, dt, 1.0 / n, 1.0 / n, euler.GAMMA, euler.EPS4)
    assert not np.array_equal(W[:, R, R], U[:, y, x])


def test_ns_window_equals_full_grid(phys):
    n = 32
    U0 = np.ascontiguousarray(tgv.initial(n))
    prm = phys.ns_params(tgv.GAMMA, tgv.MA, tgv.RE, tgv.PR, (tgv.h_of(n),) * 3)
    U = U0.copy()
    phys.ns_step(U, tgv.dt_of(n), prm)
    pts = [(0, 0, 0), (31, 5, 30), (16, 16, 16), (3, 29, 11)]
    got = sampled_oracle.ns_points(phys, U0, pts, tgv.dt_of(n), prm, 1)
    want = np.array([U[:, z, y, x] for z, y, x in pts])
    assert np.array_equal(got, want)
