"""Pins of the oracle's PDE step functions (Euler MacCormack, Navier-Stokes RK3).

Each test compares the oracle with a fact that does not come from the oracle:
discrete conservation on periodic grids, exact preservation of uniform states, the
x <-> y mirror symmetry, the closed-form amplification factor of a single Fourier
mode (the scheme is exactly linear on an entropy wave, linear to first order on an
acoustic wave and on a viscous shear wave), and the TGV initial kinetic energy.
"""
import cmath
import math

import numpy as np
import pytest

from workloads import euler, tgv

GAMMA = 1.4


@pytest.fixture(scope="module")
def phys(oracle_lib):
    from oracle import physics
    return physics


# ------------------------------------------------------------------------ Euler
def _uniform_euler(n, rho=0.7, u=0.3, v=-0.2, p=1.1):
    U = np.zeros((4, n, n))
    U[0], U[1], U[2] = rho, rho * u, rho * v
    U[3] = p / (GAMMA - 1) + 0.5 * rho * (u * u + v * v)
    return U


def test_euler_uniform_state_is_preserved(phys):
    U = _uniform_euler(24)
    ref = U.copy()
    for _ in range(5):
        phys.euler_step(U, 0.01, 1 / 24, 1 / 24, GAMMA, euler.EPS4)
    assert np.allclose(U, ref, rtol=1e-14, atol=1e-15)


def test_euler_conservation_square_problem(phys):
    n = 64
    U = euler.initial(n)
    tot0 = U.reshape(4, -1).sum(axis=1)
    scale = np.abs(U).reshape(4, -1).sum(axis=1) + 1.0
    for _ in range(10):
        dt = euler.CFL * phys.euler_dt_min(U, 1 / n, 1 / n, GAMMA)
        phys.euler_step(U, dt, 1 / n, 1 / n, GAMMA, euler.EPS4)
    tot = U.reshape(4, -1).sum(axis=1)
    assert np.all(np.abs(tot - tot0) <= 1e-13 * scale)
    assert np.all(np.isfinite(U))


def test_euler_transpose_symmetry(phys):
    """The square problem is symmetric under x <-> y (with mx <-> my); a scheme that
    treats the two axes differently (wrong lambda, G built from u) breaks it."""
    n = 48
    U = euler.initial(n)
    U[0] += 0.05 * np.outer(np.sin(2 * np.pi * np.arange(n) / n), np.sin(2 * np.pi * np.arange(n) / n))
    for _ in range(6):
        phys.euler_step(U, 0.002, 1 / n, 1 / n, GAMMA, euler.EPS4)
    assert np.allclose(U[0], U[0].T, rtol=0, atol=1e-13)
    assert np.allclose(U[3], U[3].T, rtol=0, atol=1e-13)
    assert np.allclose(U[1], U[2].T, rtol=0, atol=1e-13)
    assert np.max(np.abs(U[1])) > 1e-3   # the state did move


def _maccormack_factor(nu, theta, eps4):
    """Amplification of e^{i theta j} under one predictor-corrector step of linear
    advection with Courant number nu plus -eps4 * (fourth difference)."""
    pred = 1 - nu * (cmath.exp(1j * theta) - 1)
    corr = pred * (1 - nu * (1 - cmath.exp(-1j * theta)))
    return 0.5 * (1 + corr) - eps4 * 16 * math.sin(theta / 2) ** 4


@pytest.mark.parametrize("axis,k", [(0, 3), (1, 2)])
def test_euler_entropy_wave_closed_form(phys, axis, k):
    """rho = 1 + e sin(k x_j), constant velocity a along that axis and constant p: the
    scheme acts linearly on rho; each step multiplies the mode by the closed-form
    MacCormack factor (with the fourth-order dissipation)."""
    n, eps, a, p0, steps = 32, 1e-2, 0.6, 1.0, 15
    h = 1.0 / n
    dt = 0.4 * h
    j = np.arange(n)
    mode = np.exp(1j * 2 * np.pi * k * j / n)
    rho1 = 1.0 + eps * mode.imag
    rho = rho1[None, :] if axis == 0 else rho1[:, None]
    rho = np.broadcast_to(rho, (n, n)).copy()
    U = np.zeros((4, n, n))
    U[0] = rho
    U[1 + axis] = rho * a
    U[3] = p0 / (GAMMA - 1) + 0.5 * rho * a * a
    for _ in range(steps):
        phys.euler_step(U, dt, h, h, GAMMA, euler.EPS4)
    G = _maccormack_factor(a * dt / h, 2 * np.pi * k / n, euler.EPS4)
    expect = 1.0 + eps * (G ** steps * mode).imag
    got = U[0][0, :] if axis == 0 else U[0][:, 0]
    assert np.max(np.abs(got - expect)) <= 1e-12
    mom = U[1 + axis][0, :] if axis == 0 else U[1 + axis][:, 0]
    assert np.max(np.abs(mom - a * expect)) <= 1e-12


def test_euler_acoustic_wave_linear_response(phys):
    """A small right-running acoustic wave (rho' = e, u' = e c/rho, p' = e c^2) evolves
    with the scalar factor of Courant number (u + c) dt/dx to first order in e."""
    n, eps, steps = 40, 1e-7, 12
    rho0, p0 = 1.0, 1.0
    c = math.sqrt(GAMMA * p0 / rho0)
    h = 1.0 / n
    dt = 0.3 * h / c
    k = 2
    mode = np.exp(1j * 2 * np.pi * k * np.arange(n) / n)
    s = mode.imag
    rho = rho0 + eps * s
    u = eps * c / rho0 * s
    p = p0 + eps * c * c * s
    U = np.zeros((4, n, n))
    U[0] = rho[None, :]
    U[1] = (rho * u)[None, :]
    U[3] = (p / (GAMMA - 1) + 0.5 * rho * u * u)[None, :]
    for _ in range(steps):
        phys.euler_step(U, dt, h, h, GAMMA, euler.EPS4)
    G = _maccormack_factor(c * dt / h, 2 * np.pi * k / n, euler.EPS4)
    expect = eps * (G ** steps * mode).imag
    assert np.max(np.abs((U[0][0] - rho0) - expect)) <= 1e-4 * eps


def test_euler_dt_uniform_closed_form(phys):
    U = _uniform_euler(8, rho=0.5, u=0.4, v=-1.0, p=2.0)
    c = math.sqrt(GAMMA * 2.0 / 0.5)
    expect = min(0.1 / (0.4 + c), 0.05 / (1.0 + c))
    assert abs(phys.euler_dt_min(U, 0.1, 0.05, GAMMA) - expect) <= 1e-15 * expect


# ---------------------------------------------------------------- Navier-Stokes
def _ns_state(rho, u, v, w, p):
    E = p / (GAMMA - 1) + 0.5 * rho * (u * u + v * v + w * w)
    return np.ascontiguousarray(np.stack([rho, rho * u, rho * v, rho * w, E]).astype(np.float64))


def _d1_symbol(k, h):
    """Fourier symbol of the fourth-order central difference on sin/cos(k x)."""
    return (8 * math.sin(k * h) - math.sin(2 * k * h)) / (6 * h)


def _rk3(z):
    return 1 + z + z * z / 2 + z ** 3 / 6


def test_tgv_initial_kinetic_energy_and_momentum():
    U = tgv.initial(16)
    ke = 0.5 * (U[1] ** 2 + U[2] ** 2 + U[3] ** 2) / U[0]
    assert abs(ke.mean() - 1.0 / 8.0) <= 1e-15
    assert np.all(np.abs(U[1:4].reshape(3, -1).sum(axis=1)) <= 1e-11)


def test_ns_conservation_tgv(phys):
    n = 16
    U = np.ascontiguousarray(tgv.initial(n))
    prm = phys.ns_params(h=(tgv.h_of(n),) * 3)
    tot0 = U.reshape(5, -1).sum(axis=1)
    scale = np.abs(U).reshape(5, -1).sum(axis=1) + np.abs(U[1:4]).sum()  # momentum scale for w = 0
    for _ in range(2):
        phys.ns_step(U, tgv.dt_of(n), prm)
    tot = U.reshape(5, -1).sum(axis=1)
    assert np.all(np.abs(tot - tot0) <= 1e-13 * scale)


@pytest.mark.parametrize("axis_u,axis_vary", [(0, 1), (2, 0), (1, 2)])
def test_ns_viscous_shear_wave_closed_form(phys, axis_u, axis_vary):
    """Velocity component axis_u = e sin(k x_vary): the momentum of that component
    evolves linearly (to O(e^2)) as rho u_n = P(z)^n rho u_0, z = -mu D1(k)^2 dt,
    P the RK3 stability polynomial."""
    n, k, eps, steps = 16, 2, 1e-5, 4
    h = 2 * math.pi / n
    x = np.arange(n) * h
    grid = np.meshgrid(x, x, x, indexing="ij")        # (z, y, x)
    coord = grid[2 - axis_vary]
    vel = [np.zeros((n, n, n)) for _ in range(3)]
    vel[axis_u] = eps * np.sin(k * coord)
    p0 = 1.0 / (GAMMA * tgv.MA ** 2)
    U = _ns_state(np.ones((n, n, n)), vel[0], vel[1], vel[2], np.full((n, n, n), p0))
    mom0 = U[1 + axis_u].copy()
    prm = phys.ns_params(h=(h, h, h))
    dt = 0.05
    for _ in range(steps):
        phys.ns_step(U, dt, prm)
    z = -(1.0 / tgv.RE) * _d1_symbol(k, h) ** 2 * dt
    expect = _rk3(z) ** steps * mom0
    assert np.max(np.abs(U[1 + axis_u] - expect)) <= 1e-9 * eps
    assert abs(_rk3(z) ** steps - 1) > 1e-4   # the wave did decay


@pytest.mark.parametrize("axis", [0, 2])
def test_ns_inviscid_entropy_wave_closed_form(phys, axis):
    """Inviscid (Re <= 0), rho = 1 + e sin(k x_a), velocity a0 along axis a, constant p:
    every component's perturbation is multiplied per step by P(z), z = -i a0 D1(k) dt."""
    n, k, eps, a0, steps = 16, 1, 1e-3, 0.8, 5
    h = 2 * math.pi / n
    x = np.arange(n) * h
    grid = np.meshgrid(x, x, x, indexing="ij")
    mode = np.exp(1j * k * grid[2 - axis])
    rho = 1.0 + eps * mode.imag
    vel = [np.zeros((n, n, n)) for _ in range(3)]
    vel[axis] = np.full((n, n, n), a0)
    U = _ns_state(rho, vel[0], vel[1], vel[2], np.full((n, n, n), 50.0))
    prm = phys.ns_params(Re=0.0, h=(h, h, h))
    dt = 0.1 * h / a0
    for _ in range(steps):
        phys.ns_step(U, dt, prm)
    z = -1j * a0 * _d1_symbol(k, h) * dt
    expect = 1.0 + eps * (_rk3(z) ** steps * mode).imag
    assert np.max(np.abs(U[0] - expect)) <= 1e-12
    assert np.max(np.abs(U[1 + axis] - a0 * expect)) <= 1e-12
