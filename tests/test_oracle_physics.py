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
    ho = 1.37 * h      # spacing of the other axis: the mode must depend on h alone
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
        phys.euler_step(U, dt, h if axis == 0 else ho, ho if axis == 0 else h, GAMMA, euler.EPS4)
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


@pytest.mark.parametrize("u,v,dx,dy", [(0.4, -1.0, 0.1, 0.05), (-2.5, 0.3, 0.04, 0.1)])
def test_euler_dt_uniform_closed_form(phys, u, v, dx, dy):
    """dt of a uniform state; the first case is limited along y, the second along x."""
    U = _uniform_euler(8, rho=0.5, u=u, v=v, p=2.0)
    c = math.sqrt(GAMMA * 2.0 / 0.5)
    ax, ay = dx / (abs(u) + c), dy / (abs(v) + c)
    expect = min(ax, ay)
    assert abs(ax - ay) > 0.05 * expect
    assert abs(phys.euler_dt_min(U, dx, dy, GAMMA) - expect) <= 1e-15 * expect


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


# Closed forms of one residual evaluation on anisotropic grids: a sampled sinusoid
# sin(theta i) along axis a (grid spacing h_a) has D sin = sig cos and D cos = -sig sin
# exactly, sig = (8 sin theta - sin 2 theta) / (6 h_a); products of sinusoids reduce to
# sums of harmonics (sin^2 = (1 - cos 2t)/2, sin^3 = (3 sin t - sin 3t)/4, sin cos = sin 2t / 2).
NS_SHAPE = (8, 10, 12)               # (nz, ny, nx): every axis a different length
NS_H = (0.55, 0.7, 0.45)             # (hx, hy, hz): every axis a different spacing
NS_RE, NS_MA, NS_PR = 100.0, 0.1, 0.71


def _axis_phase(axis, m=1):
    K, J, I = np.meshgrid(*[np.arange(s) for s in NS_SHAPE], indexing="ij")
    n = NS_SHAPE[2 - axis]
    return 2 * math.pi * m / n, [I, J, K][axis]


def _sig(theta, h):
    return (8 * math.sin(theta) - math.sin(2 * theta)) / (6 * h)


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_ns_residual_heat_conduction_closed_form(phys, axis):
    """At rest with uniform pressure and T = 1 + e sin(theta i_a): mass and momentum
    residuals vanish and the energy residual is the discrete conduction term
    k D(D T) = -k sig^2 e sin(theta i_a), k = mu / ((gamma - 1) Ma^2 Pr)."""
    theta, idx = _axis_phase(axis)
    eps = 0.1
    T = 1.0 + eps * np.sin(theta * idx)
    p0 = 1.0 / (GAMMA * NS_MA ** 2)
    rho = GAMMA * NS_MA ** 2 * p0 / T
    z = np.zeros(NS_SHAPE)
    U = _ns_state(rho, z, z, z, np.full(NS_SHAPE, p0))
    prm = phys.ns_params(GAMMA, NS_MA, NS_RE, NS_PR, NS_H)
    R = phys.ns_residual(U, prm)
    kc = (1.0 / NS_RE) / ((GAMMA - 1) * NS_MA ** 2 * NS_PR)
    expect = -kc * _sig(theta, NS_H[axis]) ** 2 * eps * np.sin(theta * idx)
    scale = np.max(np.abs(expect))
    assert np.max(np.abs(R[4] - expect)) <= 1e-12 * scale
    assert np.max(np.abs(R[:4])) <= 1e-12 * scale


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_ns_residual_longitudinal_wave_closed_form(phys, axis):
    """Uniform density and pressure, velocity u_a = e sin(theta i_a) along its own axis
    (compressive, so div u and the -2/3 div u part of the stress enter):
      R_rho = -rho e s1 cos t,
      R_a   = -rho e^2 s2/2 sin 2t - (4/3) mu e s1^2 sin t,
      R_E   = -(gamma p/(gamma-1)) e s1 cos t - (rho e^3/8)(3 s1 cos t - s3 cos 3t)
              + (2/3) mu e^2 s1 s2 cos 2t,
    s_j = sig(j theta), t = theta i_a; the other momentum residuals vanish."""
    theta, idx = _axis_phase(axis)
    h = NS_H[axis]
    s1, s2, s3 = _sig(theta, h), _sig(2 * theta, h), _sig(3 * theta, h)
    eps, rho0 = 0.1, 1.0
    p0 = 1.0 / (GAMMA * NS_MA ** 2)
    t = theta * idx
    vel = [np.zeros(NS_SHAPE) for _ in range(3)]
    vel[axis] = eps * np.sin(t)
    U = _ns_state(np.full(NS_SHAPE, rho0), vel[0], vel[1], vel[2], np.full(NS_SHAPE, p0))
    prm = phys.ns_params(GAMMA, NS_MA, NS_RE, NS_PR, NS_H)
    R = phys.ns_residual(U, prm)
    mu = 1.0 / NS_RE
    e_rho = -rho0 * eps * s1 * np.cos(t)
    e_mom = -rho0 * eps ** 2 * s2 / 2 * np.sin(2 * t) - (4.0 / 3.0) * mu * eps * s1 ** 2 * np.sin(t)
    e_E = (-(GAMMA * p0 / (GAMMA - 1)) * eps * s1 * np.cos(t)
           - (rho0 * eps ** 3 / 8) * (3 * s1 * np.cos(t) - s3 * np.cos(3 * t))
           + (2.0 / 3.0) * mu * eps ** 2 * s1 * s2 * np.cos(2 * t))
    tol = 1e-12 * np.max(np.abs(e_E))
    assert np.max(np.abs(R[0] - e_rho)) <= tol
    assert np.max(np.abs(R[1 + axis] - e_mom)) <= tol
    assert np.max(np.abs(R[4] - e_E)) <= tol
    for b in range(3):
        if b != axis:
            assert np.max(np.abs(R[1 + b])) <= tol


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_ns_residual_pressure_wave_closed_form(phys, axis):
    """At rest with uniform density and p = p0 + e sin(theta i_a): only the momentum
    along a feels the pressure, R_a = -e sig cos t; the energy residual is the
    conduction of T = gamma Ma^2 p / rho, R_E = -k (gamma Ma^2 / rho) sig^2 e sin t."""
    theta, idx = _axis_phase(axis)
    sig = _sig(theta, NS_H[axis])
    eps, rho0 = 0.5, 1.3
    p0 = 1.0 / (GAMMA * NS_MA ** 2)
    t = theta * idx
    z = np.zeros(NS_SHAPE)
    U = _ns_state(np.full(NS_SHAPE, rho0), z, z, z, p0 + eps * np.sin(t))
    prm = phys.ns_params(GAMMA, NS_MA, NS_RE, NS_PR, NS_H)
    R = phys.ns_residual(U, prm)
    kc = (1.0 / NS_RE) / ((GAMMA - 1) * NS_MA ** 2 * NS_PR)
    e_mom = -eps * sig * np.cos(t)
    e_E = -kc * (GAMMA * NS_MA ** 2 / rho0) * sig ** 2 * eps * np.sin(t)
    tol = 1e-12 * p0
    assert np.max(np.abs(R[1 + axis] - e_mom)) <= tol
    assert np.max(np.abs(R[4] - e_E)) <= tol
    assert np.max(np.abs(R[0])) <= tol
    for b in range(3):
        if b != axis:
            assert np.max(np.abs(R[1 + b])) <= tol
