"""Oracle step functions of the PDE workloads (plain periodic FP64, see physics.c).

TEST INFRASTRUCTURE (see the package docstring). Arrays are numpy float64 with the
component axis first: Euler U is (4, ny, nx), Navier-Stokes U is (5, nz, ny, nx);
no halos, periodic in every axis.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import lib as _lib


def _L():
    L = _lib()
    if not getattr(L, "_phys_ready", False):
        P, I, D = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
        L.or_euler_step.argtypes = [I, I, P, D, D, D, D, D]
        L.or_euler_dt.argtypes = [I, I, P, D, D, D]
        L.or_euler_dt.restype = D
        L.or_ns_residual.argtypes = [I, I, I, P, P, P]
        L.or_ns_step.argtypes = [I, I, I, P, D, P]
        L._phys_ready = True
    return L


def _c(a):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(ctypes.c_void_p)


def euler_step(U: np.ndarray, dt: float, dx: float, dy: float, gamma: float = 1.4, eps4: float = 1.0 / 64):
    """One MacCormack step with fourth-order dissipation, in place. U: (4, ny, nx)."""
    _, ny, nx = U.shape
    _L().or_euler_step(nx, ny, _c(U), dt, dx, dy, gamma, eps4)
    return U


def euler_dt_min(U: np.ndarray, dx: float, dy: float, gamma: float = 1.4) -> float:
    """min over cells of min(dx/(|u|+c), dy/(|v|+c)); the time step is CFL times this."""
    _, ny, nx = U.shape
    return float(_L().or_euler_dt(nx, ny, _c(U), dx, dy, gamma))


def ns_params(gamma=1.4, Ma=0.1, Re=1600.0, Pr=0.71, h=(1.0, 1.0, 1.0)):
    return np.array([gamma, Ma, Re, Pr, h[0], h[1], h[2]], dtype=np.float64)


def ns_residual(U: np.ndarray, prm: np.ndarray) -> np.ndarray:
    _, nz, ny, nx = U.shape
    R = np.empty_like(U)
    _L().or_ns_residual(nx, ny, nz, _c(U), _c(prm), _c(R))
    return R


def ns_step(U: np.ndarray, dt: float, prm: np.ndarray):
    """One low-storage RK3 step (three stages), in place. U: (5, nz, ny, nx)."""
    _, nz, ny, nx = U.shape
    _L().or_ns_step(nx, ny, nz, _c(U), dt, _c(prm))
    return U
