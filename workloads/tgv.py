"""3-D compressible Navier-Stokes Taylor-Green vortex (stand-in for the OpenSBLI test case
of arXiv 1709.02125 Sec. 5.1).

Periodic cube [0, 2 pi)^3 with n^3 points (h = 2 pi / n); rho0 = V0 = L = 1, Re = 1600,
Ma = 0.1, Pr = 0.71, gamma = 1.4, p0 = 1 / (gamma Ma^2):
  u = sin x cos y cos z, v = -cos x sin y cos z, w = 0, rho = 1,
  p = p0 + (cos 2x + cos 2y)(cos 2z + 2) / 16.
Fixed time step dt = 0.5 h / (1 + 1/Ma) (no reduction inside the step, as in the
paper's OpenSBLI runs).

`chain_loops` is the user code of `steps` time steps (3 low-storage RK3 stages each)
as one loop chain for the executor. Datasets: the 5 conserved variables, the 5 RK
registers, 5 primitives (u, v, w, p, T), 12 gradients (d{u,v,w,T}/d{x,y,z}) and 15
fluxes -- 42 in all (27 with the fused residual kernel). Per stage: NS_PRIM, NS_GRAD, NS_FLUX (the 15 fluxes, 15 more
temporaries), NS_DIV (dU = A dU + dt R), NS_UPDATE (U += B dU); or, fused, NS_RHS in
place of NS_FLUX + NS_DIV. x and y are periodic inside each z-plane; z, the tiled axis, is periodic
through deep ghost planes (4 per stage) into which earlier loops extend their ranges.
"""
from __future__ import annotations

from typing import List

import numpy as np

from .spec import READ, RW, WRITE, Arg, DatSpec, Loop

GAMMA, MA, RE, PR = 1.4, 0.1, 1600.0, 0.71
RK_A = (0.0, -5.0 / 9.0, -153.0 / 128.0)
RK_B = (1.0 / 3.0, 15.0 / 16.0, 8.0 / 15.0)
REACH_PER_STAGE = 4
CONS = ["rho", "ru", "rv", "rw", "rE"]
PRIM = ["u", "v", "w", "p", "T"]
GRADS = [f"d{f}d{a}" for f in ("u", "v", "w", "T") for a in ("x", "y", "z")]
FLUXES = [f"F{m}{a}" for m in range(5) for a in ("x", "y", "z")]   # flux of component m along a


def h_of(n: int) -> float:
    return 2.0 * np.pi / n


def dt_of(n: int) -> float:
    return 0.5 * h_of(n) / (1.0 + 1.0 / MA)


def initial(n: int) -> np.ndarray:
    """Conserved state (5, n, n, n) indexed [component, z, y, x]."""
    x = np.arange(n) * h_of(n)
    Z, Y, X = np.meshgrid(x, x, x, indexing="ij")
    u = np.sin(X) * np.cos(Y) * np.cos(Z)
    v = -np.cos(X) * np.sin(Y) * np.cos(Z)
    w = np.zeros_like(u)
    p0 = 1.0 / (GAMMA * MA * MA)
    p = p0 + (np.cos(2 * X) + np.cos(2 * Y)) * (np.cos(2 * Z) + 2.0) / 16.0
    rho = np.ones_like(u)
    E = p / (GAMMA - 1.0) + 0.5 * rho * (u * u + v * v + w * w)
    return np.stack([rho, rho * u, rho * v, rho * w, E])


def ghost(steps: int) -> int:
    return REACH_PER_STAGE * 3 * steps


def datasets(n: int, steps: int = 1, dtype: str = "f64", U0: np.ndarray = None,
             mixed: bool = False, fused: bool = False) -> List[DatSpec]:
    G = ghost(steps)
    per = (0, 1, 2)
    ds = []

    def dat(name, g, init=None, dt=dtype):
        ds.append(DatSpec(name, (n, n, n), (0, 0, g), (0, 0, g), dt, per, init))

    for k, c in enumerate(CONS):
        init = None
        if U0 is not None:
            init = np.zeros((n + 2 * G, n, n))
            init[G:G + n] = U0[k]
        if mixed:
            hi = init.astype(np.float32) if init is not None else None
            lo = (init - hi.astype(np.float64)).astype(np.float32) if init is not None else None
            dat(c, G, hi)
            dat("lo_" + c, G, lo)
        else:
            dat(c, G, init)
        dat("d" + c, G - REACH_PER_STAGE, np.zeros((n + 2 * (G - REACH_PER_STAGE), n, n)))
    for c in PRIM:
        dat(c, G)
    for c in GRADS:
        dat(c, G - 2)
    if not fused:
        for c in FLUXES:
            dat(c, G - 2)
    return ds


STAR = [(0, 0, 0)] + [tuple(d * s if a == b else 0 for b in range(3)) for a in range(3) for s in (1, 2)
                      for d in (-1, 1)]


def chain_loops(n: int, steps: int = 1, mixed: bool = False, re: float = RE, fused: bool = False) -> List[Loop]:
    """`steps` RK3 steps as one chain (ranges shrink towards the last stage). fused: one
    NS_RHS loop per stage instead of NS_FLUX + NS_DIV."""
    G = ghost(steps)
    h = h_of(n)
    dt = dt_of(n)
    loops = []
    nst = 3 * steps
    full = lambda a, b: ((0, 0, a), (n, n, b))  # noqa: E731
    for st in range(nst):
        s = st % 3
        ext = REACH_PER_STAGE * (nst - 1 - st)   # reach still needed after this stage
        lo, hi = full(-ext - 4, n + ext + 4)
        loops.append(Loop("ns_prim", lo, hi, [Arg(c, READ) for c in CONS] + [Arg(c, WRITE) for c in PRIM],
                          [GAMMA, MA]))
        lo, hi = full(-ext - 2, n + ext + 2)
        loops.append(Loop("ns_grad", lo, hi, [Arg(c, READ, STAR[1:]) for c in ("u", "v", "w", "T")] +
                          [Arg(c, WRITE) for c in GRADS], [h, h, h]))
        acc = WRITE if s == 0 else RW
        if fused:
            lo, hi = full(-ext, n + ext)
            loops.append(Loop("ns_rhs", lo, hi, [Arg(c, READ, STAR[1:]) for c in CONS] +
                              [Arg(c, READ, STAR[1:]) for c in ("u", "v", "w", "p")] +
                              [Arg(c, READ, STAR[1:]) for c in GRADS] +
                              [Arg("d" + c, acc) for c in CONS],
                              [GAMMA, MA, re, PR, h, h, h, RK_A[s], dt]))
        else:
            loops.append(Loop("ns_flux", lo, hi, [Arg(c, READ, STAR[:1]) for c in CONS] +
                              [Arg(c, READ, STAR[:1]) for c in ("u", "v", "w", "p")] +
                              [Arg(c, READ, STAR[:1]) for c in GRADS] +
                              [Arg(c, WRITE, STAR[:1]) for c in FLUXES], [GAMMA, MA, re, PR]))
            lo, hi = full(-ext, n + ext)
            along = [STAR[1:5], STAR[5:9], STAR[9:13]]   # +-1, +-2 along x, y, z
            loops.append(Loop("ns_div", lo, hi, [Arg(FLUXES[3 * m + a], READ, along[a])
                                                 for m in range(5) for a in range(3)] +
                              [Arg("d" + c, acc, STAR[:1]) for c in CONS], [h, h, h, RK_A[s], dt]))
        if mixed:
            for c in CONS:
                loops.append(Loop("hilo_add", lo, hi, [Arg(c, RW), Arg("lo_" + c, RW), Arg("d" + c, READ)],
                                  [RK_B[s]]))
        else:
            loops.append(Loop("ns_update", lo, hi, [Arg(c, RW) for c in CONS] + [Arg("d" + c, READ) for c in CONS],
                              [RK_B[s]]))
    return loops


def run(ex, n: int, chains: int, steps_per_chain: int = 1, mixed: bool = False, U0: np.ndarray = None,
        fused: bool = False):
    """Drive `chains` chains of `steps_per_chain` RK3 steps on an executor `ex`."""
    U0 = initial(n) if U0 is None else U0
    for d in datasets(n, steps_per_chain, "f32" if mixed else "f64", U0, mixed, fused):
        ex.decl_dat(d)
    loops = chain_loops(n, steps_per_chain, mixed, fused=fused)
    for _ in range(chains):
        for lp in loops:
            ex.enqueue(lp)
        ex.flush()
