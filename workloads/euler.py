"""2-D compressible Euler workload (stand-in for CloverLeaf 2-D, arXiv 1709.02125 Sec. 5.1).

Ideal gas, gamma = 1.4, periodic unit square, n x n cells (dx = dy = 1/n). Background
rho = 0.2, specific internal energy e = 1.0, at rest; a centred square of side n/4
with rho = 1.0, e = 2.5. The square's edges are smoothed over `edge` cells with a tanh
profile so that the non-TVD MacCormack scheme stays positive. CFL 0.5, fourth-order
dissipation eps4 = 1/64.

`chain_loops` is the user code of one time step as a loop chain for the executor:
34 datasets -- two sets of conserved variables (ping-pong), primitives, fluxes,
predicted state, its primitives and fluxes -- and 7 loops per step, the last being the
CFL min-reduction that ends the chain. The FP64 in-place form (`inplace=True`) keeps one
set of conserved variables A and an increment set D instead: the corrector writes the
increment and four pointwise LINCOMB loops add it (A = 1*A + 1*D, no nonlinear term), so
every step is the same chain -- the repeated chain the cyclic flag asks for, under which
the increments and the other intermediates are never downloaded. The mixed form is in
place already (compensated hi + lo update). x is periodic inside each row (kernels wrap);
y, the tiled axis, is periodic through halo rows refreshed at the start of every
chain (deep ghosts), into which the loops extend their ranges.
"""
from __future__ import annotations

from typing import Dict, List, Tuple

import numpy as np

from .spec import READ, REDUCE, RW, WRITE, Arg, DatSpec, Loop, RedSpec

GAMMA = 1.4
CFL = 0.5
EPS4 = 1.0 / 64.0
SEED = 1709 + 3


def initial(n: int, edge: float = 1.5) -> np.ndarray:
    """Conserved state (4, n, n): rho, mx, my, E."""
    x = (np.arange(n) + 0.5) / n
    half = 0.125
    w = edge / n

    def prof(c):
        return 0.5 * (np.tanh((c - (0.5 - half)) / w) - np.tanh((c - (0.5 + half)) / w))

    s = np.outer(prof(x), prof(x))          # 1 inside the square, 0 outside
    rho = 0.2 + 0.8 * s
    e = 1.0 + 1.5 * s
    U = np.zeros((4, n, n))
    U[0] = rho
    U[3] = rho * e
    return U


def datasets(n: int, dtype: str = "f64", U0: np.ndarray = None, mixed: bool = False,
             steps: int = 1, inplace: bool = False) -> List[DatSpec]:
    """Datasets of the chain. Conserved sets have 2 ghost rows per step of the chain in
    y (one step reads U at y +- 2); the intermediates one row more than the widest range
    a loop computes them over."""
    per = (0, 1)
    gc = 2 * steps                 # ghost rows of the conserved variables
    gi = 2 * (steps - 1) + 1       # ghost rows of the per-step intermediates
    ds = []
    names_c = ["r", "mx", "my", "E"]

    def dat(name, hlo, hhi, init=None):
        ds.append(DatSpec(name, (n, n), (0, hlo), (0, hhi), dtype, per, init))

    def pad(a):
        out = np.zeros((n + 2 * gc, n))
        out[gc:n + gc] = a
        return out

    for k, c in enumerate(names_c):
        init = pad(U0[k]) if U0 is not None else None
        if mixed:
            hi = init.astype(np.float32) if init is not None else None
            lo = (init - hi.astype(np.float64)).astype(np.float32) if init is not None else None
            dat(f"A_{c}", gc, gc, hi)
            dat(f"L_{c}", gc, gc, lo)
            dat(f"D_{c}", gc - 2, gc - 2)
        elif inplace:
            dat(f"A_{c}", gc, gc, init)
            dat(f"D_{c}", gc - 2, gc - 2)
        else:
            dat(f"A_{c}", gc, gc, init)
            dat(f"B_{c}", gc, gc)
    for c in ("u", "v", "p"):
        dat(c, gi, gi)
    for k in range(4):
        dat(f"F{k}", gi, gi)
        dat(f"G{k}", gi, gi)
        dat(f"S{k}", gi, gi - 1)
        dat(f"H{k}", gi, gi - 1)
        dat(f"K{k}", gi, gi - 1)
    for c in ("us", "vs", "ps"):
        dat(c, gi, gi - 1)
    return ds


def chain_loops(n: int, dt: float, src: str = "A", dst: str = "B", mixed: bool = False,
                red: str = "dtmin", ext: int = 0, with_dt: bool = True, inplace: bool = False) -> List[Loop]:
    """One MacCormack step U_src -> U_dst (mixed: in-place compensated update of A/L;
    FP64 with `inplace`: A += D, src and dst ignored), computing the new state over rows
    [-ext, n + ext) (ghost rows a later step of the same chain reads), optionally followed
    by the CFL min-reduction."""
    if inplace and not mixed:
        src = dst = "A"
    lx = ly = dt / (1.0 / n)
    c = ["r", "mx", "my", "E"]
    U = [f"{src}_{k}" for k in c]
    S = [f"S{k}" for k in range(4)]
    e = ext
    loops = [
        Loop("euler_prim", (0, -e - 1), (n, n + e + 1), [Arg(u, READ) for u in U] +
             [Arg("u", WRITE), Arg("v", WRITE), Arg("p", WRITE)], [GAMMA]),
        Loop("euler_flux", (0, -e - 1), (n, n + e + 1), [Arg(u, READ) for u in U] +
             [Arg("u", READ), Arg("v", READ), Arg("p", READ)] +
             [Arg(f"F{k}", WRITE) for k in range(4)] + [Arg(f"G{k}", WRITE) for k in range(4)], []),
        Loop("euler_pred", (0, -e - 1), (n, n + e), [Arg(u, READ) for u in U] +
             [Arg(f"F{k}", READ, [(0, 0), (1, 0)]) for k in range(4)] +
             [Arg(f"G{k}", READ, [(0, 0), (0, 1)]) for k in range(4)] +
             [Arg(s, WRITE) for s in S], [lx, ly]),
        Loop("euler_prim", (0, -e - 1), (n, n + e), [Arg(s, READ) for s in S] +
             [Arg("us", WRITE), Arg("vs", WRITE), Arg("ps", WRITE)], [GAMMA]),
        Loop("euler_flux", (0, -e - 1), (n, n + e), [Arg(s, READ) for s in S] +
             [Arg("us", READ), Arg("vs", READ), Arg("ps", READ)] +
             [Arg(f"H{k}", WRITE) for k in range(4)] + [Arg(f"K{k}", WRITE) for k in range(4)], []),
    ]
    cross = [(0, 0), (1, 0), (-1, 0), (2, 0), (-2, 0), (0, 1), (0, -1), (0, 2), (0, -2)]
    corr_in = ([Arg(u, READ, cross) for u in U] + [Arg(s, READ) for s in S] +
               [Arg(f"H{k}", READ, [(0, 0), (-1, 0)]) for k in range(4)] +
               [Arg(f"K{k}", READ, [(0, 0), (0, -1)]) for k in range(4)])
    if inplace and not mixed:
        loops.append(Loop("euler_corr", (0, -e), (n, n + e), corr_in + [Arg(f"D_{k}", WRITE) for k in c],
                          [lx, ly, EPS4, 1.0]))
        for k in c:
            loops.append(Loop("lincomb", (0, -e), (n, n + e), [Arg(f"A_{k}", WRITE), Arg(f"A_{k}", READ, [(0, 0)]),
                                                              Arg(f"D_{k}", READ, [(0, 0)])], [0.0, 1.0, 1.0]))
        if with_dt:
            loops.append(Loop("euler_dt", (0, 0), (n, n), [Arg(f"A_{k}", READ) for k in c] + [Arg(red, REDUCE)],
                              [GAMMA, 1.0 / n, 1.0 / n]))
    elif not mixed:
        loops.append(Loop("euler_corr", (0, -e), (n, n + e), corr_in + [Arg(f"{dst}_{k}", WRITE) for k in c],
                          [lx, ly, EPS4, 0.0]))
        if with_dt:
            loops.append(Loop("euler_dt", (0, 0), (n, n), [Arg(f"{dst}_{k}", READ) for k in c] + [Arg(red, REDUCE)],
                              [GAMMA, 1.0 / n, 1.0 / n]))
    else:
        loops.append(Loop("euler_corr", (0, -e), (n, n + e), corr_in + [Arg(f"D_{k}", WRITE) for k in c],
                          [lx, ly, EPS4, 1.0]))
        for k in c:
            loops.append(Loop("hilo_add", (0, -e), (n, n + e), [Arg(f"A_{k}", RW), Arg(f"L_{k}", RW),
                                                                Arg(f"D_{k}", READ)], [1.0]))
        if with_dt:
            loops.append(Loop("euler_dt", (0, 0), (n, n), [Arg(f"A_{k}", READ) for k in c] +
                              [Arg(f"L_{k}", READ) for k in c] + [Arg(red, REDUCE)], [GAMMA, 1.0 / n, 1.0 / n]))
    return loops


def fixed_dt_chain(n: int, dt: float, steps: int, mixed: bool = False, src: str = "A",
                   inplace: bool = False) -> Tuple[List[Loop], str]:
    """`steps` MacCormack steps of one fixed dt as one chain with no reduction (the
    multi-timestep chains of Sec. 5.3); step j computes its new state over the ghost
    rows the remaining steps read, 2 per step. Datasets: datasets(..., steps=steps).
    Returns (loops, prefix of the final state)."""
    loops: List[Loop] = []
    a, b = src, ("B" if src == "A" else "A")
    for j in range(steps):
        loops += chain_loops(n, dt, a, b, mixed, ext=2 * (steps - 1 - j), with_dt=False, inplace=inplace)
        if not (mixed or inplace):
            a, b = b, a
    return loops, ("A" if (mixed or inplace) else a)


def totals_loops(n: int, names: List[str], reds: List[str], lo_names: List[str] = None) -> List[Loop]:
    """FP64 totals (sum over the interior) of the conserved variables (hi + lo if mixed)."""
    out = []
    for k, (nm, r) in enumerate(zip(names, reds)):
        args = [Arg(nm, READ)]
        if lo_names:
            args.append(Arg(lo_names[k], READ))
        out.append(Loop("reduce", (0, 0), (n, n), args + [Arg(r, REDUCE)], [0.0]))
    return out


def dt_loop(n: int, mixed: bool = False, src: str = "A", red: str = "dtmin") -> Loop:
    c = ["r", "mx", "my", "E"]
    args = [Arg(f"{src}_{k}", READ) for k in c]
    if mixed:
        args += [Arg(f"L_{k}", READ) for k in c]
    return Loop("euler_dt", (0, 0), (n, n), args + [Arg(red, REDUCE)], [GAMMA, 1.0 / n, 1.0 / n])


def run(ex, n: int, steps: int, mixed: bool = False, U0: np.ndarray = None, totals: bool = False,
        inplace: bool = False):
    """Drive `steps` time steps on an executor `ex` (decl_dat / decl_reduction /
    enqueue / reduce). Returns (time steps used, name prefix of the final state,
    per-step conserved totals if requested)."""
    U0 = initial(n) if U0 is None else U0
    one = mixed or inplace
    for d in datasets(n, "f32" if mixed else "f64", U0, mixed, inplace=inplace):
        ex.decl_dat(d)
    ex.decl_reduction("dtmin", "min")
    tot_names = [f"tot_{k}" for k in ("r", "mx", "my", "E")]
    for t in tot_names:
        ex.decl_reduction(t, "sum")
    ex.enqueue(dt_loop(n, mixed))
    dtmin = ex.reduce("dtmin")
    src, dst = "A", "B"
    dts, tots = [], []
    for _ in range(steps):
        dt = CFL * dtmin
        dts.append(dt)
        for lp in chain_loops(n, dt, src, dst, mixed, inplace=inplace):
            ex.enqueue(lp)
        out = "A" if one else dst
        if totals:
            for lp in totals_loops(n, [f"{out}_{k}" for k in ("r", "mx", "my", "E")], tot_names,
                                   [f"L_{k}" for k in ("r", "mx", "my", "E")] if mixed else None):
                ex.enqueue(lp)
        dtmin = ex.reduce("dtmin")
        if totals:
            tots.append([ex.reduce(t) for t in tot_names])
        if not one:
            src, dst = dst, src
    return dts, ("A" if one else src), tots
