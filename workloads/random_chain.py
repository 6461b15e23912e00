"""Synthetic random 2-D loop chain (stand-in for the many-loop, many-dataset chains
of CloverLeaf / OpenSBLI, arXiv 1709.02125 Sec. 5.1).

Recipe (all draws from numpy's PCG64 with the given seed):
  * `nfields` fields of n x n interior, halo 2, initial values U(-1, 1) everywhere
    (the halo keeps its values: a fixed Dirichlet frame);
  * `nloops` loops, each over the interior; loop l writes one field w ~ U{0..F-1}
    and reads k ~ U{1..4} distinct other fields, each through 1..5 distinct offsets
    drawn from the 25 points of [-2, 2]^2;
  * LINCOMB coefficients c ~ U(-1, 1) scaled so that sum |c| = 0.5, alpha = 0.5, so
    every loop maps [-1, 1] into [-1, 1] and values stay O(1) over many chains;
  * `nred` SUM reductions at the end of the chain over distinct seed-chosen fields.
The same chain is executed repeatedly (the workload repeats it `chains` times).
"""
from __future__ import annotations

from typing import List

import numpy as np

from .spec import READ, REDUCE, WRITE, Arg, DatSpec, Loop, RedSpec

SEED = 1709 + 2


def build(n: int = 4096, nfields: int = 24, nloops: int = 40, nred: int = 2,
          seed: int = SEED, dtype: str = "f64", with_init: bool = True):
    rng = np.random.default_rng(seed)
    loops: List[Loop] = []
    for _ in range(nloops):
        w = int(rng.integers(0, nfields))
        k = int(rng.integers(1, 5))
        others = [f for f in range(nfields) if f != w]
        ins = rng.choice(others, size=k, replace=False)
        args = [Arg(f"f{w}", WRITE)]
        for f in ins:
            npts = int(rng.integers(1, 6))
            idx = rng.choice(25, size=npts, replace=False)
            args.append(Arg(f"f{int(f)}", READ, [(int(i) % 5 - 2, int(i) // 5 - 2) for i in idx]))
        m = sum(len(a.offsets) for a in args[1:])
        c = rng.uniform(-1.0, 1.0, size=m)
        c = c * (0.5 / np.abs(c).sum())
        loops.append(Loop("lincomb", (0, 0), (n, n), args, [0.5] + [float(v) for v in c]))
    red_fields = rng.choice(nfields, size=nred, replace=False)
    reds = [RedSpec(f"sum{r}", "sum") for r in range(nred)]
    for r, f in enumerate(red_fields):
        loops.append(Loop("reduce", (0, 0), (n, n),
                          [Arg(f"f{int(f)}", READ), Arg(f"sum{r}", REDUCE)], [0.0]))
    dats = []
    init_rng = np.random.default_rng(seed + 1)
    for f in range(nfields):
        init = init_rng.uniform(-1.0, 1.0, size=(n + 4, n + 4)) if with_init else None
        dats.append(DatSpec(f"f{f}", (n, n), (2, 2), (2, 2), dtype, init=init))
    return dats, reds, loops


def footprint_bytes(n: int = 4096, nfields: int = 24, esize: int = 8) -> int:
    return nfields * (n + 4) * (n + 4) * esize


def build_general(nd: int, n: int, nfields: int, nloops: int, radius: int, seed: int, dtype: str = "f64",
                  nz: int = None):
    """Random chain on an n^2 (2-D) or n^2 x nz (3-D) grid with halo `radius`: loops read
    1-4 other fields at offsets within `radius` on every axis (same recipe as `build`).
    No initial data (zeros); used for planner sweeps, where values do not matter."""
    rng = np.random.default_rng(seed)
    nz = n if nz is None else nz
    size = (n, n) if nd == 2 else (n, n, nz)
    lo = (0,) * nd
    w = 2 * radius + 1
    loops: List[Loop] = []
    for _ in range(nloops):
        out = int(rng.integers(0, nfields))
        k = int(rng.integers(1, 5))
        ins = rng.choice([f for f in range(nfields) if f != out], size=min(k, nfields - 1), replace=False)
        args = [Arg(f"f{out}", WRITE, [(0,) * nd])]
        for f in ins:
            npts = int(rng.integers(1, 6))
            idx = rng.choice(w ** nd, size=min(npts, w ** nd), replace=False)
            offs = []
            for i in idx:
                o, r = [], int(i)
                for _a in range(nd):
                    o.append(r % w - radius)
                    r //= w
                offs.append(tuple(o))
            args.append(Arg(f"f{int(f)}", READ, offs))
        m = sum(len(a.offsets) for a in args[1:])
        c = rng.uniform(-1.0, 1.0, size=m)
        c = c * (0.5 / np.abs(c).sum())
        loops.append(Loop("lincomb", lo, size, args, [0.5] + [float(v) for v in c]))
    reds = [RedSpec("s0", "sum")]
    loops.append(Loop("reduce", lo, size, [Arg("f0", READ, [(0,) * nd]), Arg("s0", REDUCE)], [0.0]))
    dats = [DatSpec(f"f{f}", size, (radius,) * nd, (radius,) * nd, dtype) for f in range(nfields)]
    return dats, reds, loops
