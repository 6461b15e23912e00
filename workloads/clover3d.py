"""Synthetic 3-D loop chains structured like CloverLeaf 3D (arXiv 1709.02125, Sec. 5.1:
30 datasets, one time step is a chain of about 600 loops; Sec. 5.3: every 10 steps a
"summary" chain of reductions reads many datasets with little compute, the case with
poor copy/compute overlap). The application itself is not available; this recipe
reproduces its chain structure with the executor's generic kernels.

Recipe (numpy PCG64; seed 1709 + 6 draws the chain, seed 1709 + 7 the fields):
  * grid n x n x nz interior, halo 2 on every axis; 30 datasets of one element type:
    12 state fields s0..s11, U(-1, 1) everywhere (the halo is held fixed: a Dirichlet
    frame), and 18 work fields w0..w17 (zeros);
  * one time step = one chain:
      1. a prologue of 18 pointwise loops, one per work field, each defining it over
         its whole allocated extent (halos included) as a LINCOMB of 1-2 state fields
         at offset 0: every work field's first access in the chain is a full-row write
         (write-first: never uploaded, and never downloaded with the cyclic flag);
      2. `stages` stages (default 58) of `per_stage` loops (default 10) sweeping the
         axes x, y, z, x, y, z, ... (the direction sweeps of the advection). The first
         per_stage - 1 loops of a stage write a work field over the interior from 1-3
         other fields (work or state), each read through 1-4 distinct offsets along
         the stage's axis -- within +-2 in x and y stages; in a z stage only the first
         loop reaches +-1 along z and the others read at offset 0, which keeps the
         skew of one step to about one row per z stage. The last loop of a stage
         updates one state field over the interior from 2-3 work fields and one other
         state field at offset 0;
      3. one MIN reduction of s1 (a time-step-like value the user reads, ending the
         chain).
    That is 18 + 58 * 10 + 1 = 599 loops per step by default;
  * LINCOMB coefficients U(-1, 1) scaled to sum |c| = 0.5 and alpha = 0.5, so every
    loop maps [-1, 1] into [-1, 1] and values stay O(1) over many steps;
  * the summary chain: 12 reductions, one per state field -- SUM of the value for
    s0..s5, SUM of squares for s6..s9, MAX of |value| for s10, s11 -- and nothing
    else: a read-only chain.
"""
from __future__ import annotations

from typing import List, Tuple

import numpy as np

from .spec import READ, REDUCE, WRITE, Arg, DatSpec, Loop, RedSpec

SEED = 1709 + 6
NSTATE, NWORK = 12, 18
HALO = 2
SUMMARY_EVERY = 10


def datasets(n: int, nz: int, dtype: str = "f64", with_init: bool = True, seed: int = SEED + 1) -> List[DatSpec]:
    size = (n, n, nz)
    shape = (nz + 2 * HALO, n + 2 * HALO, n + 2 * HALO)
    rng = np.random.default_rng(seed)
    dats = []
    for i in range(NSTATE):
        init = rng.uniform(-1.0, 1.0, size=shape) if with_init else None
        dats.append(DatSpec(f"s{i}", size, (HALO,) * 3, (HALO,) * 3, dtype, init=init))
    for i in range(NWORK):
        dats.append(DatSpec(f"w{i}", size, (HALO,) * 3, (HALO,) * 3, dtype,
                            init=np.zeros(shape) if with_init else None))
    return dats


def footprint_bytes(n: int, nz: int, esize: int = 8) -> int:
    return (NSTATE + NWORK) * (n + 2 * HALO) ** 2 * (nz + 2 * HALO) * esize


def _coefs(rng, m: int) -> List[float]:
    c = rng.uniform(-1.0, 1.0, size=m)
    c = c * (0.5 / np.abs(c).sum())
    return [0.5] + [float(v) for v in c]


def _axis_offsets(rng, axis: int, reach: int, k: int) -> List[Tuple[int, int, int]]:
    pts = rng.choice(2 * reach + 1, size=min(k, 2 * reach + 1), replace=False)
    out = []
    for p in pts:
        o = [0, 0, 0]
        o[axis] = int(p) - reach
        out.append(tuple(o))
    return out


def step_chain(n: int, nz: int, stages: int = 58, per_stage: int = 10, seed: int = SEED):
    """(reductions, loops) of one time step."""
    rng = np.random.default_rng(seed)
    size = (n, n, nz)
    full_lo, full_hi = (-HALO,) * 3, (n + HALO, n + HALO, nz + HALO)
    zero = (0, 0, 0)
    loops: List[Loop] = []
    for w in range(NWORK):
        k = int(rng.integers(1, 3))
        src = rng.choice(NSTATE, size=k, replace=False)
        args = [Arg(f"w{w}", WRITE)] + [Arg(f"s{int(s)}", READ, [zero]) for s in src]
        loops.append(Loop("lincomb", full_lo, full_hi, args, _coefs(rng, k)))
    names = [f"w{i}" for i in range(NWORK)] + [f"s{i}" for i in range(NSTATE)]
    for st in range(stages):
        axis = st % 3
        for q in range(per_stage - 1):
            out = f"w{int(rng.integers(0, NWORK))}"
            cand = [x for x in names if x != out]
            ins = rng.choice(len(cand), size=int(rng.integers(1, 4)), replace=False)
            args = [Arg(out, WRITE)]
            for i in ins:
                npts = int(rng.integers(1, 5))
                if axis < 2:
                    offs = _axis_offsets(rng, axis, 2, npts)
                elif q == 0:
                    offs = _axis_offsets(rng, 2, 1, npts)
                else:
                    offs = [zero]
                args.append(Arg(cand[int(i)], READ, offs))
            m = sum(len(a.offsets) for a in args[1:])
            loops.append(Loop("lincomb", zero, size, args, _coefs(rng, m)))
        upd = int(rng.integers(0, NSTATE))
        ws = rng.choice(NWORK, size=int(rng.integers(2, 4)), replace=False)
        other = int(rng.choice([s for s in range(NSTATE) if s != upd]))
        args = [Arg(f"s{upd}", WRITE)] + [Arg(f"w{int(w)}", READ, [zero]) for w in ws]
        args.append(Arg(f"s{other}", READ, [zero]))
        loops.append(Loop("lincomb", zero, size, args, _coefs(rng, len(args) - 1)))
    reds = [RedSpec("dt", "min")]
    loops.append(Loop("reduce", zero, size, [Arg("s1", READ), Arg("dt", REDUCE)], [0.0]))
    return reds, loops


def summary_chain(n: int, nz: int):
    """(reductions, loops) of the summary chain: one reduction per state field."""
    size, zero = (n, n, nz), (0, 0, 0)
    reds, loops = [], []
    for i in range(NSTATE):
        op, mode = ("sum", 0.0) if i < 6 else (("sum", 2.0) if i < 10 else ("max", 1.0))
        reds.append(RedSpec(f"sm{i}", op))
        loops.append(Loop("reduce", zero, size, [Arg(f"s{i}", READ), Arg(f"sm{i}", REDUCE)], [mode]))
    return reds, loops
