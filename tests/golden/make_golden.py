"""Write the stored expected values under tests/golden/ from the oracle alone.

The paper (arXiv 1709.02125) prints no worked numeric example, so these fixtures are
regression pins of the oracle: any later change to its arithmetic shows up as a
mismatch and has to name the passage of the paper that justifies it. Inputs come from
the seeded generators in workloads/.

    python tests/golden/make_golden.py
"""
from __future__ import annotations

import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from workloads import heat, random_chain  # noqa: E402

TINY = dict(n=8, nfields=6, nloops=6, nred=2, seed=4242)


def heat_case():
    """Heat chain of Sec. 5-style config 1: 256^2, U(0,1) seed 1710, 10 steps; the ten
    max-norms (one reduction per step)."""
    dats, reds, loops = heat.build(n=256, steps=10)
    fields = oracle.make_fields(dats)
    out = oracle.run_chain(loops, fields, reds)
    return [out[r.name] for r in reds]


def tiny_case():
    """Random chain on an 8x8 grid (4 fields, 6 loops, 2 sums): every final value."""
    dats, reds, loops = random_chain.build(**TINY)
    fields = oracle.make_fields(dats)
    out = oracle.run_chain(loops, fields, reds)
    return [out[r.name] for r in reds], {d.name: fields[d.name].a.copy() for d in dats}


def euler_case():
    """Euler square problem on a 24^2 periodic grid: 3 MacCormack steps at the CFL dt of
    each state; the dts and the final conserved state."""
    from oracle import physics
    from workloads import euler
    n = 24
    U = euler.initial(n)
    dts = []
    for _ in range(3):
        dt = euler.CFL * physics.euler_dt_min(U, 1.0 / n, 1.0 / n, euler.GAMMA)
        dts.append(dt)
        physics.euler_step(U, dt, 1.0 / n, 1.0 / n, euler.GAMMA, euler.EPS4)
    return dts, U


def tgv_case():
    """Taylor-Green vortex on a 12^3 periodic grid: 2 RK3 steps of the fixed dt."""
    from oracle import physics
    from workloads import tgv
    n = 12
    U = np.ascontiguousarray(tgv.initial(n))
    prm = physics.ns_params(tgv.GAMMA, tgv.MA, tgv.RE, tgv.PR, (tgv.h_of(n),) * 3)
    for _ in range(2):
        physics.ns_step(U, tgv.dt_of(n), prm)
    return U


def main():
    oracle.build()
    dts, U = euler_case()
    with open(os.path.join(HERE, "euler24_3steps.txt"), "w") as f:
        f.write("# oracle: Euler square problem 24^2, 3 CFL steps; dts, then U (4 x 24 x 24, C order)\n")
        f.write("dts " + " ".join(f"{v:.17e}" for v in dts) + "\n")
        f.write("U " + " ".join(f"{v:.17e}" for v in U.ravel()) + "\n")
    U = tgv_case()
    with open(os.path.join(HERE, "tgv12_2steps.txt"), "w") as f:
        f.write("# oracle: Taylor-Green vortex 12^3, 2 RK3 steps of the fixed dt; U (5 x 12^3, C order)\n")
        f.write("U " + " ".join(f"{v:.17e}" for v in U.ravel()) + "\n")
    with open(os.path.join(HERE, "heat256_u01_maxnorms.txt"), "w") as f:
        f.write("# oracle: heat chain 256^2, U(0,1) seed 1710, max|u| after each of 10 steps\n")
        for v in heat_case():
            f.write(f"{v:.17e}\n")
    sums, arrs = tiny_case()
    with open(os.path.join(HERE, "random8_chain.txt"), "w") as f:
        f.write(f"# oracle: random chain {TINY}; sums, then each field (full extent, C order)\n")
        f.write("sums " + " ".join(f"{v:.17e}" for v in sums) + "\n")
        for name, a in arrs.items():
            f.write(f"{name} {a.shape[0]} {a.shape[1]} " + " ".join(f"{v:.17e}" for v in a.ravel()) + "\n")


if __name__ == "__main__":
    main()
