"""Helpers of the GPU tests: run a chain through the C ABI and compare with the oracle."""
from __future__ import annotations

import copy
from typing import Dict, List

import numpy as np


def run_gpu(dats, reds, loops, budget, h=0, depth=0, flags=0, chains=1, planner=0, ex_out=None, residency=None):
    """Declare the datasets, run `chains` repetitions of `loops` on the GPU; return
    (final arrays by name, list of per-chain reduction dicts, stats of the last chain)."""
    from paper_1709_02125_gb300 import oc
    ex = oc.Executor(budget, flags=flags, planner=planner)
    try:
        ex.set_tiling(h, depth)
        if residency is not None:
            ex.set_residency(residency)
        for d in dats:
            ex.decl_dat(d)
        for r in reds:
            ex.decl_reduction(r.name, r.op)
        per_chain = []
        for _ in range(chains):
            for lp in loops:
                ex.enqueue(lp)
            ex.flush()
            per_chain.append({r.name: ex.reduce(r.name) for r in reds})
        st = ex.stats()
        out = {d.name: ex.fetch(d.name) for d in dats}
        if ex_out is not None:
            ex_out.append(ex.plan())
    finally:
        ex.close()
    return out, per_chain, st


def run_oracle(oracle, dats, reds, loops, chains=1):
    fields = oracle.make_fields(dats)
    per_chain = [oracle.run_chain(loops, fields, reds) for _ in range(chains)]
    return {k: v.a for k, v in fields.items()}, per_chain


def rel_max(g, o):
    """Normwise relative max error max|g - o| / max|o|."""
    den = np.max(np.abs(o))
    return float(np.max(np.abs(np.asarray(g, dtype=np.float64) - o)) / (den if den > 0 else 1.0))


def rel_l2(g, o):
    den = np.linalg.norm(o.ravel())
    return float(np.linalg.norm((np.asarray(g, dtype=np.float64) - o).ravel()) / (den if den > 0 else 1.0))


def sum_bound(values_abs_sum):
    """Tolerance of a GPU sum against the compensated oracle sum: 1e-12 of sum |v|."""
    return 1e-12 * values_abs_sum
