"""Autotuner sweep: timing tables of random loop chains for training the tile planner.

Each sample is a random chain (2-D or 3-D, 8-32 fields, 8-48 loops, stencil radius 1-2,
FP32 or FP64, footprint log-uniform between --min-gb and --max-gb, device budget a
fraction 1/2 .. 1/8 of the footprint). A fresh context with OC_PLAN_AUTOTUNE runs the
chain once, which times every candidate of the grid (residency level, depth, tile
height; three interleaved rounds, median per candidate) on the GPU; the chain's
features and the timing table are written as one JSON line.

    python -m paper_1709_02125_gb300.planner_sweep --count 300 --out sweep.jsonl
"""
from __future__ import annotations

import argparse
import json
import math
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_1709_02125_gb300 import oc  # noqa: E402
from workloads import random_chain  # noqa: E402

RATIOS = (1 / 2, 1 / 3, 1 / 4, 1 / 6, 1 / 8)


def sample_chain(rng, min_gb, max_gb):
    nd = int(rng.choice([2, 3]))
    F = int(rng.integers(8, 33))
    L = int(rng.integers(8, 49))
    radius = int(rng.integers(1, 3))
    dtype = str(rng.choice(["f32", "f64"]))
    esz = 4 if dtype == "f32" else 8
    gb = math.exp(rng.uniform(math.log(min_gb), math.log(max_gb)))
    cells = gb * 1e9 / (F * esz)
    if nd == 2:
        n = int(math.sqrt(cells))
        nz = None
    else:
        n = int(round(cells ** (1 / 3)))
        nz = n
    ratio = float(rng.choice(RATIOS))
    seed = int(rng.integers(0, 2 ** 31))
    return dict(nd=nd, F=F, L=L, radius=radius, dtype=dtype, n=n, nz=nz, ratio=ratio, seed=seed)


def run_one(c, flags, repeats=1):
    """Autotune the chain `repeats` times, each on a fresh context; the first table is
    `table`, all of them `tables` (when repeats > 1), so that the timing noise between
    candidates can be measured and averaged out."""
    dats, reds, loops = random_chain.build_general(c["nd"], c["n"], c["F"], c["L"], c["radius"], c["seed"],
                                                   c["dtype"], c["nz"])
    fp = sum(int(np.prod(d.shape)) * (4 if d.dtype == "f32" else 8) for d in dats)
    budget = int(fp * c["ratio"])
    tables, tune_s = [], 0.0
    for _ in range(repeats):
        with oc.Executor(budget, flags=flags, planner=oc.OC_PLAN_AUTOTUNE) as ex:
            oc.run_chain(ex, dats, reds, loops, flush=False)
            t0 = time.perf_counter()
            ex.flush()
            tune_s += time.perf_counter() - t0
            tables.append(ex.autotune_result().tolist())
            feats = ex.features()
    row = dict(config=c, footprint=fp, budget=budget, features=[float(v) for v in feats],
               table=tables[0], tune_seconds=tune_s)
    if repeats > 1:
        row["tables"] = tables
    return row


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--count", type=int, default=300)
    ap.add_argument("--seed", type=int, default=1709 * 1000)
    ap.add_argument("--min-gb", type=float, default=0.25)
    ap.add_argument("--max-gb", type=float, default=8.0)
    ap.add_argument("--out", required=True)
    ap.add_argument("--time-limit-s", type=float, default=1e9)
    ap.add_argument("--repeats", type=int, default=1, help="autotune runs per chain (timing noise)")
    args = ap.parse_args()
    import __graft_entry__
    __graft_entry__.build()
    rng = np.random.default_rng(args.seed)
    flags = oc.OC_FLAG_CYCLIC | oc.OC_FLAG_PREFETCH
    t0 = time.perf_counter()
    with open(args.out, "a") as f:
        for i in range(args.count):
            c = sample_chain(rng, args.min_gb, args.max_gb)
            try:
                row = run_one(c, flags, args.repeats)
            except oc.OcError as e:   # a budget that cannot hold one tile: skip the sample
                print(f"sample {i}: {e}", flush=True)
                continue
            row["index"] = i
            f.write(json.dumps(row) + "\n")
            f.flush()
            if time.perf_counter() - t0 > args.time_limit_s:
                break
    print(f"done in {time.perf_counter() - t0:.1f} s", flush=True)


if __name__ == "__main__":
    main()
