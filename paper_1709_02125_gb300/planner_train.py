"""Train the tile-planner network on autotuner timing tables (planner_sweep.py output).

The network is a cost model of the two main alternatives to the fixed rule (largest
fitting tile height, depth 3): the targets are y0 = log2(t(fixed) / t(depth 4, largest
height)) and y1 = log2(t(fixed) / t(depth 3, 3/4 of the largest height)), clipped to
[-2, 2]. The planner keeps the fixed rule unless an alternative is predicted to win by
more than MARGIN (log2 units), then takes the larger predicted gain. Features are
standardised with the training split's mean and deviation. Training runs on the GPU
through liboc's MLP kernels (full-batch Adam). Evaluation: on the held-out chains, the
regret of a planner = its candidate's time / the best candidate's time - 1, for the
learned network and for the fixed rule.

    python -m paper_1709_02125_gb300.planner_train --data sweep.jsonl --out weights.json
"""
from __future__ import annotations

import argparse
import json
import math
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_1709_02125_gb300 import oc  # noqa: E402

GRID = [1.0, 0.75, 0.5, 0.375, 0.25, 0.1875, 0.125, 0.0625]
FIXED = (0, 3)   # grid index 0 (largest fitting height), depth 3


def load_rows(path):
    """Sweep rows with `table` as an array. A row autotuned several times (`tables`) gets
    the per-candidate median of its timings."""
    rows = []
    with open(path) as f:
        for line in f:
            r = json.loads(line)
            t = np.array(r["table"], dtype=np.float64)
            if len(t) == 0:
                continue
            if "tables" in r:
                reps = [np.array(x, dtype=np.float64) for x in r["tables"]]
                if all(x.shape == t.shape and np.array_equal(x[:, [0, 1, 3]], t[:, [0, 1, 3]]) for x in reps):
                    t = t.copy()
                    t[:, 2] = np.median(np.stack([x[:, 2] for x in reps]), axis=0)
            r["table"] = t
            rows.append(r)
    return rows


MARGIN = 0.03
ALT = ((0, 4), (1, 3))   # (grid index, depth) of the two alternatives


def targets(rows):
    X = np.array([r["features"] for r in rows], dtype=np.float64)
    Y = []
    for r in rows:
        t = r["table"]
        f = lookup(t, *FIXED)
        y = []
        for gi, d in ALT:
            a = lookup(t, gi, d)
            y.append(math.log2(f / a) if (f and a) else -2.0)
        Y.append(y)
    return X, np.clip(np.array(Y), -2.0, 2.0)


def choose(y):
    if max(y[0], y[1]) <= MARGIN:
        return FIXED
    return ALT[0] if y[0] >= y[1] else ALT[1]


def lookup(table, gi, depth):
    """time of candidate (grid index, depth), or None if it was not timed (did not fit)"""
    m = (table[:, 3] == gi) & (table[:, 1] == depth)
    return float(table[m, 2][0]) if m.any() else None


def regret(rows, choose):
    out = []
    for r in rows:
        t = r["table"]
        best = float(t[:, 2].min())
        gi, d = choose(r)
        ms = lookup(t, gi, d)
        if ms is None:   # candidate missing: fall back to the nearest timed height at that depth
            cand = t[t[:, 1] == d] if (t[:, 1] == d).any() else t
            ms = float(cand[np.argmin(np.abs(cand[:, 3] - gi)), 2])
        out.append(ms / best - 1.0)
    return np.array(out)


def he_init(seed):
    rng = np.random.default_rng(seed)
    parts = []
    for (o, i) in ((64, 8), (64, 0), (64, 64), (64, 0), (2, 64), (2, 0)):
        if i:
            lim = math.sqrt(6.0 / i)
            parts.append(rng.uniform(-lim, lim, size=o * i))
        else:
            parts.append(np.zeros(o))
    return np.concatenate(parts).astype(np.float32)


def train(rows_train, epochs=3000, lr=1e-3, seed=1709):
    X, Y = targets(rows_train)
    mean = X.mean(axis=0)
    std = X.std(axis=0)
    std[std == 0] = 1.0
    Xs = ((X - mean) / std).astype(np.float32)
    p, hist = oc.mlp_train(he_init(seed), Xs, Y.astype(np.float32), epochs, lr)
    return p, mean.astype(np.float32), std.astype(np.float32), hist


def evaluate(p, mean, std, rows):
    X = np.array([r["features"] for r in rows], dtype=np.float32)
    Yp = oc.mlp_forward(p, (X - mean) / std)
    learned = regret(rows, lambda r, it=iter(Yp): choose(next(it)))
    fixed = regret(rows, lambda r: FIXED)
    return learned, fixed


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--data", required=True)
    ap.add_argument("--out", required=True)
    ap.add_argument("--holdout", type=float, default=0.2)
    ap.add_argument("--epochs", type=int, default=3000)
    args = ap.parse_args()
    import __graft_entry__
    __graft_entry__.build()
    rows = load_rows(args.data)
    k = int(len(rows) * (1 - args.holdout))
    p, mean, std, hist = train(rows[:k], epochs=args.epochs)
    learned, fixed = evaluate(p, mean, std, rows[k:])
    res = {"params": p.tolist(), "mean": mean.tolist(), "std": std.tolist(), "train_chains": k,
           "heldout_chains": len(rows) - k, "final_loss": float(hist[-1]),
           "heldout_regret_learned_mean": float(learned.mean()), "heldout_regret_fixed_mean": float(fixed.mean()),
           "heldout_regret_learned_median": float(np.median(learned)),
           "heldout_regret_fixed_median": float(np.median(fixed))}
    json.dump(res, open(args.out, "w"))
    print(json.dumps({k_: v for k_, v in res.items() if k_ not in ("params", "mean", "std")}))


if __name__ == "__main__":
    main()
