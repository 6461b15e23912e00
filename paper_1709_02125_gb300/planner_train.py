"""Train the tile-planner network on autotuner timing tables (planner_sweep.py output).

A timing table has one row per grid candidate: (tile height, depth, ms, grid index, largest
fitting height, residency level), the candidate being (grid index, depth, residency index)
with residency levels RES_LEVELS (share of the budget for datasets kept resident). The
fixed rule -- the method without a planner -- is (0, 3, 0): largest fitting height,
depth 3, nothing resident.

The network is a cost model of two alternatives A0, A1 to the fixed rule: its targets are
y_k = log2(t(fixed) / t(A_k)), clipped to [-2, 2]. The alternatives are chosen on the
training split alone: the twelve pairs of candidates (largest or 3/4 height, depth 3 or 4,
any residency level) that a perfect predictor would gain most with (mean over the chains
of max(0, y0, y1)) and every pair of residency levels at the fixed tiling are
shortlisted, and the pair whose trained network has the lowest regret in a 3-fold
cross-validation over the training chains is kept. The planner keeps the fixed
rule unless an alternative is predicted to win by more than MARGIN (log2 units), then
takes the one with the larger predicted gain. Features are standardised with the
training split's mean and deviation. Training runs on the GPU through liboc's MLP kernels
(full-batch Adam). Evaluation: on the held-out chains, the regret of a planner = the time
of its candidate / the best candidate's time - 1, for the learned network and for the
fixed rule.

    python -m paper_1709_02125_gb300.planner_train --data sweep.jsonl --out weights.json
"""
from __future__ import annotations

import argparse
import itertools
import json
import math
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_1709_02125_gb300 import oc  # noqa: E402

GRID = [1.0, 0.75, 0.5, 0.25]
RES_LEVELS = [0.0, 0.25, 0.5, 0.75]
FIXED = (0, 3, 0)   # grid index 0 (largest fitting height), depth 3, nothing resident
DEFAULT_ALT = ((0, 3, 1), (0, 3, 2))
MARGIN = 0.03


def res_index(level):
    return int(np.argmin([abs(level - v) for v in RES_LEVELS]))


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
                keep = [0, 1, 3, 5] if t.shape[1] > 5 else [0, 1, 3]
                if all(x.shape == t.shape and np.array_equal(x[:, keep], t[:, keep]) for x in reps):
                    t = t.copy()
                    t[:, 2] = np.median(np.stack([x[:, 2] for x in reps]), axis=0)
            r["table"] = t
            rows.append(r)
    return rows


def lookup(table, cand):
    """Time of candidate (grid index, depth, residency index), or None if not timed. A
    residency level the autotuner skipped (it would keep no more datasets than the level
    below) stands for the one below."""
    gi, d, ri = cand
    lv = table[:, 5] if table.shape[1] > 5 else np.zeros(len(table))
    for r in range(ri, -1, -1):
        m = (table[:, 3] == gi) & (table[:, 1] == d) & (np.abs(lv - RES_LEVELS[r]) < 1e-9)
        if m.any():
            return float(table[m, 2][0])
        if r > 0 and (np.abs(lv - RES_LEVELS[r]) < 1e-9).any():
            return None   # the level was timed, this candidate at it was not
    return None


def gains(rows, cand):
    """log2(t(fixed) / t(cand)) per row (-2 when either is missing), clipped to [-2, 2]."""
    out = []
    for r in rows:
        f, a = lookup(r["table"], FIXED), lookup(r["table"], cand)
        out.append(math.log2(f / a) if (f and a) else -2.0)
    return np.clip(np.array(out), -2.0, 2.0)


def shortlist(rows, k=12):
    """Up to k pairs of candidates (grid index 0 or 1, depth 3 or 4) ranked by the mean
    gain of a perfect choice between them and the fixed rule on `rows`."""
    cands = sorted({(int(t[3]), int(t[1]), res_index(t[5] if len(t) > 5 else 0.0))
                    for r in rows for t in r["table"]
                    if int(t[3]) <= 1 and int(t[1]) in (3, 4)} - {FIXED})
    if len(cands) < 2:
        return [DEFAULT_ALT]
    G = {c: gains(rows, c) for c in cands}
    scored = [(float(np.mean(np.maximum(0.0, np.maximum(G[a], G[b])))), (a, b))
              for a, b in itertools.combinations(cands, 2)]
    scored.sort(key=lambda t: -t[0])
    out = [pair for _, pair in scored[:k]]
    # every pair of residency levels at the fixed tiling is a candidate too: residency is
    # what the fixed rule lacks most on link-bound chains
    res_only = [c for c in cands if c[0] == 0 and c[1] == 3 and c[2] > 0]
    out += [pair for pair in itertools.combinations(res_only, 2) if pair not in out]
    return out


def alternatives(rows):
    """The pair of candidates with the largest mean perfect-choice gain on `rows`."""
    return shortlist(rows, 1)[0]


def select_alternatives(rows, folds=3, epochs=1500, k=12):
    """The shortlisted pair whose network, trained on the other folds, chooses best on
    each held-out fold of `rows` (mean regret over the folds); runs on the GPU."""
    pairs = shortlist(rows, k)
    if len(pairs) == 1 or len(rows) < 3 * folds:
        return pairs[0]
    parts = [rows[i::folds] for i in range(folds)]
    best, pick = float("inf"), pairs[0]
    for pair in pairs:
        reg = []
        for f in range(folds):
            tr = [r for g, part in enumerate(parts) if g != f for r in part]
            p, mean, std, _, _ = train(tr, epochs=epochs, alts=pair)
            learned, _ = evaluate(p, mean, std, parts[f], pair)
            reg.append(learned.mean())
        if float(np.mean(reg)) < best:
            best, pick = float(np.mean(reg)), pair
    return pick


def targets(rows, alts=DEFAULT_ALT):
    X = np.array([r["features"] for r in rows], dtype=np.float64)
    Y = np.stack([gains(rows, a) for a in alts], axis=1)
    return X, Y


def choose(y, alts=DEFAULT_ALT):
    if max(y[0], y[1]) <= MARGIN:
        return FIXED
    return alts[0] if y[0] >= y[1] else alts[1]


def regret(rows, choose):
    out = []
    for r in rows:
        t = r["table"]
        best = float(t[:, 2].min())
        c = choose(r)
        ms = lookup(t, c)
        if ms is None:   # candidate missing: the nearest timed height at that depth and level
            gi, d, ri = c
            lv = t[:, 5] if t.shape[1] > 5 else np.zeros(len(t))
            sel = (t[:, 1] == d) & (np.abs(lv - RES_LEVELS[ri]) < 1e-9)
            cand = t[sel] if sel.any() else (t[t[:, 1] == d] if (t[:, 1] == d).any() else t)
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


def train(rows_train, epochs=3000, lr=1e-3, seed=1709, alts=None):
    """Returns (params, feature mean, feature std, loss history, alternatives)."""
    alts = select_alternatives(rows_train) if alts is None else alts
    X, Y = targets(rows_train, alts)
    mean = X.mean(axis=0)
    std = X.std(axis=0)
    std[std == 0] = 1.0
    Xs = ((X - mean) / std).astype(np.float32)
    p, hist = oc.mlp_train(he_init(seed), Xs, Y.astype(np.float32), epochs, lr)
    return p, mean.astype(np.float32), std.astype(np.float32), hist, alts


def install(p, mean, std, alts):
    """Load the network and its alternatives into liboc (OC_PLAN_LEARNED)."""
    oc.planner_alternatives(alts)
    oc.planner_load(p, mean, std)


def evaluate(p, mean, std, rows, alts=DEFAULT_ALT):
    X = np.array([r["features"] for r in rows], dtype=np.float32)
    Yp = oc.mlp_forward(p, (X - mean) / std)
    learned = regret(rows, lambda r, it=iter(Yp): choose(next(it), alts))
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
    p, mean, std, hist, alts = train(rows[:k], epochs=args.epochs)
    learned, fixed = evaluate(p, mean, std, rows[k:], alts)
    res = {"params": p.tolist(), "mean": mean.tolist(), "std": std.tolist(), "alternatives": alts, "train_chains": k,
           "heldout_chains": len(rows) - k, "final_loss": float(hist[-1]),
           "heldout_regret_learned_mean": float(learned.mean()), "heldout_regret_fixed_mean": float(fixed.mean()),
           "heldout_regret_learned_median": float(np.median(learned)),
           "heldout_regret_fixed_median": float(np.median(fixed))}
    json.dump(res, open(args.out, "w"))
    print(json.dumps({k_: v for k_, v in res.items() if k_ not in ("params", "mean", "std")}))


if __name__ == "__main__":
    main()
