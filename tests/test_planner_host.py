"""Host logic of the planner's training script (planner_train.py) that needs no GPU:
reading sweep rows (with repeated timings folded by their median), the two targets, the
decision rule with its margin, and the regret against the best timed candidate."""
import json
import math
import os

import numpy as np
import pytest

from paper_1709_02125_gb300 import planner_train as pt

DATA = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                    "paper_1709_02125_gb300", "planner_data", "autotune_gb300.jsonl")


def _table(ms):
    """rows (height, depth, ms, grid index, hmax, residency level): the fixed rule, 3/4 of
    its height, depth 4, and the fixed tiling with 1/4 and 1/2 of the budget resident"""
    return [[100.0, 3.0, ms[0], 0.0, 100.0, 0.0], [75.0, 3.0, ms[1], 1.0, 100.0, 0.0],
            [80.0, 4.0, ms[2], 0.0, 80.0, 0.0], [70.0, 3.0, ms[3], 0.0, 70.0, 0.25],
            [40.0, 3.0, ms[4], 0.0, 40.0, 0.5]]


def test_committed_sweep_loads():
    rows = pt.load_rows(DATA)
    raw = [json.loads(ln) for ln in open(DATA)]
    assert len(rows) == sum(1 for r in raw if r["table"])
    for r, q in zip(rows, [r for r in raw if r["table"]]):
        assert r["table"].shape[1] == 6
        assert len(r["features"]) == 8


def test_repeated_timings_fold_to_their_median(tmp_path):
    reps = [_table([10, 12, 9, 20, 5]), _table([11, 10, 30, 21, 6]), _table([30, 11, 10, 19, 4])]
    row = {"features": [0.0] * 8, "table": reps[0], "tables": reps}
    p = tmp_path / "s.jsonl"
    p.write_text(json.dumps(row) + "\n")
    (r,) = pt.load_rows(str(p))
    assert list(r["table"][:, 2]) == [11.0, 11.0, 10.0, 20.0, 5.0]
    assert list(r["table"][:, 0]) == [100.0, 75.0, 80.0, 70.0, 40.0]


def test_targets_choice_and_regret():
    rows = [{"features": [1.0] * 8, "table": np.array(_table([10, 8, 12, 9, 20]))},
            {"features": [2.0] * 8, "table": np.array(_table([10, 11, 5, 9, 4]))}]
    alts = ((0, 3, 1), (0, 3, 2))
    X, Y = pt.targets(rows, alts)
    assert Y[0] == pytest.approx([math.log2(10 / 9), math.log2(10 / 20)])
    assert Y[1] == pytest.approx([math.log2(10 / 9), math.log2(10 / 4)])
    assert pt.choose([0.02, 0.01], alts) == pt.FIXED                      # inside the margin
    assert pt.choose([0.2, 0.5], alts) == alts[1] and pt.choose([0.6, 0.5], alts) == alts[0]
    fixed = pt.regret(rows, lambda r: pt.FIXED)
    assert fixed == pytest.approx([10 / 8 - 1, 10 / 4 - 1])
    best = pt.regret(rows, lambda r: (1, 3, 0) if r is rows[0] else (0, 3, 2))
    assert best == pytest.approx([0.0, 0.0])


def test_alternatives_are_the_pair_a_perfect_choice_gains_most_with():
    """Row 1 is won by 3/4 of the height, row 2 by half of the budget resident, row 3 by
    depth 4: the pair (3/4 height, half resident) covers two rows with large gains."""
    rows = [{"features": [0.0] * 8, "table": np.array(_table(t))}
            for t in ([10, 5, 12, 11, 11], [10, 11, 12, 9, 2.5], [10, 11, 9, 11, 11])]
    assert set(pt.alternatives(rows)) == {(1, 3, 0), (0, 3, 2)}


def test_skipped_residency_level_stands_for_the_level_below():
    """The autotuner skips a residency level that keeps no more datasets than the one
    below; a candidate at the skipped level is timed as the lower level's."""
    t = np.array([[100.0, 3.0, 10.0, 0.0, 100.0, 0.0], [60.0, 3.0, 7.0, 0.0, 60.0, 0.25]])
    assert pt.lookup(t, (0, 3, 2)) == 7.0
    assert pt.lookup(t, (0, 3, 1)) == 7.0
    assert pt.lookup(t, (0, 3, 0)) == 10.0


def test_missing_candidate_falls_back_to_nearest_height():
    t = np.array([[100.0, 3.0, 10.0, 0.0, 100.0, 0.0], [50.0, 3.0, 7.0, 2.0, 100.0, 0.0]])
    r = {"features": [0.0] * 8, "table": t}
    # (grid index 1, depth 3) was not timed: the nearest timed index at depth 3 is taken,
    # the first in table order on a tie (here index 0)
    assert pt.regret([r], lambda _: (1, 3, 0))[0] == pytest.approx(10 / 7 - 1)
    assert pt.regret([r], lambda _: (2, 3, 0))[0] == 0.0
    assert pt.regret([r], lambda _: (0, 3, 0))[0] == pytest.approx(10 / 7 - 1)
