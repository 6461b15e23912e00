"""GPU tests of the tile planner: the MLP kernels against the FP64 oracle network, the
autotuner's side-effect-free trials, and the learned planner's grid snapping."""
import math

import numpy as np
import pytest

from workloads import random_chain

from gpu_helpers import run_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()


def _data(seed, n):
    rng = np.random.default_rng(seed)
    X = rng.normal(size=(n, 8)).astype(np.float32)
    T = np.stack([np.tanh(X[:, 0] - 0.5 * X[:, 3]), X[:, 1] * X[:, 2] / 2 + 3.0], axis=1).astype(np.float32)
    return X, T


def test_mlp_forward_and_gradient_match_oracle():
    from oracle import mlp
    from paper_1709_02125_gb300 import oc
    assert oc.mlp_nparams() == mlp.NPARAMS
    p = mlp.init_params(7).astype(np.float32)
    X, T = _data(8, 57)
    y = oc.mlp_forward(p, X)
    yo, _ = mlp.forward(p.astype(np.float64), X.astype(np.float64))
    assert np.max(np.abs(y - yo)) <= 1e-5 * max(1.0, np.max(np.abs(yo)))
    loss, g = oc.mlp_loss_grad(p, X, T)
    lo, go = mlp.loss_grad(p.astype(np.float64), X.astype(np.float64), T.astype(np.float64))
    assert abs(loss - lo) <= 1e-5 * lo
    assert np.linalg.norm(g - go) <= 1e-4 * np.linalg.norm(go)


def test_mlp_training_follows_oracle_adam():
    from oracle import mlp
    from paper_1709_02125_gb300 import oc
    p0 = mlp.init_params(11).astype(np.float32)
    X, T = _data(12, 64)
    lr = 1e-3
    p_gpu, hist = oc.mlp_train(p0, X, T, epochs=5, lr=lr)
    p = p0.astype(np.float64)
    m = np.zeros_like(p)
    v = np.zeros_like(p)
    for t in range(1, 6):
        L, g = mlp.loss_grad(p, X.astype(np.float64), T.astype(np.float64))
        assert abs(hist[t - 1] - L) <= 1e-4 * L
        p, m, v = mlp.adam_step(p, g, m, v, t, lr)
    # parameters whose gradient is far from zero move the same way
    assert np.mean(np.abs(p_gpu - p) <= 2e-4 + 1e-4 * np.abs(p)) > 0.99


def test_mlp_training_reduces_loss():
    from oracle import mlp
    from paper_1709_02125_gb300 import oc
    p0 = mlp.init_params(13).astype(np.float32)
    X, T = _data(14, 400)
    _, hist = oc.mlp_train(p0, X, T, epochs=800, lr=3e-3)
    assert hist[-1] < 0.05 * hist[0]


def _chain(n=512):
    dats, reds, loops = random_chain.build(n=n, nfields=12, nloops=24, seed=77, dtype="f32")
    for d in dats:
        d.init = d.init.astype(np.float32)
    return dats, reds, loops, random_chain.footprint_bytes(n, 12, 4)


def test_autotune_trials_have_no_side_effects():
    from paper_1709_02125_gb300 import oc
    dats, reds, loops, fp = _chain()
    ref, rr, _ = run_gpu(dats, reds, loops, fp // 3, chains=2)
    plans = []
    got, rg, st = run_gpu(dats, reds, loops, fp // 3, chains=2, planner=oc.OC_PLAN_AUTOTUNE, ex_out=plans)
    for d in dats:
        assert np.array_equal(ref[d.name], got[d.name]), d.name
    assert rr == rg
    with oc.Executor(fp // 3, planner=oc.OC_PLAN_AUTOTUNE) as ex:
        oc.run_chain(ex, dats, reds, loops)
        table = ex.autotune_result()
        st = ex.stats()
    # residency levels 0, 1/4, 1/2, 3/4 (those that keep datasets) x depths 2..4 x heights
    assert len(table) >= 24 and set(table[:, 1]) == {2.0, 3.0, 4.0}
    assert {0.0, 0.5} <= set(table[:, 5])
    best = table[np.argmin(table[:, 2])]
    assert st["tile_height"] == int(best[0]) and st["depth"] == int(best[1])
    assert (st["resident_dats"] > 0) == (best[5] > 0)


@pytest.mark.parametrize("bias,alts,expect", [
    ((0.5, 0.1), ((0, 4, 0), (1, 3, 0)), (0, 4, 0)),
    ((0.0, 0.4), ((0, 4, 0), (1, 3, 0)), (1, 3, 0)),
    ((-1.0, 0.02), ((0, 4, 0), (1, 3, 0)), (0, 3, 0)),
    ((0.3, 0.6), ((0, 3, 1), (0, 3, 2)), (0, 3, 2))])
def test_learned_planner_decision(bias, alts, expect):
    """A network whose outputs are its biases: y0 / y1 are the predicted log2 gains of the
    two named alternatives (grid index, depth, residency index) over the fixed rule."""
    from oracle import mlp
    from paper_1709_02125_gb300 import oc
    dats, reds, loops, fp = _chain()
    p = np.zeros(mlp.NPARAMS, dtype=np.float32)
    p[-2:] = bias
    # a wide standardisation keeps every feature of the test chain in distribution
    oc.planner_alternatives(alts)
    oc.planner_load(p, np.zeros(8), np.full(8, 1e6))
    _, _, st_l = run_gpu(dats, reds, loops, fp // 3, planner=oc.OC_PLAN_LEARNED)
    gi, depth, ri = expect
    _, _, st_f = run_gpu(dats, reds, loops, fp // 3, depth=depth, residency=(0.0, 0.25, 0.5, 0.75)[ri])
    hmax = st_f["tile_height"]
    assert st_l["depth"] == depth
    assert st_l["tile_height"] == max(1, math.floor(hmax * (1.0, 0.75)[gi] + 0.5))
    assert st_l["resident_dats"] == st_f["resident_dats"] and (st_l["resident_dats"] > 0) == (ri > 0)


def test_learned_planner_beats_fixed_rule_on_heldout_chains():
    """Train on the committed autotuner sweep (first 80 % of the chains) with the GPU
    kernels; on the held-out chains the learned planner's mean regret (time of its choice
    over the best candidate's, minus one) is below the fixed rule's."""
    import os
    from paper_1709_02125_gb300 import planner_train
    path = os.path.join(os.path.dirname(os.path.dirname(__file__)), "paper_1709_02125_gb300", "planner_data",
                        "autotune_gb300.jsonl")
    rows = planner_train.load_rows(path)
    assert len(rows) >= 100
    k = int(len(rows) * 0.8)
    p, mean, std, hist, alts = planner_train.train(rows[:k])
    assert hist[-1] < hist[0]
    learned, fixed = planner_train.evaluate(p, mean, std, rows[k:], alts)
    print(f"held-out regret: learned {learned.mean():.4f}, fixed rule {fixed.mean():.4f} "
          f"({len(rows) - k} chains; alternatives {alts})")
    assert np.all(np.isfinite(learned)) and np.all(learned >= 0)
    assert learned.mean() < fixed.mean()


def test_learned_planner_abstains_out_of_distribution():
    """Features far outside the training distribution (here: a standardisation that puts
    them at thousands of deviations): no prediction, the chain is autotuned instead."""
    from oracle import mlp
    from paper_1709_02125_gb300 import oc
    dats, reds, loops, fp = _chain()
    p = np.zeros(mlp.NPARAMS, dtype=np.float32)
    p[-2:] = (0.5, 0.1)                      # would choose an alternative if it answered
    oc.planner_load(p, np.zeros(8), np.full(8, 1e-3))
    with oc.Executor(fp // 3, planner=oc.OC_PLAN_LEARNED) as ex:
        oc.run_chain(ex, dats, reds, loops)
        table = ex.autotune_result()
        st = ex.stats()
    assert len(table) >= 24
    best = table[np.argmin(table[:, 2])]
    assert st["tile_height"] == int(best[0]) and st["depth"] == int(best[1])
