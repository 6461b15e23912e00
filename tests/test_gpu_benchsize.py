"""Parity at the sizes and settings the benchmark times (Sec. 3 sequential meaning of a
chain, through the Sec. 4 / 4.1 streamed pipeline), against the FP64 oracle.

- Headline random chain: 24 FP32 fields of 4096^2 (halo 2), 40 LINCOMB loops + 2 sums,
  device budget 1/3 of the footprint, prefetch + cyclic + graphs, learned planner, three
  chains -- exactly the benchmark's mixed+learned variant. Every field whose host copy
  the cyclic option keeps (all but the per-chain temporaries, whose first access in the
  chain is a write) is compared element by element with the oracle run from the same
  FP32-rounded initial values: relative L2 <= 1e-5 per field; every chain's two sums
  within 1e-5 of sum |v|.
- Euler 15360^2 and Taylor-Green 640^3 in the mixed form at 1/3 of the footprint (the PDE
  benchmark legs): the oracle cannot step these grids whole in test time, so it steps a
  periodic window around each sampled point (tests/sampled_oracle.py, bit-identical to the
  full-grid oracle there). Points sit on tile boundaries, on rows where a dataset's slab
  wraps, on the periodic seams and on the features of the initial state; the bar is
  1e-5 of the field's scale.
"""
import os

import numpy as np
import pytest

from workloads import euler, random_chain, tgv

import sampled_oracle
from gpu_helpers import rel_l2

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()


def _load_learned_planner():
    from paper_1709_02125_gb300 import oc, planner_train
    rows = planner_train.load_rows(os.path.join(ROOT, "paper_1709_02125_gb300", "planner_data",
                                                "autotune_gb300.jsonl"))
    k = int(len(rows) * 0.8)
    p, mean, std, _, alts = planner_train.train(rows[:k])
    planner_train.install(p, mean, std, alts)


def _write_first(loops):
    """Datasets whose first access in the chain is a write (reads of a loop count first)."""
    first = {}
    for lp in loops:
        for a in lp.args:
            if a.access in ("r", "rw") and a.name not in first:
                first[a.name] = "r"
        for a in lp.args:
            if a.access in ("w", "rw") and a.name not in first:
                first[a.name] = "w"
    return {k for k, v in first.items() if v == "w"}


def test_headline_mixed_random_chain_full_size(oracle_lib):
    from paper_1709_02125_gb300 import oc
    n, chains = 4096, 3
    dats, reds, loops = random_chain.build(n=n, dtype="f32")
    for d in dats:
        d.init = d.init.astype(np.float32)
    fp = random_chain.footprint_bytes(n, 24, 4)
    _load_learned_planner()
    flags = oc.OC_FLAG_PREFETCH | oc.OC_FLAG_CYCLIC | oc.OC_FLAG_GRAPHS
    sums = []
    with oc.Executor(int(fp / 3), flags=flags, planner=oc.OC_PLAN_LEARNED) as ex:
        for d in dats:
            ex.decl_dat(d)
        for r in reds:
            ex.decl_reduction(r.name, r.op)
        for _ in range(chains):
            for lp in loops:
                ex.enqueue(lp)
            ex.flush()
            sums.append({r.name: ex.reduce(r.name) for r in reds})
        st = ex.stats()
        got = {d.name: ex.fetch(d.name) for d in dats}
    assert st["tiles"] > 1 and st["graph_replays"] > 0 and st["prefetched_bytes"] > 0
    # the oracle from the same FP32-rounded initial values, in FP64
    fields = oracle_lib.make_fields(dats)
    osums = []
    abs_sums = []
    for _ in range(chains):
        osums.append(oracle_lib.run_chain(loops, fields, reds))
        abs_sums.append({lp.args[-1].name: float(np.abs(fields[lp.args[0].name].a).sum())
                         for lp in loops if lp.kernel == "reduce"})
    temps = _write_first(loops)
    errs = {}
    for d in dats:
        if d.name in temps:
            continue
        errs[d.name] = rel_l2(got[d.name], fields[d.name].a)
    print("headline mixed chain (24 x 4096^2, 3 chains), relative L2 per kept field: " +
          " ".join(f"{k}={v:.2e}" for k, v in errs.items()))
    print("sum errors / sum|v|: " + " ".join(
        f"{r}={abs(s[r] - o[r]) / a[r]:.2e}" for s, o, a in zip(sums, osums, abs_sums) for r in s))
    assert len(errs) >= 10
    for k, e in errs.items():
        assert e <= 1e-5, (k, e)
    for s, o, a in zip(sums, osums, abs_sums):
        for r in s:
            assert abs(s[r] - o[r]) <= 1e-5 * a[r], (r, s[r], o[r])


def _footprint(dats):
    return sum(int(np.prod(d.shape)) * (8 if d.dtype == "f64" else 4) for d in dats)


def _slow_points(plan, n, ghost, extra):
    """Interior slow-axis rows worth checking: rows next to every tile boundary of the
    plan's first loop, rows where some slab wraps (slot 0 and S - 1), the periodic seams
    and `extra`."""
    rows = set(extra) | {0, 1, n - 2, n - 1}
    rng = plan["ranges"]
    for t in range(1, plan["tiles"]):
        b = int(rng[t, 0, 0])
        rows |= {b - 1, b}
    for dp in plan["dats"]:
        S = dp["S"]
        for k in (1, 2):
            y = -ghost + k * S
            rows |= {y - 1, y}
    return sorted(r for r in rows if 0 <= r < n)


def test_euler_full_size_points(oracle_lib):
    """Euler 15360^2, mixed, 1/3 of the footprint, one CFL step (the benchmark's chain: the
    dt of the step comes from the min-reduction over the initial state). The GPU's dt is
    checked against the oracle's; the state after the step at sampled points against the
    windowed oracle stepping the oracle's own dt."""
    from oracle import physics
    from paper_1709_02125_gb300 import oc
    n = 15360
    U0 = euler.initial(n)
    fp = _footprint(euler.datasets(n, "f32", None, True))
    flags = oc.OC_FLAG_CYCLIC | oc.OC_FLAG_PREFETCH | oc.OC_FLAG_GRAPHS
    with oc.Executor(fp // 3, flags=flags) as ex:
        dts, _, _ = euler.run(ex, n, 1, mixed=True, U0=U0)
        plan = ex.plan()
        U = np.stack([ex.fetch(f"A_{k}")[2:n + 2].astype(np.float64) + ex.fetch(f"L_{k}")[2:n + 2].astype(np.float64)
                      for k in ("r", "mx", "my", "E")])
    assert plan["tiles"] > 1
    dt_o = euler.CFL * physics.euler_dt_min(U0, 1.0 / n, 1.0 / n, euler.GAMMA)
    assert abs(dts[0] - dt_o) <= 1e-6 * dt_o, (dts[0], dt_o)
    # the square (side n/4, centred) has its edges at n*3/8 and n*5/8
    e0, e1 = 3 * n // 8, 5 * n // 8
    ys = _slow_points(plan, n, 2, [e0 - 1, e0, e1 - 1, e1, n // 2])
    xs = [0, 1, e0 - 1, e0, n // 2, e1, n - 1]
    rng = np.random.default_rng(15360)
    pts = [(y, x) for y in ys for x in xs[::2]] + [(y, int(rng.integers(0, n))) for y in ys]
    want = sampled_oracle.euler_points(physics, U0, pts, dt_o, 1.0 / n, 1.0 / n, 1, euler.GAMMA, euler.EPS4)
    got = np.array([U[:, y, x] for y, x in pts])
    scale = [np.max(np.abs(U0[0])), np.max(np.abs(want[:, 1])) + 1e-30, np.max(np.abs(want[:, 2])) + 1e-30,
             np.max(np.abs(U0[3]))]
    # the momentum scale: the largest momentum the oracle gives at the sampled points,
    # which include the square's edges (where the flow starts)
    assert scale[1] > 1e-6 and scale[2] > 1e-6
    err = [float(np.max(np.abs(got[:, k] - want[:, k]))) / scale[k] for k in range(4)]
    print(f"Euler 15360^2 mixed, 1 step, {len(pts)} points: max error / scale per field "
          + " ".join(f"{c}={e:.2e}" for c, e in zip(("r", "mx", "my", "E"), err)) +
          f"; dt rel err {abs(dts[0] - dt_o) / dt_o:.2e}")
    for k in range(4):
        assert err[k] <= 1e-5, (k, err[k])


def test_tgv_full_size_points(oracle_lib):
    """Taylor-Green 640^3, mixed, 1/3 of the footprint, one RK3 step per chain (the
    benchmark's TGV chain): sampled points against the windowed oracle."""
    from oracle import physics
    from paper_1709_02125_gb300 import oc
    n = 640
    U0 = np.ascontiguousarray(tgv.initial(n))
    fp = _footprint(tgv.datasets(n, 1, "f32", None, True))
    G = tgv.ghost(1)
    flags = oc.OC_FLAG_CYCLIC | oc.OC_FLAG_PREFETCH | oc.OC_FLAG_GRAPHS
    with oc.Executor(fp // 3, flags=flags) as ex:
        tgv.run(ex, n, 1, 1, mixed=True, U0=U0)
        plan = ex.plan()
        U = [ex.fetch(c)[G:G + n].astype(np.float64) + ex.fetch("lo_" + c)[G:G + n].astype(np.float64)
             for c in tgv.CONS]
    assert plan["tiles"] > 1
    zs = _slow_points(plan, n, G, [n // 4, n // 2])
    rng = np.random.default_rng(640)
    pts = []
    for i, z in enumerate(zs):
        y = [0, n - 1, n // 2, int(rng.integers(0, n))][i % 4]
        x = [n - 1, 0, int(rng.integers(0, n)), n // 3][i % 4]
        pts.append((z, y, x))
    prm = physics.ns_params(tgv.GAMMA, tgv.MA, tgv.RE, tgv.PR, (tgv.h_of(n),) * 3)
    want = sampled_oracle.ns_points(physics, U0, pts, tgv.dt_of(n), prm, 1)
    got = np.array([[U[m][z, y, x] for m in range(5)] for z, y, x in pts])
    del U
    umax = np.max(np.abs(want[:, 1]))
    scale = [np.max(np.abs(want[:, 0])), umax, umax, umax, np.max(np.abs(want[:, 4]))]
    err = [float(np.max(np.abs(got[:, m] - want[:, m]))) / scale[m] for m in range(5)]
    print(f"TGV 640^3 mixed, 1 RK3 step, {len(pts)} points: max error / scale per field "
          + " ".join(f"{c}={e:.2e}" for c, e in zip(tgv.CONS, err)))
    for m in range(5):
        assert err[m] <= 1e-5, (tgv.CONS[m], err[m])
