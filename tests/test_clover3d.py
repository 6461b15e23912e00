"""Host-only tests of the CloverLeaf-3D-like workload (workloads/clover3d.py): its recipe,
and its plans -- a ~600-loop time-step chain and the read-only summary chain -- checked
by the brute-force legality checker and replayed on tagged slabs against the oracle
(arXiv 1709.02125, Sec. 3 / Sec. 4, and the chain structure of Sec. 5.1 / 5.3)."""
import math

import numpy as np
import pytest

from workloads import clover3d
from workloads.spec import DatSpec

import plan_sim

oc = pytest.importorskip("paper_1709_02125_gb300.oc")


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__
    __graft_entry__.build_lib()
    return oc.load()


def dry(budget, dats, reds, loops, h=0, depth=0, flags=0):
    with oc.Executor(budget, dryrun=True, flags=flags) as ex:
        ex.set_tiling(h, depth)
        oc.run_chain(ex, dats, reds, loops)
        return ex.plan(), dict(ex.names)


def _pad3(o):
    return tuple(o) + (0,) * (3 - len(o))


def test_recipe_structure():
    n, nz = 8, 40
    reds, loops = clover3d.step_chain(n, nz)
    assert len(loops) == 18 + 58 * 10 + 1
    assert [r.op for r in reds] == ["min"] and loops[-1].kernel == "reduce"
    first = {}
    zloops = 0
    for i, lp in enumerate(loops[:-1]):
        assert lp.kernel == "lincomb"
        out = lp.args[0].name
        first.setdefault(out, i)
        c = np.array(lp.params[1:])
        assert lp.params[0] == 0.5 and math.isclose(np.abs(c).sum(), 0.5, rel_tol=1e-12)
        assert len(c) == sum(len(a.offsets) for a in lp.args[1:]) <= 12
        offs = [_pad3(o) for a in lp.args[1:] for o in a.offsets]
        assert all(abs(o[0]) <= 2 and abs(o[1]) <= 2 and abs(o[2]) <= 1 for o in offs)
        assert sum(1 for o in offs if sum(v != 0 for v in o) > 1) == 0   # one axis per stage
        zloops += any(o[2] != 0 for o in offs)
        for a in lp.args[1:]:
            assert a.name != out
    # at most one z-reaching loop per z stage (19 of the 58 stages sweep z)
    assert 1 <= zloops <= 19
    # every work field is first written over its whole allocated extent (write-first)
    for w in range(clover3d.NWORK):
        lp = loops[first[f"w{w}"]]
        assert lp.lo == (-2, -2, -2) and lp.hi == (n + 2, n + 2, nz + 2)
        assert all(a.name.startswith("s") and _pad3(a.offsets[0]) == (0, 0, 0) for a in lp.args[1:])
    # a second call draws the same chain
    _, again = clover3d.step_chain(n, nz)
    assert all(a.params == b.params and a.lo == b.lo for a, b in zip(loops, again))


@pytest.mark.parametrize("frac", [3, 6])
def test_step_chain_plans_are_legal(lib, frac):
    """The full 599-loop step at 1/3 and 1/6 of the footprint: tiled, legal, and the skew
    of one step stays within about one row per z stage."""
    n, nz = 8, 200
    dats = clover3d.datasets(n, nz, with_init=False)
    reds, loops = clover3d.step_chain(n, nz)
    plan, _ = dry(clover3d.footprint_bytes(n, nz) // frac, dats, reds, loops)
    assert plan["tiles"] > 1
    plan_sim.check_legality(plan, loops)
    r = plan["ranges"]
    skew = max(int(r[0, i, 1]) for i in range(len(loops))) - int(r[0, -1, 1])
    assert 0 < skew <= 2 * 19


@pytest.mark.parametrize("h,depth,flags", [(7, 3, 0), (5, 2, "cyclic"), (9, 4, "cyclic+prefetch")])
def test_step_chain_simulation_matches_oracle(lib, oracle_lib, h, depth, flags):
    """Two time steps (the same chain twice) replayed on tagged cyclic slabs equal two
    oracle steps bit for bit. With the cyclic flag the work fields are per-chain
    temporaries (never uploaded, never downloaded), so only the state fields are
    compared there."""
    f = {0: 0, "cyclic": oc.OC_FLAG_CYCLIC, "cyclic+prefetch": oc.OC_FLAG_CYCLIC | oc.OC_FLAG_PREFETCH}[flags]
    n, nz = 8, 96
    dats = clover3d.datasets(n, nz)
    reds, loops = clover3d.step_chain(n, nz, stages=12)
    plan, names = dry(1 << 30, dats, reds, loops, h=h, depth=depth, flags=f)
    assert plan["tiles"] > 1
    plan_sim.check_legality(plan, loops)
    got, gred = plan_sim.simulate(plan, loops, dats, reds, oracle_lib, names, chains=2,
                                  prefetch=bool(f & oc.OC_FLAG_PREFETCH))
    ref = oracle_lib.make_fields(dats)
    for _ in range(2):
        rred = oracle_lib.run_chain(loops, ref, reds)
    assert gred == rred
    for d in dats:
        if f & oc.OC_FLAG_CYCLIC and d.name.startswith("w"):
            continue
        assert np.array_equal(got[d.name].a, ref[d.name].a), d.name


def test_copy_sets(lib):
    """Work fields are write-first in every step: never uploaded; with the cyclic flag
    never downloaded. Every state field the step reads is uploaded; the state fields it
    updates are downloaded."""
    n, nz = 8, 200
    dats = clover3d.datasets(n, nz, with_init=False)
    reds, loops = clover3d.step_chain(n, nz)
    updated = {lp.args[0].name for lp in loops if lp.kernel == "lincomb" and lp.args[0].name.startswith("s")}
    for flags in (0, oc.OC_FLAG_CYCLIC):
        plan, names = dry(clover3d.footprint_bytes(n, nz) // 3, dats, reds, loops, flags=flags)
        by = {d["dat"]: d for d in plan["dats"]}
        for w in range(clover3d.NWORK):
            d = by[names[f"w{w}"]]
            assert len(d["up"]) == 0
            assert (len(d["down"]) > 0) == (flags == 0)
        for s in range(clover3d.NSTATE):
            d = by.get(names[f"s{s}"])
            if d is None:
                continue
            assert len(d["up"]) > 0
            assert (len(d["down"]) > 0) == (f"s{s}" in updated)


def test_summary_chain_is_read_only_and_exact(lib, oracle_lib):
    """The summary chain uploads the 12 state fields and downloads nothing; replayed on
    tagged slabs after a step, its reductions agree with the oracle's, and the oracle's
    equal exactly rounded library sums (math.fsum) and numpy's max."""
    n, nz = 8, 96
    dats = clover3d.datasets(n, nz)
    sreds, sloops = clover3d.step_chain(n, nz, stages=6)
    plan, names = dry(1 << 30, dats, sreds, sloops, h=8, depth=3)
    got, _ = plan_sim.simulate(plan, sloops, dats, sreds, oracle_lib, names)
    after = [DatSpec(d.name, d.size, d.halo_lo, d.halo_hi, d.dtype, init=got[d.name].a.copy()) for d in dats]
    reds, loops = clover3d.summary_chain(n, nz)
    plan, names = dry(1 << 30, after, reds, loops, h=10, depth=3)
    assert plan["tiles"] > 1
    plan_sim.check_legality(plan, loops)
    by = {d["dat"]: d for d in plan["dats"]}
    assert len(by) == clover3d.NSTATE
    assert all(len(d["up"]) > 0 and len(d["down"]) == 0 for d in by.values())
    _, gred = plan_sim.simulate(plan, loops, after, reds, oracle_lib, names)
    ref = oracle_lib.make_fields(after)
    rred = oracle_lib.run_chain(loops, ref, reds)
    for r in reds:
        # the replay folds per-tile sums in tile order: equal up to rounding; max is exact
        tol = 1e-13 * max(1.0, abs(rred[r.name])) if r.op == "sum" else 0.0
        assert abs(gred[r.name] - rred[r.name]) <= tol, r.name
    for i in range(clover3d.NSTATE):
        v = got[f"s{i}"].a[2:-2, 2:-2, 2:-2].ravel()
        if i < 6:
            assert rred[f"sm{i}"] == math.fsum(v)
        elif i < 10:
            assert rred[f"sm{i}"] == math.fsum(v * v)
        else:
            assert rred[f"sm{i}"] == np.abs(v).max()
