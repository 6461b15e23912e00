"""Host-only checks of the PDE loop chains: the executor accepts their argument
layouts and stencils, and their tiled plans are legal (dry-run contexts, no GPU)."""
import numpy as np
import pytest

from workloads import euler, tgv

import plan_sim

oc = pytest.importorskip("paper_1709_02125_gb300.oc")


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__
    __graft_entry__.build_lib()
    return oc.load()


@pytest.mark.parametrize("mixed", [False, True])
@pytest.mark.parametrize("h", [3, 17])
def test_euler_chain_plan_is_legal(lib, mixed, h):
    n = 48
    with oc.Executor(1 << 30, dryrun=True) as ex:
        ex.set_tiling(h, 3)
        for d in euler.datasets(n, "f32" if mixed else "f64", None, mixed):
            ex.decl_dat(d)
        ex.decl_reduction("dtmin", "min")
        loops = euler.chain_loops(n, 1e-3, mixed=mixed)
        for lp in loops:
            ex.enqueue(lp)
        ex.flush()
        plan = ex.plan()
    assert plan["tiles"] == -(-(n + 2) // h)
    plan_sim.check_legality(plan, loops)


@pytest.mark.parametrize("steps,mixed", [(2, False), (3, False), (3, True)])
def test_euler_fixed_dt_chain_plan_is_legal(lib, steps, mixed):
    """Multi-step fixed-dt Euler chains: accepted (every range stays inside the ghost
    rows) and their tiled plans are legal."""
    n = 40
    with oc.Executor(1 << 30, dryrun=True, flags=oc.OC_FLAG_CYCLIC) as ex:
        ex.set_tiling(7, 3)
        for d in euler.datasets(n, "f32" if mixed else "f64", None, mixed, steps=steps):
            ex.decl_dat(d)
        loops, _ = euler.fixed_dt_chain(n, 1e-3, steps, mixed)
        for lp in loops:
            ex.enqueue(lp)
        ex.flush()
        plan = ex.plan()
    assert plan["tiles"] > 1
    plan_sim.check_legality(plan, loops)


@pytest.mark.parametrize("steps,mixed", [(1, False), (2, False), (1, True)])
def test_tgv_chain_plan_is_legal(lib, steps, mixed):
    n = 12
    with oc.Executor(1 << 30, dryrun=True, flags=oc.OC_FLAG_CYCLIC) as ex:
        ex.set_tiling(5, 3)
        for d in tgv.datasets(n, steps, "f32" if mixed else "f64", None, mixed):
            ex.decl_dat(d)
        loops = tgv.chain_loops(n, steps, mixed)
        for lp in loops:
            ex.enqueue(lp)
        ex.flush()
        plan = ex.plan()
        names = dict(ex.names)
    plan_sim.check_legality(plan, loops)
    by = {d["dat"]: d for d in plan["dats"]}
    # with the cyclic option only the conserved variables travel both ways
    moved_down = {n_ for n_, h in names.items() if len(by.get(h, {"down": []})["down"])}
    cons = set(tgv.CONS) | ({"lo_" + c for c in tgv.CONS} if mixed else set())
    assert moved_down == cons
    up_full = {n_ for n_, h in names.items() if any(x0 == x1 for *_, x0, x1 in by.get(h, {"up": []})["up"])}
    assert up_full == cons


def test_physics_argument_checks(lib):
    n = 16
    with oc.Executor(1 << 30, dryrun=True) as ex:
        for d in euler.datasets(n):
            ex.decl_dat(d)
        ex.decl_reduction("dtmin", "min")
        good = euler.chain_loops(n, 1e-3)
        bad_stencil = good[2]
        bad_stencil.args[4].offsets = [(0, 0), (2, 0)]
        with pytest.raises(oc.OcError) as e:
            ex.enqueue(bad_stencil)
        assert e.value.code == oc.OC_ERR_ARG
        bad_params = euler.chain_loops(n, 1e-3)[0]
        bad_params.params = []
        with pytest.raises(oc.OcError):
            ex.enqueue(bad_params)
