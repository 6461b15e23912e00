"""The PDE workloads' loop chains, evaluated loop by loop on the CPU (oracle.physics_loops):

* run in program order after the deep-ghost refresh of the periodic slow axis, the loops
  of one time step reproduce the oracle's whole-step functions (physics.c) bit for bit
  (both evaluate the same operations in the same order without contraction), which pins
  the loop-level form and the chain definitions in workloads/euler.py and tgv.py;
* the executor's tiled plans of those chains (dry-run analysis), replayed on tagged
  cyclic slabs with the same loop kernels, give the sequential results bit for bit --
  the deep ghosts, the extended ranges into them and the multi-step chains included."""
import numpy as np
import pytest

from workloads import euler, tgv

import plan_sim

EU = ["r", "mx", "my", "E"]


@pytest.fixture(scope="module")
def phys(oracle_lib):
    from oracle import physics, physics_loops
    return physics, physics_loops


def _sequential(oracle_lib, pl, dats, reds, loops, chains=1):
    fields = oracle_lib.make_fields(dats)
    out = None
    for _ in range(chains):
        pl.refresh_ghosts(fields)
        out = oracle_lib.run_chain(loops, fields, reds)
    return fields, out


def test_euler_step_chain_equals_step_function(oracle_lib, phys):
    physics, pl = phys
    from workloads.spec import RedSpec
    n = 32
    U0 = euler.initial(n)
    dt = euler.CFL * physics.euler_dt_min(U0, 1.0 / n, 1.0 / n, euler.GAMMA)
    dats = euler.datasets(n, "f64", U0)
    loops = euler.chain_loops(n, dt, "A", "B")
    f, red = _sequential(oracle_lib, pl, dats, [RedSpec("dtmin", "min")], loops)
    Uo = U0.copy()
    physics.euler_step(Uo, dt, 1.0 / n, 1.0 / n, euler.GAMMA, euler.EPS4)
    for k, c in enumerate(EU):
        assert np.array_equal(f[f"B_{c}"].a[2:n + 2], Uo[k]), c
    assert red["dtmin"] == physics.euler_dt_min(Uo, 1.0 / n, 1.0 / n, euler.GAMMA)


@pytest.mark.parametrize("steps", [2, 3])
def test_euler_fixed_dt_chain_equals_steps(oracle_lib, phys, steps):
    physics, pl = phys
    n = 24
    U0 = euler.initial(n)
    dt = 0.5 * euler.CFL * physics.euler_dt_min(U0, 1.0 / n, 1.0 / n, euler.GAMMA)
    dats = euler.datasets(n, "f64", U0, steps=steps)
    loops, src = euler.fixed_dt_chain(n, dt, steps)
    f, _ = _sequential(oracle_lib, pl, dats, [], loops)
    Uo = U0.copy()
    for _ in range(steps):
        physics.euler_step(Uo, dt, 1.0 / n, 1.0 / n, euler.GAMMA, euler.EPS4)
    G = 2 * steps
    for k, c in enumerate(EU):
        assert np.array_equal(f[f"{src}_{c}"].a[G:n + G], Uo[k]), c


@pytest.mark.parametrize("steps,fused", [(1, False), (1, True), (2, False)])
def test_tgv_chain_equals_step_function(oracle_lib, phys, steps, fused):
    physics, pl = phys
    n = 12
    U0 = np.ascontiguousarray(tgv.initial(n))
    dats = tgv.datasets(n, steps, "f64", U0, fused=fused)
    loops = tgv.chain_loops(n, steps, fused=fused)
    f, _ = _sequential(oracle_lib, pl, dats, [], loops)
    Uo = U0.copy()
    prm = physics.ns_params(tgv.GAMMA, tgv.MA, tgv.RE, tgv.PR, (tgv.h_of(n),) * 3)
    for _ in range(steps):
        physics.ns_step(Uo, tgv.dt_of(n), prm)
    G = tgv.ghost(steps)
    for m, c in enumerate(tgv.CONS):
        assert np.array_equal(f[c].a[G:G + n], Uo[m]), c


def _dry_plan(dats, reds, loops, h, depth, flags=0):
    from paper_1709_02125_gb300 import oc
    with oc.Executor(1 << 30, dryrun=True, flags=flags) as ex:
        ex.set_tiling(h, depth)
        oc.run_chain(ex, dats, reds, loops)
        return ex.plan(), dict(ex.names)


@pytest.mark.parametrize("h,depth", [(5, 3), (3, 2), (7, 4)])
def test_euler_tiled_replay_bit_exact(oracle_lib, phys, h, depth):
    physics, pl = phys
    import __graft_entry__
    __graft_entry__.build_lib()
    from workloads.spec import RedSpec
    n = 24
    U0 = euler.initial(n)
    dt = euler.CFL * physics.euler_dt_min(U0, 1.0 / n, 1.0 / n, euler.GAMMA)
    dats = euler.datasets(n, "f64", U0)
    reds = [RedSpec("dtmin", "min")]
    loops = euler.chain_loops(n, dt, "A", "B")
    plan, names = _dry_plan(dats, reds, loops, h, depth)
    assert plan["tiles"] > 1
    plan_sim.check_legality(plan, loops)
    got, gred = plan_sim.simulate(plan, loops, dats, reds, oracle_lib, names, chain_start=pl.refresh_ghosts)
    ref, rred = _sequential(oracle_lib, pl, dats, reds, loops)
    assert gred == rred
    for c in EU:
        assert np.array_equal(got[f"B_{c}"].a[2:n + 2], ref[f"B_{c}"].a[2:n + 2]), c


@pytest.mark.parametrize("steps,h", [(2, 6), (3, 5)])
def test_euler_multistep_tiled_replay_bit_exact(oracle_lib, phys, steps, h):
    physics, pl = phys
    import __graft_entry__
    __graft_entry__.build_lib()
    n = 24
    U0 = euler.initial(n)
    dt = 0.5 * euler.CFL * physics.euler_dt_min(U0, 1.0 / n, 1.0 / n, euler.GAMMA)
    dats = euler.datasets(n, "f64", U0, steps=steps)
    loops, src = euler.fixed_dt_chain(n, dt, steps)
    plan, names = _dry_plan(dats, [], loops, h, 3)
    assert plan["tiles"] > 1
    plan_sim.check_legality(plan, loops)
    got, _ = plan_sim.simulate(plan, loops, dats, [], oracle_lib, names, chains=2, chain_start=pl.refresh_ghosts)
    ref, _ = _sequential(oracle_lib, pl, dats, [], loops, chains=2)
    G = 2 * steps
    for c in EU:
        assert np.array_equal(got[f"{src}_{c}"].a[G:n + G], ref[f"{src}_{c}"].a[G:n + G]), c


@pytest.mark.parametrize("steps,fused,h", [(1, False, 4), (1, True, 5), (2, False, 7)])
def test_tgv_tiled_replay_bit_exact(oracle_lib, phys, steps, fused, h):
    physics, pl = phys
    import __graft_entry__
    __graft_entry__.build_lib()
    n = 12
    U0 = np.ascontiguousarray(tgv.initial(n))
    dats = tgv.datasets(n, steps, "f64", U0, fused=fused)
    loops = tgv.chain_loops(n, steps, fused=fused)
    plan, names = _dry_plan(dats, [], loops, h, 3)
    assert plan["tiles"] > 1
    plan_sim.check_legality(plan, loops)
    got, _ = plan_sim.simulate(plan, loops, dats, [], oracle_lib, names, chain_start=pl.refresh_ghosts)
    ref, _ = _sequential(oracle_lib, pl, dats, [], loops)
    G = tgv.ghost(steps)
    for c in tgv.CONS:
        assert np.array_equal(got[c].a[G:G + n], ref[c].a[G:G + n]), c
