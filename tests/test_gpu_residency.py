"""Partially resident datasets (oc_set_residency): a streamed plan keeps the datasets that
move the most link bytes per byte whole in the device arena across chains, and streams
the rest through slabs sized from the remaining budget. The results must not change:
the same points are computed from the same inputs (Sec. 3), so a run with residency is
bit-identical to the untiled run and within 1e-12 of the oracle, over several chains,
with the pipeline options on, across changes of the resident set, and with a periodic
slow axis whose deep ghosts are refreshed on the device."""
import numpy as np
import pytest

from workloads import euler, random_chain

from gpu_helpers import rel_max, run_gpu, run_oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()


def _write_first(loops):
    first = {}
    for lp in loops:
        for a in lp.args:
            if a.access in ("r", "rw") and a.name not in first:
                first[a.name] = "r"
        for a in lp.args:
            if a.access in ("w", "rw") and a.name not in first:
                first[a.name] = "w"
    return {k for k, v in first.items() if v == "w"}


@pytest.mark.parametrize("level,flags", [(0.25, 0), (0.5, 0), (0.5, "pcg")])
def test_residency_bit_exact(oracle_lib, level, flags):
    from paper_1709_02125_gb300 import oc
    n, chains = 300, 3
    dats, reds, loops = random_chain.build(n=n, nfields=12, nloops=24, seed=31)
    fp = random_chain.footprint_bytes(n, 12)
    f = (oc.OC_FLAG_PREFETCH | oc.OC_FLAG_CYCLIC | oc.OC_FLAG_GRAPHS) if flags == "pcg" else 0
    inc, rin, sti = run_gpu(dats, reds, loops, 4 * fp, chains=chains)
    assert sti["tiles"] == 1
    got, rgot, st = run_gpu(dats, reds, loops, fp // 3, chains=chains, flags=f, residency=level)
    assert st["tiles"] > 1 and st["resident_dats"] > 0
    assert 0 < st["resident_bytes"] <= level * (fp // 3)
    keep = [d.name for d in dats if not (f & oc.OC_FLAG_CYCLIC and d.name in _write_first(loops))]
    for nm in keep:
        assert np.array_equal(inc[nm], got[nm]), nm
    assert rin == rgot
    ref, rref = run_oracle(oracle_lib, dats, reds, loops, chains=chains)
    for nm in keep:
        assert rel_max(got[nm], ref[nm]) <= 1e-12, nm


def test_residency_changes_between_chains(oracle_lib):
    """Half the budget resident for two chains (a fetch in between), then none for one
    chain, then 35 %: datasets leaving residency go home first, the results equal four
    oracle chains."""
    from paper_1709_02125_gb300 import oc
    n = 256
    dats, reds, loops = random_chain.build(n=n, nfields=10, nloops=20, seed=12)
    fp = random_chain.footprint_bytes(n, 10)
    with oc.Executor(fp // 3) as ex:
        for d in dats:
            ex.decl_dat(d)
        for r in reds:
            ex.decl_reduction(r.name, r.op)
        counts = []
        mid = None
        for k, level in enumerate((0.5, 0.5, 0.0, 0.35)):
            ex.set_residency(level)
            for lp in loops:
                ex.enqueue(lp)
            ex.flush()
            counts.append(ex.stats()["resident_dats"])
            if k == 0:
                mid = {d.name: ex.fetch(d.name) for d in dats}
        got = {d.name: ex.fetch(d.name) for d in dats}
    assert counts[0] > 0 and counts[2] == 0 and counts[3] > 0
    ref1, _ = run_oracle(oracle_lib, dats, reds, loops, chains=1)
    ref4, _ = run_oracle(oracle_lib, dats, reds, loops, chains=4)
    for d in dats:
        assert rel_max(mid[d.name], ref1[d.name]) <= 1e-12, d.name
        assert rel_max(got[d.name], ref4[d.name]) <= 1e-12, d.name


def test_residency_periodic_slow_axis():
    """Euler (periodic in both axes: deep ghost rows refreshed every chain) with half the
    budget resident equals the untiled run bit for bit over three CFL steps."""
    from paper_1709_02125_gb300 import oc
    n, steps = 200, 3
    fp = sum(np.prod(d.shape) * 8 for d in euler.datasets(n))
    out = []
    for budget, level in ((4 * fp, None), (fp // 3, 0.5)):
        with oc.Executor(int(budget)) as ex:
            if level is not None:
                ex.set_residency(level)
            dts, pre, _ = euler.run(ex, n, steps)
            st = ex.stats()
            U = np.stack([ex.fetch(f"{pre}_{k}") for k in ("r", "mx", "my", "E")])
        out.append((U, dts, st))
    (Ui, dti, sti), (Ur, dtr, str_) = out
    assert sti["tiles"] == 1 and str_["tiles"] > 1 and str_["resident_dats"] > 0
    assert np.array_equal(Ui, Ur) and dti == dtr


def test_autotune_trials_of_periodic_resident_plans():
    """The autotuner times plans that keep periodic datasets resident before any of them
    is made resident: the trials refresh those datasets' deep ghosts at the plan's own
    arena offsets. Euler with the autotuner at a third of the footprint equals the untiled
    run bit for bit, and the trials included resident plans."""
    from paper_1709_02125_gb300 import oc
    n, steps = 200, 3
    fp = sum(np.prod(d.shape) * 8 for d in euler.datasets(n))
    out = []
    for budget, planner in ((4 * fp, oc.OC_PLAN_FIXED), (fp // 3, oc.OC_PLAN_AUTOTUNE)):
        with oc.Executor(int(budget), planner=planner) as ex:
            dts, pre, _ = euler.run(ex, n, steps)
            st = ex.stats()
            tune = ex.autotune_result() if planner == oc.OC_PLAN_AUTOTUNE else None
            U = np.stack([ex.fetch(f"{pre}_{k}") for k in ("r", "mx", "my", "E")])
        out.append((U, dts, st, tune))
    (Ui, dti, sti, _), (Ua, dta, sta, tune) = out
    assert sti["tiles"] == 1 and sta["tiles"] > 1
    assert tune is not None and np.any(tune[:, 5] > 0)   # residency levels were tried
    assert np.array_equal(Ui, Ua) and dti == dta
