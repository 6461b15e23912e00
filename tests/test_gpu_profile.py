"""GPU tests of the measurement hooks: per-kernel profiling (OC_FLAG_PROFILE) and the
per-phase time line (OC_FLAG_TRACE) must account for exactly the work of the plan, and
neither may change results."""
import numpy as np
import pytest

from workloads import random_chain

from gpu_helpers import run_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()


def _chain(n=384):
    dats, reds, loops = random_chain.build(n=n, nfields=10, nloops=16, seed=91, dtype="f32")
    for d in dats:
        d.init = d.init.astype(np.float32)
    return dats, reds, loops, random_chain.footprint_bytes(n, 10, 4)


def _expected(plan, loops, kernel):
    """(launches, algorithmic bytes) the plan issues for one kernel id: one launch per
    loop and tile with a non-empty range; each dataset argument moves its range once."""
    launches, nbytes = 0, 0.0
    for t in range(plan["tiles"]):
        for i, lp in enumerate(loops):
            s, e = plan["ranges"][t, i]
            if e <= s or lp.kernel != kernel:
                continue
            pts = (lp.hi[0] - lp.lo[0]) * (e - s)
            launches += 1
            nbytes += sum(pts * 4 * (2 if a.access == "rw" else 1) for a in lp.args if a.access != "red")
    return launches, nbytes


@pytest.mark.parametrize("graphs", [False, True])
def test_profile_counts_match_plan(graphs):
    from paper_1709_02125_gb300 import oc
    dats, reds, loops, fp = _chain()
    ref, rr, _ = run_gpu(dats, reds, loops, fp // 3, chains=2)
    flags = oc.OC_FLAG_PROFILE | (oc.OC_FLAG_GRAPHS if graphs else 0)
    with oc.Executor(fp // 3, flags=flags) as ex:
        for d in dats:
            ex.decl_dat(d)
        for r in reds:
            ex.decl_reduction(r.name, r.op)
        for _ in range(2):
            ex.kernel_stats_reset()
            for lp in loops:
                ex.enqueue(lp)
            ex.flush()
        got_red = {r.name: ex.reduce(r.name) for r in reds}
        plan = ex.plan()
        assert plan["tiles"] > 1
        for name in ("lincomb", "reduce"):
            ks = ex.kernel_stats(name)
            n_exp, b_exp = _expected(plan, loops, name)
            assert ks["launches"] == n_exp, name
            assert ks["bytes"] == pytest.approx(b_exp, rel=1e-12), name
            assert (ks["ms"] > 0) == (n_exp > 0)
        got = {d.name: ex.fetch(d.name) for d in dats}
    assert got_red == rr[-1]
    for d in dats:
        assert np.array_equal(got[d.name], ref[d.name]), d.name


def test_trace_covers_every_tile():
    from paper_1709_02125_gb300 import oc
    dats, reds, loops, fp = _chain()
    with oc.Executor(fp // 3, flags=oc.OC_FLAG_TRACE | oc.OC_FLAG_CYCLIC) as ex:
        for d in dats:
            ex.decl_dat(d)
        for r in reds:
            ex.decl_reduction(r.name, r.op)
        for lp in loops:
            ex.enqueue(lp)
        ex.flush()
        tr = ex.trace()
        st = ex.stats()
        T = ex.plan()["tiles"]
    comp = sorted(r[0] for r in tr if r[1] == "compute")
    assert comp == list(range(T))
    up = sum(r[4] for r in tr if r[1] == "upload")
    down = sum(r[4] for r in tr if r[1] == "download")
    assert up == st["h2d_bytes"] and down == st["d2h_bytes"]
    for r in tr:
        assert 0 <= r[2] <= r[3]
    # a tile's compute starts no earlier than its upload ends (tiles with nothing to
    # upload do not wait)
    ends = {r[0]: r[3] for r in tr if r[1] == "upload" and r[4] > 0}
    for r in tr:
        if r[1] == "compute" and r[0] in ends:
            assert r[2] >= ends[r[0]] - 1e-3
