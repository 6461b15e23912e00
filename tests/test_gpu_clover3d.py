"""GPU parity of the CloverLeaf-3D-like workload (workloads/clover3d.py) through the C ABI:
two 599-loop time steps and the read-only summary chain, tiled at 1/3 of the footprint
with the cyclic flag, prefetch and CUDA graphs, against the oracle and against an
untiled run.

Bars (as for the other FP64 chains): tiled == untiled bit for bit; state fields within
1e-12 normwise relative max of the oracle; the step's MIN within 1e-12; the summary sums
within 1e-12 of sum |v|."""
import numpy as np
import pytest

from workloads import clover3d

from gpu_helpers import rel_max

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()


def _gpu(n, nz, budget, flags, steps):
    from paper_1709_02125_gb300 import oc
    dats = clover3d.datasets(n, nz)
    sreds, sloops = clover3d.step_chain(n, nz)
    mreds, mloops = clover3d.summary_chain(n, nz)
    dts, tiles = [], []
    with oc.Executor(budget, flags=flags) as ex:
        for d in dats:
            ex.decl_dat(d)
        for r in sreds + mreds:
            ex.decl_reduction(r.name, r.op)
        for _ in range(steps):
            for lp in sloops:
                ex.enqueue(lp)
            dts.append(ex.reduce("dt"))
            tiles.append(ex.stats()["tiles"])
        for lp in mloops:
            ex.enqueue(lp)
        summary = {r.name: ex.reduce(r.name) for r in mreds}
        state = {f"s{i}": ex.fetch(f"s{i}") for i in range(clover3d.NSTATE)}
    return state, dts, summary, tiles


def _oracle(oracle, n, nz, steps):
    dats = clover3d.datasets(n, nz)
    sreds, sloops = clover3d.step_chain(n, nz)
    mreds, mloops = clover3d.summary_chain(n, nz)
    f = oracle.make_fields(dats)
    dts = [oracle.run_chain(sloops, f, sreds)["dt"] for _ in range(steps)]
    summary = oracle.run_chain(mloops, f, mreds)
    state = {f"s{i}": f[f"s{i}"].a for i in range(clover3d.NSTATE)}
    return state, dts, summary


def test_clover3d_two_steps_and_summary(oracle_lib):
    from paper_1709_02125_gb300 import oc
    n, nz, steps = 16, 200, 2
    fp = clover3d.footprint_bytes(n, nz)
    flags = oc.OC_FLAG_CYCLIC | oc.OC_FLAG_PREFETCH | oc.OC_FLAG_GRAPHS
    til, dtt, smt, tiles = _gpu(n, nz, fp // 3, flags, steps)
    inc, dti, smi, tin = _gpu(n, nz, 4 * fp, 0, steps)
    assert all(t > 1 for t in tiles) and all(t == 1 for t in tin)
    for k in til:
        assert np.array_equal(til[k], inc[k]), k
    assert dtt == dti and smt == smi
    ref, dto, smo = _oracle(oracle_lib, n, nz, steps)
    for k in ref:
        assert rel_max(til[k], ref[k]) <= 1e-12, k
    for a, b in zip(dtt, dto):
        assert abs(a - b) <= 1e-12 * max(1.0, abs(b))
    for i in range(clover3d.NSTATE):
        name = f"sm{i}"
        v = ref[f"s{i}"][2:-2, 2:-2, 2:-2]
        scale = float(np.sum(v * v)) if 6 <= i < 10 else float(np.abs(v).sum())
        assert abs(smt[name] - smo[name]) <= 1e-12 * max(1.0, scale), name
