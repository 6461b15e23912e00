"""The Unified Memory variant (OC_FLAG_MANAGED; Sec. 5.4 of the paper, tiling with
prefetches): stores in managed memory addressed in place by the kernels, each tile's
copies replaced by prefetches of its rows to the GPU and back. The kernels are the same,
so results equal the explicit pipeline's untiled run bit for bit and the oracle within
1e-12, with one tile or many, and on a periodic slow axis."""
import numpy as np
import pytest

from workloads import euler, random_chain

from gpu_helpers import rel_max, run_gpu, run_oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()


@pytest.mark.parametrize("frac,tiled", [(1 / 3, True), (4.0, False)])
def test_managed_random_chain(oracle_lib, frac, tiled):
    from paper_1709_02125_gb300 import oc
    n, chains = 300, 3
    dats, reds, loops = random_chain.build(n=n, nfields=12, nloops=24, seed=31)
    fp = random_chain.footprint_bytes(n, 12)
    inc, rin, _ = run_gpu(dats, reds, loops, 4 * fp, chains=chains)
    got, rgot, st = run_gpu(dats, reds, loops, int(fp * frac), chains=chains, flags=oc.OC_FLAG_MANAGED)
    assert (st["tiles"] > 1) == tiled
    assert st["h2d_bytes"] > 0 and (st["d2h_bytes"] > 0) == tiled
    for d in dats:
        assert np.array_equal(inc[d.name], got[d.name]), d.name
    assert rin == rgot
    ref, _ = run_oracle(oracle_lib, dats, reds, loops, chains=chains)
    for d in dats:
        assert rel_max(got[d.name], ref[d.name]) <= 1e-12, d.name


def test_managed_periodic_slow_axis():
    """Euler (periodic; deep ghost rows refreshed in the managed stores every chain),
    managed at a third of the footprint, equals the explicit untiled run bit for bit."""
    from paper_1709_02125_gb300 import oc
    n, steps = 200, 3
    fp = sum(np.prod(d.shape) * 8 for d in euler.datasets(n))
    out = []
    for budget, flags in ((4 * fp, 0), (fp // 3, oc.OC_FLAG_MANAGED)):
        with oc.Executor(int(budget), flags=flags) as ex:
            dts, pre, _ = euler.run(ex, n, steps)
            st = ex.stats()
            U = np.stack([ex.fetch(f"{pre}_{k}") for k in ("r", "mx", "my", "E")])
        out.append((U, dts, st))
    (Ui, dti, sti), (Um, dtm, stm) = out
    assert sti["tiles"] == 1 and stm["tiles"] > 1
    assert np.array_equal(Ui, Um) and dti == dtm
