"""Programmatic dependent launch (the kernels of a tile overlap their launches; each waits
for its predecessor before touching memory) changes no result: the same chains with the
launch attribute on (default) and off (OC_PDL=0, read at oc_init) give identical bits --
a random chain streamed through many short tiles with reductions, prefetch, cyclic slabs and
chain graphs, and the Euler step with its deep periodic ghosts and CFL reduction."""
import os

import numpy as np
import pytest

from workloads import euler, random_chain

from gpu_helpers import run_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()


def _both(fn):
    out = []
    old = os.environ.get("OC_PDL")
    try:
        for v in ("0", "1"):
            os.environ["OC_PDL"] = v
            out.append(fn())
    finally:
        if old is None:
            os.environ.pop("OC_PDL", None)
        else:
            os.environ["OC_PDL"] = old
    return out


def test_random_chain_identical_with_and_without_pdl():
    from paper_1709_02125_gb300 import oc
    n = 300
    dats, reds, loops = random_chain.build(n=n, nfields=12, nloops=24, seed=41)
    fp = random_chain.footprint_bytes(n, 12)
    flags = oc.OC_FLAG_PREFETCH | oc.OC_FLAG_CYCLIC | oc.OC_FLAG_GRAPHS
    (a, ra, sa), (b, rb, sb) = _both(lambda: run_gpu(dats, reds, loops, fp // 3, h=23, depth=3, flags=flags, chains=3))
    assert sa["tiles"] > 1 and sa["tiles"] == sb["tiles"]
    assert ra == rb
    for d in dats:
        assert np.array_equal(a[d.name], b[d.name]), d.name


def test_euler_identical_with_and_without_pdl():
    from paper_1709_02125_gb300 import oc
    n, steps = 160, 3
    fp = sum(np.prod(d.shape) * 4 for d in euler.datasets(n, "f32", None, True))
    flags = oc.OC_FLAG_PREFETCH | oc.OC_FLAG_CYCLIC | oc.OC_FLAG_GRAPHS

    def one():
        with oc.Executor(int(fp // 3), flags=flags) as ex:
            dts, pre, _ = euler.run(ex, n, steps, mixed=True)
            st = ex.stats()
            U = np.stack([ex.fetch(f"{pre}_{k}") for k in ("r", "mx", "my", "E")] +
                         [ex.fetch(f"L_{k}") for k in ("r", "mx", "my", "E")])
        return U, dts, st

    (ua, da, sa), (ub, db, sb) = _both(one)
    assert sa["tiles"] > 1
    assert da == db and np.array_equal(ua, ub)
