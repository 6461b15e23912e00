"""Failure detection on the GPU without a device fault.

- Bounded waits: with OC_TIMEOUT_S far shorter than one chain, oc_flush returns
  OC_ERR_TIMEOUT while the device work is still queued; the kernels themselves run to
  completion, oc_finalize drains them, and a new context computes the right answer.
- Injected host-side faults (oc_inject_fault): an upload copy, a download copy or a
  kernel launch of a streamed chain fails as a CUDA call would, without calling CUDA.
  The running call returns OC_ERR_CUDA with the message, oc_finalize succeeds, and a new
  context in the same process matches the oracle. One case fails a launch during the
  first execution of a chain that is being captured as a CUDA graph (two compute streams
  forked), so the capture has to end cleanly too.
"""
import os

import numpy as np
import pytest

from workloads import random_chain

from gpu_helpers import rel_max, run_gpu, run_oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()


def _chain(n=160):
    return random_chain.build(n=n, nfields=10, nloops=16, seed=44), random_chain.footprint_bytes(n, 10)


def _check_recovered(oracle_lib, dats, reds, loops, fp):
    """A fresh context after the failure computes the chain exactly as the oracle does."""
    got, sums, st = run_gpu(dats, reds, loops, fp // 3)
    assert st["tiles"] > 1
    ref, rsums = run_oracle(oracle_lib, dats, reds, loops)
    for d in dats:
        assert rel_max(got[d.name], ref[d.name]) <= 1e-12, d.name


def test_bounded_wait_times_out_then_finalizes(oracle_lib):
    from paper_1709_02125_gb300 import oc
    n = 4096
    dats, reds, loops = random_chain.build(n=n, dtype="f32")
    for d in dats:
        d.init = d.init.astype(np.float32)
    fp = random_chain.footprint_bytes(n, 24, 4)
    old = os.environ.get("OC_TIMEOUT_S")
    os.environ["OC_TIMEOUT_S"] = "1e-6"
    try:
        ex = oc.Executor(fp // 3)
    finally:
        if old is None:
            del os.environ["OC_TIMEOUT_S"]
        else:
            os.environ["OC_TIMEOUT_S"] = old
    try:
        for d in dats:
            ex.decl_dat(d)
        for r in reds:
            ex.decl_reduction(r.name, r.op)
        for lp in loops:
            ex.enqueue(lp)
        with pytest.raises(oc.OcError) as e:
            ex.flush()
        assert e.value.code == oc.OC_ERR_TIMEOUT
        assert "bounded wait expired" in str(e.value)
    finally:
        ex.close()   # oc_finalize waits for the queued chain, then frees everything
    (d2, r2, l2), fp2 = _chain()
    _check_recovered(oracle_lib, d2, r2, l2, fp2)


@pytest.mark.parametrize("site,after,graphs", [(0, 5, False), (1, 3, False), (2, 20, False), (2, 7, True)])
def test_injected_fault_fails_cleanly(oracle_lib, site, after, graphs):
    from paper_1709_02125_gb300 import oc
    (dats, reds, loops), fp = _chain()
    flags = (oc.OC_FLAG_GRAPHS | oc.OC_FLAG_PREFETCH) if graphs else 0
    ex = oc.Executor(fp // 3, flags=flags)
    try:
        for d in dats:
            ex.decl_dat(d)
        for r in reds:
            ex.decl_reduction(r.name, r.op)
        ex.inject_fault(site, after)
        for lp in loops:
            ex.enqueue(lp)
        with pytest.raises(oc.OcError) as e:
            ex.flush()
        assert e.value.code == oc.OC_ERR_CUDA
        assert "injected fault" in str(e.value)
    finally:
        ex.close()
    _check_recovered(oracle_lib, dats, reds, loops, fp)
