"""GPU parity of the PDE workloads (Euler MacCormack 2-D, Navier-Stokes TGV 3-D) against
the oracle's step functions, through the C ABI.

Bars: FP64 tiled == FP64 untiled bit for bit; FP64 against the oracle within 1e-12
normwise relative max per conserved field; FP32-stored (hi/lo compensated) runs within
1e-5 relative L2 per conserved field, with FP64 totals conserved.
"""
import numpy as np
import pytest

from workloads import euler, tgv

from gpu_helpers import rel_l2, rel_max

pytestmark = pytest.mark.gpu

EU = ["r", "mx", "my", "E"]


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()


def euler_gpu(n, steps, budget, mixed=False, h=0, flags=0, totals=False, inplace=False):
    from paper_1709_02125_gb300 import oc
    with oc.Executor(budget, flags=flags) as ex:
        ex.set_tiling(h, 3 if h else 0)
        dts, pre, tots = euler.run(ex, n, steps, mixed=mixed, totals=totals, inplace=inplace)
        st = ex.stats()
        U = np.stack([ex.fetch(f"{pre}_{k}")[2:n + 2].astype(np.float64) for k in EU])
        if mixed:
            U = U + np.stack([ex.fetch(f"L_{k}")[2:n + 2].astype(np.float64) for k in EU])
    return U, dts, st, tots


def euler_oracle(n, steps):
    from oracle import physics
    U = euler.initial(n)
    dts = []
    for _ in range(steps):
        dt = euler.CFL * physics.euler_dt_min(U, 1.0 / n, 1.0 / n, euler.GAMMA)
        dts.append(dt)
        physics.euler_step(U, dt, 1.0 / n, 1.0 / n, euler.GAMMA, euler.EPS4)
    return U, dts


def footprint(dats):
    return sum(np.prod(d.shape) * (8 if d.dtype == "f64" else 4) for d in dats)


def test_euler_fp64_tiled_untiled_oracle(oracle_lib):
    n, steps = 200, 4
    fp = footprint(euler.datasets(n))
    Ui, dti, sti, _ = euler_gpu(n, steps, 4 * fp)
    Ut, dtt, stt, _ = euler_gpu(n, steps, fp // 3)
    assert sti["tiles"] == 1 and stt["tiles"] > 1
    assert np.array_equal(Ui, Ut) and dti == dtt
    Uo, dto = euler_oracle(n, steps)
    for k in range(4):
        assert rel_max(Ut[k], Uo[k]) <= 1e-12, EU[k]
    assert np.allclose(dtt, dto, rtol=1e-12, atol=0)


def test_euler_fp64_in_place_form_under_cyclic(oracle_lib):
    """The FP64 in-place form (A += D, the same chain every step) with cyclic + prefetch +
    graphs at a third of the footprint: bit-identical to its untiled run, within 1e-12 of
    the oracle's direct MacCormack update, and its intermediates never leave the device."""
    from paper_1709_02125_gb300 import oc
    n, steps = 200, 4
    fp = footprint(euler.datasets(n, inplace=True))
    flags = oc.OC_FLAG_CYCLIC | oc.OC_FLAG_PREFETCH | oc.OC_FLAG_GRAPHS
    Ui, dti, sti, _ = euler_gpu(n, steps, 4 * fp, inplace=True)
    Ut, dtt, stt, _ = euler_gpu(n, steps, fp // 3, flags=flags, inplace=True)
    assert sti["tiles"] == 1 and stt["tiles"] > 1
    assert np.array_equal(Ui, Ut) and dti == dtt
    # one chain downloads the conserved state only: 4 datasets of at most n + 4 rows
    # of (padded) x-lines of n points
    assert stt["d2h_bytes"] <= 4 * (n + 4) * (n + 8) * 8
    Uo, dto = euler_oracle(n, steps)
    for k in range(4):
        assert rel_max(Ut[k], Uo[k]) <= 1e-12, EU[k]
    assert np.allclose(dtt, dto, rtol=1e-12, atol=0)


def test_euler_fp64_forced_small_tiles(oracle_lib):
    n, steps = 130, 3
    fp = footprint(euler.datasets(n))
    Ut, _, st, _ = euler_gpu(n, steps, 2 * fp, h=9)
    assert st["tiles"] == -(-(n + 2) // 9)
    Uo, _ = euler_oracle(n, steps)
    for k in range(4):
        assert rel_max(Ut[k], Uo[k]) <= 1e-12, EU[k]


def test_euler_mixed_error_and_totals(oracle_lib):
    from paper_1709_02125_gb300 import oc
    n, steps = 160, 6
    fp = footprint(euler.datasets(n, "f32", None, True))
    Um, dtm, st, tots = euler_gpu(n, steps, fp // 3, mixed=True, totals=True,
                                  flags=oc.OC_FLAG_CYCLIC | oc.OC_FLAG_PREFETCH | oc.OC_FLAG_GRAPHS)
    assert st["tiles"] > 1
    Uo, dto = euler_oracle(n, steps)
    errs = [rel_l2(Um[k], Uo[k]) for k in range(4)]
    print("mixed Euler, relative L2 error per conserved field:",
          " ".join(f"{EU[k]}={errs[k]:.2e}" for k in range(4)),
          f"dt rel {np.max(np.abs(np.array(dtm) - np.array(dto)) / np.array(dto)):.2e}")
    for k in range(4):
        assert errs[k] <= 1e-5, EU[k]
    U0 = euler.initial(n)
    t0 = U0.reshape(4, -1).sum(axis=1)
    scale = np.abs(U0).reshape(4, -1).sum(axis=1) + 1.0
    for t in tots:
        assert np.all(np.abs(np.array(t) - t0) <= 1e-6 * scale)
    assert np.allclose(dtm, dto, rtol=1e-5, atol=0)


def euler_fixed_gpu(n, spc, chains, dt, budget, mixed=False, h=0, flags=0):
    """`chains` chains of `spc` fixed-dt steps each (no reduction in the chain)."""
    from paper_1709_02125_gb300 import oc
    G = 2 * spc
    with oc.Executor(budget, flags=flags) as ex:
        ex.set_tiling(h, 3 if h else 0)
        for d in euler.datasets(n, "f32" if mixed else "f64", euler.initial(n), mixed, steps=spc):
            ex.decl_dat(d)
        src = "A"
        for _ in range(chains):
            loops, src = euler.fixed_dt_chain(n, dt, spc, mixed, src)
            for lp in loops:
                ex.enqueue(lp)
            ex.flush()
        st = ex.stats()
        U = np.stack([ex.fetch(f"{src}_{k}")[G:n + G].astype(np.float64) for k in EU])
        if mixed:
            U = U + np.stack([ex.fetch(f"L_{k}")[G:n + G].astype(np.float64) for k in EU])
    return U, st


@pytest.mark.parametrize("spc", [2, 3])
def test_euler_fixed_dt_multistep_chains(oracle_lib, spc):
    """Several fixed-dt steps per chain (ghost depth 2 per step): untiled == tiled bit for
    bit, both against the oracle stepping the same dt; mixed within 1e-5."""
    from oracle import physics
    n, chains = 96, 2
    U0 = euler.initial(n)
    dt = 0.5 * euler.CFL * physics.euler_dt_min(U0, 1.0 / n, 1.0 / n, euler.GAMMA)
    fp = footprint(euler.datasets(n, steps=spc))
    Ui, sti = euler_fixed_gpu(n, spc, chains, dt, 4 * fp)
    Ut, stt = euler_fixed_gpu(n, spc, chains, dt, 4 * fp, h=11)
    assert sti["tiles"] == 1 and stt["tiles"] > 1
    assert np.array_equal(Ui, Ut)
    Uo = U0.copy()
    for _ in range(spc * chains):
        physics.euler_step(Uo, dt, 1.0 / n, 1.0 / n, euler.GAMMA, euler.EPS4)
    for k in range(4):
        assert rel_max(Ut[k], Uo[k]) <= 1e-12, EU[k]
    from paper_1709_02125_gb300 import oc
    fpm = footprint(euler.datasets(n, "f32", None, True, steps=spc))
    Um, stm = euler_fixed_gpu(n, spc, chains, dt, fpm // 2, mixed=True,
                              flags=oc.OC_FLAG_CYCLIC | oc.OC_FLAG_PREFETCH | oc.OC_FLAG_GRAPHS)
    assert stm["tiles"] > 1
    for k in range(4):
        assert rel_l2(Um[k], Uo[k]) <= 1e-5, EU[k]


def tgv_gpu(n, chains, spc, budget, mixed=False, h=0, flags=0, fused=False):
    from paper_1709_02125_gb300 import oc
    G = tgv.ghost(spc)
    with oc.Executor(budget, flags=flags) as ex:
        ex.set_tiling(h, 3 if h else 0)
        tgv.run(ex, n, chains, spc, mixed=mixed, fused=fused)
        st = ex.stats()
        U = np.stack([ex.fetch(c)[G:G + n].astype(np.float64) for c in tgv.CONS])
        if mixed:
            U = U + np.stack([ex.fetch("lo_" + c)[G:G + n].astype(np.float64) for c in tgv.CONS])
    return U, st


def tgv_oracle(n, steps):
    from oracle import physics
    U = np.ascontiguousarray(tgv.initial(n))
    prm = physics.ns_params(tgv.GAMMA, tgv.MA, tgv.RE, tgv.PR, (tgv.h_of(n),) * 3)
    for _ in range(steps):
        physics.ns_step(U, tgv.dt_of(n), prm)
    return U


@pytest.mark.parametrize("spc,fused,n", [(1, False, 24), (2, False, 24), (1, True, 24), (2, False, 16)])
def test_tgv_fp64_tiled_untiled_oracle(oracle_lib, spc, fused, n):
    """(n = 16 with two steps per chain: the 24 ghost rows are deeper than the extent,
    so a ghost row takes an interior row more than one period away.)"""
    chains = 2
    fp = footprint(tgv.datasets(n, spc, fused=fused))
    Ui, sti = tgv_gpu(n, chains, spc, 4 * fp, fused=fused)
    Ut, stt = tgv_gpu(n, chains, spc, 4 * fp, h=7, fused=fused)
    assert sti["tiles"] == 1 and stt["tiles"] > 1
    assert np.array_equal(Ui, Ut)
    Uo = tgv_oracle(n, chains * spc)
    for m in range(5):
        assert rel_max(Ut[m], Uo[m]) <= 1e-12, tgv.CONS[m]


def test_tgv_mixed_error(oracle_lib):
    from paper_1709_02125_gb300 import oc
    n, chains, spc = 48, 2, 1
    fp = footprint(tgv.datasets(n, spc, "f32", None, True))
    Um, st = tgv_gpu(n, chains, spc, fp // 2, mixed=True,
                     flags=oc.OC_FLAG_CYCLIC | oc.OC_FLAG_PREFETCH | oc.OC_FLAG_GRAPHS)
    assert st["tiles"] > 1
    Uo = tgv_oracle(n, chains * spc)
    errs = {tgv.CONS[m]: rel_l2(Um[m], Uo[m]) for m in (0, 1, 2, 4)}
    print("mixed TGV, relative L2 error per conserved field:",
          " ".join(f"{k}={v:.2e}" for k, v in errs.items()),
          f"{tgv.CONS[3]} abs/max|{tgv.CONS[1]}| = {np.max(np.abs(Um[3] - Uo[3])) / np.max(np.abs(Uo[1])):.2e}")
    for m in (0, 1, 2, 4):   # w stays zero: its relative error is undefined
        assert errs[tgv.CONS[m]] <= 1e-5, tgv.CONS[m]
    assert np.max(np.abs(Um[3] - Uo[3])) <= 1e-5 * np.max(np.abs(Uo[1]))
