"""GPU parity of the out-of-core executor against the oracle (through the C ABI).

Bars: tiled and untiled FP64 runs are bit-identical (same kernels, same per-row
reduction partials); FP64 against the oracle within 1e-12 normwise relative max per
field (the kernels evaluate the documented order without contraction, so most fields
match exactly); sums within 1e-12 of sum |v|; FP32-stored runs within 1e-5 relative L2.
"""
import math

import numpy as np
import pytest

from workloads import heat, random_chain
from workloads.spec import READ, REDUCE, WRITE, Arg, DatSpec, Loop, RedSpec

from gpu_helpers import rel_l2, rel_max, run_gpu, run_oracle

pytestmark = pytest.mark.gpu

MiB = 1 << 20


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()


def _abs_sum(fields, loops, reds):
    """sum |v| over the range of each SUM reduction (bounds its rounding error)."""
    out = {}
    for lp in loops:
        if lp.kernel == "reduce":
            src = fields[lp.args[0].name]
            r = [a.name for a in lp.args if a.access == "red"][0]
            out[r] = float(np.abs(src).sum())
    return out


def test_heat_tiled_bit_exact_and_eigenmode(oracle_lib):
    dats, reds, loops = heat.build(256, 10, kind="eigen")
    inc, rin, _ = run_gpu(dats, reds, loops, 64 * MiB)
    til, rti, st = run_gpu(dats, reds, loops, MiB, h=64, depth=3)
    assert st["tiles"] == 4
    assert np.array_equal(inc["u"], til["u"])
    assert rin == rti
    ref, rref = run_oracle(oracle_lib, dats, reds, loops)
    assert rel_max(til["u"], ref["u"]) <= 1e-12
    g = 1.0 - 0.8 * math.sin(math.pi / 514) ** 2
    for s in range(10):
        expect = g ** (s + 1) * math.cos(math.pi / 514) ** 2
        assert abs(rti[0][f"max{s}"] - expect) <= 1e-13 * expect
        assert abs(rti[0][f"max{s}"] - rref[0][f"max{s}"]) <= 1e-12 * expect


def test_heat_random_four_tiles(oracle_lib):
    dats, reds, loops = heat.build(256, 10, kind="random")
    til, rti, st = run_gpu(dats, reds, loops, MiB, h=64, depth=3)
    ref, rref = run_oracle(oracle_lib, dats, reds, loops)
    assert st["tiles"] == 4 and st["h2d_bytes"] > 0
    assert rel_max(til["u"], ref["u"]) <= 1e-12
    for k, v in rref[0].items():
        assert abs(rti[0][k] - v) <= 1e-12 * abs(v)


@pytest.mark.parametrize("h,depth", [(0, 0), (1, 3), (13, 2), (29, 3), (41, 4)])
def test_random_chain_tiled_vs_untiled_vs_oracle(oracle_lib, h, depth):
    n = 300  # ragged against the 128-thread x blocks and the 4-row groups
    dats, reds, loops = random_chain.build(n=n, nfields=12, nloops=24, seed=31)
    fp = random_chain.footprint_bytes(n, 12)
    inc, rin, sti = run_gpu(dats, reds, loops, 4 * fp)
    assert sti["tiles"] == 1
    til, rti, st = run_gpu(dats, reds, loops, fp // 3 if h == 0 else 4 * fp // 5, h=h, depth=depth)
    assert st["tiles"] > 1
    for d in dats:
        assert np.array_equal(inc[d.name], til[d.name]), d.name
    assert rin == rti
    ref, rref = run_oracle(oracle_lib, dats, reds, loops)
    bounds = _abs_sum(ref, loops, reds)
    for d in dats:
        assert rel_max(til[d.name], ref[d.name]) <= 1e-12, d.name
    for k, v in rref[0].items():
        assert abs(rti[0][k] - v) <= 1e-12 * bounds[k]


def test_random_chain_repeated_with_prefetch_graphs_cyclic(oracle_lib):
    """Sec. 4.1 options on a repeated chain: results equal the plain pipeline's."""
    from paper_1709_02125_gb300 import oc
    n = 257
    dats, reds, loops = random_chain.build(n=n, nfields=10, nloops=20, seed=7)
    fp = random_chain.footprint_bytes(n, 10)
    base, rb, _ = run_gpu(dats, reds, loops, fp // 3, chains=3)
    flags = oc.OC_FLAG_PREFETCH | oc.OC_FLAG_GRAPHS | oc.OC_FLAG_CYCLIC
    opt, ro, st = run_gpu(dats, reds, loops, fp // 3, chains=3, flags=flags)
    assert st["graph_replays"] == st["tiles"]
    assert st["prefetched_bytes"] > 0
    # with the cyclic option, datasets first written in the chain are per-chain
    # temporaries whose host copies are deliberately not refreshed (Sec. 4.1)
    temps = _write_first(loops)
    assert temps
    for d in dats:
        if d.name not in temps:
            assert np.array_equal(base[d.name], opt[d.name]), d.name
    assert rb == ro
    ref, rref = run_oracle(oracle_lib, dats, reds, loops, chains=3)
    for d in dats:
        assert rel_max(base[d.name], ref[d.name]) <= 1e-12, d.name
        if d.name not in temps:
            assert rel_max(opt[d.name], ref[d.name]) <= 1e-12, d.name


def _write_first(loops):
    first = {}
    for lp in loops:
        for a in lp.args:
            if a.access == "r":
                first.setdefault(a.name, "r")
        for a in lp.args:
            if a.access == "w":
                first.setdefault(a.name, "w")
    return {k for k, v in first.items() if v == "w"}


def test_random_chain_fp32_storage_error(oracle_lib):
    n = 200
    dats, reds, loops = random_chain.build(n=n, nfields=10, nloops=24, seed=11)
    d32 = [DatSpec(d.name, d.size, d.halo_lo, d.halo_hi, "f32", init=d.init.astype(np.float32)) for d in dats]
    fp = random_chain.footprint_bytes(n, 10, 4)
    g32, r32, st = run_gpu(d32, reds, loops, fp // 3)
    assert st["tiles"] > 1
    ref, rref = run_oracle(oracle_lib, dats, reds, loops)
    errs = {d.name: rel_l2(g32[d.name], ref[d.name]) for d in dats}
    print("FP32-storage random chain, relative L2 error per field:",
          " ".join(f"{k}={v:.2e}" for k, v in errs.items()))
    for d in dats:
        assert errs[d.name] <= 1e-5, d.name


def test_random_3d_chain(oracle_lib):
    rng = np.random.default_rng(3)
    n, nz, F = 37, 45, 6
    dats = [DatSpec(f"g{f}", (n, n - 3, nz), (1, 1, 2), (1, 1, 2),
                    init=rng.uniform(-1, 1, size=(nz + 4, n - 1, n + 2))) for f in range(F)]
    loops = []
    for i in range(12):
        w = i % F
        ins = [(w + 1 + j) % F for j in range(1 + i % 3)]
        args = [Arg(f"g{w}", WRITE)]
        for f in ins:
            args.append(Arg(f"g{f}", READ, [(1, 0, -2), (0, -1, 1), (-1, 1, 0)][: 1 + (f + i) % 3]))
        m = sum(len(a.offsets) for a in args[1:])
        c = rng.uniform(-1, 1, size=m)
        c *= 0.5 / np.abs(c).sum()
        loops.append(Loop("lincomb", (0, 0, 0), (n, n - 3, nz), args, [0.5] + list(c)))
    reds = [RedSpec("s", "sum"), RedSpec("m", "max")]
    loops.append(Loop("reduce", (0, 0, 0), (n, n - 3, nz), [Arg("g1", READ), Arg("s", REDUCE)], [0.0]))
    loops.append(Loop("reduce", (0, 0, 0), (n, n - 3, nz), [Arg("g2", READ), Arg("m", REDUCE)], [1.0]))
    fp = sum(8 * np.prod(d.shape) for d in dats)
    inc, rin, _ = run_gpu(dats, reds, loops, 8 * fp)
    til, rti, st = run_gpu(dats, reds, loops, 8 * fp, h=6, depth=3)
    assert st["tiles"] == 8
    for d in dats:
        assert np.array_equal(inc[d.name], til[d.name])
    assert rin == rti
    ref, rref = run_oracle(oracle_lib, dats, reds, loops)
    for d in dats:
        assert rel_max(til[d.name], ref[d.name]) <= 1e-12
    assert rti[0]["m"] == rref[0]["m"]


def test_edge_cases(oracle_lib):
    """Empty loop ranges, single-row loops, empty reductions and one-row tiles."""
    n = 64
    rng = np.random.default_rng(9)
    dats = [DatSpec(f"e{f}", (n, n), (2, 2), (2, 2), init=rng.uniform(-1, 1, size=(n + 4, n + 4))) for f in range(3)]
    reds = [RedSpec("se", "sum"), RedSpec("me", "max"), RedSpec("s1", "sum")]
    loops = [Loop("copy", (0, 10), (n, 10), [Arg("e0", WRITE), Arg("e1", READ, [(0, 1)])]),
             Loop("lincomb", (3, 20), (n - 5, 21), [Arg("e0", WRITE), Arg("e1", READ, [(1, 2), (-2, -1)])],
                  [0.5, 0.25, -0.25]),
             Loop("reduce", (0, 5), (n, 5), [Arg("e2", READ), Arg("se", REDUCE)], [0.0]),
             Loop("reduce", (0, 0), (0, n), [Arg("e2", READ), Arg("me", REDUCE)], [0.0]),
             Loop("copy", (0, -2), (n, n + 2), [Arg("e2", WRITE), Arg("e0", READ)]),
             Loop("reduce", (0, n - 1), (n, n), [Arg("e2", READ), Arg("s1", REDUCE)], [2.0])]
    fp = 3 * (n + 4) * (n + 4) * 8
    for h, depth in ((1, 3), (1, 2), (7, 4), (0, 0)):
        got, rg, st = run_gpu(dats, reds, loops, 4 * fp if h == 0 else 16 * fp, h=h, depth=depth)
        ref, rr = run_oracle(oracle_lib, dats, reds, loops)
        for d in dats:
            assert np.array_equal(got[d.name], ref[d.name]), (d.name, h)
        assert rg[0]["se"] == 0.0 and rg[0]["me"] == -math.inf
        assert abs(rg[0]["s1"] - rr[0]["s1"]) <= 1e-13 * abs(rr[0]["s1"])


@pytest.mark.slow
def test_full_size_random_chain_at_one_third_budget(oracle_lib):
    """The benchmarked workload: 24 fields of 4096^2 FP64 (halo 2), 40 loops + 2 sums,
    budget 1/3 of the footprint, prefetch + graphs; two chains."""
    from paper_1709_02125_gb300 import oc
    dats, reds, loops = random_chain.build()
    fp = random_chain.footprint_bytes()
    flags = oc.OC_FLAG_PREFETCH | oc.OC_FLAG_GRAPHS
    got, rg, st = run_gpu(dats, reds, loops, fp // 3, chains=2, flags=flags)
    assert st["tiles"] >= 3
    ref, rr = run_oracle(oracle_lib, dats, reds, loops, chains=2)
    bounds = _abs_sum(ref, loops, reds)
    for d in dats:
        assert rel_max(got[d.name], ref[d.name]) <= 1e-12, d.name
    for c in range(2):
        for k, v in rr[c].items():
            assert abs(rg[c][k] - v) <= 1e-12 * bounds[k]


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_lincomb_many_samples(oracle_lib, dtype):
    """LINCOMB with more samples than the unrolled kernels take (25 and 64 samples run
    through the generic kernel), tiled and untiled."""
    n = 96
    rng = np.random.default_rng(21)
    F = 6
    dats = [DatSpec(f"m{f}", (n, n), (2, 2), (2, 2), init=rng.uniform(-1, 1, size=(n + 4, n + 4))) for f in range(F)]
    offs25 = [(dx, dy) for dy in range(-2, 3) for dx in range(-2, 3)]
    c = rng.uniform(-1, 1, size=64)
    loops = [Loop("lincomb", (0, 0), (n, n), [Arg("m0", WRITE), Arg("m1", READ, offs25)],
                  [0.5] + list(c[:25] * 0.5 / np.abs(c[:25]).sum())),
             Loop("lincomb", (0, 0), (n, n), [Arg("m2", WRITE)] + [Arg(f"m{f}", READ, offs25[:16]) for f in (0, 1, 3, 4)],
                  [0.5] + list(c * 0.5 / np.abs(c).sum()))]
    reds = []
    if dtype == "f32":
        dats = [DatSpec(d.name, d.size, d.halo_lo, d.halo_hi, "f32", init=d.init.astype(np.float32)) for d in dats]
    fp = F * (n + 4) * (n + 4) * (8 if dtype == "f64" else 4)
    inc, _, st_i = run_gpu(dats, reds, loops, 4 * fp)
    til, _, st_t = run_gpu(dats, reds, loops, 16 * fp, h=9, depth=3)
    assert st_i["tiles"] == 1 and st_t["tiles"] > 1
    for d in dats:
        assert np.array_equal(inc[d.name], til[d.name]), d.name
    if dtype == "f64":
        ref, _ = run_oracle(oracle_lib, dats, reds, loops)
        for d in dats:
            assert rel_max(til[d.name], ref[d.name]) <= 1e-12, d.name
