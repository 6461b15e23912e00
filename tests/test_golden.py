"""Stored expected values (tests/golden/, written by make_golden.py from the oracle).

CPU: the oracle still reproduces them (regression pin of its arithmetic).
GPU: the FP64 CUDA path, untiled and tiled, matches them within the 1e-12 bar; for the
PDE workloads (Euler 24^2, Taylor-Green 12^3) per conserved field, normwise."""
import os

import numpy as np
import pytest

from workloads import heat, random_chain

HERE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
TINY = dict(n=8, nfields=6, nloops=6, nred=2, seed=4242)


def _heat_golden():
    return [float(ln) for ln in open(os.path.join(HERE, "heat256_u01_maxnorms.txt")) if not ln.startswith("#")]


def _tiny_golden():
    sums, arrs = None, {}
    for ln in open(os.path.join(HERE, "random8_chain.txt")):
        if ln.startswith("#"):
            continue
        f = ln.split()
        if f[0] == "sums":
            sums = [float(v) for v in f[1:]]
        else:
            arrs[f[0]] = np.array([float(v) for v in f[3:]]).reshape(int(f[1]), int(f[2]))
    return sums, arrs


def _vec_golden(fname):
    out = {}
    for ln in open(os.path.join(HERE, fname)):
        if not ln.startswith("#"):
            f = ln.split()
            out[f[0]] = np.array([float(v) for v in f[1:]])
    return out


def _euler_golden():
    g = _vec_golden("euler24_3steps.txt")
    return list(g["dts"]), g["U"].reshape(4, 24, 24)


def _tgv_golden():
    return _vec_golden("tgv12_2steps.txt")["U"].reshape(5, 12, 12, 12)


def test_oracle_reproduces_euler_golden(oracle_lib):
    from oracle import physics
    from workloads import euler
    n = 24
    U = euler.initial(n)
    dts = []
    for _ in range(3):
        dt = euler.CFL * physics.euler_dt_min(U, 1.0 / n, 1.0 / n, euler.GAMMA)
        dts.append(dt)
        physics.euler_step(U, dt, 1.0 / n, 1.0 / n, euler.GAMMA, euler.EPS4)
    want_dts, want_U = _euler_golden()
    np.testing.assert_allclose(dts, want_dts, rtol=1e-15, atol=0)
    np.testing.assert_allclose(U, want_U, rtol=0, atol=1e-14)


def test_oracle_reproduces_tgv_golden(oracle_lib):
    from oracle import physics
    from workloads import tgv
    n = 12
    U = np.ascontiguousarray(tgv.initial(n))
    prm = physics.ns_params(tgv.GAMMA, tgv.MA, tgv.RE, tgv.PR, (tgv.h_of(n),) * 3)
    for _ in range(2):
        physics.ns_step(U, tgv.dt_of(n), prm)
    np.testing.assert_allclose(U, _tgv_golden(), rtol=0, atol=1e-14)


def test_oracle_reproduces_heat_golden(oracle_lib):
    dats, reds, loops = heat.build(n=256, steps=10)
    fields = oracle_lib.make_fields(dats)
    out = oracle_lib.run_chain(loops, fields, reds)
    got = [out[r.name] for r in reds]
    want = _heat_golden()
    assert len(want) == 10
    np.testing.assert_allclose(got, want, rtol=1e-15, atol=0)


def test_oracle_reproduces_random_golden(oracle_lib):
    dats, reds, loops = random_chain.build(**TINY)
    fields = oracle_lib.make_fields(dats)
    out = oracle_lib.run_chain(loops, fields, reds)
    sums, arrs = _tiny_golden()
    np.testing.assert_allclose([out[r.name] for r in reds], sums, rtol=1e-14, atol=0)
    for d in dats:
        np.testing.assert_allclose(fields[d.name].a, arrs[d.name], rtol=0, atol=1e-15)


@pytest.mark.gpu
@pytest.mark.parametrize("h", [0, 3])
def test_gpu_matches_random_golden(h):
    import __graft_entry__
    __graft_entry__.build()
    from gpu_helpers import run_gpu
    dats, reds, loops = random_chain.build(**TINY)
    budget = 4 * random_chain.footprint_bytes(TINY["n"], TINY["nfields"], 8)
    out, per_chain, st = run_gpu(dats, reds, loops, budget, h=h, depth=3 if h else 0)
    assert (st["tiles"] > 1) == (h > 0)
    sums, arrs = _tiny_golden()
    for k, r in enumerate(reds):
        assert abs(per_chain[0][r.name] - sums[k]) <= 1e-12 * max(1.0, abs(sums[k]))
    for d in dats:
        den = max(1.0, float(np.max(np.abs(arrs[d.name]))))
        assert float(np.max(np.abs(out[d.name] - arrs[d.name]))) <= 1e-12 * den, d.name


@pytest.mark.gpu
def test_gpu_matches_heat_golden():
    import __graft_entry__
    __graft_entry__.build()
    from gpu_helpers import run_gpu
    dats, reds, loops = heat.build(n=256, steps=10)
    out, per_chain, st = run_gpu(dats, reds, loops, 1 << 20, h=64, depth=3)
    assert st["tiles"] == 4
    want = _heat_golden()
    got = [per_chain[0][r.name] for r in reds]
    np.testing.assert_allclose(got, want, rtol=1e-12, atol=0)


def _rel_max(a, b):
    return float(np.max(np.abs(a - b))) / max(1e-300, float(np.max(np.abs(b))))


@pytest.mark.gpu
@pytest.mark.parametrize("h", [0, 5])
def test_gpu_matches_euler_golden(h):
    import __graft_entry__
    __graft_entry__.build()
    from test_gpu_physics import euler_gpu, footprint
    from workloads import euler
    n = 24
    U, dts, st, _ = euler_gpu(n, 3, 2 * footprint(euler.datasets(n)), h=h)
    assert (st["tiles"] > 1) == (h > 0)
    want_dts, want_U = _euler_golden()
    np.testing.assert_allclose(dts, want_dts, rtol=1e-12, atol=0)
    for k in range(4):
        assert _rel_max(U[k], want_U[k]) <= 1e-12, k


@pytest.mark.gpu
@pytest.mark.parametrize("h", [0, 5])
def test_gpu_matches_tgv_golden(h):
    import __graft_entry__
    __graft_entry__.build()
    from test_gpu_physics import footprint, tgv_gpu
    from workloads import tgv
    n = 12
    U, st = tgv_gpu(n, 2, 1, 4 * footprint(tgv.datasets(n, 1)), h=h)
    assert (st["tiles"] > 1) == (h > 0)
    want = _tgv_golden()
    for m in range(5):
        if np.max(np.abs(want[m])) > 0:
            assert _rel_max(U[m], want[m]) <= 1e-12, tgv.CONS[m]
        else:
            assert np.max(np.abs(U[m])) <= 1e-12 * np.max(np.abs(want[1])), tgv.CONS[m]
