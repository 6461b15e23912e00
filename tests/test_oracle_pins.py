"""Pins of the oracle against facts that do not come from the oracle itself.

Each test fixes the oracle's loop semantics (arXiv 1709.02125, Sec. 3: pointwise
kernels over an iteration range, reading through stencil offsets, loops in program
order) against a closed form, an invariant, or a library routine, chosen so that a
dropped term, a wrong sign or index, or a transposed axis fails at least one of them.
"""
import math

import numpy as np
import pytest

from workloads import heat
from workloads.spec import READ, REDUCE, WRITE, Arg, DatSpec, Loop, RedSpec


def _run(oracle, dats, reds, loops):
    fields = oracle.make_fields(dats)
    out = oracle.run_chain(loops, fields, reds)
    return fields, out


@pytest.mark.parametrize("nx,ny,p,q", [(48, 40, 2, 3), (33, 57, 1, 4)])
def test_heat_eigenmode_closed_form(oracle_lib, nx, ny, p, q):
    """Discrete eigenmode sin(p*pi*(x+1)/(nx+1)) sin(q*pi*(y+1)/(ny+1)) of the 5-point
    Laplacian with zero boundary decays by exactly g = 1 + 0.2(cos(p pi/(nx+1)) - 1)
    + 0.2(cos(q pi/(ny+1)) - 1) per step (rectangular grid and p != q, so a transposed
    axis or a wrong neighbour breaks it)."""
    sx = np.sin(p * np.pi * np.arange(1, nx + 1) / (nx + 1))
    sy = np.sin(q * np.pi * np.arange(1, ny + 1) / (ny + 1))
    u0 = np.zeros((ny + 2, nx + 2))
    u0[1:-1, 1:-1] = np.outer(sy, sx)
    steps = 10
    dats = [DatSpec("u", (nx, ny), (1, 1), (1, 1), init=u0),
            DatSpec("u_new", (nx, ny), (1, 1), (1, 1))]
    reds = [RedSpec(f"m{s}", "max") for s in range(steps)]
    loops = []
    for s in range(steps):
        loops += [Loop("lincomb", (0, 0), (nx, ny), [Arg("u_new", WRITE), Arg("u", READ, heat.STENCIL5)],
                       [0.0, 0.6, 0.1, 0.1, 0.1, 0.1]),
                  Loop("copy", (0, 0), (nx, ny), [Arg("u", WRITE), Arg("u_new", READ)]),
                  Loop("reduce", (0, 0), (nx, ny), [Arg("u", READ), Arg(f"m{s}", REDUCE)], [1.0])]
    fields, out = _run(oracle_lib, dats, reds, loops)
    g = 1.0 + 0.2 * (math.cos(p * math.pi / (nx + 1)) - 1.0) + 0.2 * (math.cos(q * math.pi / (ny + 1)) - 1.0)
    expect = g ** steps * u0
    got = fields["u"].a
    assert np.max(np.abs(got - expect)) <= 1e-13 * np.max(np.abs(expect))
    peak = np.max(np.abs(u0))
    for s in range(steps):
        assert abs(out[f"m{s}"] - g ** (s + 1) * peak) <= 1e-13 * peak


def test_heat_square_eigenmode_max_norm(oracle_lib):
    """The workload's own eigenmode case: max-norm after step k is
    g^k cos^2(pi/514), g = 1 - 0.8 sin^2(pi/514) (256^2 interior)."""
    dats, reds, loops = heat.build(256, 10, kind="eigen")
    _, out = _run(oracle_lib, dats, reds, loops)
    g = 1.0 - 0.8 * math.sin(math.pi / 514) ** 2
    for s in range(10):
        expect = g ** (s + 1) * math.cos(math.pi / 514) ** 2
        assert abs(out[f"max{s}"] - expect) <= 1e-13 * expect


def test_heat_maximum_principle(oracle_lib):
    """0.6 >= 0: each step is a convex combination of u and the zero boundary, so
    values stay in [0, 1] and the max-norm never increases."""
    dats, reds, loops = heat.build(64, 10, kind="random")
    fields, out = _run(oracle_lib, dats, reds, loops)
    u = fields["u"].a
    assert u.min() >= 0.0 and u.max() <= 1.0
    m = [out[f"max{s}"] for s in range(10)]
    assert all(b <= a for a, b in zip(m, m[1:]))
    assert np.all(u[0, :] == 0) and np.all(u[-1, :] == 0) and np.all(u[:, 0] == 0)


def test_lincomb_impulse_response(oracle_lib):
    """A delta input at q gives out(q - o_m) = c_m for every sample m of that input:
    pins the coefficient order, the offset signs and the axis order."""
    n = 16
    rng = np.random.default_rng(5)
    offs1 = [(1, 0), (-2, 1), (0, 2), (2, -1)]
    offs2 = [(0, -2), (1, 1)]
    c = rng.uniform(-1, 1, size=6)
    a = np.zeros((n + 4, n + 4))
    b = np.zeros((n + 4, n + 4))
    q1, q2 = (5, 7), (11, 3)       # (x, y)
    a[q1[1] + 2, q1[0] + 2] = 1.0
    b[q2[1] + 2, q2[0] + 2] = 1.0
    dats = [DatSpec("a", (n, n), (2, 2), (2, 2), init=a), DatSpec("b", (n, n), (2, 2), (2, 2), init=b),
            DatSpec("o", (n, n), (2, 2), (2, 2))]
    loops = [Loop("lincomb", (0, 0), (n, n), [Arg("o", WRITE), Arg("a", READ, offs1), Arg("b", READ, offs2)],
                  [0.0] + list(c))]
    fields, _ = _run(oracle_lib, dats, [], loops)
    o = fields["o"].a
    expect = np.zeros_like(o)
    for m, off in enumerate(offs1):
        expect[q1[1] - off[1] + 2, q1[0] - off[0] + 2] += c[m]
    for m, off in enumerate(offs2):
        expect[q2[1] - off[1] + 2, q2[0] - off[0] + 2] += c[4 + m]
    assert np.array_equal(o, expect)


@pytest.mark.parametrize("vals,npts", [((2.0, 3.0, 0.5), (1, 1, 1)), ((-1.5,), (1,)), ((0.75, -2.0), (1, 1))])
def test_lincomb_nonlinear_term_constant_fields(oracle_lib, vals, npts):
    """On constant fields the nonlinear term reduces to alpha*a*b/(1+c^2) with
    a = x0, b = x_{1 mod M}, c = x_{2 mod M}; this pins which samples it takes."""
    n = 8
    dats, args = [DatSpec("o", (n, n), (2, 2), (2, 2))], [Arg("o", WRITE)]
    for j, v in enumerate(vals):
        dats.append(DatSpec(f"i{j}", (n, n), (2, 2), (2, 2), init=np.full((n + 4, n + 4), v)))
        args.append(Arg(f"i{j}", READ, [(1, -1)]))
    c = [0.25, -0.125, 0.0625][: len(vals)]
    alpha = 0.5
    fields, _ = _run(oracle_lib, dats, [], [Loop("lincomb", (0, 0), (n, n), args, [alpha] + c)])
    M = len(vals)
    lin = sum(ci * vi for ci, vi in zip(c, vals))
    a, b, cc = vals[0], vals[1 % M], vals[2 % M]
    expect = lin + alpha * a * b / (1 + cc * cc)
    inner = fields["o"].a[2:-2, 2:-2]
    assert np.allclose(inner, expect, rtol=1e-15, atol=0)
    assert np.all(fields["o"].a[:2, :] == 0)  # halo untouched


def test_copy_shift_matches_slicing(oracle_lib):
    n = 12
    src = np.random.default_rng(1).uniform(size=(n + 4, n + 6))
    dats = [DatSpec("s", (n + 2, n), (2, 2), (2, 2), init=src), DatSpec("d", (n + 2, n), (2, 2), (2, 2))]
    loops = [Loop("copy", (1, 0), (n + 1, n - 1), [Arg("d", WRITE), Arg("s", READ, [(-2, 1)])])]
    fields, _ = _run(oracle_lib, dats, [], loops)
    expect = np.zeros_like(src)
    # d[y, x] = s[y + 1, x - 2] for x in [1, n+1), y in [0, n-1); +2 for the halo
    expect[2:n + 1, 3:n + 3] = src[3:n + 2, 1:n + 1]
    assert np.array_equal(fields["d"].a, expect)


def test_3d_geometry_matches_slicing(oracle_lib):
    """3-D datasets whose axes differ in length and in halo depth, each side: a shifted
    copy and a two-sample LINCOMB equal numpy slicing of the dense arrays (pins the
    index map of every axis against a library routine)."""
    size, hlo, hhi = (7, 5, 4), (2, 1, 3), (1, 3, 2)
    shape = tuple(size[a] + hlo[a] + hhi[a] for a in (2, 1, 0))
    rng = np.random.default_rng(11)
    a0, b0 = rng.uniform(-1, 1, size=shape), rng.uniform(-1, 1, size=shape)
    dats = [DatSpec(nm, size, hlo, hhi, init=v) for nm, v in (("a", a0), ("b", b0))]
    dats += [DatSpec("c", size, hlo, hhi), DatSpec("d", size, hlo, hhi)]
    oa, ob = (-2, 1, 2), (1, -1, -2)
    lo, hi = (0, 0, 0), size
    c0, c1 = 0.375, -1.25
    loops = [Loop("copy", lo, hi, [Arg("c", WRITE), Arg("a", READ, [oa])]),
             Loop("lincomb", lo, hi, [Arg("d", WRITE), Arg("a", READ, [oa]), Arg("b", READ, [ob])],
                  [0.0, c0, c1])]
    fields, _ = _run(oracle_lib, dats, [], loops)

    def window(arr, o):
        # interior points shifted by o (x, y, z); array axes are (z, y, x)
        return arr[hlo[2] + o[2]:hlo[2] + o[2] + size[2],
                   hlo[1] + o[1]:hlo[1] + o[1] + size[1],
                   hlo[0] + o[0]:hlo[0] + o[0] + size[0]]

    ec = np.zeros(shape)
    window(ec, (0, 0, 0))[...] = window(a0, oa)
    assert np.array_equal(fields["c"].a, ec)
    ed = np.zeros(shape)
    window(ed, (0, 0, 0))[...] = c0 * window(a0, oa) + c1 * window(b0, ob)
    assert np.array_equal(fields["d"].a, ed)


def test_chain_program_order(oracle_lib):
    """Two loops that each shift by one point compose to a shift by two (a later loop
    sees the earlier loop's writes)."""
    n = 10
    a0 = np.random.default_rng(2).uniform(size=(n + 4, n + 4))
    dats = [DatSpec("a", (n, n), (2, 2), (2, 2), init=a0), DatSpec("b", (n, n), (2, 2), (2, 2))]
    loops = [Loop("copy", (0, 0), (n, n), [Arg("b", WRITE), Arg("a", READ, [(0, 1)])]),
             Loop("copy", (0, 0), (n - 1, n - 1), [Arg("a", WRITE), Arg("b", READ, [(1, 0)])])]
    fields, _ = _run(oracle_lib, dats, [], loops)
    expect = a0.copy()
    expect[2:n + 1, 2:n + 1] = a0[3:n + 2, 3:n + 2]
    assert np.array_equal(fields["a"].a, expect)


@pytest.mark.parametrize("mode", [0, 1, 2])
def test_reductions_match_library(oracle_lib, mode):
    n = 37
    rng = np.random.default_rng(3 + mode)
    x = rng.uniform(-1, 1, size=(n + 2, n + 2)) * 1e3
    y = rng.uniform(-1, 1, size=(n + 2, n + 2))
    dats = [DatSpec("x", (n, n), (1, 1), (1, 1), init=x), DatSpec("y", (n, n), (1, 1), (1, 1), init=y)]
    reds = [RedSpec("s", "sum"), RedSpec("mx", "max"), RedSpec("mn", "min"), RedSpec("s2", "sum")]
    lo, hi = (0, 0), (n - 3, n)
    loops = [Loop("reduce", lo, hi, [Arg("x", READ), Arg(r, REDUCE)], [float(mode)]) for r in ("s", "mx", "mn")]
    loops.append(Loop("reduce", lo, hi, [Arg("x", READ), Arg("y", READ), Arg("s2", REDUCE)], [float(mode)]))
    _, out = _run(oracle_lib, dats, reds, loops)
    v = x[1:n + 1, 1:n - 2]
    v2 = x[1:n + 1, 1:n - 2] + y[1:n + 1, 1:n - 2]
    f = {0: lambda t: t, 1: np.abs, 2: lambda t: t * t}[mode]
    assert out["s"] == math.fsum(f(v).ravel())
    assert out["mx"] == f(v).max() and out["mn"] == f(v).min()
    assert abs(out["s2"] - math.fsum(f(v2).ravel())) <= 4e-16 * math.fsum(np.abs(f(v2)).ravel())


def test_out_of_extent_access_rejected(oracle_lib):
    n = 8
    dats = [DatSpec("a", (n, n), (1, 1), (1, 1)), DatSpec("b", (n, n), (1, 1), (1, 1))]
    with pytest.raises(IndexError):
        _run(oracle_lib, dats, [], [Loop("copy", (0, 0), (n, n), [Arg("b", WRITE), Arg("a", READ, [(2, 0)])])])


@pytest.mark.parametrize("nin,per", [(5, 13), (4, 25)])
def test_lincomb_more_than_64_samples(oracle_lib, nin, per):
    """65 and 100 samples (more than any fixed per-point buffer of 64): on constant fields
    v_j the loop gives sum_m c_m v_j(m) + alpha*a*b/(1+c^2) with a, b, c the first three
    samples (all of input 0 here), and leaves the halo alone."""
    n = 6
    offs = [(dx, dy) for dy in range(-2, 3) for dx in range(-2, 3)][:per]
    vals = [0.5 + 0.25 * j for j in range(nin)]
    dats, args = [DatSpec("o", (n, n), (2, 2), (2, 2))], [Arg("o", WRITE)]
    for j, v in enumerate(vals):
        dats.append(DatSpec(f"i{j}", (n, n), (2, 2), (2, 2), init=np.full((n + 4, n + 4), v)))
        args.append(Arg(f"i{j}", READ, offs))
    M = nin * per
    c = [((-1) ** m) / (8.0 * (m + 1)) for m in range(M)]
    alpha = 0.5
    fields, _ = _run(oracle_lib, dats, [], [Loop("lincomb", (0, 0), (n, n), args, [alpha] + c)])
    lin = math.fsum(c[m] * vals[m // per] for m in range(M))
    v0 = vals[0]
    expect = lin + alpha * v0 * v0 / (1 + v0 * v0)
    inner = fields["o"].a[2:-2, 2:-2]
    assert np.allclose(inner, expect, rtol=1e-14, atol=0)
    assert np.all(fields["o"].a[:2, :] == 0) and np.all(fields["o"].a[:, -2:] == 0)


def test_results_independent_of_thread_count(oracle_lib):
    """The loop kernels split lines over threads and reductions fold per-row partials in
    row order, so 1 and 4 threads give the same bits (a 2-D and a 3-D random chain)."""
    from workloads import random_chain
    rng = np.random.default_rng(77)
    cases = [random_chain.build(n=40, nfields=6, nloops=10, seed=5)]
    dats3, reds3, loops3 = random_chain.build_general(3, 10, 5, 8, 2, seed=9, nz=7)
    for d in dats3:
        d.init = rng.uniform(-1, 1, size=d.shape)
    cases.append((dats3, reds3, loops3))
    runs = []
    try:
        for nthreads in (1, 4):
            oracle_lib.set_threads(nthreads)
            out = []
            for dats, reds, loops in cases:
                fields, sums = _run(oracle_lib, dats, reds, loops)
                out.append(({k: v.a.copy() for k, v in fields.items()}, sums))
            runs.append(out)
    finally:
        oracle_lib.set_threads(oracle_lib.threads_default)
    for (f1, s1), (f4, s4) in zip(*runs):
        assert s1 == s4
        for k in f1:
            assert np.array_equal(f1[k], f4[k]), k
