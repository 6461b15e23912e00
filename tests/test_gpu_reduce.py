"""REDUCE over FP32 data (per-row partials, Sec. 3's reductions): every op and mode,
one and two sources, against values the mathematics fixes -- sums against the exactly
rounded sum of the exact terms (math.fsum over the FP64 images: v, |v| and v * v of an
FP32 v are exact in FP64), extremes exactly -- with data spread over 2^-20..2^20 and
mixed signs so that the sums cancel heavily. The FP32 form accumulates each thread's
terms as a compensated FP32 pair; the bound 1e-12 * sum |terms| is three orders above
its error and far below an uncompensated FP32 sum's. Tiled and untiled runs give the
same bits."""
import math

import numpy as np
import pytest

from workloads.spec import READ, REDUCE, Arg, DatSpec, Loop, RedSpec

from gpu_helpers import run_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()


def _data(rng, shape):
    v = rng.uniform(-1.0, 1.0, size=shape) * np.exp2(rng.integers(-20, 21, size=shape))
    return v.astype(np.float32)


CASES = [("sum", 0), ("sum", 1), ("sum", 2), ("max", 0), ("max", 1), ("max", 2),
         ("min", 0), ("min", 1), ("min", 2)]


def _terms(v, mode):
    v = np.asarray(v, dtype=np.float64)
    return v if mode == 0 else (np.abs(v) if mode == 1 else v * v)


def _expect(op, terms):
    if op == "sum":
        return math.fsum(terms.ravel().tolist())
    return float(terms.max() if op == "max" else terms.min())


def _check(op, got, terms):
    want = _expect(op, terms)
    if op == "sum":
        assert abs(got - want) <= 1e-12 * float(np.abs(terms).sum()), (got, want)
    else:
        assert got == want, (got, want)


@pytest.mark.parametrize("shape,halo", [((300, 257), (1, 2)), ((5000, 9), (2, 1)), ((37, 41, 23), (1, 1, 2))])
def test_fp32_reduce_every_op_and_mode(shape, halo):
    rng = np.random.default_rng(sum(shape))
    nd = len(shape)
    lo = halo
    hi = tuple(reversed(halo)) if nd == 2 else halo
    ext = tuple(n + a + b for n, a, b in zip(shape, lo, hi))
    init = _data(rng, tuple(reversed(ext)))
    dats = [DatSpec("u", shape, lo, hi, "f32", init=init)]
    reds, loops = [], []
    for k, (op, mode) in enumerate(CASES):
        reds.append(RedSpec(f"r{k}", op))
        loops.append(Loop("reduce", (0,) * nd, shape, [Arg("u", READ), Arg(f"r{k}", REDUCE)], [float(mode)]))
    fp = init.nbytes
    _, r_in, st_in = run_gpu(dats, reds, loops, 4 * fp)
    slow = shape[-1]
    _, r_t, st_t = run_gpu(dats, reds, loops, 4 * fp, h=max(1, slow // 5), depth=3)
    assert st_in["tiles"] == 1 and st_t["tiles"] > 1
    assert r_in == r_t
    interior = init[tuple(slice(h, h + n) for h, n in zip(reversed(lo), reversed(shape)))]
    for k, (op, mode) in enumerate(CASES):
        _check(op, r_in[0][f"r{k}"], _terms(interior, mode))


def test_fp32_two_source_reductions():
    """hi + lo sources: the plain sum takes the FP32 form (both sources term by term);
    |hi + lo| and extremes take the FP64 form (hi + lo is exact in FP64)."""
    rng = np.random.default_rng(77)
    n = 211
    hi_ = _data(rng, (n + 2, n + 2))
    lo_ = (hi_ * np.float32(2.0 ** -24) * rng.uniform(-1, 1, size=hi_.shape).astype(np.float32)).astype(np.float32)
    dats = [DatSpec("h", (n, n), (1, 1), (1, 1), "f32", init=hi_), DatSpec("l", (n, n), (1, 1), (1, 1), "f32", init=lo_)]
    cases = [("sum", 0), ("sum", 1), ("max", 1), ("min", 0)]
    reds = [RedSpec(f"r{k}", op) for k, (op, _) in enumerate(cases)]
    loops = [Loop("reduce", (0, 0), (n, n), [Arg("h", READ), Arg("l", READ), Arg(f"r{k}", REDUCE)], [float(m)])
             for k, (_, m) in enumerate(cases)]
    fp = hi_.nbytes * 2
    _, r_in, _ = run_gpu(dats, reds, loops, 4 * fp)
    _, r_t, st_t = run_gpu(dats, reds, loops, 4 * fp, h=40, depth=3)
    assert st_t["tiles"] > 1 and r_in == r_t
    v = hi_[1:-1, 1:-1].astype(np.float64) + lo_[1:-1, 1:-1].astype(np.float64)
    for k, (op, mode) in enumerate(cases):
        if op == "sum" and mode == 0:
            terms = np.concatenate([hi_[1:-1, 1:-1].ravel(), lo_[1:-1, 1:-1].ravel()]).astype(np.float64)
            _check(op, r_in[0][f"r{k}"], terms)
        else:
            _check(op, r_in[0][f"r{k}"], _terms(v, mode))


def test_fp32_sums_beyond_fp32_range():
    """Squares of values near 2^66 and sums of values near 3e38 overflow FP32 but not
    FP64: the blocks whose FP32 pair leaves the range fold again in FP64, so the results
    are the FP64 form's (finite, within the same bound)."""
    rng = np.random.default_rng(5)
    n = 130
    big = (rng.uniform(0.5, 1.0, size=(n + 2, n + 2)) * 2.0 ** 66).astype(np.float32)
    huge = (rng.uniform(0.5, 1.0, size=(n + 2, n + 2)) * 3.0e38).astype(np.float32)
    small = _data(rng, (n + 2, n + 2))
    dats = [DatSpec(nm, (n, n), (1, 1), (1, 1), "f32", init=v) for nm, v in (("b", big), ("g", huge), ("s", small))]
    cases = [("b", "sum", 2), ("b", "max", 2), ("g", "sum", 0), ("s", "sum", 2)]
    reds = [RedSpec(f"r{k}", op) for k, (_, op, _) in enumerate(cases)]
    loops = [Loop("reduce", (0, 0), (n, n), [Arg(nm, READ), Arg(f"r{k}", REDUCE)], [float(m)])
             for k, (nm, _, m) in enumerate(cases)]
    fp = 3 * big.nbytes
    _, r_in, _ = run_gpu(dats, reds, loops, 4 * fp)
    _, r_t, st_t = run_gpu(dats, reds, loops, 4 * fp, h=30, depth=3)
    assert st_t["tiles"] > 1 and r_in == r_t
    src = {"b": big, "g": huge, "s": small}
    for k, (nm, op, mode) in enumerate(cases):
        got = r_in[0][f"r{k}"]
        assert np.isfinite(got)
        _check(op, got, _terms(src[nm][1:-1, 1:-1], mode))
