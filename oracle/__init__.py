"""Oracle: plain, untiled FP64 CPU evaluation of stencil loop chains.

TEST INFRASTRUCTURE. Only `tests/`, `__graft_entry__.smoke()` and the CPU-baseline
leg of `bench.py` may import this package. It shares no code with the CUDA executor
(`paper_1709_02125_gb300`) and never imports it.

It implements the sequential meaning of a chain (arXiv 1709.02125, Sec. 3): loops run
one after another in program order over their whole iteration ranges, on full arrays
held in host memory; each kernel is evaluated pointwise as defined in `oracle.c`.
The PDE workloads (Euler, Navier-Stokes) have their own step functions in
`oracle.physics`, written with plain periodic (modular) indexing, and a loop-level form
of the same arithmetic in `oracle.physics_loops` (pinned to the step functions).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from typing import Dict, List

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "_build", "liboracle.so")
_SOURCES = ["oracle.c", "physics.c"]

_lib = None


def build(force: bool = False) -> str:
    """Compile oracle/*.c into oracle/_build/liboracle.so with gcc (OpenMP, no FMA)."""
    srcs = [os.path.join(_HERE, s) for s in _SOURCES if os.path.exists(os.path.join(_HERE, s))]
    if not force and os.path.exists(_SO):
        so_t = os.path.getmtime(_SO)
        if all(os.path.getmtime(s) <= so_t for s in srcs):
            return _SO
    os.makedirs(os.path.dirname(_SO), exist_ok=True)
    tmp = _SO + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
           "-fno-fast-math", "-o", tmp] + srcs + ["-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _SO)
    return _SO


def lib():
    """The loaded oracle library. ORACLE_LIB, when set, names a prebuilt library to load
    instead of oracle/_build/liboracle.so (the mutation tests point it at a copy of the
    oracle with one planted mistake, to show that the pins catch it)."""
    global _lib
    if _lib is None:
        path = os.environ.get("ORACLE_LIB") or build()
        L = ctypes.CDLL(path)
        P, I = ctypes.c_void_p, ctypes.c_int
        L.or_copy.argtypes = [P, P, P, P, P, P, P]
        L.or_lincomb.argtypes = [P, P, P, P, I, P, P, P, P, P, ctypes.c_double]
        L.or_lincomb.restype = I
        L.or_reduce.argtypes = [P, P, P, P, P, P, I, I]
        L.or_reduce.restype = ctypes.c_double
        L.or_threads.restype = I
        L.or_set_threads.argtypes = [I]
        L.or_set_threads.restype = None
        _lib = L
    return _lib


def threads() -> int:
    return int(lib().or_threads())


def _default_threads() -> int:
    import os as _os
    try:
        return max(1, int(_os.environ.get("OMP_NUM_THREADS", "")))
    except ValueError:
        return max(1, _os.cpu_count() or 1)


threads_default = _default_threads()


def set_threads(n: int) -> None:
    """Run the oracle's OpenMP loops on n threads from now on (results do not depend on it)."""
    lib().or_set_threads(int(n))


def _ip(a):
    return a.ctypes.data_as(ctypes.c_void_p)


class Field:
    """A dense full-extent FP64 array with its geometry (x first)."""

    def __init__(self, size, halo_lo, halo_hi, data=None):
        self.size = tuple(size)
        self.ndim = len(size)
        self.halo_lo = tuple(halo_lo)
        self.halo_hi = tuple(halo_hi)
        shape = tuple(size[a] + halo_lo[a] + halo_hi[a] for a in reversed(range(self.ndim)))
        if data is None:
            self.a = np.zeros(shape)
        else:
            self.a = np.ascontiguousarray(np.asarray(data, dtype=np.float64).reshape(shape)).copy()
        ext = [size[a] + halo_lo[a] + halo_hi[a] for a in range(self.ndim)] + [1] * (3 - self.ndim)
        hl = list(halo_lo) + [0] * (3 - self.ndim)
        self.geo = np.array(ext + hl, dtype=np.int32)

    def check(self, lo, hi, offs):
        offs = [tuple(o) + (0,) * (3 - len(o)) for o in offs]
        for a in range(self.ndim):
            omin = min(o[a] for o in offs)
            omax = max(o[a] for o in offs)
            if lo[a] < hi[a] and (lo[a] + omin < -self.halo_lo[a]
                                  or hi[a] - 1 + omax >= self.size[a] + self.halo_hi[a]):
                raise IndexError("stencil access outside the allocated extent")


def _r3(lo, hi, nd):
    lo3 = np.array(list(lo) + [0] * (3 - nd), dtype=np.int32)
    hi3 = np.array(list(hi) + [1] * (3 - nd), dtype=np.int32)
    return lo3, hi3


def _o3(offs, nd):
    return [tuple(o) + (0,) * (3 - len(o)) for o in offs]


def run_loop(loop, fields: Dict[str, Field], reds: Dict[str, float], red_ops: Dict[str, str]):
    """Evaluate one loop (a `workloads.spec.Loop`) in place on `fields`."""
    k = loop.kernel
    if k.startswith("euler_") or k.startswith("ns_"):
        from . import physics_loops
        return physics_loops.run_loop(loop, fields, reds, red_ops)
    L = lib()
    args = loop.args
    dst = fields[args[0].name] if args[0].access in ("w", "rw") else None
    nd = (dst or fields[args[0].name]).ndim
    lo3, hi3 = _r3(loop.lo, loop.hi, nd)
    for a in args:
        if a.access != "red":
            fields[a.name].check(loop.lo, loop.hi, a.offsets)
    if k == "copy":
        o = np.array(_o3(args[1].offsets, nd)[0], dtype=np.int32)
        src = fields[args[1].name]
        L.or_copy(_ip(lo3), _ip(hi3), _ip(dst.a), _ip(dst.geo), _ip(src.a), _ip(src.geo), _ip(o))
    elif k == "lincomb":
        ins = [fields[a.name] for a in args[1:]]
        ptrs = (ctypes.c_void_p * len(ins))(*[f.a.ctypes.data for f in ins])
        geos = np.concatenate([f.geo for f in ins]).astype(np.int32)
        npts = np.array([len(a.offsets) for a in args[1:]], dtype=np.int32)
        offs = np.array([o for a in args[1:] for o in _o3(a.offsets, nd)], dtype=np.int32).reshape(-1)
        coef = np.array(loop.params[1:], dtype=np.float64)
        if len(coef) != int(npts.sum()) or len(coef) < 1:
            raise ValueError("lincomb: one coefficient per sample, at least one sample")
        rc = L.or_lincomb(_ip(lo3), _ip(hi3), _ip(dst.a), _ip(dst.geo), len(ins), ptrs, _ip(geos),
                          _ip(npts), _ip(offs), _ip(coef), float(loop.params[0]))
        if rc != 0:
            raise MemoryError(f"or_lincomb failed ({rc})")
    elif k == "reduce":
        srcs = [a for a in args if a.access == "r"]
        red = [a for a in args if a.access == "red"][0].name
        a0 = fields[srcs[0].name]
        b0 = fields[srcs[1].name] if len(srcs) > 1 else None
        op = {"sum": 0, "max": 1, "min": 2}[red_ops[red]]
        v = L.or_reduce(_ip(lo3), _ip(hi3), _ip(a0.a), _ip(a0.geo),
                        _ip(b0.a) if b0 is not None else None,
                        _ip(b0.geo) if b0 is not None else None, int(loop.params[0]), op)
        if red not in reds:
            reds[red] = v
        elif op == 0:
            reds[red] = reds[red] + v
        elif op == 1:
            reds[red] = max(reds[red], v)
        else:
            reds[red] = min(reds[red], v)
    else:
        raise NotImplementedError(f"kernel {k!r}")


def make_fields(dats) -> Dict[str, Field]:
    out = {}
    for d in dats:
        f = Field(d.size, d.halo_lo, d.halo_hi, d.init)
        f.periodic = tuple(getattr(d, "periodic", ()))
        out[d.name] = f
    return out


def run_chain(loops: List, fields: Dict[str, Field], red_specs) -> Dict[str, float]:
    """Run loops in program order; return the reductions of this chain."""
    ops = {r.name: r.op for r in red_specs}
    reds: Dict[str, float] = {}
    for lp in loops:
        run_loop(lp, fields, reds, ops)
    return reds
