"""Thin ctypes binding of liboc.so (include/oc.h): argument marshalling only.

Every step of a chain -- analysis, copies, kernels, reductions -- runs inside
liboc.so. PyTorch is used only to own the device arena and the three CUDA streams.
If the library is missing, importing this module works but `load()` raises: there is
no fallback path.
"""
from __future__ import annotations

import ctypes
import os
from typing import Dict, Iterable, List, Optional, Sequence

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SO = os.path.join(HERE, "_lib", "liboc.so")

OC_OK, OC_ERR_ARG, OC_ERR_BUDGET, OC_ERR_CUDA, OC_ERR_TIMEOUT, OC_ERR_STATE, OC_ERR_NOMEM = 0, -1, -2, -3, -4, -5, -6
OC_F64, OC_F32 = 0, 1
OC_READ, OC_WRITE, OC_RW, OC_REDUCE = 1, 2, 3, 4
OC_SUM, OC_MAX, OC_MIN = 0, 1, 2
OC_FLAG_CYCLIC, OC_FLAG_PREFETCH, OC_FLAG_GRAPHS, OC_FLAG_DRYRUN, OC_FLAG_PROFILE, OC_FLAG_TRACE = \
    0x1, 0x2, 0x4, 0x8, 0x10, 0x20
OC_FLAG_MANAGED = 0x40
OC_PLAN_FIXED, OC_PLAN_AUTOTUNE, OC_PLAN_LEARNED = 0, 1, 2
OC_K_COPY, OC_K_LINCOMB, OC_K_REDUCE, OC_K_HILO_ADD = 1, 2, 3, 4

KERNELS: Dict[str, int] = {"copy": OC_K_COPY, "lincomb": OC_K_LINCOMB, "reduce": OC_K_REDUCE,
                           "hilo_add": OC_K_HILO_ADD}
ACCESS = {"r": OC_READ, "w": OC_WRITE, "rw": OC_RW, "red": OC_REDUCE}
RED_OPS = {"sum": OC_SUM, "max": OC_MAX, "min": OC_MIN}
DTYPES = {"f64": (OC_F64, np.float64), "f32": (OC_F32, np.float32)}

EXPORTS = ["oc_init", "oc_finalize", "oc_decl_dat", "oc_decl_reduction", "oc_enqueue_loop", "oc_flush",
           "oc_reduce", "oc_fetch_dat", "oc_set_flag", "oc_set_tiling", "oc_stats", "oc_last_error",
           "oc_plan_shape", "oc_plan_ranges", "oc_plan_dat", "oc_kernel_stats", "oc_kernel_stats_reset",
           "oc_trace", "oc_planner_features", "oc_autotune_result", "oc_planner_load", "oc_mlp_nparams",
           "oc_mlp_forward", "oc_mlp_loss_grad", "oc_mlp_train", "oc_numa_nodes", "oc_inject_fault", "oc_set_residency",
           "oc_planner_alternatives"]


class OcArg(ctypes.Structure):
    _fields_ = [("dat", ctypes.c_int), ("access", ctypes.c_int), ("npoints", ctypes.c_int),
                ("offsets", ctypes.POINTER(ctypes.c_int))]


class OcStats(ctypes.Structure):
    _fields_ = [("seconds", ctypes.c_double), ("cell_updates", ctypes.c_double),
                ("hbm_bytes", ctypes.c_double), ("h2d_bytes", ctypes.c_double),
                ("d2h_bytes", ctypes.c_double), ("prefetched_bytes", ctypes.c_double),
                ("tiles", ctypes.c_int), ("tile_height", ctypes.c_int), ("depth", ctypes.c_int),
                ("loops", ctypes.c_int), ("graph_replays", ctypes.c_int), ("kernel_launches", ctypes.c_int),
                ("total_seconds", ctypes.c_double), ("total_cell_updates", ctypes.c_double),
                ("total_hbm_bytes", ctypes.c_double), ("total_h2d_bytes", ctypes.c_double),
                ("total_d2h_bytes", ctypes.c_double), ("chains", ctypes.c_longlong),
                ("resident_dats", ctypes.c_int), ("pad_", ctypes.c_int), ("resident_bytes", ctypes.c_double),
                ("total_kernel_launches", ctypes.c_double)]


class OcKernelStats(ctypes.Structure):
    _fields_ = [("launches", ctypes.c_longlong), ("ms", ctypes.c_double), ("bytes", ctypes.c_double),
                ("points", ctypes.c_double)]


class OcTraceRec(ctypes.Structure):
    _fields_ = [("tile", ctypes.c_int), ("kind", ctypes.c_int), ("start_ms", ctypes.c_double),
                ("end_ms", ctypes.c_double), ("bytes", ctypes.c_double)]


class OcError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"liboc error {code}: {msg}")
        self.code = code


_lib = None


def load():
    """Load liboc.so (built by __graft_entry__.build / _build.build). Raises if absent."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(SO):
        raise ImportError(f"liboc.so not built at {SO}; run __graft_entry__.build()")
    L = ctypes.CDLL(SO)
    I, P, U = ctypes.c_int, ctypes.c_void_p, ctypes.c_uint32
    IP = ctypes.POINTER(ctypes.c_int)
    L.oc_init.argtypes = [ctypes.c_size_t, P, ctypes.c_size_t, ctypes.POINTER(P), U, I]
    L.oc_decl_dat.argtypes = [I, IP, IP, IP, I, P, I, IP]
    L.oc_decl_reduction.argtypes = [I, IP]
    L.oc_enqueue_loop.argtypes = [I, IP, IP, I, ctypes.POINTER(OcArg), ctypes.POINTER(ctypes.c_double), I]
    L.oc_reduce.argtypes = [I, ctypes.POINTER(ctypes.c_double)]
    L.oc_fetch_dat.argtypes = [I, P]
    L.oc_set_flag.argtypes = [U, I]
    L.oc_set_tiling.argtypes = [I, I]
    L.oc_stats.argtypes = [ctypes.POINTER(OcStats)]
    L.oc_last_error.restype = ctypes.c_char_p
    L.oc_plan_shape.argtypes = [IP] * 6
    L.oc_plan_ranges.argtypes = [IP]
    L.oc_plan_dat.argtypes = [I, IP, IP, IP, I, IP, IP, I, IP]
    L.oc_kernel_stats.argtypes = [I, ctypes.POINTER(OcKernelStats)]
    L.oc_kernel_stats_reset.argtypes = []
    L.oc_trace.argtypes = [ctypes.POINTER(OcTraceRec), I, IP]
    L.oc_numa_nodes.argtypes = [I, IP, IP]
    L.oc_inject_fault.argtypes = [I, ctypes.c_longlong]
    L.oc_set_residency.argtypes = [ctypes.c_double]
    L.oc_planner_alternatives.argtypes = [IP]
    FP = ctypes.POINTER(ctypes.c_float)
    DP = ctypes.POINTER(ctypes.c_double)
    L.oc_planner_features.argtypes = [FP]
    L.oc_autotune_result.argtypes = [DP, I, IP]
    L.oc_planner_load.argtypes = [FP, I, FP, FP]
    L.oc_mlp_nparams.argtypes = []
    L.oc_mlp_forward.argtypes = [FP, FP, I, FP]
    L.oc_mlp_loss_grad.argtypes = [FP, FP, FP, I, FP, DP]
    L.oc_mlp_train.argtypes = [FP, FP, FP, I, I, ctypes.c_float, FP]
    for name in EXPORTS:
        if name != "oc_last_error":
            getattr(L, name).restype = I
    _lib = L
    return L


def _check(rc: int):
    if rc != OC_OK:
        raise OcError(rc, load().oc_last_error().decode())


def _i3(v: Sequence[int]):
    a = (ctypes.c_int * 3)(*([int(x) for x in v] + [0] * (3 - len(v))))
    return a


class Executor:
    """One liboc context. `budget` bytes of device memory; `arena` a torch uint8
    CUDA tensor of at least `budget` bytes (allocated here if None and not dry-run);
    `streams` three torch.cuda.Stream objects (created here if None)."""

    def __init__(self, budget: int, flags: int = 0, planner: int = OC_PLAN_FIXED, arena=None,
                 streams=None, dryrun: bool = False):
        L = load()
        self.L = L
        self._keep = []
        ptrs = (ctypes.c_void_p * 3)()
        arena_ptr, arena_bytes = None, 0
        if dryrun:
            flags |= OC_FLAG_DRYRUN
        else:
            import torch
            if arena is None:
                arena = torch.empty(int(budget), dtype=torch.uint8, device="cuda")
            if streams is None:
                streams = [torch.cuda.Stream() for _ in range(3)]
            self._keep += [arena, streams]
            arena_ptr, arena_bytes = arena.data_ptr(), arena.numel() * arena.element_size()
            for k in range(3):
                ptrs[k] = streams[k].cuda_stream
        _check(L.oc_init(int(budget), arena_ptr, arena_bytes, ptrs, flags, planner))
        self.open = True
        self.names: Dict[str, int] = {}
        self.reds: Dict[str, int] = {}
        self.meta: Dict[int, tuple] = {}

    # -- declarations -------------------------------------------------------------
    def decl_dat(self, spec) -> int:
        """Declare a `workloads.spec.DatSpec`; returns its handle."""
        code, npdt = DTYPES[spec.dtype]
        nd = spec.ndim
        init = None
        if spec.init is not None:
            init = np.ascontiguousarray(np.asarray(spec.init, dtype=npdt).reshape(spec.shape))
        mask = 0
        for a in spec.periodic:
            mask |= 1 << a
        h = ctypes.c_int()
        _check(self.L.oc_decl_dat(nd, _i3(spec.size), _i3(spec.halo_lo), _i3(spec.halo_hi), code,
                                  init.ctypes.data if init is not None else None, mask, ctypes.byref(h)))
        self.names[spec.name] = h.value
        self.meta[h.value] = (spec.shape, npdt)
        return h.value

    def decl_reduction(self, name: str, op: str) -> int:
        h = ctypes.c_int()
        _check(self.L.oc_decl_reduction(RED_OPS[op], ctypes.byref(h)))
        self.reds[name] = h.value
        return h.value

    # -- loops --------------------------------------------------------------------
    def enqueue(self, loop, kernel_ids: Optional[Dict[str, int]] = None):
        """Queue a `workloads.spec.Loop` (names resolved through decl_* handles). The
        marshalled arguments of a Loop object are kept, so enqueueing the same object
        again (a repeated chain) costs one C call."""
        key = id(loop)
        c = self._prepared.get(key) if hasattr(self, "_prepared") else None
        if c is not None and c[0] is loop and c[1] == tuple(loop.params) and c[2] == (tuple(loop.lo), tuple(loop.hi)):
            _check(self.L.oc_enqueue_loop(*c[3]))
            return
        args = self._marshal(loop, kernel_ids)
        _check(self.L.oc_enqueue_loop(*args[0]))
        if not hasattr(self, "_prepared") or len(self._prepared) > 4096:
            self._prepared = {}
        self._prepared[key] = (loop, tuple(loop.params), (tuple(loop.lo), tuple(loop.hi)), args[0], args[1])

    def _marshal(self, loop, kernel_ids):
        kid = (kernel_ids or {}).get(loop.kernel, KERNELS.get(loop.kernel))
        if kid is None:
            from . import physics
            kid = physics.KERNELS[loop.kernel]
        n = len(loop.args)
        arr = (OcArg * n)()
        keep = []
        for j, a in enumerate(loop.args):
            if a.access == "red":
                arr[j].dat = self.reds[a.name]
                arr[j].access = OC_REDUCE
                arr[j].npoints = 0
                arr[j].offsets = None
                continue
            nd = len(loop.lo)
            offs = np.ascontiguousarray(np.array([tuple(o) + (0,) * (nd - len(o)) for o in a.offsets],
                                                 dtype=np.int32).reshape(-1))
            keep.append(offs)
            arr[j].dat = self.names[a.name]
            arr[j].access = ACCESS[a.access]
            arr[j].npoints = len(a.offsets)
            arr[j].offsets = offs.ctypes.data_as(ctypes.POINTER(ctypes.c_int))
        params = (ctypes.c_double * max(1, len(loop.params)))(*[float(p) for p in loop.params])
        call = (kid, _i3(loop.lo), _i3(loop.hi), n, arr, params, len(loop.params))
        return call, keep

    # -- execution / results ----------------------------------------------------------
    def flush(self):
        _check(self.L.oc_flush())

    def reduce(self, name: str) -> float:
        v = ctypes.c_double()
        _check(self.L.oc_reduce(self.reds[name], ctypes.byref(v)))
        return v.value

    def fetch(self, name: str) -> np.ndarray:
        h = self.names[name]
        shape, npdt = self.meta[h]
        out = np.empty(shape, dtype=npdt)
        _check(self.L.oc_fetch_dat(h, out.ctypes.data))
        return out

    def set_flag(self, flag: int, on: bool = True):
        _check(self.L.oc_set_flag(flag, 1 if on else 0))

    def set_tiling(self, tile_height: int = 0, depth: int = 0):
        _check(self.L.oc_set_tiling(int(tile_height), int(depth)))

    def set_residency(self, level: float):
        """Share of the budget for datasets kept resident across chains (< 0: planner)."""
        _check(self.L.oc_set_residency(float(level)))

    def stats(self) -> dict:
        s = OcStats()
        _check(self.L.oc_stats(ctypes.byref(s)))
        return {f: getattr(s, f) for f, _ in OcStats._fields_}

    def kernel_stats(self, kernel: str) -> dict:
        k = OcKernelStats()
        kid = KERNELS.get(kernel)
        if kid is None:
            from . import physics
            kid = physics.KERNELS[kernel]
        _check(self.L.oc_kernel_stats(kid, ctypes.byref(k)))
        return {f: getattr(k, f) for f, _ in OcKernelStats._fields_}

    def trace(self) -> list:
        """Time line of the last flush (needs OC_FLAG_TRACE): (tile, kind, start, end, bytes)."""
        n = ctypes.c_int()
        _check(self.L.oc_trace(None, 0, ctypes.byref(n)))
        arr = (OcTraceRec * max(1, n.value))()
        _check(self.L.oc_trace(arr, n.value, ctypes.byref(n)))
        kinds = ("upload", "compute", "download")
        return [(r.tile, kinds[r.kind], r.start_ms, r.end_ms, r.bytes) for r in arr[:n.value]]

    def inject_fault(self, site: int, after: int):
        """Arm a one-shot host-side failure (0 upload copy, 1 download copy, 2 launch)."""
        _check(self.L.oc_inject_fault(int(site), int(after)))

    def numa_nodes(self, name: str) -> tuple:
        """(host NUMA node of the dataset's pinned store, host node closest to the GPU)."""
        a, b = ctypes.c_int(), ctypes.c_int()
        _check(self.L.oc_numa_nodes(self.names[name], ctypes.byref(a), ctypes.byref(b)))
        return a.value, b.value

    def features(self) -> np.ndarray:
        f = np.zeros(8, dtype=np.float32)
        _check(self.L.oc_planner_features(_fp(f)))
        return f

    def autotune_result(self) -> np.ndarray:
        """rows (tile height, depth, ms, grid index, hmax, residency level) of the last
        autotuned chain"""
        n = ctypes.c_int()
        _check(self.L.oc_autotune_result(None, 0, ctypes.byref(n)))
        t = np.zeros((max(1, n.value), 6))
        _check(self.L.oc_autotune_result(t.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), n.value,
                                         ctypes.byref(n)))
        return t[:n.value]

    def kernel_stats_reset(self):
        _check(self.L.oc_kernel_stats_reset())

    def plan(self) -> dict:
        """The plan of the most recent flush: tiles, per-tile loop ranges, per-dataset
        slab rows and upload / download intervals."""
        v = [ctypes.c_int() for _ in range(6)]
        _check(self.L.oc_plan_shape(*[ctypes.byref(x) for x in v]))
        T, L_, ND, h, depth, span = [x.value for x in v]
        se = np.zeros(max(1, T * L_ * 2), dtype=np.int32)
        _check(self.L.oc_plan_ranges(se.ctypes.data_as(ctypes.POINTER(ctypes.c_int))))
        dats = []
        for k in range(ND):
            dat, S, nup, ndn = ctypes.c_int(), ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
            cap = 1 << 16
            up = np.zeros(5 * cap, dtype=np.int32)
            dn = np.zeros(5 * cap, dtype=np.int32)
            IP = ctypes.POINTER(ctypes.c_int)
            _check(self.L.oc_plan_dat(k, ctypes.byref(dat), ctypes.byref(S), up.ctypes.data_as(IP), cap,
                                      ctypes.byref(nup), dn.ctypes.data_as(IP), cap, ctypes.byref(ndn)))
            dats.append({"dat": dat.value, "S": S.value,
                         "up": up[:5 * nup.value].reshape(-1, 5).copy(),
                         "down": dn[:5 * ndn.value].reshape(-1, 5).copy()})
        return {"tiles": T, "loops": L_, "tile_height": h, "depth": depth, "slow_rows": span,
                "ranges": se[:T * L_ * 2].reshape(T, L_, 2).copy(), "dats": dats}

    def close(self):
        if self.open:
            _check(self.L.oc_finalize())
            self.open = False

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def run_chain(ex: Executor, dats, reds, loops, declare: bool = True, flush: bool = True):
    """Declare (optionally) and enqueue a chain described by workloads.spec records."""
    if declare:
        for d in dats:
            ex.decl_dat(d)
        for r in reds:
            ex.decl_reduction(r.name, r.op)
    for lp in loops:
        ex.enqueue(lp)
    if flush:
        ex.flush()


def _fp(a):
    assert a.dtype == np.float32 and a.flags.c_contiguous
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_float))


def mlp_nparams() -> int:
    return int(load().oc_mlp_nparams())


def mlp_forward(params: np.ndarray, X: np.ndarray) -> np.ndarray:
    p = np.ascontiguousarray(params, dtype=np.float32)
    x = np.ascontiguousarray(X, dtype=np.float32)
    y = np.zeros((x.shape[0], 2), dtype=np.float32)
    _check(load().oc_mlp_forward(_fp(p), _fp(x), x.shape[0], _fp(y)))
    return y


def mlp_loss_grad(params: np.ndarray, X: np.ndarray, T: np.ndarray):
    p = np.ascontiguousarray(params, dtype=np.float32)
    x = np.ascontiguousarray(X, dtype=np.float32)
    t = np.ascontiguousarray(T, dtype=np.float32)
    g = np.zeros_like(p)
    loss = ctypes.c_double()
    _check(load().oc_mlp_loss_grad(_fp(p), _fp(x), _fp(t), x.shape[0], _fp(g), ctypes.byref(loss)))
    return loss.value, g


def mlp_train(params: np.ndarray, X: np.ndarray, T: np.ndarray, epochs: int, lr: float):
    p = np.ascontiguousarray(params, dtype=np.float32).copy()
    x = np.ascontiguousarray(X, dtype=np.float32)
    t = np.ascontiguousarray(T, dtype=np.float32)
    hist = np.zeros(max(1, epochs), dtype=np.float32)
    _check(load().oc_mlp_train(_fp(p), _fp(x), _fp(t), x.shape[0], int(epochs), float(lr), _fp(hist)))
    return p, hist[:epochs]


def planner_alternatives(alts):
    """Name the two grid candidates the network predicts: ((grid, depth, residency index), ...)."""
    a = (ctypes.c_int * 6)(*[int(v) for c in alts for v in c])
    _check(load().oc_planner_alternatives(a))


def planner_load(params: np.ndarray, mean: np.ndarray, std: np.ndarray):
    p = np.ascontiguousarray(params, dtype=np.float32)
    m = np.ascontiguousarray(mean, dtype=np.float32)
    s = np.ascontiguousarray(std, dtype=np.float32)
    _check(load().oc_planner_load(_fp(p), p.size, _fp(m), _fp(s)))
