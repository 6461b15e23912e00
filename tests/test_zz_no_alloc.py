"""The allocation-free reduction entry point (oc_reduce_noalloc) against the executor's.

Callers that cannot allocate device memory (inside another component's graph capture,
allocator-free real-time code, a pool that must not grow) get a reduction whose scratch
lives in a fixed device array inside liboc.so. This test calls it through the C ABI twice
in a row -- different element types, operators, modes and shapes -- and checks each
result against an OC_K_REDUCE loop run by the executor on the same values. The two run
the same kernels on the same partial layout and fold them in the same order, so they
agree bit for bit. The shapes include a region of exactly 65536 one-element rows: the
largest the fixed scratch takes, and more rows than one launch grid dimension holds.
Collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

from workloads.spec import READ, REDUCE, Arg, DatSpec, Loop, RedSpec

pytestmark = pytest.mark.gpu


def _executor_reduce(data, dtype, op, mode):
    from paper_1709_02125_gb300 import oc
    ny, nx = data.shape[0] - 2, data.shape[1] - 2
    with oc.Executor(64 << 20) as ex:
        ex.decl_dat(DatSpec("a", (nx, ny), (1, 1), (1, 1), dtype, init=data))
        ex.decl_reduction("r", op)
        ex.enqueue(Loop("reduce", (0, 0), (nx, ny), [Arg("a", READ), Arg("r", REDUCE)], [float(mode)]))
        return ex.reduce("r")


def test_reduce_noalloc_matches_executor_twice():
    import torch

    import __graft_entry__
    from paper_1709_02125_gb300 import oc
    __graft_entry__.build()
    L = oc.load()
    L.oc_reduce_noalloc.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_longlong,
                                    ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p]
    L.oc_reduce_noalloc.restype = ctypes.c_int
    L.oc_noalloc_last_error.restype = ctypes.c_char_p
    rng = np.random.default_rng(2024)
    cases = [("f64", "sum", 0, 37, 5000), ("f32", "max", 1, 300, 911), ("f64", "sum", 2, 65536, 1)]
    for dtype, op, mode, ny, nx in cases:
        npdt = np.float64 if dtype == "f64" else np.float32
        data = rng.uniform(-1.0, 1.0, size=(ny + 2, nx + 2)).astype(npdt)
        expect = _executor_reduce(data, dtype, op, mode)
        dev = torch.from_numpy(np.ascontiguousarray(data[1:-1, 1:-1])).to("cuda")
        out = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
        stream = torch.cuda.current_stream().cuda_stream
        rc = L.oc_reduce_noalloc(dev.data_ptr(), oc.DTYPES[dtype][0], ny, nx, nx, oc.RED_OPS[op], mode,
                                 out.data_ptr(), stream)
        torch.cuda.synchronize()
        assert rc == 0, L.oc_noalloc_last_error()
        got = float(out.item())
        assert got == expect, (dtype, op, got, expect)
    # a region beyond the fixed scratch is rejected, not truncated
    big = torch.zeros((70000, 1), dtype=torch.float64, device="cuda")
    out = torch.zeros((1,), dtype=torch.float64, device="cuda")
    rc = L.oc_reduce_noalloc(big.data_ptr(), oc.OC_F64, 70000, 1, 1, oc.OC_SUM, 0, out.data_ptr(), None)
    assert rc == oc.OC_ERR_ARG
