"""Error behaviour of the C ABI (include/oc.h) that needs no GPU: every entry point returns
a status instead of aborting, calls out of order give OC_ERR_STATE, invalid arguments
give OC_ERR_ARG with a message, and a dry-run context plans but holds no data. The calls
go straight through ctypes, as a C caller would make them."""
import ctypes

import numpy as np
import pytest

oc = pytest.importorskip("paper_1709_02125_gb300.oc")


@pytest.fixture(scope="module")
def L():
    import __graft_entry__
    __graft_entry__.build_lib()
    return oc.load()


def _err(L):
    return L.oc_last_error().decode()


@pytest.fixture
def dry(L):
    ptrs = (ctypes.c_void_p * 3)()
    assert L.oc_init(1 << 20, None, 0, ptrs, oc.OC_FLAG_DRYRUN, oc.OC_PLAN_FIXED) == oc.OC_OK
    yield L
    assert L.oc_finalize() == oc.OC_OK


def test_calls_without_context_are_state_errors(L):
    h = ctypes.c_int()
    st = oc.OcStats()
    v = ctypes.c_double()
    for name, rc in (("oc_flush", L.oc_flush()), ("oc_decl_reduction", L.oc_decl_reduction(0, ctypes.byref(h))),
                     ("oc_stats", L.oc_stats(ctypes.byref(st))), ("oc_set_flag", L.oc_set_flag(1, 1)),
                     ("oc_reduce", L.oc_reduce(0, ctypes.byref(v))), ("oc_finalize", L.oc_finalize())):
        assert rc == oc.OC_ERR_STATE, name
        assert "no context" in _err(L), name


def test_second_context_is_refused(dry):
    ptrs = (ctypes.c_void_p * 3)()
    assert dry.oc_init(1 << 20, None, 0, ptrs, oc.OC_FLAG_DRYRUN, 0) == oc.OC_ERR_STATE
    assert "already exists" in _err(dry)


def test_init_argument_errors(L):
    ptrs = (ctypes.c_void_p * 3)()
    D = oc.OC_FLAG_DRYRUN
    assert L.oc_init(1 << 20, None, 0, ptrs, D, 7) == oc.OC_ERR_ARG             # planner mode
    assert L.oc_init(1 << 20, None, 4096, ptrs, D, 0) == oc.OC_ERR_ARG          # bytes, no arena
    buf = ctypes.create_string_buffer(16)
    assert L.oc_init(1 << 20, ctypes.addressof(buf), 16, ptrs, D, 0) == oc.OC_ERR_ARG  # arena < budget
    assert L.oc_flush() == oc.OC_ERR_STATE                                    # none was created


def test_init_without_a_device_is_a_cuda_error(L):
    """Without OC_FLAG_DRYRUN the context needs a device; on a machine without one the
    call fails cleanly with OC_ERR_CUDA and leaves no context behind."""
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a CUDA device is present")
    ptrs = (ctypes.c_void_p * 3)()
    assert L.oc_init(1 << 20, None, 0, ptrs, 0, 0) == oc.OC_ERR_CUDA
    assert L.oc_flush() == oc.OC_ERR_STATE


@pytest.mark.parametrize("case", ["ndim", "size", "halo", "dtype", "periodic_fast_halo", "null_out"])
def test_decl_dat_rejects(dry, case):
    i3 = oc._i3
    h = ctypes.c_int()
    args = {"ndim": (4, (8, 8, 8), (1, 1, 1), (1, 1, 1), 0, 0),
            "size": (2, (-8, 8), (1, 1), (1, 1), 0, 0),
            "halo": (2, (8, 8), (-1, 1), (1, 1), 0, 0),
            "dtype": (2, (8, 8), (1, 1), (1, 1), 7, 0),
            "periodic_fast_halo": (2, (8, 8), (1, 1), (1, 1), 0, 1),
            "null_out": (2, (8, 8), (1, 1), (1, 1), 0, 0)}[case]
    nd, size, hlo, hhi, dt, mask = args
    out = None if case == "null_out" else ctypes.byref(h)
    assert dry.oc_decl_dat(nd, i3(size), i3(hlo), i3(hhi), dt, None, mask, out) == oc.OC_ERR_ARG
    assert _err(dry).startswith("oc_decl_dat")


def test_periodic_slow_axis_may_have_halo(dry):
    """A periodic slow axis keeps its halo rows (deep ghosts refreshed every chain)."""
    h = ctypes.c_int()
    i3 = oc._i3
    assert dry.oc_decl_dat(2, i3((8, 8)), i3((0, 2)), i3((0, 2)), 0, None, 2, ctypes.byref(h)) == oc.OC_OK
    assert h.value >= 0


def test_argument_checks_of_the_other_calls(dry):
    h = ctypes.c_int()
    assert dry.oc_decl_reduction(9, ctypes.byref(h)) == oc.OC_ERR_ARG
    for height, depth in ((8, 5), (8, 1), (-3, 3)):
        assert dry.oc_set_tiling(height, depth) == oc.OC_ERR_ARG
    assert dry.oc_set_tiling(0, 0) == oc.OC_OK
    assert dry.oc_set_flag(0x1000, 1) == oc.OC_ERR_ARG
    assert dry.oc_set_flag(oc.OC_FLAG_DRYRUN, 0) == oc.OC_ERR_ARG     # not switchable
    assert dry.oc_set_flag(oc.OC_FLAG_CYCLIC, 1) == oc.OC_OK
    v = ctypes.c_double()
    assert dry.oc_reduce(99, ctypes.byref(v)) == oc.OC_ERR_ARG
    out = np.zeros(100)
    assert dry.oc_fetch_dat(99, out.ctypes.data) == oc.OC_ERR_ARG
    assert dry.oc_enqueue_loop(77, oc._i3((0, 0)), oc._i3((8, 8)), 0, None, None, 0) == oc.OC_ERR_ARG
    assert dry.oc_planner_load(None, 3, None, None) == oc.OC_ERR_ARG
    assert str(dry.oc_mlp_nparams()) in _err(dry)


def test_dry_run_plans_but_holds_no_data(dry):
    h = ctypes.c_int()
    i3 = oc._i3
    assert dry.oc_decl_dat(2, i3((8, 8)), i3((1, 1)), i3((1, 1)), 0, None, 0, ctypes.byref(h)) == oc.OC_OK
    r = ctypes.c_int()
    assert dry.oc_decl_reduction(oc.OC_SUM, ctypes.byref(r)) == oc.OC_OK
    args = (oc.OcArg * 2)()
    args[0].dat, args[0].access, args[0].npoints = h.value, oc.OC_READ, 1
    zero = (ctypes.c_int * 2)(0, 0)
    args[0].offsets = ctypes.cast(zero, ctypes.POINTER(ctypes.c_int))
    args[1].dat, args[1].access = r.value, oc.OC_REDUCE
    prm = (ctypes.c_double * 1)(0.0)
    assert dry.oc_enqueue_loop(oc.OC_K_REDUCE, i3((0, 0)), i3((8, 8)), 2, args, prm, 1) == oc.OC_OK
    assert dry.oc_flush() == oc.OC_OK
    dims = [ctypes.c_int() for _ in range(6)]
    assert dry.oc_plan_shape(*[ctypes.byref(d) for d in dims]) == oc.OC_OK
    assert dims[0].value >= 1 and dims[1].value == 1 and dims[2].value == 1
    v = ctypes.c_double()
    assert dry.oc_reduce(r.value, ctypes.byref(v)) == oc.OC_ERR_STATE
    out = np.zeros((10, 10))
    assert dry.oc_fetch_dat(h.value, out.ctypes.data) == oc.OC_ERR_STATE
    # a plan_dat call with too small capacities reports the counts it needs
    k, dat, S, nup, ndown = 0, ctypes.c_int(), ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    rc = dry.oc_plan_dat(k, ctypes.byref(dat), ctypes.byref(S), None, 0, ctypes.byref(nup), None, 0,
                         ctypes.byref(ndown))
    # (the dataset is read: it has upload intervals; it is never written: no downloads)
    assert rc == oc.OC_ERR_ARG and nup.value > 0 and ndown.value == 0
    assert dat.value == h.value
    up = (ctypes.c_int * (5 * nup.value))()
    assert dry.oc_plan_dat(k, ctypes.byref(dat), ctypes.byref(S), up, nup.value, ctypes.byref(nup), None, 0,
                           ctypes.byref(ndown)) == oc.OC_OK
    rows = sorted(y for j in range(nup.value) for y in range(up[5 * j + 1], up[5 * j + 2]))
    assert rows == list(range(0, 8))   # the interior rows the reduction reads, each once


def test_fault_hook_and_numa_query_arguments(L):
    """oc_inject_fault and oc_numa_nodes: state errors without a context, argument errors
    on a bad site or handle; a dry-run context arms the hook and plans as before (it
    issues no copy, so nothing fails) and reports no NUMA node for a store it never
    allocated."""
    a, b = ctypes.c_int(), ctypes.c_int()
    assert L.oc_inject_fault(0, 0) == oc.OC_ERR_STATE
    assert L.oc_numa_nodes(0, ctypes.byref(a), ctypes.byref(b)) == oc.OC_ERR_STATE
    ptrs = (ctypes.c_void_p * 3)()
    assert L.oc_init(1 << 20, None, 0, ptrs, oc.OC_FLAG_DRYRUN, oc.OC_PLAN_FIXED) == oc.OC_OK
    try:
        assert L.oc_inject_fault(3, 0) == oc.OC_ERR_ARG and "site" in _err(L)
        assert L.oc_inject_fault(-1, 0) == oc.OC_ERR_ARG
        for site in (0, 1, 2):
            assert L.oc_inject_fault(site, 0) == oc.OC_OK
        assert L.oc_inject_fault(0, -1) == oc.OC_OK   # disarm
        size = (ctypes.c_int * 3)(64, 64, 1)
        halo = (ctypes.c_int * 3)(1, 1, 0)
        h = ctypes.c_int()
        assert L.oc_decl_dat(2, size, halo, halo, oc.OC_F64, None, 0, ctypes.byref(h)) == oc.OC_OK
        assert L.oc_numa_nodes(h.value + 1, ctypes.byref(a), ctypes.byref(b)) == oc.OC_ERR_ARG
        assert L.oc_numa_nodes(h.value, None, ctypes.byref(b)) == oc.OC_ERR_ARG
        assert L.oc_numa_nodes(h.value, ctypes.byref(a), ctypes.byref(b)) == oc.OC_OK
        assert a.value == -1 and b.value == -1
        offs = (ctypes.c_int * 2)(0, 0)
        args = (oc.OcArg * 2)(oc.OcArg(h.value, oc.OC_WRITE, 1, offs), oc.OcArg(h.value, oc.OC_READ, 1, offs))
        lo, hi = (ctypes.c_int * 3)(0, 0, 0), (ctypes.c_int * 3)(64, 64, 1)
        assert L.oc_enqueue_loop(oc.OC_K_COPY, lo, hi, 2, args, None, 0) == oc.OC_OK
        assert L.oc_inject_fault(2, 0) == oc.OC_OK
        assert L.oc_flush() == oc.OC_OK
    finally:
        assert L.oc_finalize() == oc.OC_OK


def test_managed_flag_is_init_only_and_plans_like_the_explicit_pipeline(L):
    """OC_FLAG_MANAGED (the Unified Memory variant) is chosen at oc_init: oc_set_flag
    refuses it. A dry-run managed context plans a chain with the explicit pipeline's
    tiles (the same budget rule), without residency."""
    from workloads import random_chain
    dats, reds, loops = random_chain.build(n=128, nfields=8, nloops=12, seed=3)
    for d in dats:
        d.init = None
    fp = random_chain.footprint_bytes(128, 8)
    shapes = []
    for flags in (0, oc.OC_FLAG_MANAGED):
        with oc.Executor(fp // 3, dryrun=True, flags=flags) as ex:
            with pytest.raises(oc.OcError) as e:
                ex.set_flag(oc.OC_FLAG_MANAGED, True)
            assert e.value.code == oc.OC_ERR_ARG
            ex.set_residency(0.5)
            oc.run_chain(ex, dats, reds, loops)
            st = ex.stats()
            shapes.append((st["tiles"], st["tile_height"], st["resident_dats"]))
    assert shapes[0][2] > 0 and shapes[1][2] == 0
    with oc.Executor(fp // 3, dryrun=True, flags=oc.OC_FLAG_MANAGED) as ex:
        oc.run_chain(ex, dats, reds, loops)
        st_m = ex.stats()
    with oc.Executor(fp // 3, dryrun=True) as ex:
        oc.run_chain(ex, dats, reds, loops)
        st_e = ex.stats()
    assert (st_m["tiles"], st_m["tile_height"], st_m["depth"]) == (st_e["tiles"], st_e["tile_height"], st_e["depth"])
    assert st_m["tiles"] > 1
