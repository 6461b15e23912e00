"""The cyclic flag's promise (arXiv 1709.02125, Sec. 4.1): the chain is the one repeated,
so a dataset it writes before reading is a per-chain temporary and a streamed plan never
downloads it. A later chain that reads such a dataset first would compute from host rows
that no longer hold its values; the library refuses that chain (OC_ERR_STATE). Host-only:
dry-run contexts plan the chains and apply the same bookkeeping as a device run."""
import numpy as np
import pytest

from workloads import euler

oc = pytest.importorskip("paper_1709_02125_gb300.oc")

N = 64


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__
    __graft_entry__.build_lib()
    return oc.load()


def _footprint(dats):
    return sum(int(np.prod(d.shape)) * 8 for d in dats)


def _executor(budget, flags, inplace=False):
    ex = oc.Executor(budget, dryrun=True, flags=flags)
    for d in euler.datasets(N, "f64", None, inplace=inplace):
        ex.decl_dat(d)
    ex.decl_reduction("dtmin", "min")
    return ex


def _step(ex, src, dst, inplace=False):
    for lp in euler.chain_loops(N, 1e-4, src, dst, inplace=inplace, with_dt=False):
        ex.enqueue(lp)
    ex.flush()


def test_ping_pong_under_cyclic_is_refused(lib):
    """Chain A -> B writes B first (not downloaded); the next chain B -> A reads B first."""
    fp = _footprint(euler.datasets(N))
    with _executor(fp // 3, oc.OC_FLAG_CYCLIC) as ex:
        _step(ex, "A", "B")
        assert ex.plan()["tiles"] > 1
        with pytest.raises(oc.OcError) as e:
            _step(ex, "B", "A")
        assert e.value.code == oc.OC_ERR_STATE
        assert "cyclic" in str(e.value)


def test_ping_pong_without_cyclic_runs(lib):
    fp = _footprint(euler.datasets(N))
    with _executor(fp // 3, 0) as ex:
        for k in range(4):
            _step(ex, "A", "B") if k % 2 == 0 else _step(ex, "B", "A")


def test_in_place_form_under_cyclic_runs(lib):
    """The FP64 in-place form is the same chain every step: its state is read first, its
    increments are written first, and nothing stale is ever read."""
    fp = _footprint(euler.datasets(N, inplace=True))
    with _executor(fp // 3, oc.OC_FLAG_CYCLIC | oc.OC_FLAG_PREFETCH, inplace=True) as ex:
        for _ in range(4):
            _step(ex, "A", "A", inplace=True)
        assert ex.plan()["tiles"] > 1


def test_in_core_plans_keep_every_dataset(lib):
    """A budget that holds every dataset: the chain runs in core, its datasets are
    downloaded when they leave the device, and ping-pong under the cyclic flag is legal."""
    fp = _footprint(euler.datasets(N))
    with _executor(4 * fp, oc.OC_FLAG_CYCLIC) as ex:
        for k in range(4):
            _step(ex, "A", "B") if k % 2 == 0 else _step(ex, "B", "A")
        assert ex.plan()["tiles"] == 1


def test_stale_mark_cleared_by_a_kept_write(lib):
    """After the refusal, a chain that writes B with the cyclic flag off downloads it:
    B is current on the host again and B -> A runs."""
    fp = _footprint(euler.datasets(N))
    with _executor(fp // 3, oc.OC_FLAG_CYCLIC) as ex:
        _step(ex, "A", "B")
        with pytest.raises(oc.OcError):
            _step(ex, "B", "A")
        ex.set_flag(oc.OC_FLAG_CYCLIC, False)
        _step(ex, "A", "B")
        _step(ex, "B", "A")
