"""Host logic of bench.py that needs no GPU: the clock-sample summary (which decides
whether a run is kept), the peak denominators, the recorded-traffic lookup (which must
drop a capture once the kernel it describes has changed), the kernel names and the step
structure of a workload."""
import hashlib
import json
import os

import numpy as np
import pytest

import bench


def _clocks(lines):
    c = bench.Clocks(0)
    c.lines = list(lines)
    return c.summary()


def test_clock_summary_median_and_reasons():
    s = _clocks([
        "1965, 2070, 850.2, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
        "1980, 2070, 870.0, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "2010, 2070, 880.1, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "garbage line",
        "[N/A], 2070, 10, 0x0, Not Active, Not Active, Not Active, Not Active",
    ])
    assert s["sm_mhz"] == 1980.0 and s["sm_max_mhz"] == 2070.0
    assert s["reasons"] == ["sw_power_cap"]
    assert s["samples"] == 3


def test_clock_summary_flags_thermal_and_hw_slowdown():
    s = _clocks(["1500, 2070, 1300, 0x48, Active, Not Active, Active, Not Active"])
    assert s["reasons"] == ["hw_slowdown", "sw_thermal_slowdown"]


def test_clock_summary_without_samples():
    s = _clocks([])
    assert s["sm_mhz"] is None and s["reasons"] == ["unsampled"]


def test_peaks_measured_or_fallback(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench._peaks() == (6800.0, "fallback")
    (tmp_path / "MEASURED_PEAKS.json").write_text(json.dumps({"hbm_gbs": 6799.5, "bf16_tflops": 1900}))
    assert bench._peaks() == (6799.5, "measured")


def _traffic_root(tmp_path, kernel_text):
    csrc = tmp_path / "paper_1709_02125_gb300" / "csrc"
    csrc.mkdir(parents=True)
    (csrc / "k.cu").write_text("prologue\n// BEGIN\n" + kernel_text + "// END\nepilogue\n")
    body = "// BEGIN\n" + kernel_text
    rec = {"kernel": "k_demo<float>", "source": "k.cu", "from": "// BEGIN", "to": "// END",
           "source_sha256": hashlib.sha256(body.encode()).hexdigest(), "dram_bytes_per_launch": 1234}
    (tmp_path / "profiles").mkdir()
    (tmp_path / "profiles" / "traffic.json").write_text(json.dumps({"random/mixed_learned": rec}))
    return csrc / "k.cu"


def test_recorded_traffic_kept_while_kernel_unchanged(tmp_path, monkeypatch):
    _traffic_root(tmp_path, "x = a + b;\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    rec = bench.recorded_traffic("random", "mixed_learned")
    assert rec is not None and rec["dram_bytes_per_launch"] == 1234
    assert bench.recorded_traffic("random", "fp64_plain") is None


def test_recorded_traffic_dropped_after_kernel_change(tmp_path, monkeypatch):
    src = _traffic_root(tmp_path, "x = a + b;\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    src.write_text(src.read_text().replace("a + b", "a - b"))
    assert bench.recorded_traffic("random", "mixed_learned") is None
    # code outside the recorded markers may change freely
    src.write_text("changed prologue\n// BEGIN\nx = a + b;\n// END\nchanged epilogue\n")
    assert bench.recorded_traffic("random", "mixed_learned") is not None


def test_recorded_traffic_absent_file(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.recorded_traffic("random", "mixed_learned") is None


@pytest.mark.parametrize("name,dtype,sym", [("lincomb", "f32", "k_lincomb_ring<float>"),
                                            ("lincomb", "f64", "k_lincomb_ring<double>"),
                                            ("euler_corr", "f32", "k_euler_corr<float>")])
def test_kernel_symbol(name, dtype, sym):
    assert bench.kernel_symbol(name, dtype) == sym


def test_recorded_traffic_dropped_for_another_plan(tmp_path, monkeypatch):
    """A launch's DRAM bytes follow its rows: a record taken at one tile height (or set of
    resident datasets) is not reported for a run with another."""
    _traffic_root(tmp_path, "x = a + b;\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    p = tmp_path / "profiles" / "traffic.json"
    rec = json.loads(p.read_text())
    rec["random/mixed_learned"].update({"tile_height": 256, "resident_dats": 5})
    p.write_text(json.dumps(rec))
    assert bench.recorded_traffic("random", "mixed_learned", {"tile_height": 256, "resident_dats": 5}) is not None
    assert bench.recorded_traffic("random", "mixed_learned", {"tile_height": 410, "resident_dats": 0}) is None


def test_committed_traffic_record_points_at_real_markers():
    """The committed record names a source file and two markers that exist in it, in
    order (whether the hash still matches is the bench's decision at run time)."""
    p = os.path.join(bench.ROOT, "profiles", "traffic.json")
    for key, rec in json.load(open(p)).items():
        text = open(os.path.join(bench.ROOT, "paper_1709_02125_gb300", "csrc", rec["source"])).read()
        a, b = text.find(rec["from"]), text.find(rec["to"])
        assert 0 <= a < b, key


class _FakeExecutor:
    """Records what a bench step enqueues and reads (no library, no GPU)."""

    def __init__(self):
        self.enqueued, self.reads = [], []

    def enqueue(self, lp):
        self.enqueued.append(lp)

    def reduce(self, name):
        self.reads.append((len(self.enqueued), name))
        return 0.0

    def flush(self):
        self.reads.append((len(self.enqueued), None))


def test_clover3d_bench_step_structure():
    """One bench step of the CloverLeaf-3D-like workload: 10 time-step chains of 599
    loops, each ended by reading its MIN, then the 12-reduction summary chain."""
    from workloads import clover3d
    dats, reds, make_step, fp, ct = bench.build_workload("clover3d", False, 8)
    assert len(dats) == 30 and fp == clover3d.footprint_bytes(8, 8, 8) and ct == 8 ** 3 * 10
    assert {r.name for r in reds} == {"dt"} | {f"sm{i}" for i in range(12)}
    ex = _FakeExecutor()
    out = make_step(ex)()
    assert len(out) == 10 + 12
    assert len(ex.enqueued) == 10 * 599 + 12
    dt_reads = [k for k, nm in ex.reads if nm == "dt"]
    assert dt_reads == [599 * (i + 1) for i in range(10)]
    assert [nm for _, nm in ex.reads[10:]] == [f"sm{i}" for i in range(12)]
    mixed = bench.build_workload("clover3d", True, 8)
    assert all(d.dtype == "f32" and d.init.dtype == np.float32 for d in mixed[0])


def test_cpu_baseline_reports_threads_used_and_model(oracle_lib):
    """The CPU baseline states the threads the oracle really used (its loops split the y
    rows of a 2-D chain over the threads) beside those available and the CPU model, and a
    one-thread figure on a bounded sample."""
    b = bench.cpu_baseline(64, budget_s=0.2)
    assert b["kind"] == "oracle" and b["value"] > 0
    assert b["cores"] == min(oracle_lib.threads_default, 64) and b["threads_available"] >= 1
    assert b["one_thread"]["cores"] == 1 and b["one_thread"]["value"] > 0
    assert isinstance(b["cpu_model"], str) and b["cpu_model"]


def test_oracle_cores_used():
    from workloads import random_chain
    _, _, loops2 = random_chain.build_general(2, 16, 4, 4, 1, seed=1)
    _, _, loops3 = random_chain.build_general(3, 8, 4, 4, 1, seed=1, nz=5)
    assert bench.oracle_cores_used(loops2, 16) == 16    # 16 y rows
    assert bench.oracle_cores_used(loops2, 64) == 16
    assert bench.oracle_cores_used(loops3, 64) == 40    # 8 y rows x 5 z planes
    assert bench.oracle_cores_used(loops3, 3) == 3
