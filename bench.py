"""Benchmark of the out-of-core stencil loop-chain executor (arXiv 1709.02125).

Workload: the synthetic random 2-D loop chain -- 24 FP64 fields of 4096^2 (halo 2),
40 LINCOMB loops reading 1-4 fields at offsets within radius 2, plus 2 SUM reductions
that the user reads after every chain -- executed with a device budget of 1/3 of the
3.2 GB footprint (3x oversubscribed). One step = one chain (one oc_flush plus the two
oc_reduce reads). Metric: cell-updates/s = sum over the loops of their range points,
divided by the step time.

Variants on fresh contexts: the headline mixed+learned form (fields stored and
computed in FP32, sums in FP64, learned tile planner, prefetch and CUDA graphs), the
FP64 plain out-of-core form, FP64 with the paper's optimisations (prefetch, cyclic) and
graphs, and FP64 / FP32 in-core (budget above the footprint). Every variant times
--repeats regions of exactly --steps steps and reports the median region.

`--impl reference` times the oracle (plain untiled FP64 C; its OpenMP loops split the
(z, y) lines of every range over the host cores) on the same workload instead.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "out-of-core cell-updates/s at 3x mem: mixed+learned tiling vs FP64 plain"
UNIT = "cell-updates/s"
WORKLOAD = ("random 2-D loop chain: 24 fields x 4096^2 (halo 2), 40 LINCOMB loops (1-4 inputs, "
            "radius-2 offsets) + 2 SUM reductions per chain, device budget 1/3 of the footprint")


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class Clocks:
    """Samples nvidia-smi every 200 ms while the timed region runs."""
    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 8:
                continue
            try:
                sm.append(float(f[0]))
                mx.append(float(f[1]))
            except ValueError:
                continue
            for n, v in zip(names, f[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)), "reasons": sorted(reasons),
                "samples": len(sm)}


def link_bandwidth(torch, nbytes=1 << 30):
    """Pinned host <-> device copy GB/s (H2D, D2H, both directions at once)."""
    h = torch.empty(nbytes, dtype=torch.uint8, pin_memory=True)
    h2 = torch.empty(nbytes, dtype=torch.uint8, pin_memory=True)
    d = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    d2 = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    out = {}
    for name in ("h2d", "d2h", "duplex"):
        best = 0.0
        for _ in range(3):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            if name in ("h2d", "duplex"):
                with torch.cuda.stream(s1):
                    d.copy_(h, non_blocking=True)
            if name in ("d2h", "duplex"):
                with torch.cuda.stream(s2):
                    h2.copy_(d2, non_blocking=True)
            torch.cuda.synchronize()
            dt = time.perf_counter() - t0
            best = max(best, (2 if name == "duplex" else 1) * nbytes / dt / 1e9)
        out[f"{name}_gbs"] = round(best, 1)
    # both directions at once in 8 MiB copies issued alternately (the pipeline's copy
    # size): the rate the tile streams can reach together
    ch = 8 << 20
    best = 0.0
    for _ in range(3):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for o in range(0, nbytes, ch):
            with torch.cuda.stream(s1):
                d[o:o + ch].copy_(h[o:o + ch], non_blocking=True)
            with torch.cuda.stream(s2):
                h2[o:o + ch].copy_(d2[o:o + ch], non_blocking=True)
        torch.cuda.synchronize()
        best = max(best, 2 * nbytes / (time.perf_counter() - t0) / 1e9)
    out["duplex_8mib_gbs"] = round(best, 1)
    del h, h2, d, d2
    return out


def max_over_ranks(dist, values, device):
    """Each value's maximum over the ranks (the job takes as long as its slowest replica);
    the values themselves without a process group."""
    if dist is None:
        return list(values)
    import torch
    t = torch.tensor(list(values), dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(x) for x in t]


def job_throughput(n_ranks: int, units_per_step: float, steps: int, seconds: float) -> float:
    """Whole-job rate of N independent replicas: every rank processes the same units per
    step, and the job's time is the slowest rank's."""
    return n_ranks * units_per_step * steps / seconds


def build_workload(name: str, mixed: bool, n: int, spc: int = 1):
    """(datasets, reductions, make_step, footprint bytes, cells x timesteps per step).
    make_step(ex) returns a function running one step (one chain) on executor ex."""
    if name == "random":
        from workloads import random_chain
        dtype = "f32" if mixed else "f64"
        dats, reds, loops = random_chain.build(n=n, dtype=dtype)
        if mixed:
            for d in dats:
                d.init = d.init.astype(np.float32)
        fp = random_chain.footprint_bytes(n, 24, 4 if mixed else 8)

        def make_step(ex):
            def step():
                for lp in loops:
                    ex.enqueue(lp)
                ex.flush()
                return [ex.reduce(r.name) for r in reds]
            return step
        return dats, reds, make_step, fp, 0
    if name == "euler" and spc > 1:
        # fixed-dt mode: `spc` steps per chain and no reduction in the chain; dt is half
        # the CFL step of the initial state, computed once before the timed steps
        from workloads import euler
        # FP64: the in-place form, the same chain every step (the cyclic flag's promise)
        dats = euler.datasets(n, "f32" if mixed else "f64", euler.initial(n), mixed, steps=spc, inplace=True)
        from workloads.spec import RedSpec
        reds = [RedSpec("dtmin", "min")]

        def make_step(ex):
            state = {"src": "A", "dt": None}

            def step():
                if state["dt"] is None:
                    ex.enqueue(euler.dt_loop(n, mixed))
                    state["dt"] = 0.5 * euler.CFL * ex.reduce("dtmin")
                loops, state["src"] = euler.fixed_dt_chain(n, state["dt"], spc, mixed, state["src"], inplace=True)
                for lp in loops:
                    ex.enqueue(lp)
                ex.flush()
                return []
            return step
        fp = sum(int(np.prod(d.shape)) * (4 if d.dtype == "f32" else 8) for d in dats)
        return dats, reds, make_step, fp, n * n * spc
    if name == "euler":
        from workloads import euler
        # FP64: the in-place form, the same chain every step (the cyclic flag's promise)
        dats = euler.datasets(n, "f32" if mixed else "f64", euler.initial(n), mixed, inplace=True)
        from workloads.spec import RedSpec
        reds = [RedSpec("dtmin", "min")]

        def make_step(ex):
            state = {"dtmin": None}

            def step():
                if state["dtmin"] is None:
                    ex.enqueue(euler.dt_loop(n, mixed))
                    state["dtmin"] = ex.reduce("dtmin")
                dt = euler.CFL * state["dtmin"]
                for lp in euler.chain_loops(n, dt, "A", "A", mixed, inplace=True):
                    ex.enqueue(lp)
                state["dtmin"] = ex.reduce("dtmin")
                return [state["dtmin"]]
            return step
        fp = sum(int(np.prod(d.shape)) * (4 if d.dtype == "f32" else 8) for d in dats)
        return dats, reds, make_step, fp, n * n
    if name == "tgv":
        from workloads import tgv
        dats = tgv.datasets(n, spc, "f32" if mixed else "f64", tgv.initial(n), mixed)
        loops = tgv.chain_loops(n, spc, mixed)

        def make_step(ex):
            def step():
                for lp in loops:
                    ex.enqueue(lp)
                ex.flush()
                return []
            return step
        fp = sum(int(np.prod(d.shape)) * (4 if d.dtype == "f32" else 8) for d in dats)
        return dats, [], make_step, fp, n ** 3 * spc
    if name == "clover3d":
        # one step = SUMMARY_EVERY time steps (one chain each, ended by the MIN the user
        # reads) followed by the read-only summary chain, the cadence of Sec. 5.3
        from workloads import clover3d
        dats = clover3d.datasets(n, n, "f32" if mixed else "f64")
        if mixed:
            for d in dats:
                d.init = d.init.astype(np.float32)
        sreds, sloops = clover3d.step_chain(n, n)
        mreds, mloops = clover3d.summary_chain(n, n)

        def make_step(ex):
            def step():
                out = []
                for _ in range(clover3d.SUMMARY_EVERY):
                    for lp in sloops:
                        ex.enqueue(lp)
                    out.append(ex.reduce("dt"))
                for lp in mloops:
                    ex.enqueue(lp)
                out += [ex.reduce(r.name) for r in mreds]
                return out
            return step
        fp = clover3d.footprint_bytes(n, n, 4 if mixed else 8)
        return dats, sreds + mreds, make_step, fp, n ** 3 * clover3d.SUMMARY_EVERY
    raise ValueError(name)


def run_variant(torch, workload, name, mixed, budget_frac, flags, planner, steps, warmup, n, dist,
                profile_kernels=None, spc=1, repeats=1, trace=False):
    """Run one variant on a fresh context: `warmup` untimed steps, then `repeats` timed
    regions of exactly `steps` steps each (barrier + synchronize around each). The region
    with the median device time is the variant's figure; all regions are returned."""
    from paper_1709_02125_gb300 import oc
    dats, reds, make_step, fp, ct = build_workload(workload, mixed, n, spc)
    n_datasets = len(dats)
    first_dat = dats[0].name
    budget = int(fp * budget_frac)
    streams = [torch.cuda.Stream() for _ in range(3)]
    arena = torch.empty(budget, dtype=torch.uint8, device="cuda")
    ex = oc.Executor(budget, flags=flags, planner=planner, arena=arena, streams=streams)
    try:
        for d in dats:
            ex.decl_dat(d)
            d.init = None  # the library holds its own pinned copy
        for r in reds:
            ex.decl_reduction(r.name, r.op)
        step = make_step(ex)
        for _ in range(warmup):
            step()
        regions = []
        for _rep in range(repeats):
            s0 = ex.stats()
            torch.cuda.synchronize()
            if dist:
                dist.barrier()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(streams[1])
            t0 = time.perf_counter()
            vals = None
            for _ in range(steps):
                vals = step()
            e1.record(streams[2])
            torch.cuda.synchronize()
            wall = time.perf_counter() - t0
            dev_s = e0.elapsed_time(e1) / 1e3
            dev_s, wall = max_over_ranks(dist, [dev_s, wall], "cuda")
            s1 = ex.stats()
            launches = s1["total_kernel_launches"] - s0["total_kernel_launches"]
            regions.append({"device_s": dev_s, "wall_s": wall, "launches": launches, "vals": vals,
                            "s0": s0, "s1": s1})
        order = sorted(range(len(regions)), key=lambda k: regions[k]["device_s"])
        med = regions[order[len(order) // 2]]
        s0, s1 = med["s0"], med["s1"]
        res = {
            "dtype": "f32" if mixed else "f64", "budget_bytes": budget, "footprint_bytes": fp,
            "cells_per_step": (s1["total_cell_updates"] - s0["total_cell_updates"]) / steps,
            "cell_steps_per_step": ct,
            "hbm_bytes_per_step": (s1["total_hbm_bytes"] - s0["total_hbm_bytes"]) / steps,
            "h2d_bytes_per_step": (s1["total_h2d_bytes"] - s0["total_h2d_bytes"]) / steps,
            "d2h_bytes_per_step": (s1["total_d2h_bytes"] - s0["total_d2h_bytes"]) / steps,
            "device_s": med["device_s"], "wall_s": med["wall_s"], "tiles": s1["tiles"],
            "resident_dats": s1["resident_dats"],
            "tile_height": s1["tile_height"], "depth": s1["depth"], "kernel_launches": med["launches"],
            "graph_replays": s1["graph_replays"], "prefetched_bytes": s1["prefetched_bytes"], "sums": med["vals"],
            "regions_device_s": [r["device_s"] for r in regions], "regions_wall_s": [r["wall_s"] for r in regions],
        }
        res["n_datasets"] = n_datasets
        try:
            res["numa"] = dict(zip(("store_node", "gpu_host_node"), ex.numa_nodes(first_dat)))
        except Exception:  # noqa: BLE001 - diagnostics only
            res["numa"] = None
        if profile_kernels:
            # second pass, same steps, with every run of launches of one kernel bracketed by
            # CUDA events on the compute stream: per-kernel device time, from which the
            # dominant kernel and its average launch time are taken (kept out of the timed
            # regions because the events add host work between launches)
            ex.set_flag(oc.OC_FLAG_PROFILE, True)
            ex.kernel_stats_reset()
            for _ in range(min(steps, 10)):
                step()
            torch.cuda.synchronize()
            res["kstats"] = {k: ex.kernel_stats(k) for k in profile_kernels}
            res["kstats"] = {k: v for k, v in res["kstats"].items() if v["launches"] > 0}
            ex.set_flag(oc.OC_FLAG_PROFILE, False)
        if trace:
            # third pass with the per-tile time line (no chain graph, one compute stream):
            # the rate of every tile's upload and download as the copy engines saw it
            ex.set_flag(oc.OC_FLAG_TRACE, True)
            for _ in range(3):
                step()
            torch.cuda.synchronize()
            res["trace"] = trace_summary(ex.trace())
            ex.set_flag(oc.OC_FLAG_TRACE, False)
        return res
    finally:
        ex.close()
        del arena


def trace_summary(tr):
    """Per-tile copy rates of one traced chain: median / min / max GB/s of the tile uploads
    and downloads, the time the upload stream was busy, and the chain's span."""
    out = {}
    if not tr:
        return None
    end = max(r[3] for r in tr)
    for kind in ("upload", "download"):
        rates = [r[4] / (r[3] - r[2]) / 1e6 for r in tr if r[1] == kind and r[4] > 0 and r[3] > r[2]]
        busy = sum(r[3] - r[2] for r in tr if r[1] == kind and r[4] > 0)
        if rates:
            out[kind] = {"tiles": len(rates), "gbs_median": round(float(np.median(rates)), 1),
                         "gbs_min": round(float(min(rates)), 1), "gbs_max": round(float(max(rates)), 1),
                         "busy_ms": round(busy, 3)}
    comp = [r[3] - r[2] for r in tr if r[1] == "compute"]
    out["compute_ms_per_tile_median"] = round(float(np.median(comp)), 3) if comp else None
    out["chain_ms"] = round(end, 3)
    return out


def install_learned_planner(torch):
    """Train the planner network on the GPU from the committed autotuner sweep and load
    it; returns a summary (or None when no sweep data is present)."""
    from paper_1709_02125_gb300 import oc, planner_train
    path = os.path.join(ROOT, "paper_1709_02125_gb300", "planner_data", "autotune_gb300.jsonl")
    if not os.path.exists(path):
        return None
    rows = planner_train.load_rows(path)
    k = int(len(rows) * 0.8)
    t0 = time.perf_counter()
    p, mean, std, hist, alts = planner_train.train(rows[:k])
    train_s = time.perf_counter() - t0
    learned, fixed = planner_train.evaluate(p, mean, std, rows[k:], alts)
    planner_train.install(p, mean, std, alts)
    return {"train_chains": k, "heldout_chains": len(rows) - k, "train_s": round(train_s, 2),
            "final_loss": float(hist[-1]), "alternatives": [list(a) for a in alts],
            "heldout_regret_learned": float(learned.mean()),
            "heldout_regret_fixed": float(fixed.mean())}


def reference_main(args):
    """Time the oracle (plain untiled FP64 C with OpenMP) on the same workload."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    if args.workload != "random":
        print(json.dumps({"impl": "reference", "unavailable": "the CPU reference leg times the random-chain "
                          "workload; the other workloads are checked against the oracle in the tests but "
                          "have no timed leg"}))
        return 0
    import oracle
    from workloads import random_chain
    oracle.build()
    oracle.set_threads(oracle.threads_default)
    n = args.n
    dats, reds, loops = random_chain.build(n=n)
    fields = oracle.make_fields(dats)
    # bound the sample: rows of the slow axis processed per step
    t0 = time.perf_counter()
    oracle.run_chain(loops, fields, reds)
    one = time.perf_counter() - t0
    rows = n
    if one * (args.steps + args.warmup) > args.ref_budget_s:
        rows = max(64, int(n * args.ref_budget_s / (one * (args.steps + args.warmup + 1))))
    sub = [type(lp)(lp.kernel, lp.lo, (lp.hi[0], min(lp.hi[1], rows)), lp.args, lp.params) for lp in loops]
    for _ in range(args.warmup):
        oracle.run_chain(sub, fields, reds)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.run_chain(sub, fields, reds)
    dt = time.perf_counter() - t0
    cells = sum(np.prod([h - l for l, h in zip(lp.lo, lp.hi)]) for lp in sub) * args.steps
    v = float(cells / dt)
    cores = oracle_cores_used(sub, oracle.threads())
    sample = f"full chain (42 loops) on {n} x {rows} rows of the {n}^2 grid per step" if rows < n else \
        f"full chain (42 loops) on the full {n}^2 grid per step"
    sample += f"; {cores} thread(s): the oracle's OpenMP loops split the y rows over the threads"
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD, "n": n, "oracle_rows_per_step": rows},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def cpu_model() -> str:
    """Model name of the host CPU (lscpu, else /proc/cpuinfo, else the machine type)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.strip().lower().startswith("model name"):
                return ln.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        with open("/proc/cpuinfo") as f:
            for ln in f:
                if ln.lower().startswith("model name"):
                    return ln.split(":", 1)[1].strip()
    except OSError:
        pass
    import platform
    return platform.machine()


def oracle_cores_used(loops, threads: int) -> int:
    """Threads the oracle actually works with on a chain: its loop kernels split the (z, y)
    lines of a range over the threads, so a chain keeps min(threads, lines) of them busy."""
    lines = 1
    for lp in loops:
        n = 1
        for a in range(1, len(lp.lo)):
            n *= max(0, lp.hi[a] - lp.lo[a])
        lines = max(lines, n)
    return max(1, min(threads, lines))


def _oracle_rate(oracle, loops, fields, reds, budget_s, max_chains=8):
    """Cell-updates/s of whole chains run back to back for about budget_s seconds."""
    t0 = time.perf_counter()
    chains = cells = 0
    while (time.perf_counter() - t0 < budget_s or chains == 0) and chains < max_chains:
        oracle.run_chain(loops, fields, reds)
        chains += 1
        cells += sum(np.prod([h - l for l, h in zip(lp.lo, lp.hi)]) for lp in loops)
    dt = time.perf_counter() - t0
    return float(cells / dt), chains, dt


def cpu_baseline(n, budget_s=12.0):
    """The oracle as it stands, timed on this host at all threads (the reported value) and
    at one thread on a bounded sample (the first n/8 rows of every loop's range)."""
    import oracle
    from workloads import random_chain
    oracle.build()
    dats, reds, loops = random_chain.build(n=n)
    fields = oracle.make_fields(dats)
    threads = oracle.threads_default
    oracle.set_threads(threads)
    v_all, chains, dt = _oracle_rate(oracle, loops, fields, reds, budget_s)
    rows = max(64, n // 8)
    sub = [type(lp)(lp.kernel, lp.lo, (lp.hi[0], min(lp.hi[1], rows)), lp.args, lp.params) for lp in loops]
    oracle.set_threads(1)
    v_one, chains1, dt1 = _oracle_rate(oracle, sub, fields, reds, budget_s)
    oracle.set_threads(threads)
    return {"value": v_all, "unit": UNIT, "cores": oracle_cores_used(loops, threads), "kind": "oracle",
            "threads_available": os.cpu_count(), "cpu_model": cpu_model(),
            "sample": f"{chains} full chains (42 loops, {n}^2 grid, FP64) in {dt:.1f} s on "
                      f"{oracle_cores_used(loops, threads)} threads (the oracle's loops split the y rows "
                      f"over the threads)",
            "one_thread": {"value": v_one, "unit": UNIT, "cores": 1,
                           "sample": f"{chains1} chains on the first {rows} of {n} rows in {dt1:.1f} s"}}


WORKLOADS = {
    # name: (description, kernels whose device time the profiled pass compares, default n)
    "random": (WORKLOAD, ("lincomb", "reduce"), 4096),
    "euler": ("2-D compressible Euler (MacCormack + 4th-order dissipation), {nd} datasets, periodic square, "
              "{spc} step(s) per chain (1: the CFL min-reduction ends every chain; more: fixed dt, no "
              "reduction), device budget 1/3 of the footprint",
              ("euler_prim", "euler_flux", "euler_pred", "euler_corr", "euler_dt", "hilo_add"), 15360),
    "tgv": ("3-D compressible Navier-Stokes Taylor-Green vortex (4th-order central, low-storage RK3), "
            "{nd} datasets, {spc} RK3 step(s) per chain, device budget 1/3 of the footprint",
            ("ns_prim", "ns_grad", "ns_flux", "ns_div", "ns_update", "hilo_add"), 640),
    "clover3d": ("CloverLeaf-3D-like chains: {nd} datasets on an n^3 grid (halo 2); one step = 10 time "
                 "steps of 599 LINCOMB loops sweeping x, y, z (each ended by a MIN the user reads) plus a "
                 "read-only summary chain of 12 reductions; device budget 1/3 of the footprint",
                 ("lincomb", "reduce"), 256),
}


def kernel_symbol(name: str, dtype: str) -> str:
    """Device function behind a kernel id (LINCOMB runs as the ring-addressed kernel)."""
    t = "float" if dtype == "f32" else "double"
    return f"k_lincomb_ring<{t}>" if name == "lincomb" else f"k_{name}<{t}>"


def recorded_traffic(workload: str, variant: str, plan=None):
    """DRAM bytes per launch of the dominant kernel from a committed ncu capture
    (profiles/traffic.json), or None when the kernel's source text (between the
    recorded markers) changed since, or when the run's plan (tile height, datasets kept
    resident) differs from the captured one, since a launch's bytes follow its rows."""
    import hashlib
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    rec = json.load(open(p)).get(f"{workload}/{variant}")
    if not rec:
        return None
    text = open(os.path.join(ROOT, "paper_1709_02125_gb300", "csrc", rec["source"])).read()
    a, b = text.find(rec["from"]), text.find(rec["to"])
    if a < 0 or b < a or hashlib.sha256(text[a:b].encode()).hexdigest() != rec["source_sha256"]:
        return None
    if plan is not None:
        for k in ("tile_height", "resident_dats"):
            if k in rec and k in plan and rec[k] != plan[k]:
                return None
    return rec


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="random", choices=sorted(WORKLOADS))
    ap.add_argument("--n", type=int, default=0, help="grid size (default: the workload's)")
    ap.add_argument("--ref-budget-s", type=float, default=120.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--variants", default="mixed_learned,mixed_fixed,fp64_plain,fp64_opt,fp64_incore,mixed_incore,"
                                           "mixed_um")
    ap.add_argument("--repeats", type=int, default=5,
                    help="timed regions of --steps steps per variant; the median region is reported")
    ap.add_argument("--spc", type=int, default=1, help="tgv / euler: time steps per chain")
    args = ap.parse_args()
    desc, prof_kernels, n_default = WORKLOADS[args.workload]
    args.n = args.n or n_default
    if args.warmup < 3:
        print("warning: fewer than 3 warm-up steps", file=sys.stderr)
    if args.impl == "reference":
        return reference_main(args)

    import torch
    import __graft_entry__
    from paper_1709_02125_gb300 import oc

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    if rank == 0:
        __graft_entry__.build()
    if dist:
        dist.barrier()
    oc.load()

    link = link_bandwidth(torch)
    P, C, G = oc.OC_FLAG_PREFETCH, oc.OC_FLAG_CYCLIC, oc.OC_FLAG_GRAPHS
    variants = {
        # name: (mixed, budget / footprint, flags, planner)
        "mixed_learned": (True, 1 / 3, P | C | G, oc.OC_PLAN_LEARNED),
        "fp64_plain": (False, 1 / 3, 0, oc.OC_PLAN_FIXED),
        "fp64_opt": (False, 1 / 3, P | C | G, oc.OC_PLAN_FIXED),
        # the FP64 form with the planner's choice of tiling and residency
        "fp64_learned": (False, 1 / 3, P | C | G, oc.OC_PLAN_LEARNED),
        "fp64_tuned": (False, 1 / 3, P | C | G, oc.OC_PLAN_AUTOTUNE),
        "mixed_plain": (True, 1 / 3, 0, oc.OC_PLAN_FIXED),
        # the method without the learned planner: the fixed rule, every dataset streamed
        "mixed_fixed": (True, 1 / 3, P | C | G, oc.OC_PLAN_FIXED),
        # Unified Memory variant (Sec. 5.4): managed stores, tiles prefetched in place
        "mixed_um": (True, 1 / 3, oc.OC_FLAG_MANAGED, oc.OC_PLAN_FIXED),
        "fp64_um": (False, 1 / 3, oc.OC_FLAG_MANAGED, oc.OC_PLAN_FIXED),
        "fp64_incore": (False, 1.25, G, oc.OC_PLAN_FIXED),
        "mixed_incore": (True, 1.25, G, oc.OC_PLAN_FIXED),
    }
    learned = any(variants[v][3] == oc.OC_PLAN_LEARNED for v in args.variants.split(","))
    planner_info = install_learned_planner(torch) if learned else None
    results = {}
    clk = None
    for name in args.variants.split(","):
        mixed, frac, flags, planner = variants[name]
        if name == args.variants.split(",")[0]:
            with Clocks(local) as clk:
                results[name] = run_variant(torch, args.workload, name, mixed, frac, flags, planner, args.steps,
                                            args.warmup, args.n, dist, profile_kernels=prof_kernels, spc=args.spc,
                                            repeats=args.repeats, trace=True)
        else:
            results[name] = run_variant(torch, args.workload, name, mixed, frac, flags, planner, args.steps,
                                        args.warmup, args.n, dist, spc=args.spc, repeats=args.repeats)
    link_after = link_bandwidth(torch)
    head_name = args.variants.split(",")[0]
    head = results[head_name]
    N = world
    value = job_throughput(N, head["cells_per_step"], args.steps, head["device_s"])
    e2e_value = job_throughput(N, head["cells_per_step"], args.steps, head["wall_s"])
    hbm_peak, peak_kind = _peaks()
    kall = head.get("kstats") or {}
    roof = None
    if kall:
        top = max(kall, key=lambda k: kall[k]["ms"])
        ks = kall[top]
        total_ms = sum(v["ms"] for v in kall.values())
        achieved = ks["bytes"] / (ks["ms"] / 1e3) / 1e9
        tr = recorded_traffic(args.workload, head_name, head)
        roof = {"bound": "hbm", "kernel": kernel_symbol(top, head["dtype"]),
                "achieved": round(achieved, 1), "peak": hbm_peak, "peak_kind": peak_kind, "unit": "GB/s",
                "frac": round(achieved / hbm_peak, 4),
                "traffic": tr["dram_bytes_per_launch"] if tr else None,
                "traffic_source": tr["profile"] if tr else None,
                "launches": ks["launches"], "avg_launch_us": round(ks["ms"] / ks["launches"] * 1e3, 2),
                "algorithmic_bytes_per_launch": ks["bytes"] / ks["launches"],
                "share_of_profiled_kernel_time": round(ks["ms"] / total_ms, 4),
                "shares": {kernel_symbol(k, head["dtype"]): round(v["ms"] / total_ms, 4)
                           for k, v in sorted(kall.items(), key=lambda kv: -kv[1]["ms"])}}
    # binding roofline of the whole pipeline: HBM bytes at peak, link bytes at the link speed
    t_step = head["device_s"] / args.steps
    # the link rates are the better of the probes before and after the timed variants
    linkb = {k: max(link[k], link_after[k]) for k in link}
    terms = {"hbm": head["hbm_bytes_per_step"] / (hbm_peak * 1e9),
             "h2d": head["h2d_bytes_per_step"] / (linkb["h2d_gbs"] * 1e9),
             "d2h": head["d2h_bytes_per_step"] / (linkb["d2h_gbs"] * 1e9),
             "duplex": (head["h2d_bytes_per_step"] + head["d2h_bytes_per_step"]) / (linkb["duplex_gbs"] * 1e9)}
    binding = max(terms, key=terms.get)
    t_roof = terms[binding]
    variants_out = {}
    for k, r in results.items():
        v = job_throughput(N, r["cells_per_step"], args.steps, r["device_s"])
        variants_out[k] = {"value": v, "dtype": r["dtype"], "ms_per_step": r["device_s"] / args.steps * 1e3,
                           "resident_dats": r.get("resident_dats", 0),
                           "ms_per_step_regions": [round(x / args.steps * 1e3, 4) for x in r["regions_device_s"]],
                           "tiles": r["tiles"], "tile_height": r["tile_height"], "depth": r["depth"],
                           "h2d_bytes_per_step": r["h2d_bytes_per_step"], "d2h_bytes_per_step": r["d2h_bytes_per_step"],
                           "budget_bytes": r["budget_bytes"], "footprint_bytes": r["footprint_bytes"]}
        if r["cell_steps_per_step"]:
            variants_out[k]["cell_timesteps_per_s"] = N * r["cell_steps_per_step"] * args.steps / r["device_s"]
    for a, b in (("fp64_plain", "fp64_incore"), ("mixed_learned", "mixed_incore"), ("fp64_opt", "fp64_incore"),
                 ("fp64_learned", "fp64_incore"), ("fp64_tuned", "fp64_incore"),
                 ("mixed_fixed", "mixed_incore"), ("mixed_um", "mixed_incore"), ("fp64_um", "fp64_incore")):
        if a in variants_out and b in variants_out:
            variants_out[a]["frac_of_incore"] = variants_out[a]["value"] / variants_out[b]["value"]
    if "mixed_learned" in variants_out and "fp64_plain" in variants_out:
        variants_out["mixed_learned"]["speedup_vs_fp64_plain"] = (variants_out["mixed_learned"]["value"]
                                                                 / variants_out["fp64_plain"]["value"])
    if "mixed_learned" in variants_out and "mixed_fixed" in variants_out:
        variants_out["mixed_learned"]["speedup_vs_fixed_rule"] = (variants_out["mixed_learned"]["value"]
                                                                 / variants_out["mixed_fixed"]["value"])
    line = {
        "metric": METRIC if args.workload == "random" else f"out-of-core cell-updates/s at 3x mem ({args.workload})",
        "value": value, "unit": UNIT, "n_gpus": N, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": head["device_s"] / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": head["dtype"] + ("+f64-reductions" if head["dtype"] == "f32" else ""),
        "data": "synthetic",
        "config": {"workload": desc.format(nd=head["n_datasets"], spc=args.spc), "n": args.n, "variant": head_name,
                   "budget_bytes": head["budget_bytes"], "footprint_bytes": head["footprint_bytes"],
                   "tiles": head["tiles"], "tile_height": head["tile_height"], "depth": head["depth"],
                   "l2": "working set > 129 MB L2 (inputs streamed from host memory): no flush needed",
                   "parallelism": f"replicas x{N}"},
        "roofline": roof,
        "pipeline_roofline": {"t_roof_ms": t_roof * 1e3, "t_ms": t_step * 1e3, "frac": t_roof / t_step,
                              "binding": binding, "terms_ms": {k: round(v * 1e3, 4) for k, v in terms.items()},
                              "link": linkb, "link_before": link, "link_after": link_after, "hbm_peak_gbs": hbm_peak,
                              "numa": head.get("numa"), "trace": head.get("trace")},
        "repeats": {"regions": args.repeats, "steps_per_region": args.steps, "reported": "median region",
                    "value_min": job_throughput(N, head["cells_per_step"], args.steps, max(head["regions_device_s"])),
                    "value_max": job_throughput(N, head["cells_per_step"], args.steps, min(head["regions_device_s"])),
                    "ms_per_step_regions": [round(x / args.steps * 1e3, 4) for x in head["regions_device_s"]]},
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": head["h2d_bytes_per_step"],
                "d2h_bytes_per_step": head["d2h_bytes_per_step"] + 8 * max(1, len(head["sums"] or []))},
        "gpu_launches": int(head["kernel_launches"]),
        "clocks": clk.summary() if clk else None,
        "planner": planner_info,
        "variants": variants_out,
    }
    if rank == 0 and N == 1 and not args.no_cpu_baseline and args.workload == "random":
        line["cpu_baseline"] = cpu_baseline(args.n)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
