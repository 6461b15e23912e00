"""Test tools for tile plans (host only): a brute-force legality checker and a CPU
simulation of the cyclic-slab pipeline.

The legality checker gives every (loop, slow row) the tile that computes it and checks
that every read-after-write, write-after-read and write-after-write pair on the same
dataset row keeps program order (arXiv 1709.02125, Sec. 3: the tiled schedule must
be equivalent to executing the loops one by one).

The simulator replays a plan the way the executor does -- uploads of tile p+k,
compute of tile p, download of tile p-1 in phase p -- against slabs of S slots per
dataset whose slots carry the tag of the row they hold. Every read checks that its row
is in its slot, every phase checks that the rows touched by its three operations
occupy distinct slots, and loops run through the oracle's kernels on a gathered
window, so the final host arrays must equal a sequential oracle run bit for bit.
"""
from __future__ import annotations

import copy
from typing import Dict, List

import numpy as np


def _slow(lp):
    return len(lp.lo) - 1


def _dy(lp, a):
    """slow-axis offsets of argument a (offsets padded with zeros to the loop's rank)"""
    sa = _slow(lp)
    return [(tuple(o) + (0, 0, 0))[sa] for o in a.offsets]


def loop_rows_tile(plan, i, lo, hi):
    """tile[y - lo] for every slow row y of loop i's range [lo, hi)."""
    r = plan["ranges"]
    out = np.full(hi - lo, -1, dtype=np.int64)
    for t in range(plan["tiles"]):
        s, e = r[t, i]
        if e > s:
            assert np.all(out[s - lo:e - lo] == -1), "row computed twice"
            out[s - lo:e - lo] = t
    return out


def check_legality(plan, loops):
    """Raise AssertionError if the plan's loop ranges break program order."""
    r = plan["ranges"]
    T, L = plan["tiles"], len(loops)
    info = []
    for i, lp in enumerate(loops):
        sa = _slow(lp)
        lo, hi = lp.lo[sa], max(lp.lo[sa], lp.hi[sa])
        # partition: consecutive, monotone, covering [lo, hi)
        prev = lo
        for t in range(T):
            s, e = r[t, i]
            assert s == prev and e >= s, f"loop {i} tile {t}: range [{s},{e}) does not continue {prev}"
            prev = e
        assert prev == hi, f"loop {i} ends at {prev}, not {hi}"
        tile = loop_rows_tile(plan, i, lo, hi)
        reads, writes = {}, set()
        for a in lp.args:
            if a.access in ("r", "rw"):
                reads.setdefault(a.name, set()).update(_dy(lp, a))
            if a.access in ("w", "rw"):
                writes.add(a.name)
        info.append((lo, hi, tile, reads, writes))

    def tile_at(i, rows):
        lo, hi, tile, _, _ = info[i]
        ok = (rows >= lo) & (rows < hi)
        t = np.full(rows.shape, -1, dtype=np.int64)
        t[ok] = tile[rows[ok] - lo]
        return t, ok

    for i in range(L):
        lo_i, hi_i, tile_i, rd_i, wr_i = info[i]
        rows_i = np.arange(lo_i, hi_i)
        for j in range(i + 1, L):
            lo_j, hi_j, tile_j, rd_j, wr_j = info[j]
            rows_j = np.arange(lo_j, hi_j)
            for D in wr_i:
                # RAW: j reads row y+dy that i writes
                for dy in rd_j.get(D, ()):
                    ti, ok = tile_at(i, rows_j + dy)
                    assert np.all(ti[ok] <= tile_j[ok]), f"RAW violated: loop {i} -> {j} on {D}"
                # WAW
                if D in wr_j:
                    ti, ok = tile_at(i, rows_j)
                    assert np.all(ti[ok] <= tile_j[ok]), f"WAW violated: loop {i} -> {j} on {D}"
            for D, dys in rd_i.items():
                if D not in wr_j:
                    continue
                # WAR: i reads row y+dy that j later writes
                for dy in dys:
                    tj, ok = tile_at(j, rows_i + dy)
                    assert np.all(tile_i[ok] <= tj[ok]), f"WAR violated: loop {i} -> {j} on {D}"


def simulate(plan, loops, dats, reds, oracle, handle_of: Dict[str, int], chains: int = 1,
             prefetch: bool = False, stats: Dict = None, chain_start=None):
    """Replay the plan with tagged cyclic slabs for `chains` repetitions of the chain;
    returns (fields, reductions of the last chain).

    With `prefetch`, the speculative prefetch of Sec. 4.1 is replayed as the executor
    issues it: once phase T - 2 of a chain is done, every dataset whose tile-0 upload rows
    all sit in slots not used by rows live in phases T - 1 and T, and none of which is
    downloaded in those phases, has those rows copied from the host into its slab; the
    next chain skips them. The simulation checks that the prefetched slots stay untouched
    until the next chain reads them.

    `chain_start(host)`, if given, runs on the host fields before each chain's first copy
    (the executor refreshes the deep ghost rows of periodic datasets there)."""
    T, k = plan["tiles"], plan["depth"] - 2
    by_handle = {d["dat"]: d for d in plan["dats"]}
    specs = {d.name: d for d in dats}
    host = oracle.make_fields(dats)
    name_of = {h: n for n, h in handle_of.items()}
    slabs = {}
    for d in plan["dats"]:
        spec = specs[name_of[d["dat"]]]
        sa = spec.ndim - 1
        y0 = -spec.halo_lo[sa]
        row_shape = host[spec.name].a.shape[1:]
        slabs[spec.name] = {"S": d["S"], "y0": y0, "data": np.full((d["S"],) + row_shape, np.nan),
                            "tag": np.full(d["S"], -10 ** 9, dtype=np.int64), "plan": d}
    red_ops = {r.name: r.op for r in reds}
    red_vals: Dict[str, float] = {}

    def slot(sl, y):
        return (y - sl["y0"]) % sl["S"]

    def phase_rows(p):
        """rows touched in phase p per dataset: uploads of p+k, compute of p, downloads of p-1"""
        rows = {n: set() for n in slabs}
        for n, sl in slabs.items():
            for t, a, b, _, _ in sl["plan"]["up"]:
                if t == p + k:
                    rows[n].update(range(a, b))
            for t, a, b, _, _ in sl["plan"]["down"]:
                if t == p - 1:
                    rows[n].update(range(a, b))
        if 0 <= p < T:
            for i, lp in enumerate(loops):
                s, e = plan["ranges"][p, i]
                if e <= s:
                    continue
                sa = _slow(lp)
                for a in lp.args:
                    if a.access == "red":
                        continue
                    dys = _dy(lp, a) if a.access in ("r", "rw") else [0]
                    rows[a.name].update(range(s + min(dys), e + max(dys)))
        return rows

    # phases in which each row of each dataset is live (upload ... download), for the
    # prefetch rule
    last_live = {n: {} for n in slabs}
    for p in range(-k, T + 1):
        for n, rows in phase_rows(p).items():
            for y in rows:
                last_live[n][y] = max(last_live[n].get(y, p), p)

    def prefetch_rows():
        out = {}
        for n, sl in slabs.items():
            busy = {slot(sl, y) for y, pe in last_live[n].items() if pe >= T - 1}
            late_dl = {y for t, a, b, _, _ in sl["plan"]["down"] if t >= T - 2 for y in range(a, b)}
            ivs = [(a, b, x0, x1) for t, a, b, x0, x1 in sl["plan"]["up"] if t == 0]
            rows = [(y, x0, x1) for a, b, x0, x1 in ivs for y in range(a, b)]
            if rows and all(slot(sl, y) not in busy and y not in late_dl for y, _, _ in rows):
                out[n] = rows
        return out

    def upload_row(n, sl, y, x0, x1):
        hx = specs[n].halo_lo[0]
        row = host[n].a[y - sl["y0"]]
        if x0 < x1:
            # first written over [x0, x1): only the other columns travel; the written
            # part holds garbage until then
            new = np.full_like(row, np.nan)
            new[..., :x0 + hx] = row[..., :x0 + hx]
            new[..., x1 + hx:] = row[..., x1 + hx:]
            row = new
        sl["data"][slot(sl, y)] = row
        sl["tag"][slot(sl, y)] = y

    have = {}   # rows prefetched for the next chain, per dataset
    for c in range(chains):
        red_vals = {}
        if chain_start is not None:
            chain_start(host)
        have = _run_chain(plan, loops, T, k, slabs, host, specs, red_ops, red_vals, oracle, slot, phase_rows,
                          upload_row, have, prefetch and c + 1 < chains, prefetch_rows, stats)
    return host, red_vals


def _run_chain(plan, loops, T, k, slabs, host, specs, red_ops, red_vals, oracle, slot, phase_rows,
               upload_row, have, do_prefetch, prefetch_rows, stats):
    pf = {}
    pf_slots = {}
    for p in range(-k, T + 1):
        if do_prefetch and p == T - 1:
            # phase T - 2 is done: the prefetch goes in while phases T - 1 and T run
            pf = prefetch_rows()
            for n, rows in pf.items():
                sl = slabs[n]
                for y, x0, x1 in rows:
                    upload_row(n, sl, y, x0, x1)
                pf_slots[n] = {slot(sl, y) for y, _, _ in rows}
                if stats is not None:
                    stats["prefetched_rows"] = stats.get("prefetched_rows", 0) + len(rows)
        if pf_slots and p >= T - 1:
            for n, rows in phase_rows(p).items():
                hit = {slot(slabs[n], y) for y in rows} & pf_slots.get(n, set())
                assert not hit, f"phase {p}: a live row of {n} uses a prefetched slot"
        # all rows the three concurrent operations of this phase touch hold distinct slots
        for n, rows in phase_rows(p).items():
            sl = slabs[n]
            slots = [slot(sl, y) for y in rows]
            assert len(set(slots)) == len(slots), f"phase {p}: two live rows of {n} share a slot"
        u = p + k
        if 0 <= u < T:
            for n, sl in slabs.items():
                skip = {y for y, _, _ in have.get(n, [])} if u == 0 else set()
                for t, a, b, x0, x1 in sl["plan"]["up"]:
                    if t == u:
                        for y in range(a, b):
                            if y in skip:
                                # prefetched by the previous chain: still in its slot
                                assert sl["tag"][slot(sl, y)] == y, f"prefetched row {y} of {n} was overwritten"
                                continue
                            upload_row(n, sl, y, x0, x1)
        if 0 <= p < T:
            for i, lp in enumerate(loops):
                s, e = plan["ranges"][p, i]
                if e <= s:
                    continue
                sa = _slow(lp)
                win = {}
                for a in lp.args:
                    if a.access == "red" or a.name in win:
                        continue
                    sl = slabs[a.name]
                    dys = [0]
                    for b in lp.args:
                        if b.name == a.name and b.access in ("r", "rw"):
                            dys += _dy(lp, b)
                    f = copy.copy(host[a.name])
                    f.a = np.full_like(host[a.name].a, np.nan)
                    for y in range(s + min(dys), e + max(dys)):
                        reading = any(b.name == a.name and b.access in ("r", "rw") for b in lp.args)
                        if reading or y in range(s, e):
                            if sl["tag"][slot(sl, y)] == y:
                                f.a[y - sl["y0"]] = sl["data"][slot(sl, y)]
                            elif reading and y in _read_rows(lp, a.name, s, e, sa):
                                raise AssertionError(f"tile {p} loop {i}: row {y} of {a.name} not resident")
                    win[a.name] = f
                sub = copy.copy(lp)
                sub.lo = tuple(lp.lo[:sa]) + (s,)
                sub.hi = tuple(lp.hi[:sa]) + (e,)
                part: Dict[str, float] = {}
                oracle.run_loop(sub, win, part, red_ops)
                for rn, v in part.items():
                    if rn not in red_vals:
                        red_vals[rn] = v
                    elif red_ops[rn] == "sum":
                        red_vals[rn] += v
                    elif red_ops[rn] == "max":
                        red_vals[rn] = max(red_vals[rn], v)
                    else:
                        red_vals[rn] = min(red_vals[rn], v)
                for a in lp.args:
                    if a.access in ("w", "rw"):
                        sl = slabs[a.name]
                        for y in range(s, e):
                            sl["data"][slot(sl, y)] = win[a.name].a[y - sl["y0"]]
                            sl["tag"][slot(sl, y)] = y
        q = p - 1
        if 0 <= q < T:
            for n, sl in slabs.items():
                for t, a, b, _, _ in sl["plan"]["down"]:
                    if t == q:
                        for y in range(a, b):
                            assert sl["tag"][slot(sl, y)] == y, f"download of {n} row {y}: slot holds another row"
                            host[n].a[y - sl["y0"]] = sl["data"][slot(sl, y)]
    return pf


def _read_rows(lp, name, s, e, sa):
    rows = set()
    for b in lp.args:
        if b.name == name and b.access in ("r", "rw"):
            for dy in _dy(lp, b):
                rows.update(range(s + dy, e + dy))
    return rows
