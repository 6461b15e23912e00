"""Mutation check of the host-side tests of the chain analysis.

The skew analysis, footprints, copy sets and slab sizes of liboc.so (arXiv 1709.02125,
Sec. 3 and Sec. 4) are checked on the CPU by a brute-force legality checker and by
replaying plans on tagged slabs (test_analysis.py, test_physics_plans.py). Each case
here plants one mistake in a copy of analysis.cpp (a dependency rule dropped, a reach
ignored, a copy-set or slab-size rule broken), relinks the library with it and runs
those tests against it; they must fail for every mutant. Nothing here runs on a GPU:
the plans are built by dry-run contexts.
"""
import concurrent.futures as cf
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1709_02125_gb300", "csrc")
TESTS = ["tests/test_analysis.py", "tests/test_physics_plans.py"]

PS_PE = ("int ps = dp.need_up[r] ? dp.first[r] - k : dp.first[r];\n"
         "            int pe = dp.dl[r] ? dp.last[r] + 1 : dp.last[r];")

# (id, exact original text of analysis.cpp (must occur once), replacement)
MUTANTS = [
    # skewed tiling (Sec. 3): the RAW / WAR / WAW rules of the backward sweep
    ("raw_rule_dropped", "if (is_write(ar.access)) e = std::max(e, std::max(RE[d], WE[d]));",
     "if (is_write(ar.access)) e = std::max(e, WE[d]);"),
    ("waw_rule_dropped", "if (is_write(ar.access)) e = std::max(e, std::max(RE[d], WE[d]));",
     "if (is_write(ar.access)) e = std::max(e, RE[d]);"),
    ("war_rule_dropped", "if (is_read(ar.access) && WE[d] > NEG) e = std::max(e, WE[d] - ar.rmin[sa]);",
     "(void)NEG;"),
    ("war_reach_sign", "if (is_read(ar.access) && WE[d] > NEG) e = std::max(e, WE[d] - ar.rmin[sa]);",
     "if (is_read(ar.access) && WE[d] > NEG) e = std::max(e, WE[d] + ar.rmin[sa]);"),
    ("raw_reach_ignored", "if (is_read(ar.access)) RE[d] = std::max(RE[d], e + ar.rmax[sa]);",
     "if (is_read(ar.access)) RE[d] = std::max(RE[d], e);"),
    ("writer_end_not_recorded", "if (is_write(ar.access)) WE[d] = std::max(WE[d], e);", "(void)0;"),
    # (dropping the clamp e >= e of the previous tile is an equivalent mutant: the sweep
    # already gives monotone ends, since b grows with t and so do the later loops' ends)
    # footprints (Sec. 4): rows a tile touches
    ("footprint_reach_ignored",
     "if (is_read(ar.access)) mark(dp, t, (long long)s + ar.rmin[sa], (long long)e + ar.rmax[sa]);",
     "if (is_read(ar.access)) mark(dp, t, s, e);"),
    ("footprint_lower_reach_ignored",
     "if (is_read(ar.access)) mark(dp, t, (long long)s + ar.rmin[sa], (long long)e + ar.rmax[sa]);",
     "if (is_read(ar.access)) mark(dp, t, s, (long long)e + ar.rmax[sa]);"),
    ("first_tile_overwritten", "if (dp.first[r] < 0) dp.first[r] = t;", "dp.first[r] = t;"),
    # copy sets (Sec. 4.1): write-first rows are not uploaded, read-only rows not downloaded
    ("read_first_upper_reach_ignored",
     "long long b = std::min<long long>((long long)hi + ar.rmax[sa], (long long)dp.y0 + dp.nrows);",
     "long long b = std::min<long long>((long long)hi, (long long)dp.y0 + dp.nrows);"),
    ("read_first_lower_reach_ignored",
     "long long a = std::max<long long>((long long)lo + ar.rmin[sa], dp.y0);",
     "long long a = std::max<long long>((long long)lo, dp.y0);"),
    ("partial_write_taken_as_full", "uint8_t st = full_row_write(lp, dd) ? 1 : 2;", "uint8_t st = 1;"),
    ("full_row_ignores_halo", "if (lp.lo[a] > -d.hlo[a] || lp.hi[a] < d.size[a] + d.hhi[a]) return false;",
     "if (lp.lo[a] > 0 || lp.hi[a] < d.size[a]) return false;"),
    ("strip_rows_not_uploaded", "dp.need_up[r] = st == 2 ? 1 : (st == 3 ? 2 : 0);",
     "dp.need_up[r] = st == 2 ? 1 : 0;"),
    ("strip_columns_wrong", "dp.wx0[r] = std::max(lp.lo[0], -dd.hlo[0]);", "dp.wx0[r] = std::max(lp.lo[0], 0);"),
    ("cyclic_skips_read_first_downloads", "dp.dl[r] = written[d][r] && !(cyclic && dfirst[d] == 1);",
     "dp.dl[r] = written[d][r] && !(cyclic && dfirst[d] != 0);"),
    ("cyclic_per_row_first_write", "dp.dl[r] = written[d][r] && !(cyclic && dfirst[d] == 1);",
     "dp.dl[r] = written[d][r] && !(cyclic && (st == 1 || st == 3));"),
    ("read_only_downloaded", "dp.dl[r] = written[d][r] && !(cyclic && dfirst[d] == 1);",
     "dp.dl[r] = !(cyclic && dfirst[d] == 1);"),
    ("first_access_reads_ignored", "if (ar.access != OC_REDUCE && is_read(ar.access) && !dfirst[P.dat_index[ar.dat]])\n                dfirst[P.dat_index[ar.dat]] = 2;",
     "if (false)\n                dfirst[P.dat_index[ar.dat]] = 2;"),
    ("copy_groups_merge_tiles", "while (r < dp.nrows && need[r] == kind && tile[r] == t && key(r) == kx) ++r;",
     "while (r < dp.nrows && need[r] == kind && key(r) == kx) ++r;"),
    # slab sizes (cyclic slots): rows live in one pipeline phase must fit
    ("slab_ignores_upload_lookahead", PS_PE,
     "int ps = dp.first[r];\n            int pe = dp.dl[r] ? dp.last[r] + 1 : dp.last[r];"),
    ("slab_ignores_download_phase", PS_PE,
     "int ps = dp.need_up[r] ? dp.first[r] - k : dp.first[r];\n            int pe = dp.last[r];"),
    ("prefetch_slots_not_checked", "return d1 >= ll && d1 + rl <= Sc;", "return d1 >= 0;"),
    ("prefetch_hull_misses_live_rows", "if (pe >= T - 1) { lea = std::min(lea, r); leb = std::max(leb, r + 1); }",
     "if (pe >= T) { lea = std::min(lea, r); leb = std::max(leb, r + 1); }"),
    # budget fit: the largest tile height whose arena fits
    ("budget_search_inverted", "if (fits(mid)) lo = mid; else hi = mid;", "if (fits(mid)) hi = mid; else lo = mid;"),
]


def _nvcc():
    return os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")


def _build_mutant(tmp, old, new):
    from paper_1709_02125_gb300 import _build
    text = open(os.path.join(CSRC, "analysis.cpp")).read()
    if old:
        assert text.count(old) == 1, f"mutant text must occur once in analysis.cpp: {old!r}"
        text = text.replace(old, new)
    src = os.path.join(tmp, "analysis.cpp")
    with open(src, "w") as fh:
        # the copy sits outside csrc/: its relative includes are made absolute
        fh.write(text.replace('#include "../../include/oc.h"', f'#include "{os.path.join(ROOT, "include", "oc.h")}"')
                 .replace('#include "oc_internal.h"', f'#include "{os.path.join(CSRC, "oc_internal.h")}"'))
    obj = os.path.join(tmp, "analysis.o")
    subprocess.run([_nvcc(), "-x", "cu"] + _build._flags() + ["-c", src, "-o", obj], check=True,
                   capture_output=True)
    objs = [obj if s == "analysis.cpp" else os.path.join(_build.OUT_DIR, "obj", s + ".o") for s in _build.SOURCES]
    so = os.path.join(tmp, "liboc_mutant.so")
    subprocess.run([_nvcc()] + _build.ARCH + ["-shared", "-o", so] + objs, check=True, capture_output=True)
    return so


_RUNNER = """
import sys
sys.path[:0] = [{root!r}, {tests!r}]
from paper_1709_02125_gb300 import oc
oc.SO = {so!r}
import pytest
sys.exit(pytest.main({tests_list!r} + ["-x", "-q", "-p", "no:cacheprovider", "-m", "not gpu"]))
"""


def _case(tmp, old, new):
    so = _build_mutant(tmp, old, new)
    code = _RUNNER.format(root=ROOT, tests=os.path.join(ROOT, "tests"), so=so, tests_list=TESTS)
    r = subprocess.run([sys.executable, "-c", code], cwd=ROOT, capture_output=True, text=True, timeout=900,
                       env=dict(os.environ, OMP_NUM_THREADS="1"))
    return r.returncode, r.stdout[-1500:]


@pytest.fixture(scope="module")
def outcomes(tmp_path_factory):
    import __graft_entry__
    __graft_entry__.build_lib()          # the other objects the mutants link against
    base = tmp_path_factory.mktemp("analysis_mutants")
    jobs = [("unmutated", "", "")] + MUTANTS

    def run(job):
        mid, old, new = job
        tmp = os.path.join(str(base), mid)
        os.makedirs(tmp)
        return mid, _case(tmp, old, new)

    with cf.ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 2)) as ex:
        return dict(ex.map(run, jobs))


def test_unmutated_copy_passes(outcomes):
    rc, out = outcomes["unmutated"]
    assert rc == 0, out


@pytest.mark.parametrize("mid", [m[0] for m in MUTANTS])
def test_analysis_tests_catch_mutant(outcomes, mid):
    rc, out = outcomes[mid]
    assert rc == 1, f"mutant {mid} survived the analysis tests:\n{out}"
