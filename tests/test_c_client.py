"""The C ABI used from plain C: include/oc.h compiles as C99 with warnings as errors, and
a C program linked against liboc.so (tests/c/abi_dryrun.c) plans the heat chain in a
dry-run context, with the same plan the Python binding gets for the same chain."""
import os
import subprocess

import numpy as np
import pytest

from workloads import heat

import plan_sim

oc = pytest.importorskip("paper_1709_02125_gb300.oc")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
INC = os.path.join(ROOT, "include")


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__
    return __graft_entry__.build_lib()


@pytest.mark.parametrize("header", ["oc.h", "oc_physics.h"])
def test_headers_are_plain_c99(tmp_path, header):
    src = tmp_path / "inc.c"
    src.write_text(f'#include "{header}"\nint main(void) {{ return 0; }}\n')
    subprocess.run(["gcc", "-std=c99", "-pedantic", "-Wall", "-Wextra", "-Werror", f"-I{INC}", "-c", str(src),
                    "-o", str(tmp_path / "inc.o")], check=True)


def test_c_client_plans_like_the_binding(lib, tmp_path):
    exe = tmp_path / "abi_dryrun"
    libdir = os.path.dirname(lib)
    subprocess.run(["gcc", "-std=c99", "-Wall", "-Werror", f"-I{INC}", os.path.join(ROOT, "tests", "c", "abi_dryrun.c"),
                    "-o", str(exe), f"-L{libdir}", "-l:liboc.so", f"-Wl,-rpath,{libdir}"], check=True)
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stderr
    lines = r.stdout.splitlines()
    head = lines[0].split()
    T, L = int(head[1]), int(head[3])
    assert (T, L, int(head[5]), int(head[7]), int(head[9])) == (4, 30, 2, 64, 3)
    se = np.zeros((T, L, 2), dtype=np.int64)
    for ln in lines[1:]:
        _, t, i, s, e = ln.split()
        se[int(t), int(i)] = (int(s), int(e))
    dats, reds, loops = heat.build(256, 10)
    with oc.Executor(1 << 20, dryrun=True) as ex:
        ex.set_tiling(64, 3)
        oc.run_chain(ex, dats, reds, loops)
        plan = ex.plan()
    assert np.array_equal(plan["ranges"], se)
    plan_sim.check_legality({"tiles": T, "ranges": se}, loops)
