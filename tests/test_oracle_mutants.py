"""Mutation check of the oracle's pins.

Each case plants one plausible mistake in a copy of the oracle's source (a dropped
term, a wrong sign, index, axis or coefficient, a transposed operand) and runs the
independent pins against that copy: for the C library (built into a temporary library
and loaded through ORACLE_LIB) test_oracle_pins.py for the loop kernels and
test_oracle_physics.py for the PDE step functions; for the numpy modules (the mutated
module stands in for oracle.mlp or oracle.physics_loops) test_oracle_mlp.py and the
step-equality tests of test_physics_loops.py. The pins must fail for every mutant. The golden fixtures are left out on purpose: they are the
oracle's own output and would catch any change trivially.

The mistakes are planted on the CPU only; nothing here touches the CUDA path.
"""
import concurrent.futures as cf
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
ORACLE = os.path.join(ROOT, "oracle")

PINS = {"oracle.c": "tests/test_oracle_pins.py", "physics.c": "tests/test_oracle_physics.py"}

# (id, file, exact original text (must occur once), replacement)
MUTANTS = [
    # ---- loop kernels (Sec. 3: pointwise kernels through stencil offsets)
    ("copy_offset_sign", "oracle.c",
     "src[at(sg, x + o[0], y + o[1], z + o[2])]", "src[at(sg, x - o[0], y - o[1], z - o[2])]"),
    ("copy_offset_axes", "oracle.c",
     "src[at(sg, x + o[0], y + o[1], z + o[2])]", "src[at(sg, x + o[1], y + o[0], z + o[2])]"),
    ("lincomb_offset_axes", "oracle.c",
     "at(sg + 6 * j, x + o[0], y + o[1], z + o[2])", "at(sg + 6 * j, x + o[1], y + o[0], z + o[2])"),
    ("lincomb_offset_sign_y", "oracle.c",
     "at(sg + 6 * j, x + o[0], y + o[1], z + o[2])", "at(sg + 6 * j, x + o[0], y - o[1], z + o[2])"),
    ("lincomb_dropped_sample", "oracle.c",
     "for (m = 1; m < M; ++m) acc", "for (m = 2; m < M; ++m) acc"),
    ("lincomb_first_coef", "oracle.c",
     "double acc = coef[0] * xs[0];", "double acc = coef[1 % M] * xs[0];"),
    ("lincomb_nonlinear_sign", "oracle.c",
     "acc = acc + ((alpha * a) * b)", "acc = acc - ((alpha * a) * b)"),
    ("lincomb_nonlinear_operand", "oracle.c",
     "/ (1.0 + c * c)", "/ (1.0 + b * b)"),
    ("lincomb_nonlinear_index", "oracle.c",
     "b = xs[1 % M], c = xs[2 % M]", "b = xs[2 % M], c = xs[1 % M]"),
    ("lincomb_nonlinear_square", "oracle.c",
     "/ (1.0 + c * c)", "/ (1.0 + c)"),
    ("geometry_halo_index", "oracle.c",
     "(size_t)(x + g[3])", "(size_t)(x + g[4])"),
    ("geometry_extent_index", "oracle.c",
     "(size_t)(z + g[5]) * (size_t)g[1]", "(size_t)(z + g[5]) * (size_t)g[0]"),
    ("reduce_abs_dropped", "oracle.c",
     "if (mode == 1) v = fabs(v);", "if (mode == 1) v = v;"),
    ("reduce_square", "oracle.c",
     "else if (mode == 2) v = v * v;", "else if (mode == 2) v = fabs(v);"),
    ("reduce_second_source_sign", "oracle.c",
     "if (b) v = v + b[at(bg, x, y, z)];", "if (b) v = v - b[at(bg, x, y, z)];"),
    ("reduce_min_is_max", "oracle.c",
     "else m = v < m ? v : m;", "else m = v > m ? v : m;"),
    ("reduce_rows_skipped", "oracle.c",
     "for (k = 0; k < nr; ++k) {\n        if (op == 0)", "for (k = 1; k < nr; ++k) {\n        if (op == 0)"),
    ("reduce_row_range", "oracle.c",
     "for (int x = lo[0]; x < hi[0]; ++x) {\n                    double v",
     "for (int x = lo[0] + 1; x < hi[0]; ++x) {\n                    double v"),
    ("reduce_row_split_overlap", "oracle.c",
     "y1 = three ? hi[1] : r0 + k + 1;", "y1 = three ? hi[1] : r0 + k + 2;"),
    # ---- Euler (Sec. 5.1 stand-in: MacCormack with fourth-order dissipation)
    ("euler_pressure_dropped_term", "physics.c",
     "double p = (gamma - 1.0) * (E[q] - 0.5 * (mx[q] * u + my[q] * v));",
     "double p = (gamma - 1.0) * (E[q] - 0.5 * (mx[q] * u));"),
    ("euler_gamma", "physics.c",
     "double p = (gamma - 1.0) * (E[q]", "double p = gamma * (E[q]"),
    ("euler_flux_x_pressure", "physics.c",
     "F[N + q] = mx[q] * u + p;", "F[N + q] = mx[q] * u;"),
    ("euler_flux_y_pressure_axis", "physics.c",
     "G[N + q] = my[q] * u;\n        G[2 * N + q] = my[q] * v + p;",
     "G[N + q] = my[q] * u + p;\n        G[2 * N + q] = my[q] * v;"),
    ("euler_flux_energy_velocity", "physics.c",
     "G[3 * N + q] = (E[q] + p) * v;", "G[3 * N + q] = (E[q] + p) * u;"),
    ("euler_flux_energy_pressure", "physics.c",
     "F[3 * N + q] = (E[q] + p) * u;", "F[3 * N + q] = E[q] * u;"),
    ("euler_predictor_backward", "physics.c",
     "lx * (Fk[IX2(i + 1, j)] - Fk[IX2(i, j)])", "lx * (Fk[IX2(i, j)] - Fk[IX2(i - 1, j)])"),
    ("euler_predictor_sign_y", "physics.c",
     "- ly * (Gk[IX2(i, j + 1)] - Gk[IX2(i, j)]);", "+ ly * (Gk[IX2(i, j + 1)] - Gk[IX2(i, j)]);"),
    ("euler_corrector_forward_y", "physics.c",
     "- ly * (Gk[IX2(i, j)] - Gk[IX2(i, j - 1)]))", "- ly * (Gk[IX2(i, j + 1)] - Gk[IX2(i, j)]))"),
    ("euler_corrector_uses_U", "physics.c",
     "0.5 * (Uk[IX2(i, j)] + Us[k * N + IX2(i, j)]", "0.5 * (Uk[IX2(i, j)] + Uk[IX2(i, j)]"),
    ("euler_corrector_lx_ly", "physics.c",
     "- lx * (Fk[IX2(i, j)] - Fk[IX2(i - 1, j)])", "- ly * (Fk[IX2(i, j)] - Fk[IX2(i - 1, j)])"),
    ("euler_dissipation_sign", "physics.c",
     "- eps4 * (d4x + d4y);", "+ eps4 * (d4x + d4y);"),
    ("euler_dissipation_y_dropped", "physics.c",
     "- eps4 * (d4x + d4y);", "- eps4 * d4x;"),
    ("euler_dissipation_coef", "physics.c",
     "double d4x = Uk[IX2(i - 2, j)] - 4.0 * Uk[IX2(i - 1, j)] + 6.0 * Uk[IX2(i, j)]",
     "double d4x = Uk[IX2(i - 2, j)] - 4.0 * Uk[IX2(i - 1, j)] + 5.0 * Uk[IX2(i, j)]"),
    ("euler_dissipation_y_axis", "physics.c",
     "double d4y = Uk[IX2(i, j - 2)] - 4.0 * Uk[IX2(i, j - 1)]",
     "double d4y = Uk[IX2(i - 2, j)] - 4.0 * Uk[IX2(i - 1, j)]"),
    ("euler_dt_sound_speed", "physics.c",
     "double a = dx / (fabs(u) + c), b = dy / (fabs(v) + c);",
     "double a = dx / (fabs(u) + c), b = dy / (fabs(v) + 0.5 * c);"),
    ("euler_dt_spacing", "physics.c",
     "b = dy / (fabs(v) + c);", "b = dx / (fabs(v) + c);"),
    ("euler_dt_velocity_axis", "physics.c",
     "double a = dx / (fabs(u) + c)", "double a = dx / (fabs(v) + c)"),
    ("euler_dt_gamma", "physics.c",
     "double c = sqrt(gamma * p / r);", "double c = sqrt(p / r);"),
    # ---- Navier-Stokes (Sec. 5.1 stand-in: fourth-order central, low-storage RK3)
    ("ns_d1_coefficient", "physics.c",
     "return ((fm2 - 8.0 * fm1) + (8.0 * fp1 - fp2)) / (12.0 * h);",
     "return ((fm2 - 6.0 * fm1) + (6.0 * fp1 - fp2)) / (8.0 * h);"),
    ("ns_d1_spacing", "physics.c",
     "D[(3 * f + a) * N + c] = d1(src, nx, ny, nz, i, j, k, a, h[a]);",
     "D[(3 * f + a) * N + c] = d1(src, nx, ny, nz, i, j, k, a, h[0]);"),
    ("ns_residual_sign", "physics.c",
     "r = r - ((fm2 - 8.0 * fm1) + (8.0 * fp1 - fp2)) / (12.0 * h[a]);",
     "r = r + ((fm2 - 8.0 * fm1) + (8.0 * fp1 - fp2)) / (12.0 * h[a]);"),
    ("ns_residual_coefficient", "physics.c",
     "r = r - ((fm2 - 8.0 * fm1) + (8.0 * fp1 - fp2)) / (12.0 * h[a]);",
     "r = r - ((fm2 - 6.0 * fm1) + (6.0 * fp1 - fp2)) / (12.0 * h[a]);"),
    ("ns_pressure_w_dropped", "physics.c",
     "0.5 * (U[N + q] * u + U[2 * N + q] * v + U[3 * N + q] * w)",
     "0.5 * (U[N + q] * u + U[2 * N + q] * v)"),
    ("ns_temperature_gamma", "physics.c",
     "W[4 * N + q] = gamma * Ma * Ma * p / r;", "W[4 * N + q] = Ma * Ma * p / r;"),
    ("ns_conductivity_gamma", "physics.c",
     "const double kc = mu / ((gamma - 1.0) * Ma * Ma * Pr);",
     "const double kc = mu / (gamma * Ma * Ma * Pr);"),
    ("ns_conductivity_prandtl", "physics.c",
     "const double kc = mu / ((gamma - 1.0) * Ma * Ma * Pr);",
     "const double kc = mu * Pr / ((gamma - 1.0) * Ma * Ma);"),
    ("ns_heat_flux_dropped", "physics.c",
     "- kc * D[(9 + a) * N + c];", ";"),
    ("ns_heat_flux_sign", "physics.c",
     "- kc * D[(9 + a) * N + c];", "+ kc * D[(9 + a) * N + c];"),
    ("ns_heat_flux_gradient", "physics.c",
     "- kc * D[(9 + a) * N + c];", "- kc * D[(6 + a) * N + c];"),
    ("ns_viscosity", "physics.c",
     "const double mu = Re > 0 ? 1.0 / Re : 0.0;", "const double mu = Re > 0 ? 2.0 / Re : 0.0;"),
    ("ns_stress_transpose_dropped", "physics.c",
     "mu * (D[(3 * b + a) * N + c] + D[(3 * a + b) * N + c]", "mu * (2.0 * D[(3 * b + a) * N + c]"),
    ("ns_stress_two_thirds", "physics.c",
     "(2.0 / 3.0) * div", "(1.0 / 3.0) * div"),
    ("ns_divergence_term_dropped", "physics.c",
     "const double div = D[0 * N + c] + D[4 * N + c] + D[8 * N + c];",
     "const double div = D[0 * N + c] + D[4 * N + c];"),
    ("ns_momentum_pressure_axis", "physics.c",
     "(m - 1 == a ? p : 0.0)", "(m == a ? p : 0.0)"),
    ("ns_momentum_stress_sign", "physics.c",
     "+ (m - 1 == a ? p : 0.0) - tau[m - 1];", "+ (m - 1 == a ? p : 0.0) + tau[m - 1];"),
    ("ns_energy_viscous_work_dropped", "physics.c",
     "- (vel[0] * tau[0] + vel[1] * tau[1] + vel[2] * tau[2])", "- (vel[0] * tau[0])"),
    ("ns_energy_pressure_work", "physics.c",
     "return (U[4 * N + c] + p) * vel[a]", "return U[4 * N + c] * vel[a]"),
    ("ns_mass_flux_axis", "physics.c",
     "if (m == 0) return U[(size_t)(a + 1) * N + c];", "if (m == 0) return U[(size_t)(1) * N + c];"),
    ("ns_rk3_A", "physics.c",
     "{0.0, -5.0 / 9.0, -153.0 / 128.0}", "{0.0, -5.0 / 8.0, -153.0 / 128.0}"),
    ("ns_rk3_B", "physics.c",
     "{1.0 / 3.0, 15.0 / 16.0, 8.0 / 15.0}", "{1.0 / 3.0, 15.0 / 16.0, 7.0 / 15.0}"),
    ("ns_rk3_stage_order", "physics.c",
     "dU[q] = A[s] * dU[q] + dt * R[q];", "dU[q] = A[s] * dU[q] + B[s] * dt * R[q];"),
]


# planner-network oracle (oracle/mlp.py), pinned by test_oracle_mlp.py
MLP_MUTANTS = [
    ("mlp_relu2_dropped", "a2 = np.maximum(z2, 0.0)", "a2 = z2"),
    ("mlp_W2_transposed", "z2 = a1 @ w[\"W2\"].T + w[\"b2\"]", "z2 = a1 @ w[\"W2\"] + w[\"b2\"]"),
    ("mlp_b1_dropped", "z1 = X @ w[\"W1\"].T + w[\"b1\"]", "z1 = X @ w[\"W1\"].T"),
    ("mlp_layer_order", "y = a2 @ w[\"W3\"].T + w[\"b3\"]", "y = a1 @ w[\"W3\"].T + w[\"b3\"]"),
    ("mlp_loss_half", "return float(np.sum((y - np.asarray(T, dtype=np.float64)) ** 2) / (2 * len(X)))",
     "return float(np.sum((y - np.asarray(T, dtype=np.float64)) ** 2) / len(X))"),
    ("mlp_grad_no_mean", "dy = (y - np.asarray(T, dtype=np.float64)) / n", "dy = y - np.asarray(T, dtype=np.float64)"),
    ("mlp_grad_mask_layer", "dz2 = (dy @ w[\"W3\"]) * (z2 > 0)", "dz2 = (dy @ w[\"W3\"]) * (z1 > 0)"),
    ("mlp_grad_W1_input", "g[\"W1\"], g[\"b1\"] = dz1.T @ X, dz1.sum(axis=0)",
     "g[\"W1\"], g[\"b1\"] = dz1.T @ X, dz2.sum(axis=0)"),
    ("mlp_grad_W2_operand", "g[\"W2\"], g[\"b2\"] = dz2.T @ a1", "g[\"W2\"], g[\"b2\"] = dz2.T @ z1"),
    ("mlp_adam_second_moment_bias", "vh = v / (1 - b2 ** t)", "vh = v / (1 - b2)"),
    ("mlp_adam_first_moment_bias", "mh = m / (1 - b1 ** t)", "mh = m"),
    ("mlp_adam_sqrt", "np.sqrt(vh) + eps", "vh + eps"),
    ("mlp_adam_decay", "m = b1 * m + (1 - b1) * g", "m = b1 * m + g"),
    ("mlp_adam_sign", "return p - lr * mh", "return p + lr * mh"),
]

# loop-level PDE oracle (oracle/physics_loops.py), pinned bit for bit to the whole-step
# functions by the "equals" tests of test_physics_loops.py
LOOP_MUTANTS = [
    ("loops_euler_pressure_term", "p = (gamma - 1.0) * (E - 0.5 * (mx * u + my * v))",
     "p = (gamma - 1.0) * (E - 0.5 * (mx * u))"),
    ("loops_euler_flux_pressure", "Fv = (mx, mx * u + p, mx * v, (E + p) * u)", "Fv = (mx, mx * u, mx * v, (E + p) * u)"),
    ("loops_euler_pred_sign", "(U - lx * dF) - ly * dG", "(U - lx * dF) + ly * dG"),
    ("loops_euler_corr_d4", "((m2 - 4.0 * m1) + 6.0 * U)", "((m2 - 4.0 * m1) + 5.0 * U)"),
    ("loops_euler_corr_backward", "_get(g[8 + c], lo, hi, (-1, 0))", "_get(g[8 + c], lo, hi, (1, 0))"),
    ("loops_euler_corr_state", "first = (U + S) if mode == 0.0", "first = (S + S) if mode == 0.0"),
    ("loops_euler_dt_gamma", "c = np.sqrt(gamma * p / rho)", "c = np.sqrt(p / rho)"),
    ("loops_ns_temperature", "T = gamma * Ma * Ma * p / rho", "T = Ma * Ma * p / rho"),
    ("loops_ns_divergence", "div = (D[0] + D[4]) + D[8]", "div = D[0] + D[4]"),
    ("loops_ns_heat_flux_sign", "- kc * D[9 + a]", "+ kc * D[9 + a]"),
    ("loops_d1_coefficient", "((fm2 - 8.0 * fm1) + (8.0 * fp1 - fp2)) / (12.0 * h)",
     "((fm2 - 6.0 * fm1) + (6.0 * fp1 - fp2)) / (12.0 * h)"),
    ("loops_rk_register", "Acoef * _get(out, lo, hi) + dt * r", "_get(out, lo, hi) + dt * r"),
    ("loops_rk_update", "_get(g[m], lo, hi) + B * _get(g[5 + m], lo, hi)", "_get(g[m], lo, hi) + _get(g[5 + m], lo, hi)"),
    ("loops_fast_axis_wrap", "r = np.mod(r, f.size[a])", "r = np.clip(r, 0, f.size[a] - 1)"),
    ("loops_ghost_rows", "f.a[r] = f.a[(y % n) + h0]", "f.a[r] = f.a[min(max(y, 0), n - 1) + h0]"),
]

_PY_RUNNER = """
import importlib.util, sys
sys.path[:0] = [{root!r}, {tests!r}]
import oracle
spec = importlib.util.spec_from_file_location("oracle.{mod}", {path!r})
mod = importlib.util.module_from_spec(spec)
spec.loader.exec_module(mod)
sys.modules["oracle.{mod}"] = mod
setattr(oracle, {mod!r}, mod)
import pytest
sys.exit(pytest.main({pins!r} + ["-x", "-q", "-p", "no:cacheprovider", "-m", "not gpu"]))
"""

PY_PINS = {"mlp": ["tests/test_oracle_mlp.py"], "physics_loops": ["tests/test_physics_loops.py", "-k", "equals"]}


def _run_py_pins(tmp, module, old, new):
    """Run the pins of the numpy oracle module `module` with a mutated copy standing in
    for it."""
    text = open(os.path.join(ORACLE, module + ".py")).read()
    if old:
        assert text.count(old) == 1, f"mutant text must occur once in {module}.py: {old!r}"
        text = text.replace(old, new)
    path = os.path.join(tmp, module + "_mutant.py")
    with open(path, "w") as fh:
        fh.write(text)
    code = _PY_RUNNER.format(root=ROOT, tests=os.path.join(ROOT, "tests"), mod=module, path=path,
                             pins=PY_PINS[module])
    return subprocess.run([sys.executable, "-c", code], cwd=ROOT, capture_output=True, text=True, timeout=600)


def _run_mlp_pins(tmp, old, new):
    return _run_py_pins(tmp, "mlp", old, new)


def _run_loop_pins(tmp, old, new):
    return _run_py_pins(tmp, "physics_loops", old, new)


def _build_mutant(tmp, fname, old, new):
    srcs = []
    for f in ("oracle.c", "physics.c"):
        text = open(os.path.join(ORACLE, f)).read()
        if f == fname:
            assert text.count(old) == 1, f"mutant text must occur once in {f}: {old!r}"
            text = text.replace(old, new)
        path = os.path.join(tmp, f)
        with open(path, "w") as fh:
            fh.write(text)
        srcs.append(path)
    so = os.path.join(tmp, "liboracle_mutant.so")
    subprocess.run(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
                    "-fno-fast-math", "-o", so] + srcs + ["-lm"], check=True)
    return so


def _run_pins(pins, lib):
    env = dict(os.environ, ORACLE_LIB=lib, OMP_NUM_THREADS="1")
    return subprocess.run([sys.executable, "-m", "pytest", pins, "-x", "-q", "-p", "no:cacheprovider",
                           "-m", "not gpu"], cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)


def _c_case(tmp, fname, old, new):
    so = _build_mutant(tmp, fname, old, new)
    files = [PINS[fname]] if fname else sorted(set(PINS.values()))
    rcs, out = [], ""
    for pins in files:
        r = _run_pins(pins, so)
        rcs.append(r.returncode)
        out += r.stdout[-1500:]
    return max(rcs), out


@pytest.fixture(scope="module")
def outcomes(tmp_path_factory):
    """(exit status, output tail) of every case, keyed by id; the cases are independent
    subprocesses and run concurrently."""
    jobs = {"c_unmutated": (_c_case, "", "", ""), "mlp_unmutated": (_run_mlp_pins, "", ""),
            "loops_unmutated": (_run_loop_pins, "", "")}
    for mid, old, new in LOOP_MUTANTS:
        jobs[mid] = (_run_loop_pins, old, new)
    for mid, fname, old, new in MUTANTS:
        jobs[mid] = (_c_case, fname, old, new)
    for mid, old, new in MLP_MUTANTS:
        jobs[mid] = (_run_mlp_pins, old, new)

    base = tmp_path_factory.mktemp("mutants")

    def run(item):
        mid, (fn, *args) = item
        tmp = os.path.join(str(base), mid)
        os.makedirs(tmp)
        r = fn(tmp, *args)
        return mid, (r if isinstance(r, tuple) else (r.returncode, r.stdout[-1500:]))

    with cf.ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 2)) as ex:
        return dict(ex.map(run, jobs.items()))


def test_unmutated_copies_pass_the_pins(outcomes):
    """The harness itself: the unchanged sources, built and loaded the same way, pass
    every pin."""
    for mid in ("c_unmutated", "mlp_unmutated", "loops_unmutated"):
        rc, out = outcomes[mid]
        assert rc == 0, out


@pytest.mark.parametrize("mid", [m[0] for m in MUTANTS] + [m[0] for m in MLP_MUTANTS] + [m[0] for m in LOOP_MUTANTS])
def test_pins_catch_mutant(outcomes, mid):
    rc, out = outcomes[mid]
    # exit status 1: a test failed (not a collection or usage error)
    assert rc == 1, f"mutant {mid} survived the pins:\n{out}"
