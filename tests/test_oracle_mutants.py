"""Planted mistakes in the oracle.

Each entry below is a plausible slip in oracle/pc_oracle.c -- a dropped term,
a wrong sign, factor or index, a transposed operand, a step applied on the
wrong side -- written into a copy of the source, which is compiled on its own.
The oracle's independent pins (closed forms, finite differences, library
least squares and eigenvalues, brute-force windows and minimisation, the
values the paper prints for its synthetic objects) must fail on every copy;
the stored snapshot of the oracle's own output is left out, since it was
written by the oracle itself and would catch any change.  The unchanged source
built the same way must pass them (the control)."""
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "pc_oracle.c")
PINS = ["tests/test_oracle_pins.py", "tests/test_oracle_outputs.py",
        "tests/test_oracle_golden.py::test_table1_synthetic_expected_values"]

# name: (text of the source, the slip written in its place)
MUTANTS = {
    # step 1, back-projection (Sec. 3.2)
    "backproject_y_over_fx": ("P[1] = ((double)v - p->cy) * z / p->fy;",
                              "P[1] = ((double)v - p->cy) * z / p->fx;"),
    "backproject_without_cx": ("P[0] = ((double)u - p->cx) * z / p->fx;",
                               "P[0] = ((double)u) * z / p->fx;"),
    # step 2, initial normal (Sec. 3.2.1)
    "normal_sign_of_b": ("n[0] = -a * s; n[1] = -b * s; n[2] = s;",
                         "n[0] = -a * s; n[1] = b * s; n[2] = s;"),
    "normal_inverse_transposed": ("const double a = (m11 * v0s - m01 * v1s) / det;",
                                  "const double a = (m00 * v0s - m01 * v1s) / det;"),
    "normal_mean_over_n_minus_1": ("const double mx = sx / cnt, my = sy / cnt, mz = sz / cnt;",
                                   "const double mx = sx / (cnt - 1), my = sy / cnt, mz = sz / cnt;"),
    # step 3, frame (Sec. 3.2.2)
    "frame_rotates_the_wrong_way": ("const double w[3] = {n[1], -n[0], 0.0};",
                                    "const double w[3] = {-n[1], n[0], 0.0};"),
    "rotation_exp_sign_of_sine": ("R[i] += s * K[i] + c1 * K2[i];",
                                  "R[i] += -s * K[i] + c1 * K2[i];"),
    # step 4, residual (Sec. 3.1.2, Eq. quad and error_func)
    "quadric_without_half_on_A": ("Q[0] = A / 2.0;  Q[1] = B / 2.0;",
                                  "Q[0] = A;  Q[1] = B / 2.0;"),
    "offset_sign": ("E[4 * 2 + 3] = tz;", "E[4 * 2 + 3] = -tz;"),
    # step 5, Jacobian (Sec. 3.2.3)
    "jacobian_rotation_without_2": ("j[a] = 2.0 * dot4(QEp, dEp);", "j[a] = dot4(QEp, dEp);"),
    "jacobian_B_one_sided": ("if (q == 1) { dQ[1] = 0.5; dQ[4] = 0.5; }", "if (q == 1) { dQ[1] = 0.5; }"),
    # step 6, weights (Eq. weighting_function)
    "weight_of_abs_eps": ("return p->k / (p->k + e2);", "return p->k / (p->k + fabs(eps));"),
    "rejection_strict": ("if (p->reject && !(e2 <= p->reject_ratio * mse)) return 0.0;",
                         "if (p->reject && !(e2 < p->reject_ratio * mse)) return 0.0;"),
    # step 7, normal equations, solve and update (Eq. iter_reweighted_update)
    "normal_matrix_diagonal_only": ("N[6 * a + c] += ji[a] * w * ji[c];", "N[6 * a + c] += ji[a] * w * ji[a];"),
    "rhs_without_jacobian": ("rhs[a] += ji[a] * w * eps[i];", "rhs[a] += w * eps[i];"),
    "forward_substitution_transposed": ("for (int k = 0; k < i; k++) s -= L[6 * i + k] * z[k];",
                                        "for (int k = 0; k < i; k++) s -= L[6 * k + i] * z[k];"),
    "solution_not_unscaled": ("for (int i = 0; i < 6; i++) b[i] = D[i] * y[i];",
                              "for (int i = 0; i < 6; i++) b[i] = y[i];"),
    "update_sign_of_A": ("*A -= b[3];", "*A += b[3];"),
    "rotation_update_on_the_right": ("mat3_mul(Rd, R, Rn);", "mat3_mul(R, Rd, Rn);"),
    # step 8, principal curvatures (Sec. 3.1.2)
    "principal_order_swapped": ("*k1 = T1 + T2;\n    *k2 = T1 - T2;", "*k1 = T1 - T2;\n    *k2 = T1 + T2;"),
    "principal_without_B": ("const double T2 = sqrt(h * h + B * B);", "const double T2 = sqrt(h * h);"),
    # window and p'
    "window_without_centre": ("const int u = u0 + du, v = v0 + dv;\n            if (u < 0",
                              "const int u = u0 + du, v = v0 + dv;\n            if (du == 0 && dv == 0) continue;\n"
                              "            if (u < 0"),
    "window_stride_start": ("for (int dv = -(r / s) * s; dv <= r; dv += s)", "for (int dv = -r; dv <= r; dv += s)"),
    "points_not_centred": ("for (int c = 0; c < 3; c++) pts[3 * i + c] = Pi[c] - P0[c];",
                           "for (int c = 0; c < 3; c++) pts[3 * i + c] = Pi[c];"),
    # step 9, refined normal (Sec. 3.2.4)
    "refined_normal_from_row_1": ("res->normal[0] = R[6]; res->normal[1] = R[7]; res->normal[2] = R[8];",
                                  "res->normal[0] = R[3]; res->normal[1] = R[4]; res->normal[2] = R[5];"),
}


def _build(src_text, where):
    os.makedirs(where, exist_ok=True)
    c = os.path.join(where, "pc_oracle_copy.c")
    so = os.path.join(where, "liboracle_copy.so")
    with open(c, "w") as f:
        f.write(src_text)
    subprocess.run(["gcc", "-O2", "-std=c99", "-ffp-contract=off", "-fPIC", "-shared", "-D_DEFAULT_SOURCE",
                    c, "-o", so, "-lm"], check=True, capture_output=True)
    return so


def _run_pins(lib):
    env = dict(os.environ, PC_ORACLE_LIB=lib)
    return subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider", *PINS],
                          cwd=ROOT, env=env, capture_output=True, text=True, timeout=900)


@pytest.fixture(scope="module")
def source():
    if shutil.which("gcc") is None:
        pytest.skip("gcc is needed to build the planted copies")
    with open(SRC) as f:
        return f.read()


@pytest.fixture(scope="module")
def outcomes(source, tmp_path_factory):
    """Builds the control and every planted copy and runs the pins on each,
    several at a time (separate processes); name -> completed pytest run."""
    from concurrent.futures import ThreadPoolExecutor
    base = str(tmp_path_factory.mktemp("planted"))
    jobs = {"control": source}
    for name, (old, new) in MUTANTS.items():
        assert source.count(old) == 1, f"{name}: the text to replace must occur exactly once"
        jobs[name] = source.replace(old, new)

    def one(item):
        name, text = item
        return name, _run_pins(_build(text, os.path.join(base, name)))

    with ThreadPoolExecutor(max_workers=max(1, min(8, os.cpu_count() or 1))) as ex:
        return dict(ex.map(one, jobs.items()))


def test_control_copy_passes_the_pins(outcomes):
    r = outcomes["control"]
    assert r.returncode == 0, r.stdout[-3000:]


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_catch_planted_mistake(outcomes, name):
    r = outcomes[name]
    # pytest exits 1 when tests ran and some failed
    assert r.returncode == 1, f"{name} was not caught by any pin:\n{r.stdout[-3000:]}"
