"""Planted mistakes: each plausible slip in the oracle must make a pin fail.

Every case copies ``oracle/elbm_oracle.c`` into a temporary directory, plants
one mistake (a dropped term, a flipped sign, a wrong set, a transposed operand,
a wrong constant), rebuilds it there and runs the pin tests named for it against
the mutated copy.  The case passes only if those pins FAIL.  Nothing here touches
a GPU; the committed oracle is never modified.
"""
import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "elbm_oracle.c")

P = "tests/test_oracle_pins.py"
F = "tests/test_oracle_field.py"
A = "tests/test_oracle_adjoint.py"

# name: (original text, planted text, pins expected to catch it)
MUTANTS = {
    "a_drops_h3_term": ("h * h * beta * beta * x3 * xi * xi / 20.0 -",
                        "h * h * beta * beta * x3 * xi * xi / 20.0 - 0.0 *",
                        [P + "::test_H_theorem_alpha_higher"]),
    "a_x4_sign": ("x3 / 6.0 - h * beta * x3 * xi / 12.0", "x3 / 6.0 + h * beta * x3 * xi / 12.0",
                  [P + "::test_quadratic_bounds_sextic_and_root_order"]),
    "b_omega_plus_sign": ("b -= f[i] * (2.0 * aL", "b += f[i] * (2.0 * aL",
                          [P + "::test_coefficients_from_quadratures"]),
    "b_denominator_without_beta": ("double k = (b_variant == 1) ? aL : aL * beta;", "double k = aL;",
                                   [P + "::test_coefficients_from_quadratures"]),
    "c_denominator_coefficient": ("60.0 + 90.0 * xi + 36.0 * xi * xi",
                                  "60.0 + 90.0 * xi + 30.0 * xi * xi",
                                  [P + "::test_coefficients_from_quadratures"]),
    "c1_denominator_sign": ("2.0 * x[i] * x[i] / (2.0 + x[i])", "2.0 * x[i] * x[i] / (2.0 - x[i])",
                            [P + "::test_coefficients_from_quadratures"]),
    "a1_wrong_set": ("if (x[i] < 0.0) a1 +=", "if (x[i] > 0.0) a1 +=",
                     [P + "::test_lower_order_split_identity"]),
    "a2_beta_power": ("a2 *= beta * beta;", "a2 *= beta;",
                      [P + "::test_quadratic_bounds_sextic_and_root_order"]),
    "root_discriminant_sign": ("return 2.0 * c / (b + sqrt(b * b - 4.0 * a * c));",
                               "return 2.0 * c / (b + sqrt(b * b + 4.0 * a * c));",
                               [P + "::test_quadratic_bounds_sextic_and_root_order"]),
    "weights": ("{1.0 / 6.0, 4.0 / 6.0, 1.0 / 6.0}", "{1.0 / 6.0, 2.0 / 3.0 + 1e-9, 1.0 / 6.0}",
                [P + "::test_weight_moment_conditions"]),
    "z_denominator_sign": ("(2.0 * u[a] + s) / (1.0 - u[a])", "(2.0 * u[a] + s) / (1.0 + u[a])",
                           [P + "::test_equilibrium_has_the_prescribed_moments"]),
    "upsilon_sign": ("Y[a] = 2.0 - s;", "Y[a] = 2.0 + s - 2.0 * s * s + 1.0;",
                     [P + "::test_equilibrium_has_the_prescribed_moments"]),
    "stream_direction": ("or_wrap(xx - c[i * D + 0], nx);\n                    int64_t sy = or_wrap(y - c[i * D + 1], ny);\n"
                         "                    int64_t sz = (D == 3) ? or_wrap(z - c[i * D + 2], nz) : 0;\n"
                         "                    fout",
                         "or_wrap(xx + c[i * D + 0], nx);\n                    int64_t sy = or_wrap(y - c[i * D + 1], ny);\n"
                         "                    int64_t sz = (D == 3) ? or_wrap(z - c[i * D + 2], nz) : 0;\n"
                         "                    fout",
                         [F + "::test_stream_moves_along_velocity"]),
    "clamp_rule": ("r.alpha = (1.0 + r.alpha_max) / 2.0;", "r.alpha = r.alpha_max;",
                   [P + "::test_positivity_clamp"]),
    "relax_drops_beta": ("fstar[i] = f[i] + alpha * beta * (feq[i] - f[i]);",
                         "fstar[i] = f[i] + alpha * (feq[i] - f[i]);",
                         [P + "::test_deltaH_closed_form_matches_direct_difference"]),
    "cutoff_threshold": ("r.xabsmax < OR_CUTOFF", "r.xabsmax <= 2e-3",
                         [P + "::test_cutoff_and_equilibrium"]),
    "newton_derivative": ("s += f[i] * x[i] * (log1p(alpha * x[i]) - log1p(x[i]));",
                          "s += f[i] * x[i] * (log1p(alpha * x[i]) - log1p(x[i])) * 1.5;",
                          [P + "::test_alpha_elbm_is_mirror_root"]),
    "g_series_sign": ("((k % 2 == 0) ? 1.0 : -1.0)", "((k % 2 == 0) ? 1.0 : 1.0)",
                      [P + "::test_d1q2_mirror_root_is_two"]),
    "moments_velocity_index": ("m[a] += f[i] * c[i * D + a];", "m[a] += f[i] * c[i * D + (D - 1 - a)];",
                               [P + "::test_equilibrium_has_the_prescribed_moments"]),
    "force_not_divided_by_rho": ("v[a] = u[a] + force[a] / rho;", "v[a] = u[a] + force[a];",
                                 [A + "::test_force_term_moments"]),
    "force_sign": ("f[i] += feq1[i] - feq0[i];", "f[i] += feq0[i] - feq1[i];",
                   [A + "::test_uniform_flow_accelerates_linearly"]),
    "entropy_drops_minus_one": ("H += f[i] * (log(f[i] / w[i]) - 1.0);", "H += f[i] * log(f[i] / w[i]);",
                                [P + "::test_H_of_uniform_rest_states"]),
    "iterate1_newton_sign": ("return alpha_lower - or_F(Q, f, x, alpha_lower) / or_dF(Q, f, x, alpha_lower);",
                             "return alpha_lower + or_F(Q, f, x, alpha_lower) / or_dF(Q, f, x, alpha_lower);",
                             [P + "::test_iterate1_and_table3_magnitudes"]),
    "kinetic_energy_half": ("L += 0.5 * rho * uu;", "L += rho * uu;",
                            [A + "::test_kinetic_energy_of_uniform_flows"]),
    "adjoint_push_direction": ("g_t[(int64_t)i * N + (sz * ny + sy) * nx + sx] = h[i];",
                               "g_t[(int64_t)i * N + n] = h[i];",
                               [A + "::test_step_adjoint_transpose_identity"]),
}


def _run(name, tmp):
    old, new, targets = MUTANTS[name]
    src = open(SRC).read()
    assert src.count(old) == 1, f"{name}: anchor text not unique in the oracle"
    d = os.path.join(tmp, name)
    os.makedirs(os.path.join(d, "oracle"))
    open(os.path.join(d, "oracle", "elbm_oracle.c"), "w").write(src.replace(old, new))
    shutil.copy(os.path.join(ROOT, "oracle", "__init__.py"), os.path.join(d, "oracle", "__init__.py"))
    env = dict(os.environ, PYTHONPATH=d + os.pathsep + ROOT, OMP_NUM_THREADS="1")
    cmd = [sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider", "--rootdir", d,
           "-c", os.devnull] + [os.path.join(ROOT, t) for t in targets]
    r = subprocess.run(cmd, env=env, capture_output=True, text=True, cwd=d, timeout=300)
    return name, r.returncode, r.stdout[-2000:]


def test_every_planted_mistake_is_caught(tmp_path):
    with ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 2)) as ex:
        results = list(ex.map(lambda n: _run(n, str(tmp_path)), list(MUTANTS)))
    survived = [(n, out) for n, rc, out in results if rc != 1]
    assert not survived, "mutants not caught by their pins:\n" + "\n".join(
        f"--- {n}\n{out}" for n, out in survived)
