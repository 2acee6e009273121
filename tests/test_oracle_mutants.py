"""The oracle's pins must catch plausible mistakes.

Each case plants one mistake (a dropped term, a flipped sign, a wrong
exponent or coefficient, a transposed operand, a broken level or active-set
rule) in a COPY of the oracle's C source, builds it in a temporary directory
and runs the pin suite against it in a subprocess; the suite must fail.
Nothing here touches the real oracle or any GPU.
"""
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "nbody_oracle.c")

MUTANTS = {
    "jerk_drops_3dw_term": ("gm * (w[c] / s3 - 3.0 * dw * d[c] / s5)", "gm * (w[c] / s3)"),
    "jerk_wrong_coefficient": ("gm * (w[c] / s3 - 3.0 * dw * d[c] / s5)", "gm * (w[c] / s3 - 2.0 * dw * d[c] / s5)"),
    "separation_sign": ("double d[3], w[3];\n            for (int c = 0; c < 3; c++) {\n                d[c] = pos[3 * j + c] - pos[3 * i + c];",
                        "double d[3], w[3];\n            for (int c = 0; c < 3; c++) {\n                d[c] = pos[3 * i + c] - pos[3 * j + c];"),
    "velocity_transposed": ("w[c] = vel[3 * j + c] - vel[3 * i + c];\n            }\n            double s2",
                            "w[c] = vel[3 * i + c] - vel[3 * j + c];\n            }\n            double s2"),
    "force_exponent": ("double s3 = s2 * s;", "double s3 = s2;"),
    "softening_dropped": ("d[2] * d[2] + eps2;\n            double s = sqrt(s2);", "d[2] * d[2];\n            double s = sqrt(s2);"),
    "potential_sign": ("nsum_add(&p, -gm / s);", "nsum_add(&p, gm / s);"),
    "self_term_kept": ("if (j == i) continue;\n            double d[3], w[3];\n",
                       "if (j == i && eps == 0.0) continue;\n            double d[3], w[3];\n"),
    "predictor_jerk_coefficient": ("jerk[q] * t * t * t / 6.0", "jerk[q] * t * t * t / 2.0"),
    "predictor_velocity_term": ("vp[q] = vel[q] + acc[q] * t + jerk[q] * t * t / 2.0;", "vp[q] = vel[q] + acc[q] * t;"),
    "corrector_a2_swapped": ("t * (4.0 * j0[q] + 2.0 * j1[q])", "t * (2.0 * j0[q] + 4.0 * j1[q])"),
    "corrector_a3_coefficient": ("(12.0 * da + 6.0 * t * (j0[q] + j1[q]))", "(6.0 * da + 6.0 * t * (j0[q] + j1[q]))"),
    "corrector_x_term": ("a3 * t5 / 120.0", "a3 * t5 / 24.0"),
    "corrector_end_snap": ("a2_end[q] = a2 + a3 * t;", "a2_end[q] = a2;"),
    "aarseth_square_dropped": ("double num = na * n2 + nj * nj;", "double num = na * n2 + nj;"),
    "level_growth_unsynchronised": ("if (t_new_ticks % step2 == 0) return Ld;", "return Ld;"),
    "level_rounds_up": ("L = 1 - e;", "L = -e;"),
    "active_set_all": ("if (t[i] + ((int64_t)1 << (tick_exp - level[i])) == t_next)", "if (1)"),
    "tau_sign": ("tau[i] = ldexp((double)(t_next - t[i]), -tick_exp);", "tau[i] = ldexp((double)(t[i] - t_next), -tick_exp);"),
    "energy_pair_mass": ("nsum_add(&p, -G * mass[i] * mass[j] / s);", "nsum_add(&p, -G * mass[j] / s);"),
    "kinetic_factor": ("nsum_add(&k, 0.5 * mass[i] * v2);", "nsum_add(&k, mass[i] * v2);"),
    "angular_momentum_sign": ("(r[0] * v[1] - r[1] * v[0])", "(r[1] * v[0] - r[0] * v[1])"),
    "leapfrog_full_kick": ("const double h = 0.5 * dt;", "const double h = dt;"),
    "leapfrog_second_kick_dropped": ("""        oracle_force(n, pos, vel, mass, G, eps, n, idx, acc, NULL, NULL);
        oracle_kick(n, vel, acc, h);""", """        oracle_force(n, pos, vel, mass, G, eps, n, idx, acc, NULL, NULL);"""),
    "snap_alpha_coefficient": ("- 6.0 * alpha * J - 3.0 * beta * A", "- 3.0 * alpha * J - 3.0 * beta * A"),
    "snap_beta_without_alpha2": ("double beta = (ww + du) / s2 + alpha * alpha;", "double beta = (ww + du) / s2;"),
    "snap_target_acceleration_dropped": ("u[c] = acc_src[3 * j + c] - acc_src[3 * i + c];", "u[c] = acc_src[3 * j + c];"),
    "hermite6_corrector_h2_coefficient": ("- t2 / 10.0 * (j1[i] - j0[i])", "- t2 / 12.0 * (j1[i] - j0[i])"),
    "hermite6_crackle_coefficient": ("crackle[i] = (60.0 * D", "crackle[i] = (30.0 * D"),
    "hermite6_predictor_crackle_dropped": ("+ s[i] * h4 / 24.0 + c[i] * h5 / 120.0;", "+ s[i] * h4 / 24.0;"),
    "hermite6_predictor_acc_crackle_coefficient": ("ap[i] = a[i] + j[i] * h + s[i] * h2 / 2.0 + c[i] * h3 / 6.0;",
                                                   "ap[i] = a[i] + j[i] * h + s[i] * h2 / 2.0 + c[i] * h3 / 2.0;"),
    "hermite6_predictor_velocity_snap_dropped": ("vp[i] = v[i] + a[i] * h + j[i] * h2 / 2.0 + s[i] * h3 / 6.0",
                                                 "vp[i] = v[i] + a[i] * h + j[i] * h2 / 2.0"),
    "hermite6_dt_exponent": ("return eta * cbrt(A1 / A4);", "return eta * sqrt(A1 / A4);"),
    "leapfrog_drift_before_kick": ("""        oracle_kick(n, vel, acc, h);
        oracle_drift(n, pos, vel, dt);""", """        oracle_drift(n, pos, vel, dt);
        oracle_kick(n, vel, acc, h);"""),
}


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_catch_mutant(name, tmp_path):
    if shutil.which("gcc") is None:
        pytest.skip("gcc not available")
    old, new = MUTANTS[name]
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutation anchor not found once: {old!r}"
    mut = tmp_path / "oracle_mut.c"
    mut.write_text(src.replace(old, new))
    lib = tmp_path / "liboracle_mut.so"
    subprocess.run(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp",
                    "-ffp-contract=off", str(mut), "-o", str(lib), "-lm"], check=True)
    env = dict(os.environ, NBODY_ORACLE_LIB=str(lib), OMP_NUM_THREADS="2")
    # the stored-values check pins the oracle to its own earlier output, not
    # to an independent fact, so it does not count here
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                        "-k", "not stored_values",
                        os.path.join(ROOT, "tests", "test_oracle_pins.py")],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode != 0, f"mutant {name} survived the pins:\n{r.stdout[-2000:]}"
