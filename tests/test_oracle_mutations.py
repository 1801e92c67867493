"""Mutation check of the oracle's pins: each case plants one plausible mistake (a wrong coefficient, sign,
index or spacing) in a copy of the oracle's C source, compiles it, and runs the pins meant to catch it
against that copy in a separate process; every planted mistake must make them fail, and the unmodified
copy must pass the same pins. The mistakes are planted in the oracle only, on the CPU."""
import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

# (name, source file, text, planted text, test file, pins (pytest -k))
MUTATIONS = [
    ("linear_weight", "hydro_oracle.c", "double a0 = 0.1 / (", "double a0 = 0.2 / (", "test_oracle_pins.py",
     "linear_weights_are_the_textbook_ones or weno5_matches_first_principles"),
    ("indicator_coefficient", "hydro_oracle.c", "double beta1 = 13.0 / 12.0 *", "double beta1 = 13.0 / 11.0 *",
     "test_oracle_pins.py", "weno5_matches_first_principles"),
    ("candidate_value", "hydro_oracle.c", "q[1] = (-b + 5.0 * c + 2.0 * d) / 6.0;",
     "q[1] = (-b + 5.0 * c + 2.0 * d) / 5.0;", "test_oracle_pins.py", "weno5_exact_for_quadratics_and_odd"),
    ("split_sign", "hydro_oracle.c", "fm[cc * m + k] = 0.5 * (F[cc] - alpha * Uc[cc]);",
     "fm[cc * m + k] = 0.5 * (F[cc] + alpha * Uc[cc]);", "test_oracle_pins.py", "cylindrical_divergence_closed_form"),
    ("geometric_source_index", "hydro_oracle.c", "S[2] = -(mx * v) / r;", "S[2] = -(mx * u) / r;",
     "test_oracle_pins.py", "cylindrical_divergence_closed_form"),
    ("gravity_work_term", "hydro_oracle.c", "S[3] += my * c->gravity;", "S[3] += mx * c->gravity;",
     "test_oracle_pins.py", "moving_gravity_source_closed_form"),
    ("rk3_stage_weights", "hydro_oracle.c", "U2[k] = 0.75 * U[k] + 0.25 * (U1[k] + dt * L[k]);",
     "U2[k] = 0.7 * U[k] + 0.3 * (U1[k] + dt * L[k]);", "test_oracle_pins.py", "third_order_in_time"),
    ("cfl_spacing", "hydro_oracle.c", "*dt = c->cfl * (dx < dy ? dx : dy) / s;",
     "*dt = c->cfl * (dx > dy ? dx : dy) / s;", "test_oracle_pins.py", "alpha_and_dt_on_a_designed_state"),
    ("flame_direction", "hydro_oracle.c", "double H = (u * gx + v * gy) - sf * sqrt(gx * gx + gy * gy);",
     "double H = (u * gx + v * gy) + sf * sqrt(gx * gx + gy * gy);", "test_oracle_pins.py",
     "level_set_plane_front_moves_at_flame_speed"),
    ("totals_radius", "hydro_oracle.c", "two_pi * (c->x0 + (i + 0.5) * dx) * dx * dy",
     "two_pi * (c->x0 + (i + 1.0) * dx) * dx * dy", "test_oracle_pins.py", "totals_closed_forms"),
    ("front_point_spacing", "hydro_oracle_reinit.inc", "px[m] = xa + dx * (a / (a - b));",
     "px[m] = xa + dy * (a / (a - b));", "test_oracle_reinit.py", "tilted_front_on_unequal_spacing"),
    ("poisson_east_west", "hydro_oracle_poisson.inc", "aE = rp / (r * dr * dr), aW = rm / (r * dr * dr)",
     "aE = rm / (r * dr * dr), aW = rp / (r * dr * dr)", "test_oracle_poisson.py", "uniform_sphere_potential"),
    ("poisson_mirror_mass", "hydro_oracle_poisson.inc", "const double M = zsym ? 2.0 * mass : mass;",
     "const double M = mass;", "test_oracle_poisson.py", "reflecting_plane_matches_mirrored_full_domain"),
    ("roe_average_weights", "hydro_oracle_char.inc", "const double un = (s[0] * vn[0] + s[1] * vn[1]) / den;",
     "const double un = (s[1] * vn[0] + s[0] * vn[1]) / den;", "test_oracle_char.py", "roe_eigen_system"),
    ("left_eigenvector_sign", "hydro_oracle_char.inc", "{1.0 - b2, b1 * un, b1 * ut, -b1},",
     "{1.0 + b2, b1 * un, b1 * ut, -b1},", "test_oracle_char.py", "roe_eigen_system"),
    ("adjoint_indicator_derivative", "hydro_oracle_adjoint.inc", "const double dbeta = 13.0 / 6.0 * sk[k]",
     "const double dbeta = 13.0 / 12.0 * sk[k]", "test_oracle_adjoint.py", "weno5_gradient_matches_finite_differences"),
    ("adjoint_gravity_term", "hydro_oracle_adjoint.inc", "g[0] += c->gravity * mu[2 * n + k];",
     "g[0] += c->gravity * mu[3 * n + k];", "test_oracle_adjoint.py", "rhs_adjoint_dot_product"),
    ("blend_offset", "hydro_oracle_reinit.inc", "const double d0 = 3.0 * delta, w = delta / 3.0;",
     "const double d0 = 2.0 * delta, w = delta / 3.0;", "test_oracle_reinit.py", "blend_weight_properties"),
    ("rk5_coefficient", "hydro_oracle.c", "{0.0, 0.0, 0.16352294089771, 0.0, 0.0},",
     "{0.0, 0.0, 0.16552294089771, 0.0, 0.0},", "test_oracle_pins.py", "five_stage_scheme_third_order_in_time"),
    ("roche_sign", "hydro_oracle_poisson.inc", "{ return -grav_const * M / sqrt(r * r + z * z); }",
     "{ return grav_const * M / sqrt(r * r + z * z); }", "test_oracle_poisson.py", "uniform_sphere_potential"),
]


def _copy(dst, mutation=None):
    shutil.copytree(os.path.join(ROOT, "oracle"), os.path.join(dst, "oracle"),
                    ignore=shutil.ignore_patterns("_build", "__pycache__"))
    if mutation:
        _, fname, old, new, _, _ = mutation
        path = os.path.join(dst, "oracle", fname)
        src = open(path).read()
        assert src.count(old) == 1, (fname, old)
        open(path, "w").write(src.replace(old, new))
    # the copy must compile: a planted mistake is wrong arithmetic, not broken code
    env = dict(os.environ, PYTHONPATH=ROOT)
    r = subprocess.run([sys.executable, "-c", "import oracle, sys; oracle.build(); print(oracle.__file__)"],
                       cwd=dst, env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    assert r.stdout.strip().startswith(os.path.join(dst, "oracle")), r.stdout  # the copy, not the tree's


def _pins(dst, testfile, kexpr):
    env = dict(os.environ, PYTHONPATH=ROOT, OMP_NUM_THREADS="2")
    return subprocess.run([sys.executable, "-m", "pytest", os.path.join(ROOT, "tests", testfile), "-q", "-x",
                           "-k", kexpr, "-m", "not gpu", "-p", "no:cacheprovider"],
                          cwd=dst, env=env, capture_output=True, text=True, timeout=600)


def test_every_planted_mistake_fails_a_pin(tmp_path):
    base = str(tmp_path / "base")
    os.makedirs(base)
    _copy(base)

    def run(mutation):
        d = str(tmp_path / mutation[0])
        os.makedirs(d)
        _copy(d, mutation)
        clean = _pins(base, mutation[4], mutation[5])
        planted = _pins(d, mutation[4], mutation[5])
        return mutation[0], clean, planted

    with cf.ThreadPoolExecutor(max_workers=4) as ex:
        results = list(ex.map(run, MUTATIONS))
    for name, clean, planted in results:
        assert clean.returncode == 0, (name, clean.stdout[-1500:])
        assert "passed" in clean.stdout and " 0 passed" not in clean.stdout, (name, clean.stdout[-500:])
        assert planted.returncode == 1 and "failed" in planted.stdout, (name, planted.stdout[-1500:])
