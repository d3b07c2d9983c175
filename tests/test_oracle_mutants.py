"""Planted mistakes: each test compiles a copy of the oracle with one
plausible error (a dropped term, a wrong sign, a transposed operand, a wrong
constant) and checks that the pins of the named test file fail against it.
The identity copy must pass, so failures come from the planted mistake.
CPU only; the mistakes live only in temporary copies."""
import os
import subprocess
import sys
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "vbd_oracle.c")

# (name, text in vbd_oracle.c, replacement, pin file that must catch it)
MUTANTS = [
    ("hessian_skew_sign", "cross3(gl, gk, gx);", "cross3(gk, gl, gx);", "test_oracle_element.py"),
    ("hessian_drops_lambda_cc", "+ lam * ck[r] * cl[s]", "", "test_oracle_element.py"),
    ("alpha_one", "1.0 + mu / lam", "1.0", "test_oracle_element.py"),
    ("lame_without_mu_shift", "E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu)) + *mu;",
     "E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu));", "test_oracle_element.py"),
    ("F_uses_B_transposed", "acc += Ds[r * 3 + a] * B[a * 3 + s];", "acc += Ds[r * 3 + a] * B[s * 3 + a];",
     "test_oracle_element.py"),
    ("mass_over_three", "density[j] * m->V[j] / 4.0", "density[j] * m->V[j] / 3.0", "test_oracle_element.py"),
    ("inertia_gravity_sign", "+ h * h * p->gravity[r];", "- h * h * p->gravity[r];", "test_oracle_solver.py"),
    ("adaptive_clamp_top", "if (a_ext_comp > gnorm) atil = 1.0;", "if (a_ext_comp > gnorm) atil = 0.0;",
     "test_oracle_solver.py"),
    ("chebyshev_omega2_sign", "2.0 / (2.0 - rho * rho)", "2.0 / (2.0 + rho * rho)", "test_oracle_solver.py"),
    ("chebyshev_no_collision_skip", "if (n >= 2 && !m->pinned[i] && !coll[i])", "if (n >= 2 && !m->pinned[i])",
     "test_oracle_solver.py"),
    ("velocity_times_h", "double vn = (x[q] - xt[q]) / h;", "double vn = (x[q] - xt[q]) * h;",
     "test_oracle_solver.py"),
    ("contact_force_sign", "f[r] += p->k_c * d * nh[k][r];", "f[r] -= p->k_c * d * nh[k][r];",
     "test_oracle_solver.py"),
    ("damping_force_sign", "f[r] -= p->k_d / h * Hel[r * 3 + s]", "f[r] += p->k_d / h * Hel[r * 3 + s]",
     "test_oracle_solver.py"),
    ("colouring_tie_break", "return (i > j) - (i < j);\n}\n\n/* Returns", "return (i < j) - (i > j);\n}\n\n/* Returns",
     "test_oracle_solver.py"),
    ("friction_pushes_along_motion", "f[r] -= c * ut[r];", "f[r] += c * ut[r];", "test_oracle_friction.py"),
    ("line_search_accepts_increase", "<= G0) ok = 1;", ">= G0) ok = 1;", "test_oracle_variants.py"),
    ("self_contact_corner_force_sign", "f[r] -= p->k_c * d * wk * nn[r];", "f[r] += p->k_c * d * wk * nn[r];",
     "test_oracle_collision.py"),
    ("self_contact_corner_drops_weight", "double wk = w[corner];", "double wk = 1.0;", "test_oracle_collision.py"),
    ("self_contact_corner_hessian_linear_weight", "p->k_c * wk * wk * nn[r] * nn[c]", "p->k_c * wk * nn[r] * nn[c]",
     "test_oracle_collision.py"),
    ("closest_point_unclamped_edge", "if (tt > 1.0) tt = 1.0;", "", "test_oracle_collision.py"),
    ("inside_test_counts_own_tets", "if (t[0] == a || t[1] == a || t[2] == a || t[3] == a) continue;", "",
     "test_oracle_collision.py"),
    ("inside_test_sign", "if (l < 0.0) return 0;", "if (l > 0.0) return 0;", "test_oracle_collision.py"),
    ("self_friction_corner_unweighted", "x, xt, -wk, f, H);", "x, xt, -1.0, f, H);", "test_oracle_collision.py"),
    ("self_friction_relative_motion_sign", "dlt[r] -= w[k] * (x[3 * v[k] + r]", "dlt[r] += w[k] * (x[3 * v[k] + r]",
     "test_oracle_collision.py"),
    ("wall_offset_sign", "c[k++] = n[3];", "c[k++] = -n[3];", "test_oracle_walls.py"),
    ("wall_normal_not_normalised", "for (int r = 0; r < 3; ++r) nh[k][r] = n[r] / nn;",
     "for (int r = 0; r < 3; ++r) nh[k][r] = n[r];", "test_oracle_walls.py"),
    ("walls_skip_the_last", "for (int w = 0; w < p->n_walls && w < ORC_MAX_WALLS; ++w)",
     "for (int w = 0; w + 1 < p->n_walls && w < ORC_MAX_WALLS; ++w)", "test_oracle_walls.py"),
    ("wall_friction_first_normal", "plane_friction(p, h, nh[k], x + 3 * i", "plane_friction(p, h, nh[0], x + 3 * i",
     "test_oracle_walls.py"),
    ("wall_energy_dropped",
     "    for (int k = 0; k < np; ++k) {\n        double d = c[k] - dot3(x + 3 * i, nh[k]);\n"
     "        if (d > 0.0) G += 0.5",
     "    for (int k = 0; k < 0; ++k) {\n        double d = c[k] - dot3(x + 3 * i, nh[k]);\n"
     "        if (d > 0.0) G += 0.5",
     "test_oracle_walls.py"),
    ("subspace_guess_not_projected", "        if (m->sub_dim[i] < 3) {\n            /* a subspace-constrained",
     "        if (0) {\n            /* a subspace-constrained", "test_oracle_subspace.py"),
    ("subspace_rhs_first_axis", "b[a] = dot3(q + 3 * a, f);", "b[a] = dot3(q, f);", "test_oracle_subspace.py"),
    ("subspace_step_first_axis_only",
     "    for (int a = 0; a < L; ++a)\n        for (int r = 0; r < 3; ++r) dx[r] +=",
     "    for (int a = 0; a < 1; ++a)\n        for (int r = 0; r < 3; ++r) dx[r] +=", "test_oracle_subspace.py"),
    ("subspace_2x2_solve_sign", "dz[1] = (A[0] * b[1] - A[2] * b[0]) / det;",
     "dz[1] = (A[0] * b[1] + A[2] * b[0]) / det;", "test_oracle_subspace.py"),
    ("plane_basis_not_orthogonalised", "for (int r = 0; r < 3; ++r) e[r] -= en * d[r];", "",
     "test_oracle_subspace.py"),
    ("ccd_cubic_term_dropped", "cross3(A[1], B[2], tmp); c[1] += dot3(A[0], tmp);", "", "test_oracle_ccd.py"),
    ("ccd_inside_test_two_weights", "if (w[0] >= 0.0 && w[1] >= 0.0 && w[2] >= 0.0) return t;",
     "if (w[0] >= 0.0 && w[1] >= 0.0) return t;", "test_oracle_ccd.py"),
    ("ccd_latest_impact_wins", "if (t >= 0.0 && t < best - 1e-5) {",
     "if (t >= 0.0 && (best > 1.5 || t > best + 1e-5)) {", "test_oracle_ccd.py"),
    ("ccd_pair_uses_nearest_point", "    if (m->contact_ccd[a]) {\n        /* CCD pair",
     "    if (0) {\n        /* CCD pair", "test_oracle_ccd.py"),
    ("ee_crossing_parameters_swapped", "double s = dot3(wg, n) / nn, u = dot3(we, n) / nn;",
     "double s = dot3(we, n) / nn, u = dot3(wg, n) / nn;", "test_oracle_ccd.py"),
    ("ee_depth_weights_sign", "c[0] = -(1.0 - s); c[1] = -s; c[2] = 1.0 - u; c[3] = u;",
     "c[0] = 1.0 - s; c[1] = s; c[2] = -(1.0 - u); c[3] = -u;", "test_oracle_ccd.py"),
    ("ee_pair_not_carried", "if (ee_depth(m, e, x, v, c) > 0.0) m->ee_carried[e] = 1;", "if (0) m->ee_carried[e] = 1;",
     "test_oracle_ccd.py"),
    ("ee_crossing_test_one_segment", "if (s >= 0.0 && s <= 1.0 && u >= 0.0 && u <= 1.0) {",
     "if (s >= 0.0 && s <= 1.0) {", "test_oracle_ccd.py"),
    ("ee_parallel_threshold_loosened", "if (nn > 0.01 * dot3(e, e) * dot3(g, g)) {",
     "if (nn > 0.0001 * dot3(e, e) * dot3(g, g)) {", "test_oracle_ccd.py"),
]


def _run_pins(src_text, pin_file):
    with tempfile.TemporaryDirectory() as tmp:
        c = os.path.join(tmp, "vbd_oracle.c")
        with open(c, "w") as f:
            f.write(src_text)
        lib = os.path.join(tmp, "libmutant.so")
        subprocess.check_call(["gcc", "-std=c99", "-O2", "-fPIC", "-shared", "-fno-fast-math",
                               "-ffp-contract=off", "-I", os.path.join(ROOT, "oracle"), "-o", lib, c, "-lm"])
        env = dict(os.environ, VBD_ORACLE_LIB=lib)
        res = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                              os.path.join(ROOT, "tests", pin_file)], env=env, cwd=ROOT,
                             capture_output=True, text=True, timeout=600)
        return res.returncode


def test_identity_copy_passes():
    src = open(SRC).read()
    for pin in ("test_oracle_element.py", "test_oracle_solver.py", "test_oracle_collision.py",
                "test_oracle_walls.py", "test_oracle_subspace.py", "test_oracle_ccd.py"):
        assert _run_pins(src, pin) == 0, pin


@pytest.mark.parametrize("name,old,new,pin", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_pins_catch_planted_mistake(name, old, new, pin):
    src = open(SRC).read()
    assert src.count(old) >= 1, "mutation target missing: %s" % name
    assert _run_pins(src.replace(old, new), pin) != 0, "%s was not caught by %s" % (name, pin)
