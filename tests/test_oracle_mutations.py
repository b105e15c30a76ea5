"""The pins must catch plausible mistakes in the oracle.

Each case plants one mistake in a copy of ``oracle/o3g_oracle.c`` (a dropped
term, a wrong sign, a transposed operand, a wrong index, a strict bound, a
wrong order), builds the copy on the CPU and runs the pins of
``test_oracle_pins.py`` that cover that part; at least one must fail.  The
committed oracle itself is untouched.
"""
from __future__ import annotations

import importlib.util
import os
import shutil

import pytest

import oracle
from tests import test_oracle_pins as pins

ORACLE_DIR = os.path.dirname(os.path.abspath(oracle.__file__))

# (name, text in o3g_oracle.c, planted replacement, pins to run: (function, params))
NN = [("test_nn_matches_numpy_bruteforce_bitexact", (257, 1000, 0.2, )),
      ("test_nn_matches_numpy_bruteforce_bitexact", (1500, 700, 0.5)),
      ("test_nn_radius_boundary_inclusive", ()), ("test_nn_golden_tiny", ())]
EQ = [("test_jacobian_matches_finite_differences", ()), ("test_normal_equations_equal_gauss_newton_of_fd_jacobian", ()),
      ("test_normal_equations_symmetric_psd_and_sign_invariant", ()), ("test_planar_closed_form_golden", ())]
SOLVE = [("test_ldlt_matches_numpy_solve_on_spd", ()), ("test_ldlt_frozen_pivot_solves_reduced_system", ()),
         ("test_one_gauss_newton_step_matches_lstsq", ())]
ICP = [("test_icp_recovers_known_transform_noise_free", ()), ("test_delta_T_is_intrinsic_zyx_euler", ()),
       ("test_one_gauss_newton_step_matches_lstsq", ())]
NRM = [("test_normals_on_sphere_are_radial_and_oriented", ()), ("test_normals_match_eigh_of_neighbour_covariance", ()),
       ("test_jacobi_matches_numpy_eigh", ())]
P2P = [("test_rigid_align_matches_svd_kabsch", (0.01, 10.0, 0.1)), ("test_icp_point_to_point_recovers_noise_free", ()),
       ("test_jacobi4_matches_numpy_eigh", ())]
VOX = [("test_voxel_downsample_matches_numpy_bitexact", (20000, 0.1, 1.0)), ("test_voxel_downsample_properties", ()),
       ("test_voxel_downsample_edge_cases", ())]
GRID = [("test_grid_nn_partners_at_the_radius_anywhere_in_a_cell", ()), ("test_grid_nn_on_a_lattice_at_the_radius", ()),
        ("test_grid_nn_equals_bruteforce_bitexact", (3000, 3000, 0.05, 1.0))]
EVAL = [("test_evaluate_poses_matches_independent_bruteforce", ())]
KNN = [("test_knn_matches_numpy_bruteforce", ()), ("test_knn_radius_boundary_and_ties", ())]

MUTATIONS = [
    ("nn tie keeps the last index", "if (best < 0 || d2 < best_d2) {", "if (best < 0 || d2 <= best_d2) {", NN),
    ("nn radius strict", "if (!(d2 <= c->r2)) continue;", "if (!(d2 < c->r2)) continue;", NN),
    ("nn distance drops dz", "return (dx * dx + dy * dy) + dz * dz;", "return (dx * dx + dy * dy);", NN),
    ("jacobian wrong sign", "J[1] = pz * nx - px * nz;", "J[1] = px * nz - pz * nx;", EQ),
    ("residual wrong sign", "double dx = px - (double)q[0], dy = py - (double)q[1], dz = pz - (double)q[2];",
     "double dx = (double)q[0] - px, dy = (double)q[1] - py, dz = (double)q[2] - pz;", EQ),
    ("J^T r dropped", "      b[a] += J[a] * r;", "      b[a] += 0.0 * r;", EQ),
    ("J^T J transposed operand", "A[6 * a + c] += J[a] * J[c];", "A[6 * a + c] += J[a] * J[a];", EQ),
    ("solve without the minus sign", "double v = -b[i];", "double v = b[i];", SOLVE),
    ("solve wrong L index", "v -= L[i][m] * L[k][m] * D[m];", "v -= L[i][m] * L[i][m] * D[m];", SOLVE),
    ("frozen pivot rule dropped", "frozen[k] = !(s > thr);", "frozen[k] = 0;", SOLVE),
    ("euler order swapped", "mat3_mul(Rz, RyRx, R);", "mat3_mul(RyRx, Rz, R);", ICP),
    ("update sin sign", "double Rx[9] = {1, 0, 0, 0, ca, -sa, 0, sa, ca};",
     "double Rx[9] = {1, 0, 0, 0, ca, sa, 0, -sa, ca};", ICP),
    ("covariance not divided", "for (int k = 0; k < 9; ++k) C[k] /= (double)m;",
     "for (int k = 0; k < 9; ++k) C[k] /= 1.0;", [("test_jacobi_matches_numpy_eigh", ()),
                                                   ("test_normals_match_eigh_of_neighbour_covariance", ())]),
    ("normal orientation flipped", "if (facing < 0.0)", "if (facing > 0.0)", NRM),
    ("jacobi rotation sign", "double theta = (a[3 * q + q] - a[3 * p + p]) / (2.0 * apq);",
     "double theta = (a[3 * p + p] - a[3 * q + q]) / (2.0 * apq);", NRM),
    ("horn uses the smallest eigenvalue", "if (ev[k] > ev[k1]) k1 = k;", "if (ev[k] < ev[k1]) k1 = k;", P2P),
    ("horn translation sign", "dT[4 * r + 3] = mq[r] - (R[3 * r]", "dT[4 * r + 3] = mq[r] + (R[3 * r]", P2P),
    ("voxel index rounds", "float q = floorf(p[d] / voxel);", "float q = roundf(p[d] / voxel);", VOX),
    ("voxel centroid off by one", "out[3 * nv + d] = (float)(s[d] / (double)(b - a));",
     "out[3 * nv + d] = (float)(s[d] / (double)(b - a + 1));", VOX),
    ("grid cell narrower than r", "g->inv_h = 1.0 / (1.01 * (double)r_max);",
     "g->inv_h = 1.0 / (0.999 * (double)r_max);", GRID),
    ("grid drops a neighbour layer", "for (int dz = -1; dz <= 1; ++dz)", "for (int dz = -1; dz <= 0; ++dz)", GRID),
    ("knn ties to the higher index", "  if (x->d2 > y->d2) return 1;\n  return (x->j > y->j) - (x->j < y->j);",
     "  if (x->d2 > y->d2) return 1;\n  return (x->j < y->j) - (x->j > y->j);", KNN),
    ("knn ordered by index only", "  if (x->d2 < y->d2) return -1;\n  if (x->d2 > y->d2) return 1;\n", "", KNN),
    ("knn radius strict", "      if (d2 <= c->r2) {\n        buf[m].d2 = d2;", "      if (d2 < c->r2) {\n        buf[m].d2 = d2;",
     KNN),
    ("knn keeps one too few", "int64_t keep = m < c->max_nn ? m : c->max_nn;",
     "int64_t keep = m < c->max_nn ? m : c->max_nn - 1;", KNN),
    ("evaluation counts unmatched", "    if (corr[i] >= 0) {\n        sum_d2 += (double)d2[i];\n        ++count;\n      }\n    out_count",
     "    if (corr[i] >= -1) {\n        sum_d2 += (double)d2[i];\n        ++count;\n      }\n    out_count", EVAL),
]


def _mutant(tmp_path, name, old, new):
    src = open(os.path.join(ORACLE_DIR, "o3g_oracle.c")).read()
    assert src.count(old) >= 1, f"mutation site not found: {name}"
    d = tmp_path / name.replace(" ", "_").replace("^", "")
    d.mkdir()
    (d / "o3g_oracle.c").write_text(src.replace(old, new, 1))
    shutil.copy(os.path.join(ORACLE_DIR, "__init__.py"), d / "__init__.py")
    spec = importlib.util.spec_from_file_location(f"oracle_mutant_{d.name}", d / "__init__.py",
                                                  submodule_search_locations=[str(d)])
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    mod.build(force=True)
    return mod


@pytest.mark.parametrize("name,old,new,checks", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_planted_mistake_fails_a_pin(tmp_path, name, old, new, checks):
    mod = _mutant(tmp_path, name, old, new)
    failed = []
    for fn, params in checks:
        try:
            getattr(pins, fn)(mod, *params)
        except Exception as e:  # an assertion, or the mutant rejecting its own input
            failed.append((fn, type(e).__name__))
    assert failed, f"no pin caught the planted mistake '{name}'"


def test_unmutated_copy_passes_the_same_pins(tmp_path):
    """Control: the harness itself does not make pins fail (an identical copy passes every check used above)."""
    mod = _mutant(tmp_path, "control", "if (facing < 0.0)", "if (facing < 0.0)")
    seen = set()
    for _, _, _, checks in MUTATIONS:
        for fn, params in checks:
            if (fn, params) in seen:
                continue
            seen.add((fn, params))
            getattr(pins, fn)(mod, *params)
