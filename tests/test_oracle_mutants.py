"""The pins are strong enough: each plausible mistake, planted in a copy of
the oracle source and compiled on the CPU, makes at least one pin fail.

The mistakes are ones a reader of the paper could make: the other quad
diagonal (Eq. 3), a signed or halved Jacobian (Eq. 4), the barycentric roles
swapped when mapping back to uv (Eq. 5), the footprint covariance or
normalisation wrong, the printed "+" of Eq. 11's line term, the "d_x"
projection cosine of App. B, a reversed arc, a wrong clip root (Alg. 1) and a
misplaced per-triangle kernel sample, and a collapsed normal triangle
treated as a point at its centroid.  For the cluster hierarchy (Eq. 7-8,
App. A): the other cluster diagonal or hat functions, an unweighted fit, the
squared residual, a cluster Jacobian without its 2^(2l) scale, swapped
barycentric roles or corners, and a cut on the wrong footprint size.  For
the disk and box kernels: a 3-sigma disk, the box sheared by the upper
Cholesky factor, and the box normalised as a unit square.  For the Eq. 6
clamp and sampling: a replacement of area eps, a Jacobian of eps / 2, an
untruncated sampling radius, a transposed Cholesky factor and the other
diagonal for the sample's triangle.  For the GGX fit (Eq. 12): the printed
form without its parentheses, a wrong fit observation, a halved cross term
and a box filter normalised by the side instead of the area.
"""

import os

import pytest

import oracle
import test_oracle_cluster as cpins  # noqa: E402
import test_oracle_pins as pins  # noqa: E402

SRC = os.path.join(os.path.dirname(oracle.__file__), "pndf_oracle.c")

PNDF_PINS = [pins.test_affine_closed_form, pins.test_mass_invariant, pins.test_binning_converges,
             pins.test_transpose_symmetry]
AREA_PINS = [pins.test_stokes_matches_area_quadrature, pins.test_projarea_normal_incidence_is_shoelace,
             pins.test_projarea_uv_form, pins.test_projarea_uv_form_collapsed_triangles]


def cluster_dense_fit_level3(m):
    cpins.test_fit_matches_dense_least_squares(m, 3, 1, 1)


def cluster_mass_all_cut(m):
    cpins.test_cluster_mass_invariant(m, 1e9)


def cluster_mass_mixed(m):
    cpins.test_cluster_mass_invariant(m, "mixed")


def affine_disk(m):
    pins.test_affine_closed_form_disk_box(m, 1)


def affine_box(m):
    pins.test_affine_closed_form_disk_box(m, 2)


def mass_disk(m):
    pins.test_mass_invariant_disk_box(m, 1)


def mass_box(m):
    pins.test_mass_invariant_disk_box(m, 2)


KERNEL_PINS = [affine_disk, affine_box, mass_disk, mass_box, pins.test_binning_box_kernel]

import test_oracle_sampling as spins  # noqa: E402


def samples_on_triangles(m):
    spins.test_samples_lie_on_their_triangles(m, 0)


SAMPLING_PINS = [spins.test_clamp_keeps_the_mass_of_flat_triangles, spins.test_sample_frequencies_follow_the_kernel,
                 samples_on_triangles, spins.test_binned_samples_match_clamped_pndf]

import test_oracle_ggx as gpins  # noqa: E402


def ggx_node_P_0p3(m):
    gpins.test_node_P_matches_uv_quadrature(m, 0.3)


GGX_PINS = [gpins.test_fit_recovers_a_ggx_omega, gpins.test_flat_map_has_zero_omega, ggx_node_P_0p3,
            gpins.test_lambda_is_ggx_smith_for_isotropic_omega, gpins.test_interpolation_properties,
            gpins.test_shadow_masking_flat_and_backfacing]

CLUSTER_PINS = [cpins.test_fit_recovers_piecewise_linear_data, cluster_dense_fit_level3, cluster_mass_all_cut,
                cluster_mass_mixed, cpins.test_cluster_binning_with_anisotropic_cut,
                cpins.test_cluster_transpose_symmetry, cpins.test_piecewise_linear_map_is_unchanged_by_any_cut]

MUTANTS = {
    "other_diagonal": (
        [("ax = i; ay = j; bx = i + 1; by = j; cx = i; cy = j + 1;\n                    na = n0; nb = n1; nc = n2;",
          "ax = i; ay = j; bx = i + 1; by = j; cx = i + 1; cy = j + 1;\n                    na = n0; nb = n1; nc = n3;"),
         ("ax = i + 1; ay = j + 1; bx = i; by = j + 1; cx = i + 1; cy = j;\n                    na = n3; nb = n2; nc = n1;",
          "ax = i + 1; ay = j + 1; bx = i; by = j + 1; cx = i; cy = j;\n                    na = n3; nb = n2; nc = n0;")],
        PNDF_PINS),
    "signed_jacobian": ([("double J = fabs(A2);", "double J = A2;")], PNDF_PINS),
    "area_not_twice_area": ([("D += norm * exp(-0.5 * q) / J;", "D += norm * exp(-0.5 * q) / (0.5 * J);")], PNDF_PINS),
    "bary_roles_swapped": ([("double ux = ax * l0 + bx * l1 + cx * l2;", "double ux = ax * l0 + bx * l2 + cx * l1;"),
                            ("double uy = ay * l0 + by * l1 + cy * l2;", "double uy = ay * l0 + by * l2 + cy * l1;")],
                           PNDF_PINS),
    "inverse_cov_sign": ([("double ia = syy / det, ib = -sxy / det, ic = sxx / det;\n    double norm = 1.0 / (2.0 * M_PI * sqrt(det));\n    int i0, i1, j0, j1;\n    quad_range(N, x, y, sxx, syy, &i0, &i1, &j0, &j1);\n    double D = 0.0;",
                           "double ia = syy / det, ib = sxy / det, ic = sxx / det;\n    double norm = 1.0 / (2.0 * M_PI * sqrt(det));\n    int i0, i1, j0, j1;\n    quad_range(N, x, y, sxx, syy, &i0, &i1, &j0, &j1);\n    double D = 0.0;")],
                         PNDF_PINS),
    "kernel_missing_2pi": ([("double norm = 1.0 / (2.0 * M_PI * sqrt(det));\n    int i0, i1, j0, j1;\n    quad_range(N, x, y, sxx, syy, &i0, &i1, &j0, &j1);\n    double D = 0.0;",
                             "double norm = 1.0 / (sqrt(det));\n    int i0, i1, j0, j1;\n    quad_range(N, x, y, sxx, syy, &i0, &i1, &j0, &j1);\n    double D = 0.0;")],
                           PNDF_PINS),
    "line_term_plus_sign": ([("return tz - tx;", "return tz + tx;")], AREA_PINS),
    "projection_cosine_dx": ([("double tx = 0.5 * wx * r2 * dy *", "double tx = 0.5 * wx * r2 * dx *")], AREA_PINS),
    "arc_reversed": ([("return 0.5 * (Fasin(e[1]) - Fasin(s[1]));", "return 0.5 * (Fasin(s[1]) - Fasin(e[1]));")],
                     AREA_PINS),
    "clip_start_uses_t1": ([("oa[0] = a[0] * (1.0 - t0) + b[0] * t0;\n            oa[1] = a[1] * (1.0 - t0) + b[1] * t0;",
                             "oa[0] = a[0] * (1.0 - t1) + b[0] * t1;\n            oa[1] = a[1] * (1.0 - t1) + b[1] * t1;")],
                           AREA_PINS),
    "collapsed_as_centroid_point": ([("P += k * collapsed_uv_form(a, b, cc, w, c, s, gl_x, gl_w, ngl);",
                                      "P += k * 0.5 * visible_cos_ratio((a[0] + b[0] + cc[0]) / 3.0, "
                                      "(a[1] + b[1] + cc[1]) / 3.0, w);")], AREA_PINS),
    "kernel_at_wrong_centroid": ([("double gx = i + (tri == 0 ? 1.0 / 3.0 : 2.0 / 3.0) - x;",
                                   "double gx = i + (tri == 0 ? 2.0 / 3.0 : 1.0 / 3.0) - x;")], AREA_PINS),
    # disk and box footprint kernels
    "disk_radius_3_sigma": ([("return q <= 2.25 ? 1.0 / (2.25 * M_PI * sqrt(det)) : 0.0;",
                              "return q <= 9.0 ? 1.0 / (2.25 * M_PI * sqrt(det)) : 0.0;")], KERNEL_PINS),
    "box_upper_cholesky": ([("double v1 = dx / l11, v2 = (dy - l21 * v1) / l22;",
                             "double v2 = dy / l11, v1 = (dx - l21 * v2) / l22;")], KERNEL_PINS),
    "box_norm_unit_square": ([("return vm <= 1.5 ? 1.0 / (9.0 * sqrt(det)) : 0.0;",
                               "return vm <= 1.5 ? 1.0 / (4.0 * sqrt(det)) : 0.0;")], KERNEL_PINS),
    # Jacobian clamp (Eq. 6) and sampling
    "eqtri_area_eps": ([("double side = sqrt(2.0 * eps / sqrt(3.0));", "double side = sqrt(4.0 * eps / sqrt(3.0));")],
                       SAMPLING_PINS),
    "clamp_jacobian_half_eps": ([("if (jac_eps > 0.0 && J < jac_eps) J = jac_eps;",
                                  "if (jac_eps > 0.0 && J < jac_eps) J = 0.5 * jac_eps;")], SAMPLING_PINS),
    "sampler_untruncated": ([("sqrt(-2.0 * log(1.0 - u1 * (1.0 - exp(-8.0))))", "sqrt(-2.0 * log(1.0 - u1))")],
                            SAMPLING_PINS),
    "sampler_cholesky_transposed": ([("double ux = x + l11 * v1, uy = y + l21 * v1 + l22 * v2;",
                                      "double ux = x + l11 * v1 + l21 * v2, uy = y + l22 * v2;")], SAMPLING_PINS),
    "sampler_other_diagonal": ([("int tri = fu + fv < 1.0 ? 0 : 1;", "int tri = fu < fv ? 0 : 1;")], SAMPLING_PINS),
    # GGX projected-area fit per mip node (Eq. 12) and shadow-masking
    "ggx_printed_parentheses": ([("return 0.5 * (w[2] + sqrt(fmax(w[2] * w[2] + q, 0.0)));",
                                  "return 0.5 * w[2] + sqrt(fmax(w[2] * w[2] + q, 0.0));")], GGX_PINS),
    "ggx_fit_observation": ([("double ak = t * t - wz * wz;", "double ak = 4.0 * P[k] * P[k] - wz * wz;")], GGX_PINS),
    "ggx_fit_cross_term": ([("double row[3] = {wx * wx, 2.0 * wx * wy, wy * wy};",
                             "double row[3] = {wx * wx, wx * wy, wy * wy};")], GGX_PINS),
    "ggx_box_area": ([("for (int k = 0; k < K; ++k) P[k] /= (double)a * (double)a;",
                       "for (int k = 0; k < K; ++k) P[k] /= (double)a;")], GGX_PINS),
    # cluster hierarchy (Eq. 7-8, App. A) and the tau cut
    "cluster_fit_main_diagonal": ([("        phi[0] = 1.0 - s - t; phi[1] = s; phi[2] = t; phi[3] = 0.0;",
                                    "        phi[0] = 1.0 - s; phi[1] = s - t; phi[2] = 0.0; phi[3] = t;"),
                                   ("        phi[0] = 0.0; phi[1] = 1.0 - t; phi[2] = 1.0 - s; phi[3] = s + t - 1.0;",
                                    "        phi[0] = 1.0 - t; phi[1] = 0.0; phi[2] = t - s; phi[3] = s;"),
                                   ("int upper = cs + ct > 1.0;", "int upper = ct > cs;")], CLUSTER_PINS),
    "cluster_fit_upper_hats_swapped": ([("phi[0] = 0.0; phi[1] = 1.0 - t; phi[2] = 1.0 - s;",
                                         "phi[0] = 0.0; phi[1] = 1.0 - s; phi[2] = 1.0 - t;")], CLUSTER_PINS),
    "cluster_fit_unweighted": ([("double w = (0.5 / 3.0) / fmax(cr, ORACLE_JAC_EPS);", "double w = (0.5 / 3.0);")],
                               CLUSTER_PINS),
    "cluster_residual_squared": ([("*e = sqrt(mf.F);", "*e = mf.F;")], CLUSTER_PINS),
    "cluster_jacobian_unscaled": ([("double J = fabs(A2) / (scale * scale);", "double J = fabs(A2);")], CLUSTER_PINS),
    "cluster_uv_roles_swapped": ([("double ux = uv[0][0] * l0 + uv[1][0] * l1 + uv[2][0] * l2;",
                                   "double ux = uv[0][0] * l0 + uv[1][0] * l2 + uv[2][0] * l1;"),
                                  ("double uy = uv[0][1] * l0 + uv[1][1] * l1 + uv[2][1] * l2;",
                                   "double uy = uv[0][1] * l0 + uv[1][1] * l2 + uv[2][1] * l1;")], CLUSTER_PINS),
    "cluster_upper_corners_swapped": ([("double nv1[3][2] = {{c[6], c[7]}, {c[4], c[5]}, {c[2], c[3]}};",
                                        "double nv1[3][2] = {{c[6], c[7]}, {c[2], c[3]}, {c[4], c[5]}};")],
                                      CLUSTER_PINS),
    "cut_on_max_radius": ([("Q.theta = Q.rx * Q.ry * tau;", "Q.theta = fmax(Q.rx, Q.ry) * fmax(Q.rx, Q.ry) * tau;")],
                          CLUSTER_PINS),
}


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(name, tmp_path):
    edits, which = MUTANTS[name]
    src = open(SRC).read()
    for old, new in edits:
        assert src.count(old) == 1, (name, old)
        src = src.replace(old, new)
    path = tmp_path / f"{name}.c"
    path.write_text(src)
    mutant = oracle.Oracle(oracle.build(force=True, src=str(path), out=str(tmp_path / f"{name}.so")))
    caught = []
    for pin in which:
        try:
            pin(mutant)
        except AssertionError:
            caught.append(pin.__name__)
    assert caught, f"no pin caught mutant {name}"
