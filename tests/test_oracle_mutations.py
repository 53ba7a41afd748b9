"""Planted mistakes in a scratch copy of the oracle (CPU only): each must make
at least one oracle pin fail.  Shows that the pins constrain the dropped-term,
wrong-sign, wrong-index and transposed-operand errors they are meant to."""
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PINS = ["tests/test_oracle_coeffs.py", "tests/test_oracle_scheme.py", "tests/test_oracle_bruteforce.py",
        "tests/test_oracle_adi.py", "tests/test_oracle_refresh.py"]

MUTATIONS = {
    "cross_term_sign": ("- EXT(u, a + 1, b - 1, mx)\n                - EXT(u, a - 1, b + 1, mx)",
                        "+ EXT(u, a + 1, b - 1, mx)\n                - EXT(u, a - 1, b + 1, mx)"),
    "source_time_index": ("double tk = T + k * dt;\n            double sk",
                          "double tk = T + (k + 1) * dt;\n            double sk"),
    "upwind_direction": ("ux = nu > 0.0 ? (uc - uW) / g->dx : (uE - uc) / g->dx;",
                         "ux = nu < 0.0 ? (uc - uW) / g->dx : (uE - uc) / g->dx;"),
    "edge_weight_sign": ("e->gL[b + 1] = ((-0.5 - rx) * A[0]", "e->gL[b + 1] = ((-0.5 + rx) * A[0]"),
    "C0_dropped_term": ("- g->hy * g->hy * Uyy / 24.0", ""),
    "ghost_corner_order": ("for (int b = -1; b <= ny + 1; ++b) {\n        double gl",
                           "for (int b = 0; b <= ny; ++b) {\n        double gl"),
    "trapezoid_weight": ("double wb = (b == 0 || b == ny) ? 0.5 : 1.0;", "double wb = (b == 0) ? 0.5 : 1.0;"),
    "nu_sign": ("out[3] = Vxi - c_xi;", "out[3] = Vxi + c_xi;"),
    "jacobian_derivative": ("double Jeta = xab * yb + xa * ybb - xbb * ya - xb * yab;",
                            "double Jeta = xab * yb + xa * ybb + xbb * ya - xb * yab;"),
    "transposed_metric": ("double a[2] = { yb, -xb }, b[2] = { -ya, xa };",
                          "double a[2] = { yb, -xb }, b[2] = { -xa, ya };"),
    "periodic_wrap": ("return ((i % n) + n) % n;", "return i < 0 ? 0 : (i >= n ? n - 1 : i);"),
    "adi_mixed_dropped": ("+ h * (op_part(P, g, c, u, a, b, 1) + op_part(P, g, c, u, a, b, 2) + f);",
                          "+ h * (op_part(P, g, c, u, a, b, 1) + f);"),
    "adi_full_half_step": ("double h = 0.5 * dt;\n    double sm", "double h = dt;\n    double sm"),
    "adi_source_time": ("double sm = orc_time_factor(P, tk + h);", "double sm = orc_time_factor(P, tk);"),
    "adi_reaction_split": ("return c[0] * uxx - c[3] * ux + 0.5 * c[5] * uc;",
                           "return c[0] * uxx - c[3] * ux + c[5] * uc;"),
    "adi_eta_upwind": ("else uy = c[4] > 0.0 ? (uc - uS) / g->dy : (uN - uc) / g->dy;",
                       "else uy = c[4] < 0.0 ? (uc - uS) / g->dy : (uN - uc) / g->dy;"),
    "adi_line_ghost_sign": ("EXT(u, -1, line, g->mx) = EXT(u, 1, line, g->mx) - 2.0 * g->dx * gl;",
                            "EXT(u, -1, line, g->mx) = EXT(u, 1, line, g->mx) + 2.0 * g->dx * gl;"),
    "adi_explicit_direction": ("+ h * (op_part(P, g, c, u, a, b, 1) + op_part(P, g, c, u, a, b, 2) + f);",
                               "+ h * (op_part(P, g, c, u, a, b, 0) + op_part(P, g, c, u, a, b, 2) + f);"),
    "refresh_stale_estimate": ("V[g.j * nxp + g.i] = U[g.j * nxp + g.i] + dR[p];",
                               "V[g.j * nxp + g.i] = U[g.j * nxp + g.i];"),
    "refresh_boundary_time": ("orc_apply_bc(P, V, Tq);", "orc_apply_bc(P, V, T);"),
    "refresh_subburst_time": ("double tk = Tq + k * dt;\n                    fill_ghosts(&g, &eq, up, 0);",
                              "double tk = T + k * dt;\n                    fill_ghosts(&g, &eq, up, 0);"),
    "refresh_split_ghost_data": ("eq.gL[k] -= e0[p].gL[k]; eq.gR[k] -= e0[p].gR[k];",
                                 "eq.gR[k] -= e0[p].gR[k];"),
    "lift_bias_divisor": ("return (g->dx * g->dx * Uxx + g->dy * g->dy * Uyy) / 12.0;",
                          "return (g->dx * g->dx * Uxx + g->dy * g->dy * Uyy) / 6.0;"),
    "macro_rate_cross_dropped": ("+ fabs(c[1]) / (g.Dx * g.Dy) + fabs(c[3]) / g.Dx", "+ fabs(c[3]) / g.Dx"),
    "micro_rate_reaction_dropped": ("+ fabs(c[1]) / (hx * hy) + fabs(c[5]);", "+ fabs(c[1]) / (hx * hy);"),
    "project_boundary_time": ("+ dtm * F;\n    }\n    orc_apply_bc(P, U, t + dtm);", "+ dtm * F;\n    }\n    orc_apply_bc(P, U, t);"),
    "tanh_map_curvature_sign": ("*X2 = -2.0 * s * s * sech2 * th / (T * L);", "*X2 = 2.0 * s * s * sech2 * th / (T * L);"),
    "radial_curvature_factor": ("rho2 = -4.0 * sr * sr * sech2 * th / T;", "rho2 = -2.0 * sr * sr * sech2 * th / T;"),
    "source_amplitude_index": ("P->src_amp[p] : 1.0;", "P->src_amp[0] : 1.0;"),
    "sine_map_curvature_sign": ("o[6] = -lam * M_PI * sin(M_PI * xi);", "o[6] = lam * M_PI * sin(M_PI * xi);"),
    "mms_cross_term_dropped": (" + 2.0 * M_PI * M_PI * ph[1] * cx * cy;", ";"),
    "mms_reaction_sign": ("+ (ph[11] - ph[12]) * S;", "+ (ph[12] - ph[11]) * S;"),
    "mms_convection_swapped": ("M_PI * (ph[9] * cx * sy + ph[10] * sx * cy)", "M_PI * (ph[10] * cx * sy + ph[9] * sx * cy)"),
    "sin_diffusivity_gradient": ("gx += P->ds * k2 * cos(k2 * x) * sy;", "gx += P->ds * k2 * cos(k2 * y) * sy;"),
    "fourier_diffusivity_gradient": ("gx += ck * (ct * A * dB - st / r * dA * B);", "gx += ck * (ct * A * dB + st / r * dA * B);"),
    "velocity_divergence_index": ("o[11] = P->va[1] + P->vb[2];", "o[11] = P->va[1] + P->vb[1];"),
    "time_factor_sin_cos": ("case ORC_TIME_SIN: return sin(P->tc * t);", "case ORC_TIME_SIN: return cos(P->tc * t);"),
    "lift_cross_factor": ("+ 0.5 * (s * s * Uxx + 2.0 * s * t * Uxy + t * t * Uyy);",
                          "+ 0.5 * (s * s * Uxx + s * t * Uxy + t * t * Uyy);"),
    "lift_eta_slope_operand": ("double Uy = (S[1][2] - S[1][0]) / (2.0 * g->Dy);",
                               "double Uy = (S[2][1] - S[0][1]) / (2.0 * g->Dy);"),
    "edge_top_middle_sign": ("e->gT[a + 1] = ((-0.5 + ry) * B[0] - 2.0 * ry * B[1]", "e->gT[a + 1] = ((-0.5 + ry) * B[0] + 2.0 * ry * B[1]"),
    "edge_row_offset": ("double t = -0.5 * g->hy + b * g->dy;\n        double A[3];",
                        "double t = 0.5 * g->hy + b * g->dy;\n        double A[3];"),
    "ghost_top_sign": ("EXT(u, a, ny + 1, g->mx) = EXT(u, a, ny - 1, g->mx) + 2.0 * g->dy * gt;",
                       "EXT(u, a, ny + 1, g->mx) = EXT(u, a, ny - 1, g->mx) - 2.0 * g->dy * gt;"),
    "lagrange_node": ("double nodes[3] = { -D, 0.0, D };", "double nodes[3] = { -D, 0.0, 2.0 * D };"),
    "sampled_patch_index": ("dU[s] = run_patch(P, U, sel[s], c, t, P->k_micro, dt, form, NULL);",
                            "dU[s] = run_patch(P, U, s, c, t, P->k_micro, dt, form, NULL);"),
    "refresh_macro_bias_omitted": ("            if (P->restrict_mode == ORC_RESTRICT_MACRO) d += lift_trapezoid_bias(&g, &e0[p]);\n"
                                   "            U[g.j * nxp + g.i] = U[g.j * nxp + g.i] + dtm * (d / tau);",
                                   "            U[g.j * nxp + g.i] = U[g.j * nxp + g.i] + dtm * (d / tau);"),
    "boundary_top_row_dropped": ("int bnd = (j == 0 || j == ny - 1) || (!P->periodic_xi && (i == 0 || i == nx - 1));\n            if (!bnd) continue;",
                                 "int bnd = (j == 0) || (!P->periodic_xi && (i == 0 || i == nx - 1));\n            if (!bnd) continue;"),
    "boundary_periodic_sides_set": ("int bnd = (j == 0 || j == ny - 1) || (!P->periodic_xi && (i == 0 || i == nx - 1));\n            if (!bnd) continue;",
                                    "int bnd = (j == 0 || j == ny - 1) || (i == 0 || i == nx - 1);\n            if (!bnd) continue;"),
    "bump_periodic_factor": ("double fx = P->periodic_xi ? (1.0 + 0.5 * cos(xi)) : sin(M_PI * zx);",
                             "double fx = P->periodic_xi ? (1.0 + 0.5 * sin(xi)) : sin(M_PI * zx);"),
    "bump_eta_factor": ("val = fx * sin(M_PI * zy);", "val = fx * sin(M_PI * zy * 0.5);"),
    "manufactured_solution_growth": ("case ORC_SOL_SINPROD_DECAY: return exp(-t) * sin(M_PI * x) * sin(M_PI * y);",
                                     "case ORC_SOL_SINPROD_DECAY: return exp(t) * sin(M_PI * x) * sin(M_PI * y);"),
    "gauss_source_width": ("return exp(-(x * x + y * y));", "return exp(-0.5 * (x * x + y * y));"),
    "fourier_radial_frequency": ("double B = cos(k * M_PI * rho), dB = -k * M_PI * sin(k * M_PI * rho) / (rb - ra);",
                                 "double B = cos(k * M_PI * rho * 0.5), dB = -0.5 * k * M_PI * sin(k * M_PI * rho * 0.5) / (rb - ra);"),
    "fourier_phase_sign": ("double A = cos(k * th + ph), dA = -k * sin(k * th + ph);",
                           "double A = cos(k * th - ph), dA = -k * sin(k * th - ph);"),
    "adi_xi_central_scale": ("if (P->conv == ORC_CONV_CENTRAL) ux = (uE - uW) / (2.0 * g->dx);\n        else ux = c[3]",
                             "if (P->conv == ORC_CONV_CENTRAL) ux = (uE - uW) / g->dx;\n        else ux = c[3]"),
    "projection_tau": ("U[g.j * nx + g.i] = U[g.j * nx + g.i] + dtm * (dU[p] / tau);",
                       "U[g.j * nx + g.i] = U[g.j * nx + g.i] + dtm * dU[p];"),
}

# mistakes in the initial fields and the full-domain solver, caught by pins of
# the convergence file (run by node id: the rest of that file is slow)
CONV_PINS = ["tests/test_oracle_convergence.py::test_bessel_roots_match_scipy",
             "tests/test_oracle_convergence.py::test_bessel_mode_field_solves_the_heat_equation",
             "tests/test_oracle_convergence.py::test_full_domain_step_is_exact_on_quadratics",
             "tests/test_oracle_convergence.py::test_annulus_initial_data_of_section_4_2",
             "tests/test_oracle_convergence.py::test_paper_table7_annulus"]
MUTATIONS_CONV = {
    "bessel_angular_factor": ("* orc_bessel_Z(k, mu[k - 1], prm[1], r) * cos(k * th)",
                              "* orc_bessel_Z(k, mu[k - 1], prm[1], r) * sin(k * th)"),
    "bessel_decay_diffusivity": ("* exp(-P->d0 * mu[k - 1] * mu[k - 1] * t);", "* exp(-mu[k - 1] * mu[k - 1] * t);"),
    "annulus_initial_angular_factor": ("val = (r - prm[0]) * (prm[1] - r) * sin(th);",
                                       "val = (r - prm[0]) * (prm[1] - r) * cos(th);"),
    "full_domain_cross_sign": ("double uxy = (uNE - uSE - uNW + uSW) / (4.0 * hx * hy);",
                               "double uxy = (uNE - uSE + uNW + uSW) / (4.0 * hx * hy);"),
    "full_domain_source_time": ("double st = orc_time_factor(P, t);", "double st = orc_time_factor(P, t + dt);"),
    "bessel_root_index": ("if (++found == which) {", "if (++found == which + 1) {"),
    "full_domain_boundary_time": ("un[o] = orc_exact(P, m[0], m[1], tn);", "un[o] = orc_exact(P, m[0], m[1], tn - dt);"),
}


def _caught(tmp_path, name, old, new, pins):
    src = open(os.path.join(ROOT, "oracle", "pd_oracle.c")).read()
    assert old in src, "mutation anchor missing: " + name
    d = tmp_path / name
    d.mkdir()
    (d / "pd_oracle.c").write_text(src.replace(old, new, 1))
    shutil.copy(os.path.join(ROOT, "oracle", "pd_oracle.h"), d)
    so = str(d / "lib.so")
    subprocess.run(["gcc", "-O2", "-std=c11", "-D_DEFAULT_SOURCE", "-ffp-contract=off", "-fopenmp",
                    "-fPIC", "-shared", "-o", so, str(d / "pd_oracle.c"), "-lm"], check=True)
    env = dict(os.environ, ORC_SO_OVERRIDE=so)
    r = subprocess.run([sys.executable, "-m", "pytest", "-q", "-x", "-p", "no:cacheprovider"] + pins,
                       cwd=ROOT, env=env, capture_output=True, text=True)
    assert r.returncode != 0, "planted mistake %s passed every pin:\n%s" % (name, r.stdout[-2000:])


@pytest.mark.parametrize("name", sorted(MUTATIONS_CONV))
def test_planted_mistake_in_fields_or_full_domain_is_caught(tmp_path, name):
    old, new = MUTATIONS_CONV[name]
    _caught(tmp_path, name, old, new, CONV_PINS)


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_planted_mistake_is_caught(tmp_path, name):
    old, new = MUTATIONS[name]
    _caught(tmp_path, name, old, new, PINS)
