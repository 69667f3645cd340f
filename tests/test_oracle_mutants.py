"""Plant plausible mistakes in copies of the oracle source and check that a pin fails.

Each mutant is one textual edit of oracle/pxst_oracle.c (a swapped weight, a wrong sign,
a transposed index, a dropped term, an off-by-one rounding, a changed tie-break); the copy
is compiled into a temporary directory and every pin is run against it. A mutant that no
pin catches means the pins leave that part of the oracle unchecked.
"""
import os
import subprocess

import pytest

import oracle
import pins

SRC = os.path.join(os.path.dirname(oracle.__file__), "pxst_oracle.c")

MUTANTS = {
    "weights_swapped": ("wt[1] = (1.0 - x) * y;\n    wt[2] = x * (1.0 - y);",
                        "wt[1] = x * (1.0 - y);\n    wt[2] = (1.0 - x) * y;"),
    "weight_uses_wrong_fraction": ("wt[3] = x * y;", "wt[3] = x * x;"),
    "scatter_adds_delta": ("const double a = u[p] - delta[2 * n + 0];",
                           "const double a = u[p] + delta[2 * n + 0];"),
    "scatter_transposed_delta": ("const double b = u[P + p] - delta[2 * n + 1];",
                                 "const double b = u[P + p] - delta[2 * n + 0];"),
    "scatter_den_not_squared": ("w[ii * Rx + jj] += wt[k] * m * Wv * Wv;",
                                "w[ii * Rx + jj] += wt[k] * m * Wv;"),
    "no_normalisation": ("Iref[c] = (w[c] > 0.0) ? Iref[c] / w[c] : 0.0;",
                         "Iref[c] = (w[c] > 0.0) ? Iref[c] : 0.0;"),
    "gather_not_renormalised": ("*out = num / den;", "*out = num;"),
    "gather_ignores_coverage": ("if (!(wc > 0.0)) continue;", "(void)wc;"),
    "candidate_adds_delta": ("double q0 = (double)(*ci + a) - c->delta[2 * n + 0];",
                             "double q0 = (double)(*ci + a) + c->delta[2 * n + 0];"),
    "error_without_whitefield": ("const double d = I - Wv * R;", "const double d = I - R;"),
    "var_dropped": ("var += v * v;", "var += 1.0;"),
    "centre_truncated": ("*ci = (int64_t)floor(c->u[p] + 0.5);", "*ci = (int64_t)floor(c->u[p]);"),
    "tie_break_last": ("if (e[k] < e[best]) best = k;", "if (e[k] <= e[best]) best = k;"),
    "fit_cross_term_sign": ("da = (-2.0 * c5 * c1 + c4 * c2) / det;",
                            "da = (-2.0 * c5 * c1 - c4 * c2) / det;"),
    "fit_curvature_wrong": ("double c3 = (a2 - 2.0 * (s - a2)) / 6.0;",
                            "double c3 = (a2 - 2.0 * (s - a2)) / 4.0;"),
    "fallback_parabola_sign": ("if (k > 0.0) db = (fm - fp) / (2.0 * k);",
                               "if (k > 0.0) db = (fp - fm) / (2.0 * k);"),
    "refterms_not_squared": ("t += R * R;", "t += R;"),
    "invalid_frame_counted": ("if (!pxst_oracle_gather(c->Iref, c->w, c->Ry, c->Rx, q0, q1, &R)) continue;",
                              "if (!pxst_oracle_gather(c->Iref, c->w, c->Ry, c->Rx, q0, q1, &R)) R = 0.0;"),
    "pixel_var_dropped": ("s2 += v * v;", "s2 += 1.0;"),
    "frac_step_halved": ("const double c0 = u0 + (double)a / sub, c1 = u1 + (double)b / sub;",
                         "const double c0 = u0 + (double)a / (2 * sub), c1 = u1 + (double)b / sub;"),
    "frac_adds_delta": ("if (!pxst_oracle_gather(Iref, w, Ry, Rx, c0 - delta[2 * n], c1 - delta[2 * n + 1], &R))",
                        "if (!pxst_oracle_gather(Iref, w, Ry, Rx, c0 + delta[2 * n], c1 - delta[2 * n + 1], &R))"),
    "contrast_not_normalised": ("return sqrt(s2 / (double)n) / mean;", "return sqrt(s2 / (double)n);"),
    "sweep_scale_inverted": ("us[p] = u[pc] + sy[ky] * (u[p] - u[pc]);", "us[p] = u[pc] + (u[p] - u[pc]) / sy[ky];"),
    "filter_unnormalised": ("u_out[p] = num0 / den;", "u_out[p] = num0;"),
    "filter_ignores_mask": ("if (!M[q]) continue;", "(void)q;"),
    "filter_width_halved": ("const double g = exp(-(double)(a * a + b * b) / (2.0 * sigma * sigma));",
                            "const double g = exp(-(double)(a * a + b * b) / (sigma * sigma));"),
    "error_not_normalised": ("const double eps = var > 0.0 ? d * d / var : d * d;", "const double eps = d * d;"),
    "error_plane_unnormalised": ("ref_err[c] = den[c] > 0.0 ? num[c] / den[c] : 0.0;",
                                 "ref_err[c] = den[c] > 0.0 ? num[c] : 0.0;"),
    "error_plane_adds_delta": ("const double q0 = u[p] - delta[2 * n], q1 = u[P + p] - delta[2 * n + 1];",
                               "const double q0 = u[p] + delta[2 * n], q1 = u[P + p] - delta[2 * n + 1];"),
    "translation_shift_sign": ("const double q0 = u[p] - (delta[2 * n] + a), q1 = u[P + p] - (delta[2 * n + 1] + b);",
                               "const double q0 = u[p] - (delta[2 * n] - a), q1 = u[P + p] - (delta[2 * n + 1] + b);"),
    "translation_sum_not_mean": ("e[(a + Ty) * wx + (b + Tx)] = cnt > 0 ? sum / (double)cnt : INFINITY;",
                                 "e[(a + Ty) * wx + (b + Tx)] = cnt > 0 ? sum : INFINITY;"),
    "translation_update_sign": ("delta_out[2 * n + 1] = delta_in[2 * n + 1] + (double)(ib - Tx) + db;",
                                "delta_out[2 * n + 1] = delta_in[2 * n + 1] - (double)(ib - Tx) + db;"),
    "integrate_central_not_halved": ("off[0] = 1; c[0] = 0.5; off[1] = -1; c[1] = -0.5; return 2;",
                                     "off[0] = 1; c[0] = 1.0; off[1] = -1; c[1] = -1.0; return 2;"),
    "integrate_second_order_wrong": ("off[0] = 0; c[0] = -1.5; off[1] = 1; c[1] = 2.0; off[2] = 2; c[2] = -0.5; return 3;",
                                     "off[0] = 0; c[0] = -1.0; off[1] = 1; c[1] = 1.0; off[2] = 2; c[2] = 0.0; return 3;"),
    "integrate_backward_sign": ("off[0] = 0; c[0] = 1.5; off[1] = -1; c[1] = -2.0; off[2] = -2; c[2] = 0.5; return 3;",
                                "off[0] = 0; c[0] = -1.5; off[1] = -1; c[1] = 2.0; off[2] = -2; c[2] = -0.5; return 3;"),
    "integrate_transposed_gradient": ("const long step = a == 0 ? nx : 1;\n                int off[3];\n                double c[3];\n                const int n = integ_stencil(ny, nx, M, i, j, a, off, c);\n                double v = 0.0;",
                                      "const long step = a == 0 ? 1 : nx;\n                int off[3];\n                double c[3];\n                const int n = integ_stencil(ny, nx, M, i, j, a, off, c);\n                double v = 0.0;"),
    "integrate_cg_beta_sign": ("for (size_t p = 0; p < P; ++p) d[p] = r[p] + beta * d[p];",
                               "for (size_t p = 0; p < P; ++p) d[p] = r[p] - beta * d[p];"),
    "integrate_keeps_input": ("u_out[a * P + p] = integ_stencil(ny, nx, M, i, j, a, off, c) ? g[a * P + p] : u_in[a * P + p];",
                              "u_out[a * P + p] = u_in[a * P + p];"),
}


@pytest.fixture(scope="module")
def source():
    with open(SRC) as fh:
        return fh.read()


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_some_pin_catches_the_mutant(name, source, tmp_path):
    old, new = MUTANTS[name]
    assert source.count(old) == 1, f"mutation site for {name} not found exactly once"
    src = tmp_path / "mutant.c"
    src.write_text(source.replace(old, new))
    so = tmp_path / "libmutant.so"
    subprocess.run(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fopenmp", "-shared", "-fPIC",
                    "-o", str(so), str(src), "-lm"], check=True)
    L = oracle.load_variant(str(so))
    caught = []
    for pin in pins.ALL_PINS:
        try:
            pin(L)
        except (AssertionError, ValueError):
            caught.append(pin.__name__)
    assert caught, f"no pin catches mutant {name}"
