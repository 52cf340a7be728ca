"""Mutation check of the oracle pins: plant plausible mistakes in copies of the oracle's C
source (a flipped convolution, a dropped mask, a wrong sign, factor, weight or update) and
check that the pin suite fails for every one of them.  The mistakes are planted on the CPU,
in the oracle only."""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "misr_oracle.c")

MUTANTS = {
    "convolution_flipped": ("int bu = cu - a;", "int bu = cu + a;"),
    "blur_padding_dropped": ("if (bu < 0 || bu >= H) continue;", "/* row padding dropped */"),
    "shift_sign": ("int u = bu + ty, v = bv + tx;", "int u = bu - ty, v = bv + tx;"),
    "bilinear_weights_swapped": ("const double wy[2] = {1.0 - P->fy[k], P->fy[k]}, wx[2] = {1.0 - P->fx[k], P->fx[k]};",
                                 "const double wy[2] = {P->fy[k], 1.0 - P->fy[k]}, wx[2] = {1.0 - P->fx[k], P->fx[k]};"),
    "bilinear_second_tap_offset": ("const int u = bu + P->ty[k] + p;", "const int u = bu + P->ty[k] - p;"),
    "gamma_exponent": ("return pow(P->btv_alpha, dx + dy);", "return pow(P->btv_alpha, dx > dy ? dx : dy);"),
    "btv_window_short": ("for (int dy = 0; dy < P->btv_w; ++dy) {\n        for (int dx = 0; dx < P->btv_w; ++dx) {\n            if (dx == 0 && dy == 0) continue;\n#pragma omp parallel for schedule(static)\n            for (int u = 0; u < H; ++u) {\n                double s = 0;\n                if (u + dy < H)",
                         "for (int dy = 0; dy < P->btv_w - 1; ++dy) {\n        for (int dx = 0; dx < P->btv_w; ++dx) {\n            if (dx == 0 && dy == 0) continue;\n#pragma omp parallel for schedule(static)\n            for (int u = 0; u < H; ++u) {\n                double s = 0;\n                if (u + dy < H)"),
    "dpsi_sign": ("if (eps > 0) return t / sqrt(t * t + eps * eps);", "if (eps > 0) return -t / sqrt(t * t + eps * eps);"),
    "d2psi_power": ("return eps * eps / (s * sqrt(s));", "return eps * eps / s;"),
    "grad_factor_2_dropped": ("for (long i = 0; i < n; ++i) g[i] += 2.0 * t[i];", "for (long i = 0; i < n; ++i) g[i] += t[i];"),
    "hessvec_factor": ("for (long i = 0; i < n; ++i) out[i] += (l1 ? 1.0 : 2.0) * t[i];",
                       "for (long i = 0; i < n; ++i) out[i] += (l1 ? 1.0 : 1.0) * t[i];"),
    "l1_gradient_factor_2_kept": ("for (long i = 0; i < n; ++i) g[i] += t[i];", "for (long i = 0; i < n; ++i) g[i] += 2.0 * t[i];"),
    "l1_hessian_weight_dropped": ("for (long i = 0; i < m; ++i) e[i] *= d2psi(ex[i] - y[k * m + i], P->data_eps);",
                                  "for (long i = 0; i < m; ++i) e[i] *= 1.0;"),
    "l1_value_squared": ("s += l1 ? psi(t, ed) : t * t;", "s += l1 ? t * t : t * t;"),
    "beta_fletcher_reeves": ("const double beta = (rr_new - rr_cross) / mu;", "const double beta = rr_new / dot(r, r, n);"),
    "lambda_not_reduced": ("if (Delta >= 0.75) lam = lam / 4.0;", "if (Delta >= 0.75) lam = lam / 2.0;"),
    "delta_not_scaled": ("delta += (lam - lam_bar) * pn2;", "delta += 0.0 * (lam - lam_bar) * pn2;"),
    # Moller's scale increase after a poor step (step 8) and the lambda_bar it works against
    "lambda_raise_times_4": ("if (Delta < 0.25) lam = lam + delta * (1.0 - Delta) / pn2;",
                             "if (Delta < 0.25) lam = 4.0 * lam + delta * (1.0 - Delta) / pn2;"),
    "lambda_raise_sign": ("if (Delta < 0.25) lam = lam + delta * (1.0 - Delta) / pn2;",
                          "if (Delta < 0.25) lam = lam + delta * (1.0 + Delta) / pn2;"),
    "lambda_bar_left_at_0": ("lam_bar = lam;\n            success = 0;", "lam_bar = 0.0;\n            success = 0;"),
    "negative_curvature_branch_always": ("if (delta <= 0) {", "if (delta <= 0 || it >= 0) {"),
    "shift_add_no_average": ("x0[i] = cnt[i] > 0 ? x0[i] / cnt[i] : 0.0;", "x0[i] = x0[i];"),
    "binning_weight_1_over_f": ("const double wd = 1.0 / ((double)nb * nb);", "const double wd = 1.0 / (double)nb;"),
    "binning_block_backwards": ("const int cu = f * i + a2, cv = f * j + b2;   /* pixel of B's output */",
                                "const int cu = f * i - a2, cv = f * j + b2;   /* pixel of B's output */"),
    "binned_adjoint_weight_dropped": ("const double ev = wd * e[(long)i * P->w + j];",
                                      "const double ev = e[(long)i * P->w + j];"),
    "log_convert_no_clamp": ("double c = counts[i] < 1 ? 1.0 : (double)counts[i];", "double c = (double)counts[i] + 1e-300;"),
}


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_catch_mutant(name, tmp_path):
    old, new = MUTANTS[name]
    src = open(SRC).read()
    assert src.count(old) >= 1, f"mutation anchor for {name} not found"
    mut = src.replace(old, new, 1)
    cfile = tmp_path / "misr_oracle.c"
    cfile.write_text(mut)
    (tmp_path / "misr_oracle.h").write_text(open(os.path.join(ROOT, "oracle", "misr_oracle.h")).read())
    lib = tmp_path / "libmut.so"
    subprocess.run(["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-o", str(lib), str(cfile), "-lm"],
                   check=True, capture_output=True)
    env = dict(os.environ, MISR_ORACLE_LIB=str(lib))
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                        os.path.join(ROOT, "tests", "test_oracle_pins.py")],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode != 0, f"mutant {name} survived the pin suite"
