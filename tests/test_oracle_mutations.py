"""Plants single mistakes in a copy of the oracle source and checks that the pin aimed at
each one fails.  CPU only: every mutant is compiled with gcc and run on the host."""
import os
import subprocess
import sys

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(os.path.dirname(HERE), "oracle", "lbm_oracle.c")

# name: (original text, planted mistake, pin expected to catch it)
MUTATIONS = {
    "delta_s_factor": ("double ds = 1.5 * o->p.W;", "double ds = 1.0;", "marangoni_convection"),
    "theta_sign": ("double theta = 4.0 * ph * (1.0 - ph) / o->p.W;\n            double pop[QMAX];",
                   "double theta = -4.0 * ph * (1.0 - ph) / o->p.W;\n            double pop[QMAX];",
                   "flat_interface"),
    "capillary_sign": ("double Fsx = ds * (-sg * g2 * dv * nxv", "double Fsx = ds * (sg * g2 * dv * nxv", "laplace"),
    "pressure_force_sign": ("double Fpx = -dpx, Fpy = -dpy;", "double Fpx = dpx, Fpy = dpy;", "two_layer_poiseuille"),
    "half_force_velocity": ("double ux = (sx + 0.5 * CS2 * Ftx) / (rho * CS2);",
                            "double ux = (sx + CS2 * Ftx) / (rho * CS2);", "poiseuille"),
    "source_weight": ("out[m] = e[m] + w * (eq[m] - e[m]) + (1.0 - 0.5 * w) * s[m];",
                      "out[m] = e[m] + w * (eq[m] - e[m]) + s[m];", "flow_source"),
    "split_rates_swapped": ("double w2s = 1.0, w2d = omega_nu;", "double w2s = omega_nu, w2d = 1.0;", "split"),
    "equilibrium_22": ("-(c2 * (ux * ux + uy * uy) + ux * ux * uy * uy)};", "-(c2 * (ux * ux + uy * uy))};",
                       "matching_principle"),
    "equilibrium_21": ("-uy * uy, -ux * uy, ax * uy, ay * ux,", "-uy * uy, -ux * uy, ay * uy, ay * ux,",
                       "matching_principle"),
    "source_11": ("s[5] = c2 * (Fpx * uy + Fpy * ux) + ux * uy * G;", "s[5] = c2 * (Fpx * ux + Fpy * uy) + ux * uy * G;",
                  "two_layer_poiseuille"),
    "source_20_factor": ("s[3] = 2.0 * c2 * Fpx * ux + (ux * ux + c2) * G;", "s[3] = c2 * Fpx * ux + (ux * ux + c2) * G;",
                         "continuous_source"),
    "source_02_component": ("s[4] = 2.0 * c2 * Fpy * uy + (uy * uy + c2) * G;",
                            "s[4] = 2.0 * c2 * Fpy * uy + (ux * ux + c2) * G;", "continuous_source"),
    "source_11_gamma_term": ("s[5] = c2 * (Fpx * uy + Fpy * ux) + ux * uy * G;", "s[5] = c2 * (Fpx * uy + Fpy * ux);",
                             "continuous_source"),
    "shift_sign": ("ipow(-ux, m - p) * ipow(-uy, n - q);", "ipow(ux, m - p) * ipow(-uy, n - q);", "central_moment_shift"),
    "specular_as_bounce_back": ("int am = find_dir(o->Qf, EX[a], -EY[a]);", "int am = find_dir(o->Qf, -EX[a], -EY[a]);",
                                "streaming_routes"),
    "anti_bounce_back_sign": ("o->hpre[IDX(a, j, i)] = -o->h[IDX(oh, j, i)] + 2.0 * weight(o->Qh, a) * Tw;",
                              "o->hpre[IDX(a, j, i)] = o->h[IDX(oh, j, i)] + 0.0 * weight(o->Qh, a) * Tw;",
                              "streaming_routes"),
    "wall_crossing_point": ("double xc = (double)i - 0.5 * (double)EX[a];", "double xc = (double)i + 0.5 * (double)EX[a];",
                            "link_crossing"),
    "temperature_ghost": ("if (j < 0) T = 2.0 * T_bottom(o, (double)i) - o->T[FLD(0, i)];",
                          "if (j < 0) T = o->T[FLD(0, i)];", "up_to_the_walls"),
    "viscosity_interp": ("return o->muA + phi * (o->muB - o->muA); }", "return o->muB + phi * (o->muA - o->muB); }",
                         "two_layer_poiseuille"),
    "viscosity_rate": ("double omega_nu = 1.0 / (nu / CS2 + 0.5);", "double omega_nu = 1.0 / (nu / CS2 + 1.0);",
                       "shear_mode"),
    "phase_rate_y": ("double w = (m == 1 || m == 2) ? omega_phi : 1.0;", "double w = (m == 1) ? omega_phi : 1.0;",
                     "phase_collision"),
    "curvature_components": ("dv += weight(9, a) * (EX[a] * o->nxs[e] + EY[a] * o->nys[e]);",
                             "dv += weight(9, a) * (EX[a] * o->nys[e] + EY[a] * o->nxs[e]);", "laplace"),
    "marangoni_projection": ("g2 * ((1.0 - nxv * nxv) * dsx - nxv * nyv * dsy));",
                             "g2 * ((1.0 - nyv * nyv) * dsx - nxv * nyv * dsy));", "marangoni_convection"),
    "energy_equilibrium_22": ("0.0, 0.0, 0.0, CS2 * CS2 * T};\n    to_central(B, ux, uy, pop, k);\n    for (int m = 0; m < B->Q; ++m) {\n        double w = (m == 1 || m == 2) ? omega_T",
                              "0.0, 0.0, 0.0, CS2 * T};\n    to_central(B, ux, uy, pop, k);\n    for (int m = 0; m < B->Q; ++m) {\n        double w = (m == 1 || m == 2) ? omega_T",
                              "energy_collision"),
}


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_pin_catches_planted_mistake(name, tmp_path):
    original, planted, pin = MUTATIONS[name]
    base = open(SRC).read()
    assert base.count(original) == 1, f"mutation site for {name} not found exactly once"
    mutant = tmp_path / "lbm_oracle.c"
    mutant.write_text(base.replace(original, planted))
    env = dict(os.environ, LBM_ORACLE_SRC=str(mutant))
    r = subprocess.run([sys.executable, "-m", "pytest", os.path.join(HERE, "test_oracle_pins.py"), "-q", "-x",
                        "-p", "no:cacheprovider", "-k", pin], env=env, capture_output=True, text=True,
                       cwd=os.path.dirname(HERE), timeout=600)
    assert r.returncode == 1 and "failed" in r.stdout, f"pin '{pin}' did not catch {name}:\n{r.stdout[-800:]}"
