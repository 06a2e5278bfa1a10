"""Mutation check of the oracle's pins: each case plants one plausible
mistake in a copy of the oracle source (a dropped term, a wrong sign, a
swapped operand or index), builds it, and requires that the pin suite fails
on it.  Runs on the CPU only; the real oracle is never modified."""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "hydro_oracle.c")
PINS = [os.path.join(ROOT, "tests", "test_oracle_riemann.py"),
        os.path.join(ROOT, "tests", "test_oracle_scheme.py"),
        os.path.join(ROOT, "tests", "test_oracle_variants.py")]

MUTANTS = {
    "trace_drops_pressure_gradient": ("dW[1] = half * (u * D[1] + D[3] / rho);",
                                      "dW[1] = half * (u * D[1]);"),
    "trace_drops_compression": ("dW[0] = half * (u * D[0] + rho * D[1]);",
                                "dW[0] = half * (u * D[0]);"),
    "trace_wrong_sign_pressure_row": ("dW[3] = half * (P->gamma * p * D[1] + u * D[3]);",
                                      "dW[3] = half * (P->gamma * p * D[1] - u * D[3]);"),
    "trace_faces_swapped": ("WL[q] = W0[q] - 0.5 * D[q] + dW[q];",
                            "WL[q] = W0[q] + 0.5 * D[q] + dW[q];"),
    "minmod_takes_larger": ("if (a > 0.0 && b > 0.0) return (a < b) ? a : b;",
                            "if (a > 0.0 && b > 0.0) return (a > b) ? a : b;"),
    "shock_B_inverted": ("double B = (g - 1.0) / (g + 1.0) * pk;",
                         "double B = (g + 1.0) / (g - 1.0) * pk;"),
    "rarefaction_exponent": ("*f = 2.0 * ck / (g - 1.0) * (pow(r, (g - 1.0) / (2.0 * g)) - 1.0);",
                             "*f = 2.0 * ck / (g - 1.0) * (pow(r, (g + 1.0) / (2.0 * g)) - 1.0);"),
    "ustar_sign": ("*ustar = 0.5 * (ul + ur) + 0.5 * (fr - fl);",
                   "*ustar = 0.5 * (ul + ur) + 0.5 * (fl - fr);"),
    "newton_sign": ("p = p - (fl + fr + (ur - ul)) / (dfl + dfr);",
                    "p = p - (fl + fr - (ur - ul)) / (dfl + dfr);"),
    "tangential_from_wrong_side": ("        W[2] = WL[2];\n", "        W[2] = WR[2];\n"),
    "left_shock_density": ("W[0] = rl * (pr_ + G6) / (G6 * pr_ + 1.0);",
                           "W[0] = rl * (G6 * pr_ + 1.0) / (pr_ + G6);"),
    "fan_sign": ("double c = 2.0 / (g + 1.0) * (cl + 0.5 * (g - 1.0) * (ul - xi));",
                 "double c = 2.0 / (g + 1.0) * (cl - 0.5 * (g - 1.0) * (ul - xi));"),
    "flux_tangential": ("F[2] = rho * un * ut;", "F[2] = rho * un * un;"),
    "flux_energy_drops_p": ("F[3] = un * (E + p);", "F[3] = un * E;"),
    "update_sign": ("out[i][q] = line[i + 2][q] - dtdx * (F[i + 1][q] - F[i][q]);",
                    "out[i][q] = line[i + 2][q] + dtdx * (F[i + 1][q] - F[i][q]);"),
    "reflect_without_flip": ("if (bc == ORC_BC_REFLECT) *flip = 1;", "if (bc == ORC_BC_REFLECT) *flip = 0;"),
    "periodic_off_by_one": ("if (bc == ORC_BC_PERIODIC) return (k < 0) ? k + n : k - n;",
                            "if (bc == ORC_BC_PERIODIC) return (k < 0) ? k + n - 1 : k - n;"),
    "pressure_drops_kinetic_half": ("double eint = U[3] - 0.5 * rho * (un * un + ut * ut);",
                                    "double eint = U[3] - rho * (un * un + ut * ut);"),
    "cfl_sums_speeds": ("double s = ((au > av) ? au : av) + c;", "double s = au + av + c;"),
    "sweep_order_swapped": ("if (((step0 + s) & 1) == 0) {", "if (((step0 + s) & 1) == 1) {"),
    "pressure_floor_linear_in_c": ("double pmin = rho * P->c_floor * P->c_floor / P->gamma;",
                                   "double pmin = rho * P->c_floor / P->gamma;"),
    "density_floor_ignored": ("return (rho < P->rho_floor) ? P->rho_floor : rho;", "return rho;"),
    "riemann_floor_drops_gamma": ("return P->rho_floor * P->c_floor * P->c_floor / P->gamma;",
                                  "return P->rho_floor * P->c_floor * P->c_floor;"),
    "two_shock_flag_ignored": ("if (p > pk || P->riemann == ORC_RIEMANN_TWO_SHOCK) {", "if (p > pk) {"),
    "mc_without_central": ("    if (fabs(2.0 * a) < m) m = fabs(2.0 * a);\n",
                           "    m = fabs(2.0 * a);\n"),
    "mc_sign_lost": ("    return (a > 0.0) ? m : -m;", "    return m;"),
    "no_slope_is_minmod": ("    if (P->slope == ORC_SLOPE_NONE) return 0.0;\n", ""),
    "char_eigvec_sign": ("double r1[4] = {1.0, -c / rho, 0.0, c * c}", "double r1[4] = {1.0, c / rho, 0.0, c * c}"),
    "char_amplitude_half": ("a[3] = rho / (2.0 * c) * D[1] + D[3] / (2.0 * c * c);",
                            "a[3] = rho / (2.0 * c) * D[1] + D[3] / (c * c);"),
    "char_nu_sign": ("if (lam[k] > 0.0) WR[q] += 0.5 * (1.0 - nu) * a[k] * r[k][q];",
                     "if (lam[k] > 0.0) WR[q] += 0.5 * (1.0 + nu) * a[k] * r[k][q];"),
    "char_all_waves_right": ("if (lam[k] > 0.0) WR[q]", "if (1) WR[q]"),
}


@pytest.mark.slow
@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_kill_mutant(name, tmp_path):
    old, new = MUTANTS[name]
    src = open(SRC).read()
    assert src.count(old) >= 1, f"mutation site for {name} not found"
    mut = tmp_path / "mutant.c"
    mut.write_text(src.replace(old, new, 1))
    so = tmp_path / "mutant.so"
    subprocess.run(["gcc", "-O2", "-ffp-contract=off", "-std=c11", "-fPIC", "-shared",
                    "-o", str(so), str(mut), "-lm"], check=True)
    env = dict(os.environ, ORACLE_LIB=str(so))
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                        *PINS], cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode != 0, f"mutant {name} survived the pins:\n{r.stdout[-2000:]}"
