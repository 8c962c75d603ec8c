"""Planted mistakes: each one is a plausible error in the oracle (a dropped
term, a wrong sign, a swapped index or operand); a copy of the oracle with
the mistake is built and the oracle's pins are run against it -- at least
one pin must fail for every mistake.  The mistakes are planted only in
copies of the C source built under oracle/_build/mutants/, on the CPU."""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
ORACLE = os.path.join(ROOT, "oracle")
OUT = os.path.join(ORACLE, "_build", "mutants")
PINS = ["tests/test_golden.py", "tests/test_oracle_boundaries.py", "tests/test_oracle_pointwise.py",
        "tests/test_oracle_scheme.py"]
MLP_PINS = ["tests/test_oracle_mlp.py"]
HO_PINS = ["tests/test_oracle_high_order.py"]

# (name, file, original text, planted text, pin files).  Not listed: a
# change to the sign factors of minmod4's last two arguments, which is an
# equivalent mistake for the arguments MP5 passes (4a - b and 4b - a of one
# sign force a and b to that sign).
MUTANTS = [
    ("uct_diffusion_sign", "echo_oracle.c", "+ da * (Bb[1] - Bb[0]) - db * (Ba[1] - Ba[0])",
     "- da * (Bb[1] - Bb[0]) - db * (Ba[1] - Ba[0])", PINS),
    ("uct_weight_swap", "echo_oracle.c", "wLR = apa * amb / den;", "wLR = ama * apb / den;", PINS),
    ("c2p_dropped_sb_term", "echo_oracle.c", "- SB * SB / (2.0 * Z * Z) - U;", "- U;", PINS),
    ("mp5_coefficient", "echo_oracle.c", "47.0 * u0", "46.0 * u0", PINS),
    ("flux_dropped_magnetic_stress", "echo_oracle.c", "- bu[d] * bl[j];", ";", PINS),
    ("ks_shift_scaling", "echo_oracle.c", "beta[0] = z / (1.0 + z) / r;", "beta[0] = z / (1.0 + z);", PINS),
    ("emf_side_labels", "echo_oracle.c", "Est[s][t] = -(vta * Bb[s] - vtb * Ba[t]);",
     "Est[s][t] = -(vta * Bb[t] - vtb * Ba[s]);", PINS),
    ("source_index_swap", "echo_oracle.c", "st += Wij * dbe[j][i];", "st += Wij * dbe[i][j];", PINS),
    ("source_dropped_lapse_term", "echo_oracle.c", "s -= U * dal[i];", ";", PINS),
    ("fast_speed_dropped_cross_term", "echo_oracle.c", "double a2 = cs2 + ca2 - cs2 * ca2;",
     "double a2 = cs2 + ca2;", PINS),
    ("mlp_dropped_activation", "mlp_oracle.c", "a2[k] = tanh(s);", "a2[k] = s;", MLP_PINS),
    ("guard_lower_cell_only", "echo_oracle.c", "for (int side = 0; side < 2; ++side) {\n                        int *t = side",
     "for (int side = 0; side < 1; ++side) {\n                        int *t = side", HO_PINS),
    ("guard_without_reassembly", "echo_oracle.c", "replaced += guard_revert(c, G);\n        assemble(c, G);",
     "replaced += guard_revert(c, G);", HO_PINS),
    ("guard_stage_weight", "echo_oracle.c", "(stage == 1 ? 0.75 : 1.0 / 3.0)", "(stage == 1 ? 0.25 : 1.0 / 3.0)",
     HO_PINS),
    ("ho_dropped_fourth_difference", "echo_oracle.c", "return f5[2] - d2 / 24.0 + 3.0 * d4 / 640.0;",
     "return f5[2] - d2 / 24.0;", HO_PINS),
    ("ho_emf_correction_direction", "echo_oracle.c", "const double *Eb = c->order ? G->Ec[b][1] : G->E[b];",
     "const double *Eb = c->order ? G->Ec[b][0] : G->E[b];", HO_PINS),
    ("ho_point_value_weight", "echo_oracle.c", "90.0 * u0", "91.0 * u0", HO_PINS),
    ("ho_centre_weight", "echo_oracle.c", "150.0 * b6[2] + 150.0 * b6[3]", "150.0 * b6[2] + 149.0 * b6[3]",
     HO_PINS),
    ("c2p_derivative_factor", "echo_oracle.c", "double dv2 = -2.0 * (S2", "double dv2 = -1.0 * (S2", PINS),
    ("c2p_recovery_sign", "echo_oracle.c", "vl[j] = (S[j] + SB * Bl[j] / Z) / (Z + B2);",
     "vl[j] = (S[j] - SB * Bl[j] / Z) / (Z + B2);", PINS),
    ("rk3_stage_weights", "echo_oracle.c", "u[id] = 0.75 * u0[id] + 0.25 * (u[id] + dt * l[id]);",
     "u[id] = 0.25 * u0[id] + 0.75 * (u[id] + dt * l[id]);", PINS),
    ("ct_curl_sign", "echo_oracle.c", "G->LB[d][id] = -(dEb_da - dEa_db);", "G->LB[d][id] = (dEb_da - dEa_db);",
     PINS),
    ("cfl_max_instead_of_sum", "echo_oracle.c", "s += fmax(fabs(lp), fabs(lm)) / c->dx[d];",
     "s = fmax(s, fmax(fabs(lp), fabs(lm)) / c->dx[d]);", PINS),
    ("hll_diffusion_sign", "echo_oracle.c", "- ap * am * (UR[q] - UL[q])) / s;", "+ ap * am * (UR[q] - UL[q])) / s;",
     PINS),
    ("mp5_limiter_alpha", "echo_oracle.c", "double uul = u0 + MP5_ALPHA * (u0 - um1);",
     "double uul = u0 + 2.0 * (u0 - um1);", PINS),
    ("mp5_lc_coefficient", "echo_oracle.c", "4.0 / 3.0 * dMm", "3.0 / 4.0 * dMm", PINS),
    ("mp5_curvature_side", "echo_oracle.c", "double dMp = minmod4(4.0 * d0 - dp1, 4.0 * dp1 - d0, d0, dp1);",
     "double dMp = minmod4(4.0 * d0 - dm1, 4.0 * dm1 - d0, d0, dm1);", PINS),
    ("mp5_minmod4_dropped_operand", "echo_oracle.c", "fmin(fmin(fabs(w), fabs(x)), fmin(fabs(y), fabs(z)))",
     "fmin(fmin(fabs(w), fabs(x)), fabs(y))", PINS),
    ("mp5_bounds_min_max", "echo_oracle.c", "double umin = fmax(fmin(fmin(u0, up1), umd)",
     "double umin = fmin(fmin(fmin(u0, up1), umd)", PINS),
    ("mp5_test_direction", "echo_oracle.c", "if ((uor - u0) * (uor - ump) <= MP5_EPS)",
     "if ((uor - u0) * (uor - ump) >= MP5_EPS)", PINS),
    ("adam_bias_correction_constant", "mlp_oracle.c", "double c1 = 1.0 - pow(b1, t), c2", "double c1 = 1.0 - b1, c2",
     MLP_PINS),
    ("bc_outflow_offset", "echo_oracle.c", "return side == 0 ? lo : hi;", "return side == 0 ? lo + 1 : hi;", PINS),
    ("bc_axis_mirror_offset", "echo_oracle.c", "return side == 0 ? 2 * NG - 1 - i : 2 * (NG + n) - 1 - i;",
     "return side == 0 ? 2 * NG - i : 2 * (NG + n) - 1 - i;", PINS),
    ("bc_axis_no_flip", "echo_oracle.c", "if (flip && ((comp == d) != (dens != 0)))", "if (flip && comp == -2)", PINS),
    ("bc_axis_density_even", "echo_oracle.c", "if (flip && ((comp == d) != (dens != 0)))", "if (flip && comp == d)", PINS),
    ("coord_centre_shift", "echo_oracle.c", "+ 0.5 + off) * c->dx[d];", "+ off) * c->dx[d];", PINS),
    ("floor_power_sign", "echo_oracle.c", "return f0 * pow(exp(x1), pw);", "return f0 * pow(exp(x1), -pw);", PINS),
    ("c2p_v2_term", "echo_oracle.c", "SB * SB * (2.0 * Z + B2)) / (Z * Z * ZB * ZB)",
     "SB * SB * (Z + B2)) / (Z * Z * ZB * ZB)", PINS),
    ("p2c_dropped_vb", "echo_oracle.c", "0.5 * (B2 + B2 * v2 - vB * vB)", "0.5 * (B2 + B2 * v2)", PINS),
    ("speeds_shift_sign", "echo_oracle.c", "*lp = m->alpha / den * (vd * (1.0 - a2) + sq) - m->beta[d];",
     "*lp = m->alpha / den * (vd * (1.0 - a2) + sq) + m->beta[d];", PINS),
    ("flux_tau_shift_sign", "echo_oracle.c", "F[4] = m->alpha * (Su[d] - C[0] * v[d]) - m->beta[d] * C[4];",
     "F[4] = m->alpha * (Su[d] - C[0] * v[d]) + m->beta[d] * C[4];", PINS),
    ("divb_spacing", "echo_oracle.c", "dv += (bf[1] - bf[0]) / c->dx[d];", "dv += (bf[1] - bf[0]) / c->dx[0];",
     PINS),
    ("energy_total_component", "echo_oracle.c", "sT += G.U[4][id] * dV;", "sT += G.U[3][id] * dV;", PINS),
    ("source_derivative_weight", "echo_oracle.c", "double wts[6] = {-1.0, 9.0, -45.0, 45.0, -9.0, 1.0};",
     "double wts[6] = {-1.0, 9.0, -45.0, 45.0, -9.0, 0.0};", PINS),
    ("source_tau_lapse_sign", "echo_oracle.c", "st -= Su[j] * dal[j];", "st += Su[j] * dal[j];", PINS),
    ("source_magnetic_pressure", "echo_oracle.c", "(p + 0.5 * b2) * m->gi[i][j]", "(p + b2) * m->gi[i][j]", PINS),
    ("emf_transport_shift_sign", "echo_oracle.c", "double vta = alpha * va[s][t] - beta[a];",
     "double vta = alpha * va[s][t] + beta[a];", PINS),
    ("ks_polar_metric", "echo_oracle.c", "g[1][1] = sig;", "g[1][1] = r * r;", PINS),
    ("face_fallback_dropped", "echo_oracle.c", "if (!(Ps[0] > 0.0) || !(Ps[4] > 0.0) || !(v2 < 1.0)) {",
     "if (0) {", PINS),
    ("face_fallback_wrong_cell", "echo_oracle.c", "size_t src = cid[side == 0 ? 2 : 3];", "size_t src = cid[3];",
     PINS),
    ("ho_second_difference_sign", "echo_oracle.c", "double d2 = f5[1] - 2.0 * f5[2] + f5[3];",
     "double d2 = f5[1] - 2.0 * f5[2] - f5[3];", HO_PINS),
    ("ho_flux_stencil_offset", "echo_oracle.c", "                            t[d] += s - 2;\n                            f5[s] = G->F[d][q]",
     "                            t[d] += s - 1;\n                            f5[s] = G->F[d][q]", HO_PINS),
    ("cell_centre_field_one_face", "echo_oracle.c",
     "Bc[d] = 0.5 * (G->B[d][IDX(G, i, j, k)] + G->B[d][IDX(G, t[0], t[1], t[2])]) / sqrtg;",
     "Bc[d] = G->B[d][IDX(G, i, j, k)] / sqrtg;", PINS),
    ("floor_reset_skipped", "echo_oracle.c", "                if (reset) {", "                if (0) {", PINS),
    ("p2c_momentum_sign", "echo_oracle.c", "C[1 + j] = (Zw + B2) * vl[j] - vB * Bl[j];",
     "C[1 + j] = (Zw + B2) * vl[j] + vB * Bl[j];", PINS),
    ("speeds_root_metric_term", "echo_oracle.c", "((1.0 - v2 * a2) * m->gi[d][d] - (1.0 - a2) * vd * vd)",
     "((1.0 - v2 * a2) - (1.0 - a2) * vd * vd)", PINS),
    ("mlp_loss_weight", "mlp_oracle.c", "double wgt[NO] = {1.0, 1.0, w2};", "double wgt[NO] = {1.0, 1.0, 1.0};",
     MLP_PINS),
    ("mlp_standardisation", "mlp_oracle.c", "xs[i] = (x[i] - mu[i]) / sd[i];", "xs[i] = (x[i] - mu[i]) * sd[i];",
     MLP_PINS),
    ("c2p_pressure_dropped_root", "echo_oracle.c", "double p = gg * (Z * (1.0 - v2) - D * sq);",
     "double p = gg * (Z * (1.0 - v2) - D);", PINS),
]


def _build(name, fname, old, new):
    srcs = {}
    for f in ("echo_oracle.c", "mlp_oracle.c"):
        with open(os.path.join(ORACLE, f)) as fh:
            srcs[f] = fh.read()
    assert srcs[fname].count(old) >= 1, f"anchor of {name} not found"
    srcs[fname] = srcs[fname].replace(old, new, 1)
    d = os.path.join(OUT, name)
    os.makedirs(d, exist_ok=True)
    paths = []
    for f, txt in srcs.items():
        p = os.path.join(d, f)
        with open(p, "w") as fh:
            fh.write(txt)
        paths.append(p)
    lib = os.path.join(d, "liboracle_mutant.so")
    subprocess.run(["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared", "-fopenmp",
                    "-std=c11", "-w", "-o", lib, *paths, "-lm"], check=True, capture_output=True, text=True)
    return lib


@pytest.mark.parametrize("name,fname,old,new,pins", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_planted_mistake_fails_a_pin(name, fname, old, new, pins):
    lib = _build(name, fname, old, new)
    env = dict(os.environ, ECHO_ORACLE_LIB=lib)
    r = subprocess.run([sys.executable, "-m", "pytest", *pins, "-x", "-q", "-p", "no:cacheprovider",
                        "-m", "not gpu"], cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 1, f"{name}: no pin failed\n{r.stdout[-1500:]}"
    assert " failed" in r.stdout, r.stdout[-1500:]
