"""The oracle pins catch plausible mistakes.

Each case plants one mistake in a copy of the oracle source (a sign, a
weight, a coefficient, a dropped term, a boundary rule), builds it on the CPU
and runs the pin that must fail on it.  This is what makes the pins evidence:
a pin suite that passes on a broken oracle would prove nothing.
"""
import concurrent.futures
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "eulbfs_oracle.c")
PINS = "tests/test_oracle_pins.py::"
AXI = "tests/test_oracle_axisymmetric.py::"
HYS = "tests/test_oracle_hysteresis.py::"
STR = "tests/test_oracle_streaming.py::"
BRT = "tests/test_oracle_brute_force.py::"

# (name, original text, planted text, pin that must fail)
MUTATIONS = [
    ("f_star_sign_R3", "const double fstar = feqf + (1.0 - 1.0 / (2.0 * tau_f)) * fneqm;",
     "const double fstar = feqf - (1.0 - 1.0 / (2.0 * tau_f)) * fneqm;", "test_simple_shear_viscous_flux"),
    ("gamma_one_R8", "const double Gamma = CS2 * (eu / CS2", "const double Gamma = CS2 * (1.0 + eu / CS2",
     "test_uniform_state_euler_fluxes"),
    ("diagonal_weight", "1.0 / 36, 1.0 / 36, 1.0 / 36, 1.0 / 36};", "1.0 / 36, 1.0 / 36, 1.0 / 36, 1.0 / 30};",
     "test_equilibria_moments"),
    ("rk3_coefficient", "0.75 * s->Wn[k][c] + 0.25 * s->W[k][c]", "0.7 * s->Wn[k][c] + 0.3 * s->W[k][c]",
     "test_rk3_mode_decay"),
    ("phase_source_sign", "FE[4] = C * kv * s->dFs[c];", "FE[4] = -C * kv * s->dFs[c];", "test_volume_change_sources"),
    ("phase_source_gated_twice", "FE[4] = C * kv * s->dFs[c];", "FE[4] = C * kv * D;",
     "test_volume_change_sources_in_a_mixed_cell"),
    ("pressure_source_sign", "rho * CS2 * kv * D;\n", "- rho * CS2 * kv * D;\n", "test_volume_change_sources"),
    ("muc_sign_R5", "- s->kappa * lap;", "+ s->kappa * lap;", "test_flat_interface_equilibrium"),
    ("surface_tension_sign", "const double Fsx = -Fl * C * s->grx[P_MUC][q];",
     "const double Fsx = Fl * C * s->grx[P_MUC][q];", "test_three_phase_expansion_law"),
    ("ibm_force_sign", "const double Fix = -rho * u * D, Fiy = -rho * v * D;",
     "const double Fix = rho * u * D, Fiy = rho * v * D;", "test_freezing_momentum_decay"),
    ("enthalpy_source_dropped", "FE[0] = Cp * T * divu;", "FE[0] = 0.0 * divu;", "test_three_phase_expansion_law"),
    ("density_gradient_source_dropped",
     "FE[1] = u * (s->grx[P_RHO][q] * CS2) + v * (s->gry[P_RHO][q] * CS2) +", "FE[1] = 0.0 +",
     "test_three_phase_expansion_law"),
    ("gravity_sign", "FE[3] = CS2 * (Fsy + rho * s->P.gy + Fiy);", "FE[3] = CS2 * (Fsy - rho * s->P.gy + Fiy);",
     "test_hydrostatic_pressure"),
    ("tau_h_heat_capacity", "const double tau_h = 0.5 + lamf / (rho_f * s->Cref * CS2 * s->dth);",
     "const double tau_h = 0.5 + lamf / (rho_f * Cpf * CS2 * s->dth);", "test_pure_conduction_face_flux"),
    ("reconstruction_offset_sign", "+ (y - (cj + 0.5)) * s->gry[f][q];", "- (y - (cj + 0.5)) * s->gry[f][q];",
     "test_linear_temperature_convective_diffusive_flux"),
    ("tie_rule_R7", "q[a][f] = 0.5 * (recon(s, f, Li, Lj, sx, sy) + recon(s, f, Ri, Rj, sx, sy));",
     "q[a][f] = recon(s, f, Li, Lj, sx, sy);", "test_mirror_symmetry"),
    ("geq_rest_coefficient", "if (a == 0) return C - muc * Qg * (1.0 - WA[0]) / CS2;",
     "if (a == 0) return C - muc * Qg * (1.0 - WA[0]);", "test_equilibria_moments"),
    ("heq_quadratic", "(Cref / Cp + eu / CS2 + eu * eu / (2.0 * CS2 * CS2) - uu / (2.0 * CS2));",
     "(Cref / Cp + eu / CS2 + eu * eu / (2.0 * CS2) - uu / (2.0 * CS2));", "test_equilibria_moments"),
    ("solid_branch_heat_capacity", "*T = H / cps;", "*T = H / cpl;", "test_enthalpy_inversion_values"),
    ("wetting_sign_R11", "return vm + (2.0 * k - 1.0) * (4.0 * cth", "return vm - (2.0 * k - 1.0) * (4.0 * cth",
     "test_contact_angle"),
    ("dirichlet_ghost", "2.0 * sd->Tw - vm : vm;", "sd->Tw : vm;", "test_neumann_two_phase_front"),
    ("noslip_tangential", "if (sd->flow == OR_BC_NOSLIP) return -vm;",
     "if (sd->flow == OR_BC_NOSLIP) return f == normal_f ? -vm : vm;", "test_poiseuille_profile"),
    ("rigid_solid_R15", "const double keep = 1.0 - solid_gate(&s->P, s->W[4][c]) * (1.0 - Fl);", "const double keep = 1.0;",
     "test_rigid_solid"),
    ("lagged_rate_R14", "s->dFs[c] = (Fs - s->Fsp[c]) / dt;", "s->dFs[c] = 0.5 * (Fs - s->Fsp[c]) / dt;",
     "test_freezing_momentum_decay"),
    # axisymmetric form (reading R24 and the r-weighted balance of Eq. 52)
    ("axi_planar_divergence", "for (int k = 0; k < 5; ++k) divF[k] = (re * fe[k] - rw * fw[k]) / rc + (fn[k] - fs[k]);",
     "for (int k = 0; k < 5; ++k) divF[k] = (fe[k] - fw[k]) + (fn[k] - fs[k]);",
     AXI + "test_cylinder_conduction_mode_decay"),
    ("axi_hoop_pressure_dropped", "FE[2] += CS2 * (s->prim[P_P][q] - s->dtf",
     "FE[2] += CS2 * (0.0 * s->prim[P_P][q] - s->dtf",
     AXI + "test_uniform_pressure_is_force_free"),
    ("axi_hoop_pressure_not_advanced", "s->prim[P_P][q] - s->dtf * divF[1] -", "s->prim[P_P][q] -",
     AXI + "test_uniform_radial_expansion"),
    ("axi_hoop_pressure_not_advanced_stability", "s->prim[P_P][q] - s->dtf * divF[1] -", "s->prim[P_P][q] -",
     AXI + "test_resting_drop_in_light_gas_stays_bounded"),
    ("axi_hoop_viscous_dropped", "2.0 * s->prim[P_MU][q] * u / rc) / rc;", "0.0 * s->prim[P_MU][q] * u / rc) / rc;",
     AXI + "test_stagnation_flow_residual_linear_part_vanishes"),
    ("axi_streamed_source_R24", "const double Sp = -dts * rho_f * CS2 * q[0][P_U] / xf;", "const double Sp = 0.0;",
     AXI + "test_stagnation_flow_residual_linear_part_vanishes"),
    ("axi_planar_velocity_divergence", "divu = (re * fe[5] - rw * fw[5]) / rc + (fn[5] - fs[5]);",
     "divu = (fe[5] - fw[5]) + (fn[5] - fs[5]);", AXI + "test_stagnation_flow_residual_linear_part_vanishes"),
    ("axi_laplacian_face_radius", "lap = (((i + 1.0) * (C[PI(s, i + 1, j)] - c) - i * (c - C[PI(s, i - 1, j)])) / rc)",
     "lap = (((i + 0.5) * (C[PI(s, i + 1, j)] - c) - (i + 0.5) * (c - C[PI(s, i - 1, j)])) / rc)",
     AXI + "test_laplacian_of_r_squared"),
    ("axi_volume_weight", "const double w = s->N.axisymmetric ? (c % s->nx) + 0.5 : 1.0;",
     "const double w = s->N.axisymmetric ? (c % s->nx) + 1.0 : 1.0;", AXI + "test_sphere_volume_and_gibbs_thomson"),
    # contact-angle hysteresis (reading R25)
    ("hysteresis_normal_sign", "const double dn = CAT(l0, tc) - CAT(l1, tc);",
     "const double dn = CAT(l1, tc) - CAT(l0, tc);", HYS + "test_contact_line_pinned_inside_window"),
    ("hysteresis_tangential_dropped", "const double g = sqrt(dn * dn + dt * dt);", "const double g = fabs(dn) + 0.0 * dt;",
     HYS + "test_contact_line_pinned_inside_window"),
    ("hysteresis_limits_swapped", "return c < lo ? lo : (c > hi ? hi : c);", "return c < hi ? hi : (c > lo ? lo : c);",
     HYS + "test_limits_act_as_static_angles_outside_window"),
    # per-distribution streaming steps (reading R26)
    ("streaming_h_points_from_f", "else surrounding(s, xf, yf, nxv, nyv, Li, Lj, Ri, Rj, s->dth, qh);",
     "else surrounding(s, xf, yf, nxv, nyv, Li, Lj, Ri, Rj, s->dtf, qh);", STR + "test_conduction_flux_hand_expanded"),
    ("streaming_g_points_from_f", "else surrounding(s, xf, yf, nxv, nyv, Li, Lj, Ri, Rj, s->dtg, qg);",
     "else surrounding(s, xf, yf, nxv, nyv, Li, Lj, Ri, Rj, s->dtf, qg);", STR + "test_phase_field_fluxes_with_steps"),
    ("streaming_tau_f_step", "const double tau_f = 0.5 + muf / (rho_f * CS2 * s->dtf);",
     "const double tau_f = 0.5 + muf / (rho_f * CS2 * s->dth);", STR + "test_shear_flux_independent_of_steps"),
    ("streaming_Qg_step", "s->Qg = P->Mc / ((P->tau_g - 0.5) * s->dtg);", "s->Qg = P->Mc / ((P->tau_g - 0.5) * s->dtf);",
     STR + "test_phase_field_fluxes_with_steps"),
    ("streaming_hoop_step", "FE[2] += CS2 * (s->prim[P_P][q] - s->dtf * divF[1] -",
     "FE[2] += CS2 * (s->prim[P_P][q] - s->dth * divF[1] -", STR + "test_axisymmetric_radial_expansion_with_steps"),
    # cross terms that only fields varying together expose (brute-force pin)
    ("surrounding_feq_face_density", "feqs[a] = or_feq(a, qf[a][P_P], qf[a][P_RHO], qf[a][P_U], qf[a][P_V]);",
     "feqs[a] = or_feq(a, qf[a][P_P], rho_f, qf[a][P_U], qf[a][P_V]);", BRT + "test_face_flux_matches_brute_force"),
    ("feqm_surrounding_density", "feqms[a] = or_feqm(a, qf[a][P_P], rho_f, qf[a][P_U], qf[a][P_V]);",
     "feqms[a] = or_feqm(a, qf[a][P_P], qf[a][P_RHO], qf[a][P_U], qf[a][P_V]);",
     BRT + "test_face_flux_matches_brute_force"),
    ("heq_face_heat_capacity",
     "heqs[a] = or_heq(a, qh[a][P_H], qh[a][P_T], qh[a][P_CP], s->Cref, qh[a][P_U], qh[a][P_V]);",
     "heqs[a] = or_heq(a, qh[a][P_H], qh[a][P_T], Cpf, s->Cref, qh[a][P_U], qh[a][P_V]);",
     BRT + "test_face_flux_matches_brute_force"),
    # Eq. 5-7 as printed (literal_eq7)
    ("literal_liquidus_enthalpy_gated", "*Hl = P->l.cp * P->Tl + P->L;", "*Hl = *cpl * P->Tl + P->L;",
     "test_literal_eq7_closure_values"),
    ("literal_mixture_drops_liquid_fraction", "return Fs * gs + (1.0 - Fs) * Ct * gl", "return Fs * gs + Ct * gl",
     "test_literal_eq7_closure_values"),
    ("literal_sources_gated", "return P->literal_eq7 ? 1.0 : clamp01(C);", "return clamp01(C);",
     BRT + "test_literal_eq7_matches_brute_force"),
]


def _run_mutant(name, orig, planted, pin, workdir):
    """Build the oracle with one planted mistake and run its pin; returns
    (anchor found, pin exit code, pin output)."""
    src = open(SRC).read()
    if src.count(orig) != 1:
        return False, None, ""
    mut_c = os.path.join(workdir, name + ".c")
    mut_so = os.path.join(workdir, "lib" + name + ".so")
    with open(mut_c, "w") as f:
        f.write(src.replace(orig, planted))
    subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-std=c99", "-fPIC", "-shared", "-D_DEFAULT_SOURCE",
                           "-I", os.path.join(ROOT, "oracle"), "-o", mut_so, mut_c, "-lm"])
    env = dict(os.environ, EULBFS_ORACLE_LIB=mut_so)
    node = pin if "::" in pin else PINS + pin
    r = subprocess.run([sys.executable, "-m", "pytest", "-q", "-x", "-p", "no:cacheprovider", node],
                       env=env, cwd=ROOT, capture_output=True, text=True, timeout=600)
    return True, r.returncode, r.stdout[-2000:]


@pytest.fixture(scope="module")
def mutant_results(tmp_path_factory):
    """All mutants built and their pins run concurrently (each in its own
    process), so the suite costs about one pin run per core."""
    workdir = str(tmp_path_factory.mktemp("mutants"))
    with concurrent.futures.ThreadPoolExecutor(max_workers=max(1, min(8, os.cpu_count() or 1))) as ex:
        futs = {m[0]: ex.submit(_run_mutant, *m, workdir) for m in MUTATIONS}
        return {k: f.result() for k, f in futs.items()}


@pytest.mark.parametrize("name,orig,planted,pin", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_pin_catches_planted_mistake(name, orig, planted, pin, mutant_results):
    found, code, out = mutant_results[name]
    assert found, f"mutation anchor for {name} not found exactly once"
    assert code != 0, f"pin {pin} passed on an oracle with '{name}' planted:\n{out}"
