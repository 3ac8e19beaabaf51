"""Planted mistakes: copies of the oracle with one plausible error each (a dropped or wrong
coefficient, a flipped sign, a transposed operand, a wrong index) must fail at least one pin.
This checks that the pins constrain the oracle; the oracle itself is never modified."""
import math

import numpy as np
import pytest

import test_oracle_mrs as TM
import test_oracle_rod as TR
import test_oracle_rot as TS


def fails(fn, *a):
    try:
        fn(*a)
    except AssertionError:
        return True
    return False


MRS_PINS = [
    lambda o: TM.test_stokeslet_solves_regularized_stokes(o, 0.3),
    lambda o: TM.test_stokeslet_solves_regularized_stokes(o, 1.0),
    lambda o: TM.test_angular_velocity_is_half_curl(o, 0.5),
    lambda o: TM.test_angular_velocity_is_half_curl(o, 4.0),
    lambda o: TM.test_far_field_recovers_singular_kernels(o),
    lambda o: TM.test_self_term_closed_form(o),
    lambda o: TM.test_mobility_symmetric_psd(o, "rod", 1.5),
    lambda o: TM.test_equivariances(o),
    lambda o: TM.test_two_point_case_exact(o, ("1/3", "1/5", "-1/7")),
]

MRS_MUTANTS = {
    "H1_coefficient": [("H[0] = (r2 + 2.0 * e2)", "H[0] = (r2 + 1.0 * e2)")],
    "H2_power": [("H[1] = 1.0 / (8.0 * ORC_PI * d15);", "H[1] = 1.0 / (8.0 * ORC_PI * d25);")],
    "H3_coefficient": [("H[2] = (2.0 * r2 + 5.0 * e2)", "H[2] = (2.0 * r2 + 4.0 * e2)")],
    "H4_sign": [("- 7.0 * e2 * r2", "+ 7.0 * e2 * r2")],
    "H4_dropped_term": [("- 2.0 * r2 * r2)", ")")],
    "H5_coefficient": [("H[4] = (6.0 * r2 + 21.0 * e2)", "H[4] = (6.0 * r2 + 12.0 * e2)")],
    "rotlet_sign": [("nxr[c] * H[2]", "-nxr[c] * H[2]")],
    "cross_transposed": [("cross3(fj, r, fxr);", "cross3(r, fj, fxr);")],
    "separation_sign": [("r[0] = xt[3*i + 0] - X[3*j + 0];", "r[0] = X[3*j + 0] - xt[3*i + 0];")],
    "dipole_dot_index": [("const double nr = dot3(nj, r);", "const double nr = dot3(fj, r);")],
    "viscosity_dropped": [("u[3*i + c] = ui[c] / mu;", "u[3*i + c] = ui[c];")],
}


@pytest.mark.parametrize("name", sorted(MRS_MUTANTS))
def test_mrs_mutant_is_caught(name):
    import oracle
    v = oracle.variant(MRS_MUTANTS[name], "mrs_" + name)
    assert any(fails(pin, v) for pin in MRS_PINS), name


ROD_PINS = [
    lambda o: TR.test_force_is_minus_energy_gradient(o),
    lambda o: TR.test_torque_is_minus_energy_rotation_derivative(o),
    lambda o: TR.test_total_force_and_torque_vanish(o),
    lambda o: TR.test_initial_sinusoid_forces_vanish_at_second_order(o),
    lambda o: TR.test_objectivity(o),
    lambda o: TR.test_energy_decreases_under_euler_flow(o),
    lambda o: TR.test_convergence_order(o, 1, 2),
    lambda o: TR.test_rodrigues_update_matches_library_rotation(o),
]

ROD_MUTANTS = {
    "force_sign": [("gk[q] += Fs[3*k + q]; mk[q] += Ns[3*k + q];",
                    "gk[q] -= Fs[3*k + q]; mk[q] += Ns[3*k + q];")],
    "half_cross_term": [("for (int q = 0; q < 3; ++q) mk[q] += 0.5 * cr[q];\n            }\n            if (k > 0)",
                         "for (int q = 0; q < 3; ++q) mk[q] += 1.0 * cr[q];\n            }\n            if (k > 0)")],
    "moment_index": [("const double Ni = p->a[i] * (dot3(dD, Dh + 3*l) - Om[i]);",
                      "const double Ni = p->a[i] * (dot3(dD, Dh + 3*j) - Om[i]);")],
    "stretch_reference": [("(jj == 2 ? 1.0 : 0.0)", "(jj == 1 ? 1.0 : 0.0)")],
    "mid_frame_unrotated": [("Dh[3*i + r] = S[3*r + 0] * Dk[3*i + 0] + S[3*r + 1] * Dk[3*i + 1] + S[3*r + 2] * Dk[3*i + 2];",
                             "Dh[3*i + r] = Dk[3*i + r];")],
    "rodrigues_sign": [("ct * Di[q] + st * exD[q]", "ct * Di[q] - st * exD[q]")],
    "rk2_stage_time": [("t + 0.5 * dt, g, m, u, w);", "t, g, m, u, w);"),
                       ("Xh[q] = X[q] + u[q] * (0.5 * dt);", "Xh[q] = X[q] + u[q] * (1.0 * dt);")],
}


@pytest.mark.parametrize("name", sorted(ROD_MUTANTS))
def test_rod_mutant_is_caught(name):
    import oracle
    v = oracle.variant(ROD_MUTANTS[name], "rod_" + name)
    assert any(fails(pin, v) for pin in ROD_PINS), name


SQRT_MUTANTS = {
    "skew_sign": [("+ sh * K[3*r + q];", "- sh * K[3*r + q];")],
    "full_angle": [("const double ch = cos(0.5 * theta), sh = sin(0.5 * theta);",
                    "const double ch = cos(theta), sh = sin(theta);")],
    "axis_index": [("const double v[3] = { R[7] - R[5], R[2] - R[6], R[3] - R[1] };",
                    "const double v[3] = { R[5] - R[7], R[2] - R[6], R[3] - R[1] };")],
    "near_pi_sign": [("if (dot3(nv, v) < 0.0)", "if (dot3(nv, v) > 0.0)")],
}


@pytest.mark.parametrize("name", sorted(SQRT_MUTANTS))
def test_sqrt_mutant_is_caught(name):
    import oracle
    v = oracle.variant(SQRT_MUTANTS[name], "sqrt_" + name)
    pins = [lambda o: TS.test_paper_sweep_accuracy_and_table2(o),
            lambda o: TS.test_matches_scipy_sqrtm_away_from_pi(o),
            lambda o: TS.test_endpoints(o)]
    assert any(fails(pin, v) for pin in pins), name
