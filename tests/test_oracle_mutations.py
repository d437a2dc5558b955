"""The oracle's pins are sharp enough: plant plausible mistakes in copies of the
oracle source (on the CPU), rebuild, and check that some pin fails for each.

Each mutation is a one-token slip of the kind a restatement of the paper could
contain: a wrong sign, a dropped factor, a transposed index, a wrong time level.
"""
from __future__ import annotations

import os
import tempfile

import pytest

import oracle
from tests import test_oracle as T
from tests import test_oracle_adjoint as TA
from tests import test_oracle_subcycle as TS

# (name, original text, planted text)
MUTATIONS = [
    ("cross product sign", "r[0] = a[1] * b[2] - a[2] * b[1];", "r[0] = a[2] * b[1] - a[1] * b[2];"),
    ("TSC centre weight", "w[1] = 0.75 - d * d;", "w[1] = 0.75 - 0.5 * d * d;"),
    ("TSC side weight", "w[2] = 0.5 * (0.5 + d) * (0.5 + d);", "w[2] = 0.5 * (0.5 - d) * (0.5 + d);"),
    ("CIC weight swap", "w[0] = 1.0 - f;\n        w[1] = f;", "w[0] = f;\n        w[1] = 1.0 - f;"),
    ("second half kick dropped", "u1[q] = up[q] + h * E[q];", "u1[q] = up[q];"),
    ("h without the 1/2", "return K * p->dt / 2.0;", "return K * p->dt;"),
    ("c/c~ inverted in the push", "double K = (p->c_tilde / p->c)", "double K = (p->c / p->c_tilde)"),
    ("momentum source sign", "Q[4 + q] = -Nq * (E[q] + bxB[q]);", "Q[4 + q] = Nq * (E[q] + bxB[q]);"),
    ("E dropped from momentum source", "Q[4 + q] = -Nq * (E[q] + bxB[q]);", "Q[4 + q] = -Nq * bxB[q];"),
    ("beta_bar at the new gamma", "bbar[q] = (up[q] + um[q]) / (2.0 * gm);", "bbar[q] = (up[q] + um[q]) / (g1 + g0);"),
    ("energy source at the mid gamma", "Q[7] = -Nq * p->c * dot(E, sum) / (g1 + g0);", "Q[7] = -Nq * p->c * dot(E, sum) / (2.0 * gm);"),
    ("current at the old momentum", "Q[1 + q] = Nq * p->c * u1[q] / g1;", "Q[1 + q] = Nq * p->c * u1[q] / g0;"),
    ("drift with the old gamma", "adv * u1[0] / g1, p->nx);", "adv * u1[0] / g0, p->nx);"),
    ("drift with true c", "double adv = p->dt * p->c_tilde / p->dx;", "double adv = p->dt * p->c / p->dx;"),
    ("rotation vector t not divided by gamma", "t[q] = h * B[q] / *gm;", "t[q] = h * B[q];"),
    ("gather index transposed", "int64_t node = ((int64_t)kz * p->ny + ky) * p->nx + kx;\n                for (int q = 0; q < 6; ++q)",
     "int64_t node = ((int64_t)kx * p->ny + ky) * p->nx + kz;\n                for (int q = 0; q < 6; ++q)"),
    ("energy density missing c", "Q[4] = N * g * m * p->c * p->c;", "Q[4] = N * g * m * p->c;"),
    ("total momentum missing m", "out[1 + q] += N * m * p->c * u[q];", "out[1 + q] += N * p->c * u[q];"),
    ("cell key x/y swapped", "(lz * bin + ly) * bin + lx;", "(lz * bin + lx) * bin + ly;"),
    ("carry into the wrong cell", "int ci = *cell + (int)k;", "int ci = *cell - (int)k;"),
    ("TSC anchor at the lower node", "if (shape == 2 && f >= 0.5)", "if (shape == 2 && f > 1.0)"),
    ("losses without c~/c", "double rate = (p->c_tilde / p->c) * sigma", "double rate = sigma"),
    ("losses at gamma not beta", "double beta = sqrt(dot(u, u)) / g;", "double beta = g;"),
    ("tangent: TSC weight slope sign", "dw[1] = -2.0 * d;", "dw[1] = 2.0 * d;"),
    ("tangent: y weight derivative along x", "w[0][a] * dw[1][b] * w[2][c] * dxj[1] +",
     "w[0][a] * dw[1][b] * w[2][c] * dxj[0] +"),
    ("tangent: rotation vector without its gamma term",
     "dtt[q] = h * dB[q] / gm - h * B[q] * dgm / (gm * gm);", "dtt[q] = h * dB[q] / gm;"),
    ("tangent: drift without the gamma term",
     "dxj[q] += adv * (du1[q] / g1 - u1[q] * dg1 / (g1 * g1));", "dxj[q] += adv * du1[q] / g1;"),
    ("sub-cycling: gyro limit without c~/c", "double omega = ((p->c_tilde / p->c) * fabs(p->q_over_m) / p->c)",
     "double omega = (fabs(p->q_over_m) / p->c)"),
    ("sub-cycling: gyro limit without gamma", "* bmag / g;", "* bmag;"),
    ("sub-cycling: Courant limit at the true c", "double t_cross = (p->dx / p->c_tilde) / beta;",
     "double t_cross = (p->dx / p->c) / beta;"),
    ("sub-cycling: deposit weight not averaged", "double wsub = ldexp(P->w[j], -k);", "double wsub = P->w[j];"),
    ("sub-cycling: boundary level rejected", "while (k < max_level && dts > limit)",
     "while (k < max_level && dts >= limit)"),
    ("sub-cycling: loss limit without c~/c", "double t_loss = (1.0 / ((p->c_tilde / p->c) * sigma_nn * p->c)) / beta;",
     "double t_loss = (1.0 / (sigma_nn * p->c)) / beta;"),
    ("tangent: deposit weights frozen", "dG[q * ncell + nodes[k]] += dWk[k] * S[q] + Wk[k] * dS[q];",
     "dG[q * ncell + nodes[k]] += Wk[k] * dS[q];"),
    ("c~/c applied twice in the push", "double K = (p->c_tilde / p->c)",
     "double K = (p->c_tilde / p->c) * (p->c_tilde / p->c)"),
]

PINS = [
    lambda: [T.test_weights_match_textbook_bspline(s) for s in (1, 2)],
    lambda: [T.test_weights_moments(s) for s in (1, 2)],
    lambda: [T.test_gather_bruteforce(s) for s in (1, 2)],
    T.test_pure_electric_kick_exact,
    T.test_pure_electric_acceleration_orbit,
    T.test_rotation_preserves_norm_and_uses_beta_bar,
    T.test_gyration_discrete_closed_form,
    T.test_gyrofrequency_scales_with_c_tilde,
    T.test_exb_drift_velocity,
    lambda: [T.test_deposit_bruteforce_and_momentum_exchange(s) for s in (1, 2)],
    lambda: [T.test_conserved_momentum_and_energy(s) for s in (1, 2)],
    lambda: [T.test_state_moments_bruteforce(s) for s in (1, 2)],
    T.test_drift_carry_keeps_offsets_in_range,
    T.test_moments_change_with_c_in_time_units,
    lambda: T.test_cell_key_bijective_and_bin_major((5, 6, 7), 2),
    lambda: T.test_cell_key_bijective_and_bin_major((8, 8, 8), 8),
    lambda: [T.test_anchor_node_is_floor_or_nearest(s) for s in (1, 2)],
    T.test_losses_closed_form_uniform_density,
    T.test_losses_per_distance_independent_of_c_tilde,
    lambda: TA.test_tangent_fd_static(steps=6, n_dirs=2),
    TS.test_level_rule,
    TS.test_gyro_level_and_phase_closed_form,
    TS.test_courant_level_and_straight_line,
    TS.test_loss_limit_level,
    lambda: TS.test_exchange_identities_subcycled(2),
    T.test_comoving_gas_zero_net_force,
    T.test_moving_waves_c_tilde_independent_statistics,
]

# Mistakes that the two statistical pins of Sec. 2 must catch on their own:
# c~-independence of the steady state in moving waves, and no net force on a
# comoving gas.
NAMED = [
    ("drift with true c", T.test_moving_waves_c_tilde_independent_statistics),
    ("E dropped from momentum source", T.test_comoving_gas_zero_net_force),
    ("c~/c applied twice in the push", T.test_comoving_gas_zero_net_force),
]


def _mutated(name):
    orig, planted = {m[0]: m[1:] for m in MUTATIONS}[name]
    src = oracle.source()
    assert src.count(orig) == 1, f"mutation anchor not unique: {name}"
    return src.replace(orig, planted)


@pytest.mark.parametrize("name,orig,planted", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_planted_mistake_is_caught(name, orig, planted):
    bad = _mutated(name)
    with tempfile.TemporaryDirectory() as d:
        so = oracle.compile_source(bad, os.path.join(d, "mut.so"))
        caught = False
        with oracle.use_library(so):
            for pin in PINS:
                try:
                    pin()
                except AssertionError:
                    caught = True
                    break
        assert caught, f"no pin caught the planted mistake: {name}"


@pytest.mark.parametrize("name,pin", NAMED, ids=[f"{m} / {p.__name__}" for m, p in NAMED])
def test_statistical_pin_catches_its_mistake(name, pin):
    with tempfile.TemporaryDirectory() as d:
        so = oracle.compile_source(_mutated(name), os.path.join(d, "mut.so"))
        with oracle.use_library(so):
            with pytest.raises(AssertionError):
                pin()
