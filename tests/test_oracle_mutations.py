"""The oracle's pins are strong enough to catch plausible mistakes.

Each case plants one mistake (a dropped term, a wrong sign, a swapped index
or operand, a changed constant) in a copy of the oracle's C source, builds
it on the CPU, and checks that at least one of the named pin tests fails.
Nothing here touches the GPU or the CUDA planner.
"""
import os
import subprocess

import pytest

import oracle

from tests import test_oracle_dynamics as dyn
from tests import test_oracle_geometry as geo
from tests import test_oracle_refine as ref
from tests import test_oracle_remap as rmp
from tests import test_oracle_revalidate as rv
from tests import test_oracle_sampling as smp
from tests import test_oracle_steps as stp

SRC = os.path.join(os.path.dirname(oracle.__file__), "kpx_oracle.c")

MUTATIONS = [
    ("philox_swap_products", "uint32_t n0 = hi1 ^ c1 ^ k0;", "uint32_t n0 = hi0 ^ c1 ^ k0;",
     [smp.test_philox_known_answers]),
    ("philox_key_bump", "k1 += W1;", "k1 += W0;", [smp.test_philox_known_answers]),
    ("sample_shift", "(float)(w[i] >> 8) * 0x1p-24f", "(float)(w[i] >> 9) * 0x1p-23f",
     [smp.test_sample_wiring_against_kat]),
    ("sample_k_word", "(uint64_t)w[P->m] * range", "(uint64_t)w[P->m - 1] * range",
     [smp.test_sample_wiring_against_kat]),
    ("sample_counter_order", "uint32_t ctr[4] = {iter, node, sample, 0u};",
     "uint32_t ctr[4] = {node, iter, sample, 0u};", [smp.test_seed_words_and_counter_fields]),
    ("euler_half_step", "x_next[i] = x[i] + h * k1[i];", "x_next[i] = x[i] + 0.5 * h * k1[i];",
     [dyn.test_di_euler_closed_form]),
    ("rk4_weight", "2.0 * k3[i] + k4[i]", "1.0 * k3[i] + k4[i]",
     [dyn.test_di_rk4_exact_for_quadratic, dyn.test_dubins_circle_convergence_orders]),
    ("rk4_stage", "tmp[i] = x[i] + h * k3[i];", "tmp[i] = x[i] + 0.5 * h * k3[i];",
     [dyn.test_di_rk4_exact_for_quadratic, dyn.test_dubins_circle_convergence_orders]),
    ("dubins_sin_cos", "dx[0] = v * cos(psi) * cos(gam);", "dx[0] = v * sin(psi) * cos(gam);",
     [dyn.test_dubins_straight_flight]),
    ("dubins_climb", "dx[2] = v * sin(gam);", "dx[2] = v * cos(gam);", [dyn.test_dubins_straight_flight]),
    ("quad_r13_sign", "double r13 = cpsi * sth * cphi + spsi * sphi;",
     "double r13 = cpsi * sth * cphi - spsi * sphi;", [dyn.test_quad_rotation_column_hand_values]),
    ("quad_r23_sign", "double r23 = spsi * sth * cphi - cpsi * sphi;",
     "double r23 = spsi * sth * cphi + cpsi * sphi;", [dyn.test_quad_rotation_column_hand_values]),
    ("quad_gravity", "dx[8] = a * r33 - g;", "dx[8] = a * r33 + g;", [dyn.test_quad_free_fall_and_hover]),
    ("quad_W_row2", "dx[4] = cphi * q - sphi * r;", "dx[4] = cphi * q + sphi * r;",
     [dyn.test_quad_euler_rates_hand_values]),
    ("quad_W_row1", "dx[3] = p + sphi * tth * q + cphi * tth * r;", "dx[3] = p + sphi * tth * r + cphi * tth * q;",
     [dyn.test_quad_euler_rates_hand_values]),
    ("quad_gyro_sign", "dx[9] = (u[1] - (Jz - Jy) * q * r) / Jx;", "dx[9] = (u[1] + (Jz - Jy) * q * r) / Jx;",
     [dyn.test_quad_gyroscopic_term]),
    ("quad_inertia_index", "dx[10] = (u[2] - (Jx - Jz) * r * p) / Jy;", "dx[10] = (u[2] - (Jx - Jz) * r * p) / Jx;",
     [dyn.test_quad_gyroscopic_term]),
    ("path_drop_dz", "len += sqrt(dx * dx + dy * dy + dz * dz);", "len += sqrt(dx * dx + dy * dy);",
     [dyn.test_edge_costs]),
    ("effort_square", "e += t * t;", "e += t;", [dyn.test_edge_costs]),
    ("open_box", "if (x[0] >= o[0] && x[0] <= o[3]", "if (x[0] > o[0] && x[0] <= o[3]",
     [geo.test_closed_boxes_and_bounds]),
    ("workspace_open", "if (!(x[a] >= P->ws_lo[a] && x[a] <= P->ws_hi[a])) return 0;",
     "if (!(x[a] > P->ws_lo[a] && x[a] <= P->ws_hi[a])) return 0;", [geo.test_closed_boxes_and_bounds]),
    ("cheb_min", "double e = lo > hi ? lo : hi;", "double e = lo < hi ? lo : hi;",
     [geo.test_margin_and_clearance_hand_values]),
    ("region_no_clamp_hi", "if (c > bins - 1) c = bins - 1;", "(void)0;", [geo.test_region_map_hand_values]),
    ("region_radix_order", "id = id * bins + c;", "id = id + c * bins;", [geo.test_region_map_hand_values]),
    ("region_no_wrap", "xf = xf - w;", "xf = xf;", [geo.test_region_yaw_wrap]),
    ("goal_open_ball", "return d2 <= P->goal_r * P->goal_r;", "return d2 < P->goal_r * P->goal_r;",
     [geo.test_goal_ball]),
    ("select_no_filter", "if (key[c] == region_key[region[c]]) winners[w++] = c;", "winners[w++] = c;",
     [stp.test_select_winners_min_ties_and_filter]),
    ("select_no_restore", "region_key[r] = region_snap[r];", "(void)r;", [stp.test_select_winners_capacity]),
    ("append_no_region_key", "region_key[cregion[k]] = key[id];", "(void)id;",
     [stp.test_append_rows_keys_and_solution]),
    ("append_key_slot_id", "key[id] = kpo_pack_key((float)ccost[k], (uint32_t)id);",
     "key[id] = kpo_pack_key((float)ccost[k], (uint32_t)k);", [stp.test_append_rows_keys_and_solution]),
    ("append_goal_any", "if (cgoal[k] && key[id] < *goal_key) {", "if (key[id] < *goal_key) {",
     [stp.test_append_rows_keys_and_solution]),
    ("prune_rule2_drops_best", "if (icount[i] > i_max && best) continue;", "if (icount[i] > i_max) continue;",
     [stp.test_prune_reactivation_after_imax]),
    ("prune_terminal_skip_dropped", "if (set[i] == KPO_SET_T) continue;", "(void)0;",
     [stp.test_prune_inactive_not_best_goes_terminal_and_t_is_permanent]),
    ("prune_parent_only", "for (int32_t p = parent[i]; p >= 0; p = parent[p]) {",
     "for (int32_t p = parent[i]; p >= 0; p = -1) {", [stp.test_prune_ancestor_chain_is_strict_and_reaches_root]),
    ("compact_off_by_one", "if (mask[i]) I[acc++] = i;", "if (mask[i] && i + 1 < n) I[acc++] = i;",
     [stp.test_compaction_paper_example]),
    # refinement objective and its reverse-mode gradient
    ("box_inside_sign", "return -best;", "return best;", [ref.test_box_distance_hand_values]),
    ("box_outside_norm", "grad[a] = (p[a] - q[a]) / d;", "grad[a] = (p[a] - q[a]);",
     [ref.test_box_distance_hand_values]),
    ("vjp_phi_row1_sign", "gx[3] += a[3] * (cphi * tth * q - sphi * tth * r);",
     "gx[3] += a[3] * (cphi * tth * q + sphi * tth * r);", [ref.test_gradient_matches_central_differences]),
    ("vjp_thrust_column", "gu[0] = (a[6] * r13 + a[7] * r23 + a[8] * r33) / mass;",
     "gu[0] = (a[6] * r13 + a[7] * r23 + a[8] * r13) / mass;", [ref.test_thrust_gradient_at_hover_closed_form]),
    ("vjp_torque_index", "gu[3] = a[11] / Jz;", "gu[3] = a[10] / Jz;", [ref.test_gradient_matches_central_differences]),
    ("vjp_gyro_drop", "gx[9] += -a[11] * (Jy - Jx) * q / Jz;", "(void)0;",
     [ref.test_gradient_matches_central_differences]),
    ("rk4_adjoint_weight", "ak2[i] = h / 3.0 * lam[i];", "ak2[i] = h / 6.0 * lam[i];",
     [ref.test_gradient_matches_central_differences, ref.test_thrust_gradient_at_hover_closed_form]),
    ("rk4_adjoint_stage", "ak3[i] += h * g[i];", "ak3[i] += 0.5 * h * g[i];",
     [ref.test_gradient_matches_central_differences]),
    ("penalty_grad_sign", "g3[a] -= s * gd[a];", "g3[a] += s * gd[a];", [ref.test_gradient_matches_central_differences]),
    ("effort_grad_factor", "g4[0] += dur * R->w_effort * 2.0 * (u[0] - mg) / (mg * mg);",
     "g4[0] += dur * R->w_effort * (u[0] - mg) / (mg * mg);", [ref.test_effort_cost_and_gradient_closed_form]),
    ("goal_grad_factor", "lam[a] = 2.0 * R->w_goal * e;", "lam[a] = R->w_goal * e;",
     [ref.test_thrust_gradient_at_hover_closed_form]),
    ("softplus_scale", "return (t > 0.0 ? t + log1p(exp(-t)) : log1p(exp(t))) / beta;",
     "return (t > 0.0 ? t + log1p(exp(-t)) : log1p(exp(t)));", [ref.test_penalty_value_by_hand]),
    ("validate_no_check", "if (!kpo_point_valid(P, x)) ok = 0;", "(void)0;", [ref.test_validate_controls]),
    # FP64 re-validation of a returned trajectory and the returned trajectory itself
    ("revalidate_always_ok", "return (clear >= -1e-4 && *goal_slack >= -1e-4 && worst <= 1e-4) ? 1 : 0;",
     "return 1;", [rv.test_revalidate_rejects_one_point_in_thin_box, rv.test_revalidate_rejects_missing_the_goal]),
    ("revalidate_no_step_clearance",
     "for (int k = 1; k <= kdone; ++k) clear = fmin(clear, kpo_point_clearance(P, traj + (int64_t)k * n));",
     "(void)kdone;", [rv.test_revalidate_rejects_one_point_in_thin_box]),
    ("revalidate_no_goal_test", "clear >= -1e-4 && *goal_slack >= -1e-4 && worst <= 1e-4",
     "clear >= -1e-4 && worst <= 1e-4", [rv.test_revalidate_rejects_missing_the_goal]),
    ("revalidate_goal_slack_sign", "*goal_slack = P->goal_r - sqrt(d2);", "*goal_slack = sqrt(d2) - P->goal_r;",
     [rv.test_revalidate_accepts_valid_flight, rv.test_revalidate_rejects_missing_the_goal]),
    ("revalidate_no_consistency", "clear >= -1e-4 && *goal_slack >= -1e-4 && worst <= 1e-4",
     "clear >= -1e-4 && *goal_slack >= -1e-4", [rv.test_revalidate_rejects_inconsistent_stored_state]),
    ("revalidate_start_unchecked", "clear = fmin(clear, kpo_point_clearance(P, states));", "(void)0;",
     [rv.test_revalidate_rejects_start_in_box]),
    ("revalidate_cost_last_only", "total += ec;", "total = ec;", [rv.test_revalidate_accepts_valid_flight]),
    ("revalidate_goal_on_previous_state", "const double* xl = states + (int64_t)len * n;",
     "const double* xl = states + (int64_t)(len - 1) * n;", [rv.test_revalidate_rejects_missing_the_goal]),
    ("revalidate_tolerance_loose", "return (clear >= -1e-4 && *goal_slack >= -1e-4 && worst <= 1e-4)",
     "return (clear >= -1e-2 && *goal_slack >= -1e-2 && worst <= 1e-2)",
     [rv.test_revalidate_rejects_one_point_in_thin_box, rv.test_revalidate_rejects_missing_the_goal,
      rv.test_revalidate_rejects_inconsistent_stored_state]),
    ("best_traj_steps_of_parent", "steps[k - 1] = v->K[p];", "steps[k - 1] = v->K[v->parent[p]];",
     [rv.test_best_trajectory_is_the_parent_walk]),
    ("best_traj_cost_of_parent", "*out_cost = v->cost[id];", "*out_cost = v->cost[v->parent[id]];",
     [rv.test_best_trajectory_is_the_parent_walk]),
    ("best_traj_skips_goal_node", "int32_t id = (int32_t)(v->goal_key & 0xFFFFFFFFu);",
     "int32_t id = v->parent[(int32_t)(v->goal_key & 0xFFFFFFFFu)];", [rv.test_best_trajectory_is_the_parent_walk]),
    ("best_traj_controls_shift", "controls[(int64_t)(k - 1) * v->m + d] = v->u[(int64_t)p * v->m + d];",
     "controls[(int64_t)(k - 1) * v->m + d] = v->u[(int64_t)v->parent[p] * v->m + d];",
     [rv.test_best_trajectory_is_the_parent_walk]),
    # region remap (adaptive delta)
    ("remap_terminal_holds_region", "if (set[i] != KPO_SET_T && key[i] < region_key[region[i]])",
     "if (key[i] < region_key[region[i]])", [rmp.test_remap_hand_example]),
    ("remap_terminal_dominated", "dominated[i] = (set[i] != KPO_SET_T && key[i] != region_key[region[i]])",
     "dominated[i] = (key[i] != region_key[region[i]])", [rmp.test_remap_hand_example]),
]


@pytest.fixture(scope="module")
def src_text():
    with open(SRC) as f:
        return f.read()


@pytest.mark.parametrize("name,old,new,pins", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_planted_mistake_is_caught(name, old, new, pins, src_text, tmp_path, monkeypatch):
    assert src_text.count(old) >= 1, "mutation anchor not found: " + name
    mutated = src_text.replace(old, new, 1)
    csrc = tmp_path / "kpx_oracle.c"
    csrc.write_text(mutated)
    hdr = os.path.join(os.path.dirname(SRC), "kpx_oracle.h")
    (tmp_path / "kpx_oracle.h").write_text(open(hdr).read())
    so = tmp_path / ("lib_%s.so" % name)
    subprocess.run(["gcc", "-O2", "-std=c11", "-D_DEFAULT_SOURCE", "-fPIC", "-shared", "-ffp-contract=off",
                    "-o", str(so), str(csrc), "-lm"], check=True, capture_output=True)
    monkeypatch.setattr(oracle, "_lib", oracle.load_library(str(so)))
    failures = 0
    for pin in pins:
        try:
            pin(oracle)
        except AssertionError:
            failures += 1
    assert failures >= 1, "planted mistake %s went unnoticed" % name
