"""Mutation check of the oracle's pins.

Each entry below plants one plausible mistake in a scratch copy of
oracle/oracle.c: a dropped term, a wrong sign, index or coefficient, a
transposed operand, a changed comparison.  The copy is compiled into a
temporary library, and the pins named beside the mistake run against it in
a child pytest process (ORACLE_LIB points the oracle package at the copy).
The check passes only if the child run fails, i.e. some pin catches the
mistake.  The unmodified source, compiled the same way, must pass every pin
named here, so a failure of a planted copy is due to its mistake.

Snippets must occur exactly once in the source; when the oracle changes, an
entry that no longer matches fails loudly instead of testing nothing.
"""
import concurrent.futures as cf
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "oracle.c")

P = "tests/test_oracle_pins.py::"
H = "tests/test_oracle_hilbert.py::"
S = "tests/test_oracle_sph.py::"
L = "tests/test_oracle_learned_mac.py::"
F = "tests/test_oracle_leapfrog.py::"
SO = "tests/test_oracle_softening.py::"
KD = ("            vel[4 * i + a] = vel[4 * i + a] + acc[4 * i + a] * dt_kick;\n"
      "            pos[4 * i + a] = pos[4 * i + a] + vel[4 * i + a] * dt_drift;")

# name: (snippet, replacement, pins expected to catch it)
MUTATIONS = {
    "direct_softening_exponent": (
        "const double mr3 = m * rinv * rinv * rinv;\n            ax += mr3 * dx;",
        "const double mr3 = m * rinv * rinv;\n            ax += mr3 * dx;",
        [P + "test_two_body_closed_form", P + "test_direct_gradient_of_potential"]),
    "direct_potential_sign": (
        "            phi -= m * rinv;",
        "            phi += m * rinv;",
        [P + "test_two_body_closed_form", P + "test_direct_gradient_of_potential"]),
    "direct_self_index": (
        "if (j == skip) continue;",
        "if (j == skip - 1) continue;",
        [P + "test_two_body_closed_form", P + "test_direct_momentum_conservation"]),
    "bbox_degenerate_side": (
        "if (!(L > 0.0f) || !isfinite(inv)) L = 1.0f;",
        "(void)inv;",
        [P + "test_bbox_degenerate"]),
    "morton_bit_order": (
        ": (or_spread3(x, nbits) << 2) | (or_spread3(y, nbits) << 1) | or_spread3(z, nbits);",
        ": (or_spread3(z, nbits) << 2) | (or_spread3(y, nbits) << 1) | or_spread3(x, nbits);",
        [P + "test_morton_golden", P + "test_morton_random_vs_independent"]),
    "key_rounding_not_truncation": (
        "uint32_t ci = (uint32_t)q;",
        "uint32_t ci = (uint32_t)(q + 0.5f);",
        [P + "test_morton_golden", P + "test_morton_random_vs_independent"]),
    "sort_not_stable": (
        "if (keys[a[j]] < keys[a[i]]) tmp[k++] = a[j++];",
        "if (keys[a[j]] <= keys[a[i]]) tmp[k++] = a[j++];",
        [P + "test_sort_matches_numpy_stable"]),
    "tree_leaf_rule": (
        "if (count[v] <= n_leaf || l == max_level) {",
        "if (count[v] < n_leaf || l == max_level) {",
        [P + "test_tree_matches_definition", P + "test_tree_coincident_particles"]),
    "s_eff_theta_placement": (
        "const double t = lside / theta + s;",
        "const double t = lside * theta + s;",
        [P + "test_s_eff_hand_example"]),
    "s_eff_offset_dropped": (
        "const double t = lside / theta + s;",
        "const double t = lside / theta;",
        [P + "test_s_eff_hand_example"]),
    "moment_cross_term": (
        "q[4] += m * y0 * y2;",
        "q[4] += m * y0 * y1;",
        [P + "test_moments_root_and_parallel_axis", P + "test_multipole_convergence_orders"]),
    "quadrupole_potential_sign": (
        "acc[3] -= 0.5 * (3.0 * q * g5 - T * g3);",
        "acc[3] += 0.5 * (3.0 * q * g5 - T * g3);",
        [P + "test_quadrupole_gradient", P + "test_quadrupole_textbook_at_zero_softening"]),
    "quadrupole_coefficient": (
        "const double c = 1.5 * T * g5 - 7.5 * q * g7;",
        "const double c = 1.5 * T * g5 - 5.0 * q * g7;",
        [P + "test_quadrupole_gradient", P + "test_quadrupole_textbook_at_zero_softening"]),
    "quadrupole_transposed_operand": (
        "const double Ir1 = qd[3] * rx + qd[1] * ry + qd[5] * rz;",
        "const double Ir1 = qd[3] * rx + qd[1] * ry + qd[4] * rz;",
        [P + "test_quadrupole_gradient", P + "test_quadrupole_textbook_at_zero_softening"]),
    "group_box_distance": (
        "if (c[a] < lo[a]) t = lo[a] - c[a];\n                else if (c[a] > hi[a]) t = c[a] - hi[a];\n"
        "                d2 += t * t;\n            }\n            const double S = s_eff[v];\n"
        "            const int holds_member",
        "if (c[a] < lo[a]) t = hi[a] - c[a];\n                else if (c[a] > hi[a]) t = c[a] - hi[a];\n"
        "                d2 += t * t;\n            }\n            const double S = s_eff[v];\n"
        "            const int holds_member",
        [P + "test_group_criterion_is_conservative", P + "test_group_walk_follows_the_pinned_lists"]),
    "group_member_nodes_accepted": (
        "const int holds_member = first[v] < ge && (int64_t)first[v] + count[v] > gb;\n"
        "            if (!holds_member) {\n                const double mg",
        "const int holds_member = 0;\n"
        "            if (!holds_member) {\n                const double mg",
        [P + "test_nodes_holding_members_are_opened", P + "test_group_walk_follows_the_pinned_lists"]),
    "groups_not_greedy": (
        "if (run_first >= 0 && run_count + count[ch] <= G) {",
        "if (run_first >= 0 && run_count + count[ch] < G) {",
        [P + "test_groups_greedy_maximal"]),
    "hilbert_gray_step_dropped": (
        "    w[1] ^= w[0];\n    w[2] ^= w[1];\n    uint32_t g = 0;",
        "    w[1] ^= w[0];\n    uint32_t g = 0;",
        [H + "test_first_level_is_gray_code", H + "test_level3_curve_is_face_connected"]),
    "hilbert_reflection_axis": (
        "w[0] ^= low;                              /* reflect */",
        "w[1] ^= low;                              /* reflect */",
        [H + "test_level3_curve_is_face_connected", H + "test_deep_curve_face_connected_and_invertible"]),
    "hilbert_inverse_axis_order": (
        "for (int a = 2; a >= 0; a--) {",
        "for (int a = 0; a < 3; a++) {",
        [H + "test_deep_curve_face_connected_and_invertible"]),
    "sph_kernel_coefficient": (
        "if (q <= 0.5) return c * (1.0 - 6.0 * q * q + 6.0 * q * q * q);",
        "if (q <= 0.5) return c * (1.0 - 6.0 * q * q + 5.0 * q * q * q);",
        [S + "test_kernel_normalised_and_continuous"]),
    "sph_radius_not_strict": (
        "if (r2 < h2) {",
        "if (r2 <= h2) {",
        [S + "test_lattice_counts_and_density"]),
    "sph_self_term_dropped": (
        "double r = (double)pos[4 * i + 3] * or_sph_kernel(0.0, hi);",
        "double r = 0.0;",
        [S + "test_lattice_counts_and_density"]),
    "bf16_truncates": (
        "u += 0x7fffu + lsb;",
        "u += 0u * lsb;",
        [L + "test_forward_bf16_emulation"]),
    "adam_no_bias_correction": (
        "P[k] -= lr * (m[k] / c1) / (sqrt(v[k] / c2) + eps);",
        "P[k] -= lr * m[k] / (sqrt(v[k]) + eps);",
        [L + "test_adam_closed_form"]),
    "pp_softening_doubled": (
        "    const double r2 = dx * dx + dy * dy + dz * dz + e2;\n    const double rinv = 1.0 / sqrt(r2);",
        "    const double r2 = dx * dx + dy * dy + dz * dz + 2.0 * e2;\n    const double rinv = 1.0 / sqrt(r2);",
        [P + "test_theta_to_zero_equals_direct"]),
    "particle_walk_self_term": (
        "if (first[v] != i) {",
        "if (first[v] != i || 1) {",
        [P + "test_theta_to_zero_equals_direct"]),
    "particle_walk_cells_always_softened": (
        "const double e2c = unsoftened_pc ? 0.0 : e2;",
        "const double e2c = e2;",
        [P + "test_particle_walk_unsoftened_cells"]),
    "com_not_divided_by_mass": (
        "cx = sx / M;",
        "cx = sx;",
        [P + "test_moments_root_and_parallel_axis"]),
    "cell_centre_off_by_half": (
        "const double gx = (double)box[0] + (px + 0.5) * lside;",
        "const double gx = (double)box[0] + px * lside;",
        [P + "test_s_eff_hand_example"]),
    "tree_digit_shift": (
        "const int shift = 3 * (max_level - 1 - l);",
        "const int shift = 3 * (max_level - l);",
        [P + "test_tree_matches_definition"]),
    "groups_chunk_size": (
        "OR_EMIT(first[ch] + k, (count[ch] - k < G) ? (count[ch] - k) : G);",
        "OR_EMIT(first[ch] + k, (count[ch] - k < G) ? (count[ch] - k) : G - 1);",
        [P + "test_groups_cut_oversized_leaves_into_chunks_of_G"]),
    "feature_group_radius": (
        "r2 += 0.25 * (hi[a] - lo[a]) * (hi[a] - lo[a]);",
        "r2 += 0.5 * (hi[a] - lo[a]) * (hi[a] - lo[a]);",
        [L + "test_features_hand_case"]),
    "feature_anisotropy_cross_terms": (
        "sqrt(a0 * a0 + a1 * a1 + a2 * a2 + 2 * (qd[3] * qd[3] + qd[4] * qd[4] + qd[5] * qd[5]))",
        "sqrt(a0 * a0 + a1 * a1 + a2 * a2 + (qd[3] * qd[3] + qd[4] * qd[4] + qd[5] * qd[5]))",
        [L + "test_features_hand_case"]),
    "label_against_total_not_node": (
        "const double e = sqrt(dx * dx + dy * dy + dz * dz) / a_tot[i];",
        "const double e = sqrt(dx * dx + dy * dy + dz * dz);",
        [L + "test_labels_exact_cases"]),
    "deep_key_scale": (
        "const float inv = (1024.0f / box[3]) * (float)(1u << (max_level - 10));",
        "const float inv = (1024.0f / box[3]) * (float)(1u << (max_level - 11));",
        [P + "test_deep_keys_extend_shallow_keys", P + "test_deep_keys_hand_corners"]),
    "cell_centre_axes_swapped": (
        "const double px = cell[0] >> (max_level - l), py = cell[1] >> (max_level - l),",
        "const double px = cell[1] >> (max_level - l), py = cell[0] >> (max_level - l),",
        [P + "test_s_eff_hand_example", H + "test_same_octree_for_both_orders"]),
    "sph_kernel_outer_piece": (
        "if (q <= 1.0) return c * 2.0 * (1.0 - q) * (1.0 - q) * (1.0 - q);",
        "if (q <= 1.0) return c * 2.0 * (1.0 - q) * (1.0 - q);",
        [S + "test_kernel_normalised_and_continuous"]),
    "term_magnitude_distance_dropped": (
        "acc[4] += fabs(mr3) * sqrt(dx * dx + dy * dy + dz * dz);",
        "acc[4] += fabs(mr3);",
        [P + "test_term_magnitude_sum"]),
    "learned_network_decision_inverted": (
        "accept = yh < ltau;",
        "accept = yh > ltau;",
        [L + "test_learned_walk_limits"]),
    "learned_fallback_theta": (
        "const double t = side[v] / theta_fb + (s > 0 ? s : 0);",
        "const double t = side[v] / theta_guard + (s > 0 ? s : 0);",
        [L + "test_learned_walk_limits"]),
    "learned_guard_ignores_members": (
        "const int member = first[v] < ge && (int64_t)first[v] + count[v] > gb;\n            int accept = 0;",
        "const int member = 0;\n            int accept = 0;",
        [L + "test_learned_walk_limits"]),
    "particle_walk_leaf_of_one_as_cell": (
        "            if (count[v] == 1) {",
        "            if (count[v] == 0) {",
        [P + "test_particle_walk_single_particle_leaves_are_particles"]),
    "particle_walk_holds_target_ignored": (
        "const int holds_i = first[v] <= i && i < (int64_t)first[v] + count[v];",
        "const int holds_i = 0;",
        [P + "test_particle_walk_equals_group_walk_of_single_particles"]),
    "groups_root_chunks": (
        "OR_EMIT(first[0] + k, (count[0] - k < G) ? (count[0] - k) : G);",
        "OR_EMIT(first[0] + k, G);",
        [P + "test_groups_of_a_root_leaf"]),
    "feature_mass_fraction_base": (
        "f[1] = (cm[3] > 0 && mtot > 0) ? log10(cm[3] / mtot) : -30.0;",
        "f[1] = (cm[3] > 0 && mtot > 0) ? log(cm[3] / mtot) : -30.0;",
        [L + "test_features_hand_case"]),
    "feature_level_scale": (
        "f[4] = level / 10.0;",
        "f[4] = level / 21.0;",
        [L + "test_features_hand_case"]),
    "relu_gradient_gate": (
        "dh2[k] = h2[k] > 0 ? dy * W3[k] : 0;",
        "dh2[k] = dy * W3[k];",
        [L + "test_loss_weights_and_gradient"]),
    "adam_second_moment": (
        "v[k] = b2 * v[k] + (1 - b2) * g[k] * g[k];",
        "v[k] = b2 * v[k] + (1 - b2) * fabs(g[k]);",
        [L + "test_adam_closed_form"]),
    "training_pairs_no_descent": (
        "if (worst > descend_above && nchild[v] > 0)",
        "if (worst > descend_above && nchild[v] < 0)",
        [L + "test_labels_exact_cases"]),
    "learned_range_check_dropped": (
        "if (f[k] < fmin[k] || f[k] > fmax[k]) inrange = 0;",
        "if (f[k] < fmin[k] && f[k] > fmax[k]) inrange = 0;",
        [L + "test_learned_walk_limits"]),
    "learned_fallback_offset": (
        "const double s = sqrt(S) - side[v] / theta_guard;",
        "const double s = sqrt(S);",
        [L + "test_learned_walk_limits"]),
    "bbox_side_smallest_extent": (
        "        if (d > L) L = d;",
        "        if (d < L || L == 0.0f) L = d;",
        [P + "test_bbox_matches_numpy", P + "test_morton_golden"]),
    "hilbert_inverse_gray_decode": (
        "const uint32_t g = w[2] >> 1;                          /* Gray decode */",
        "const uint32_t g = w[2] >> 2;                          /* Gray decode */",
        [H + "test_deep_curve_face_connected_and_invertible"]),
    "morton_decode_axis": (
        "        c[0] = or_compact3(key >> 2, nbits);",
        "        c[0] = or_compact3(key >> 1, nbits);",
        [P + "test_s_eff_hand_example"]),
    "tree_child_level": (
        "                level[nn] = l + 1;",
        "                level[nn] = l;",
        [P + "test_tree_matches_definition"]),
    "cell_side_per_level": (
        "const double lside = (double)box[3] / (double)(1u << l);",
        "const double lside = (double)box[3] / (double)(1u << (l + 1));",
        [P + "test_s_eff_hand_example"]),
    "massless_node_centre": (
        "            cx = gx;",
        "            cx = 0.0;",
        [P + "test_massless_node_takes_cell_centre"]),
    "cell_monopole_sign": (
        "    acc[0] -= M * g3 * rx;",
        "    acc[0] += M * g3 * rx;",
        [P + "test_quadrupole_gradient", P + "test_multipole_convergence_orders"]),
    "pp_force_sign": (
        "    acc[0] += mr3 * dx;",
        "    acc[0] -= mr3 * dx;",
        [P + "test_theta_to_zero_equals_direct"]),
    "quadrupole_g7_exponent": (
        "const double g5 = g3 * g2, g7 = g5 * g2;",
        "const double g5 = g3 * g2, g7 = g5 * g1;",
        [P + "test_quadrupole_gradient", P + "test_quadrupole_textbook_at_zero_softening"]),
    "cell_potential_sign": (
        "    acc[3] -= M * g1;",
        "    acc[3] += M * g1;",
        [P + "test_quadrupole_gradient", P + "test_multipole_convergence_orders"]),
    "pp_potential_sign": (
        "    acc[3] -= m * rinv;",
        "    acc[3] += m * rinv;",
        [P + "test_theta_to_zero_equals_direct"]),
    "pp_softening_exponent": (
        "    const double mr3 = m * rinv * rinv * rinv;\n    acc[0] += mr3 * dx;",
        "    const double mr3 = m * rinv * rinv;\n    acc[0] += mr3 * dx;",
        [P + "test_theta_to_zero_equals_direct"]),
    "s_eff_not_squared": (
        "        s_eff[v] = t * t;",
        "        s_eff[v] = t;",
        [P + "test_s_eff_hand_example"]),
    "moment_diagonal_term": (
        "                q[0] += m * y0 * y0;",
        "                q[0] += m * y0 * y1;",
        [P + "test_moments_root_and_parallel_axis", P + "test_multipole_convergence_orders"]),
    "groups_run_not_reset": (
        "                    run_first = -1;",
        "                    (void)0;",
        [P + "test_groups_partition", P + "test_groups_greedy_maximal"]),
    "groups_oversized_child_not_chunked": (
        "                    if (nchild[ch] == 0)",
        "                    if (nchild[ch] < 0)",
        [P + "test_groups_cut_oversized_leaves_into_chunks_of_G", P + "test_groups_partition"]),
    "particle_walk_cell_count": (
        "                cpc++;",
        "                cpc += 2;",
        [P + "test_particle_walk_single_particle_leaves_are_particles",
         P + "test_particle_walk_equals_group_walk_of_single_particles"]),
    "sph_count_increment": (
        "                c++;",
        "                c += (r2 > 0.0f);",
        [S + "test_coincident_particles_are_neighbours"]),
    "loss_weight_on_wrong_side": (
        "const double w = (yh < Y[i]) ? under_weight : 1.0;",
        "const double w = (yh > Y[i]) ? under_weight : 1.0;",
        [L + "test_loss_weights_and_gradient"]),
    "leapfrog_drift_with_old_velocity": (
        KD,
        "            pos[4 * i + a] = pos[4 * i + a] + vel[4 * i + a] * dt_drift;\n"
        "            vel[4 * i + a] = vel[4 * i + a] + acc[4 * i + a] * dt_kick;",
        [F + "test_one_update_by_hand", F + "test_harmonic_oscillator_closed_form"]),
    "leapfrog_kick_sign": (
        "vel[4 * i + a] + acc[4 * i + a] * dt_kick;",
        "vel[4 * i + a] - acc[4 * i + a] * dt_kick;",
        [F + "test_harmonic_oscillator_closed_form", F + "test_two_body_circular_orbit"]),
    "leapfrog_steps_swapped": (
        KD,
        "            vel[4 * i + a] = vel[4 * i + a] + acc[4 * i + a] * dt_drift;\n"
        "            pos[4 * i + a] = pos[4 * i + a] + vel[4 * i + a] * dt_kick;",
        [F + "test_harmonic_oscillator_closed_form", F + "test_two_body_circular_orbit"]),
    "leapfrog_component_index": (
        "acc[4 * i + a] * dt_kick;",
        "acc[4 * i + (a + 1) % 3] * dt_kick;",
        [F + "test_one_update_by_hand", F + "test_two_body_circular_orbit"]),
    "softening_pair_not_symmetrized": (
        "const double r2 = dx * dx + dy * dy + dz * dz + 0.5 * (ei * ei + ej * ej);",
        "const double r2 = dx * dx + dy * dy + dz * dz + ej * ej;",
        [SO + "test_two_bodies_closed_form_and_symmetry", SO + "test_momentum_is_conserved"]),
    "softening_cell_unweighted_mean": (
        "            sm += m;\n            se += m * e * e;",
        "            sm += (m != 0.0);\n            se += (m != 0.0) * e * e;",
        [SO + "test_cell_softening_is_the_mass_weighted_mean",
         SO + "test_cell_softening_cancels_the_first_order_term"]),
    "softening_cell_term_target_only": (
        "(unsoftened_pc ? 0.0 : 0.5 * (ei2 + e2bar[v]))",
        "(unsoftened_pc ? 0.0 : ei2)",
        [SO + "test_particle_walk_cell_term_uses_the_pair_mean"]),
    "softening_particle_node_target_only": (
        "spos + 4 * (int64_t)first[v], eps_s ? 0.5 * (ei2 + ej * ej) : e2, acc);",
        "spos + 4 * (int64_t)first[v], eps_s ? ei2 : e2, acc);",
        [SO + "test_particle_walk_at_theta_to_zero_is_the_direct_sum"]),
}


def _pins(ids):
    env = dict(os.environ)
    return subprocess.run([sys.executable, "-m", "pytest", "-q", "-x", "-p", "no:cacheprovider", "-m", "not gpu"]
                          + ids, cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)


@pytest.fixture(scope="module")
def mutants(tmp_path_factory):
    from oracle import build as ob
    src = open(SRC).read()
    d = tmp_path_factory.mktemp("oracle_mutants")

    def one(item):
        name, (old, new, _) = item
        if name == "_control":
            text = src
        else:
            assert src.count(old) == 1, "snippet of %s occurs %d times" % (name, src.count(old))
            text = src.replace(old, new)
        c = d / (name + ".c")
        c.write_text(text)
        out = str(d / (name + ".so"))
        ok, err = ob.compile_to(str(c), out)
        assert ok, name + ": " + err
        return name, out

    items = list(MUTATIONS.items()) + [("_control", ("", "", []))]
    with cf.ThreadPoolExecutor(8) as ex:
        return dict(ex.map(one, items))


def test_unmodified_oracle_passes_the_named_pins(mutants, monkeypatch):
    ids = sorted({t for _, _, ts in MUTATIONS.values() for t in ts})
    monkeypatch.setenv("ORACLE_LIB", mutants["_control"])
    r = _pins(ids)
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-2000:]


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_planted_mistake_fails_a_pin(mutants, monkeypatch, name):
    monkeypatch.setenv("ORACLE_LIB", mutants[name])
    r = _pins(MUTATIONS[name][2])
    assert r.returncode != 0, "no pin caught the planted mistake %r:\n%s" % (name, r.stdout[-2000:])
