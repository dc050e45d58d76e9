"""The oracle's pins are sharp: each entry below plants one plausible mistake (a dropped term, a wrong sign,
index, bound or operand) in a copy of the oracle's C source, rebuilds the copy, and runs the pins meant to
catch it, which must fail.  The unchanged copy passes the same pins first, so a failure is the mistake's.

CPU only; the copies build and run in parallel, one OpenMP thread each.
"""
import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PRIM = "tests/test_oracle_primitives.py::"
METH = "tests/test_oracle_method.py::"

# (file, original text, planted text, pins that must catch it)
MUTANTS = [
    # bilinear sampling (exact on affine ramps; clamped at the border)
    ("oracle_core.c", "out[c] = (1.0 - fy) * ((1.0 - fx) * a + fx * b) + fy * ((1.0 - fx) * d + fx * e);",
     "out[c] = (1.0 - fx) * ((1.0 - fy) * a + fy * b) + fx * ((1.0 - fy) * d + fy * e);",
     [PRIM + "test_bilinear_reproduces_affine_ramp"]),
    ("oracle_core.c", "    if (X > W - 1) X = W - 1;\n", "",
     [PRIM + "test_bilinear_integer_points_and_clamping"]),
    # warped patch cost (eq. 3 over a patch): a dropped channel, the plane's offset taken from p instead of G(p)
    ("oracle_core.c", "            sum += fabs(a[0] - s[0]) + fabs(a[1] - s[1]) + fabs(a[2] - s[2]);\n        }\n    }",
     "            sum += fabs(a[0] - s[0]) + fabs(a[1] - s[1]);\n        }\n    }",
     [PRIM + "test_identity_and_translation_planes_reduce_to_square_patch",
      PRIM + "test_warped_cost_closed_form_on_projective_ramp"]),
    ("oracle_core.c", "X = px + vx + (gx - gpx);", "X = px + vx + (gx - px);",
     [PRIM + "test_warped_cost_closed_form_on_projective_ramp"]),
    # PatchMatch: random initial targets inside the frame; propagation from all four neighbours
    ("oracle_core.c", "ty = (int)(w[1] % (uint32_t)H);", "ty = (int)(w[1] % (uint32_t)W);",
     [METH + "test_pm_init_targets_inside_frame_and_deterministic"]),
    ("oracle_core.c", "NY[4] = {0, 0, -1, 1};\n            for (int k = 0; k < 4; ++k) {\n                int nx",
     "NY[4] = {0, 0, -1, -1};\n            for (int k = 0; k < 4; ++k) {\n                int nx",
     [METH + "test_propagation_takes_offsets_from_each_of_the_four_neighbours"]),
    # homography solvers: a wrong index in a DLT row
    ("oracle_planes.c", "double r1[9] = {x, y, 1, 0, 0, 0, -u * x, -u * y, -u};",
     "double r1[9] = {x, y, 1, 0, 0, 0, -u * x, -v * y, -u};",
     [PRIM + "test_minimal_and_refit_recover_generating_homography"]),
    # Philox-4x32-10 (known answers), the window grid, RANSAC ties and refit acceptance
    ("oracle_core.c", "uint64_t p0 = (uint64_t)0xD2511F53u * c0;", "uint64_t p0 = (uint64_t)0xD2511F53u * c1;",
     [PRIM + "test_philox_known_answers"]),
    ("oracle_core.c", "if (mi[id2 * ORC_MI + ORC_MI_VALID]) return mh + (size_t)id2 * 9;\n    if (mi[id1",
     "if (mi[id1 * ORC_MI + ORC_MI_VALID]) return mh + (size_t)id1 * 9;\n    if (mi[id1",
     [METH + "test_distortion_plane_is_the_home_window_model"]),
    ("oracle_core.c", "if (last + s < n) {", "if (last + s <= n) {",
     [PRIM + "test_grid_counts_and_overlap", PRIM + "test_cell_totals_of_the_two_workloads"]),
    ("oracle_planes.c", "if (scores[k] > bscore) {", "if (scores[k] >= bscore) {",
     [PRIM + "test_ransac_ties_keep_the_lowest_hypothesis"]),
    ("oracle_planes.c", "if (rscore >= bscore) {", "if (rscore > bscore) {",
     [PRIM + "test_ransac_recovers_integer_affine_with_outliers"]),
    ("oracle_planes.c", "if (stage == 2 && !resid[i]) continue;", ";",
     [PRIM + "test_residual_stage_fits_only_the_masked_matches"]),
    # Hartley normalisation of the DLT: no centring; a scale that is not rotation invariant
    ("oracle_planes.c", "    mx /= n;\n    my /= n;\n    for (int i = 0; i < n; ++i) d += hypot",
     "    mx = 0;\n    my = 0;\n    for (int i = 0; i < n; ++i) d += hypot",
     [PRIM + "test_normalised_dlt_is_similarity_covariant"]),
    ("oracle_planes.c", "d += hypot(p[2 * i] - mx, p[2 * i + 1] - my);", "d += fabs(p[2 * i] - mx);",
     [PRIM + "test_normalised_dlt_is_similarity_covariant"]),
    # plane validity (R12, R14)
    ("oracle_planes.c", "int valid = count >= P->min_inliers && 5 * count >= N;",
     "int valid = count >= P->min_inliers && count >= N / 5;", [PRIM + "test_plane_validity_support_orientation_and_scale"]),
    ("oracle_planes.c", "int valid = count >= P->min_inliers && 5 * count >= N;",
     "int valid = count > P->min_inliers && 5 * count >= N;", [PRIM + "test_plane_validity_support_orientation_and_scale"]),
    ("oracle_planes.c", "double cxs[4] = {x0 - r, x0 + s - 1 + r, x0 - r, x0 + s - 1 + r};",
     "double cxs[4] = {x0, x0 + s - 1, x0, x0 + s - 1};", [PRIM + "test_plane_validity_denominator_on_the_grown_window"]),
    ("oracle_planes.c", "if (!(sc >= P->scale_min && sc <= P->scale_max)) valid = 0;",
     "if (!(sc >= P->scale_min)) valid = 0;", [PRIM + "test_plane_validity_support_orientation_and_scale"]),
    ("oracle_planes.c", "double sc = sqrt(det);", "double sc = det;",
     [PRIM + "test_plane_validity_support_orientation_and_scale", PRIM + "test_plane_validity_denominator_on_the_grown_window"]),
    ("oracle_planes.c", "if (!valid) mi[ORC_MI_FLAGS] |= ORC_F_BAD_GEOM;", ";",
     [PRIM + "test_plane_validity_support_orientation_and_scale"]),
    # assignment (eq. 3-4, R23, R24)
    ("oracle_planes.c", "if (!(d < P->eps)) continue;\n                    if (bm >= 0 && near_colour",
     "if (!(d <= P->eps)) continue;\n                    if (bm >= 0 && near_colour", [METH + "test_assignment_rules_on_hand_built_windows"]),
    ("oracle_planes.c", "if (d < bL - ORC_L_TIE) {\n                        bL = d;\n                        bm = id;",
     "if (d < bL) {\n                        bL = d;\n                        bm = id;", [METH + "test_assignment_rules_on_hand_built_windows"]),
    ("oracle_planes.c", "if (!in_frame(P, X, Y)) continue;\n                    double d = delta_at(P, src, tgt, x, y, X, Y);\n                    if (near_colour(d, P->eps)) a = 1;",
     "double d = delta_at(P, src, tgt, x, y, X, Y);\n                    if (near_colour(d, P->eps)) a = 1;",
     [METH + "test_assignment_rules_on_hand_built_windows"]),
    ("oracle_planes.c", "if (!mi[id * ORC_MI + ORC_MI_VALID]) continue;\n                    const double* Hm = mh + (size_t)id * 9;\n                    double X, Y;",
     "const double* Hm = mh + (size_t)id * 9;\n                    double X, Y;", [METH + "test_assignment_rules_on_hand_built_windows"]),
    ("oracle_planes.c", "int id = (g->base + cell) * 2 + (stage - 1);", "int id = (g->base + cell) * 2;",
     [METH + "test_assignment_rules_on_hand_built_windows"]),
    ("oracle_planes.c", "    if (!(w > 0)) return 0;\n    *X", "    if (w == 0) return 0;\n    *X",
     [METH + "test_assignment_rules_on_hand_built_windows", METH + "test_edge_aware_fill_evaluates_the_seed_plane_at_the_pixel"]),
    ("oracle_planes.c", "return (fabs(a[0] - s[0]) + fabs(a[1] - s[1]) + fabs(a[2] - s[2])) / 3.0;",
     "return (fabs(a[0] - s[0]) + fabs(a[1] - s[1]) + fabs(a[2] - s[2])) / 2.0;",
     [METH + "test_assignment_rules_on_hand_built_windows"]),
    # occlusion cues (Sec. 3.4)
    ("oracle_planes.c", "f[ORC_MI_NSYM] < P->eta * f[ORC_MI_NASSIGN]", "f[ORC_MI_NSYM] > P->eta * f[ORC_MI_NASSIGN]",
     [METH + "test_symmetry_cue_discards_asymmetric_plane", METH + "test_single_plane_scene_is_recovered_and_assigned"]),
    ("oracle_planes.c", "if (f[ORC_MI_NRC] < P->kappa * f[ORC_MI_COUNT]) {", "if (0) {",
     [METH + "test_overlap_cue_discards_colour_inconsistent_plane"]),
    ("oracle_planes.c", "double ex = lfx[i] + ofx[j]", "double ex = lfx[i] - ofx[j]",
     [METH + "test_symmetry_cue_discards_asymmetric_plane", METH + "test_single_plane_scene_is_recovered_and_assigned"]),
    ("oracle_planes.c",
     "            mi[m * ORC_MI + ORC_MI_NASSIGN]++;\n            double tx = x + lfx[i] + 0.5, ty = y + lfy[i] + 0.5;",
     "            mi[m * ORC_MI + ORC_MI_NASSIGN]++;\n            double tx = x + lfx[i], ty = y + lfy[i];",
     [METH + "test_symmetry_count_reads_the_target_rounded_half_up"]),
    ("oracle_planes.c", "if (!(e2 < t2)) lose[i] = 1;", "if (e2 < t2) lose[i] = 1;",
     [METH + "test_many_to_one_flags_the_worse_of_two_motions"]),
    ("oracle_planes.c",
     "        if (lm[i] < 0) continue;\n        int x = i % W, y = i / W;\n        double tx = x + lfx[i] + 0.5, ty = y + lfy[i] + 0.5;",
     "        if (lm[i] < 0) continue;\n        int x = i % W, y = i / W;\n        double tx = x + lfx[i], ty = y + lfy[i];",
     [METH + "test_many_to_one_targets_round_half_up"]),
    ("oracle_planes.c", "double ex = lfx[i] - lfx[w]", "double ex = lfx[i] + lfx[w]",
     [METH + "test_many_to_one_flags_the_worse_of_two_motions"]),
    # merge and NNF update (Sec. 3.3, 3.3.1)
    ("oracle_planes.c", "lL[i] < aL[i] - P->beta) {", "lL[i] < aL[i] + P->beta) {",
     [METH + "test_merge_keeps_coarse_unless_clearly_better_and_nnf_update_rounds_half_up"]),
    ("oracle_planes.c", "vx[i] = (int)floor(afx[i] + 0.5);", "vx[i] = (int)afx[i];",
     [METH + "test_merge_keeps_coarse_unless_clearly_better_and_nnf_update_rounds_half_up"]),
    # model-propagation fill (Sec. 3.4.1): neighbours, and the colour bound
    ("oracle_planes.c", "NY[4] = {0, 0, -1, 1};\n                int bm = -1, nd", "NY[4] = {0, 0, -1, -1};\n                int bm = -1, nd",
     [METH + "test_fill_front_advances_one_pixel_per_jacobi_iteration"]),
    ("oracle_planes.c", "(fabs(d - bL) <= ORC_L_TIE && m < bm)", "(fabs(d - bL) <= ORC_L_TIE && m > bm)",
     [METH + "test_fill_takes_the_lowest_model_id_among_equal_neighbours"]),
    ("oracle_planes.c", "if (!in_frame(P, X, Y)) continue;\n                    double d = delta_at(P, src, tgt, x, y, X, Y);\n"
     "                    if (amb && near_colour(d, P->eps)) a = 1;", "double d = delta_at(P, src, tgt, x, y, X, Y);",
     [METH + "test_fill_takes_the_lowest_model_id_among_equal_neighbours"]),
    # final map (Sec. 3.4.1, R20, R23) and the edge-aware fill (R28)
    ("oracle_planes.c", "int o = am[i] < 0 || (cue[i] & ORC_CUE_M2O);", "int o = am[i] < 0;",
     [METH + "test_final_map_flow_source_and_occlusion_rule_on_hand_built_state"]),
    ("oracle_planes.c", "if (!(d < P->occ_thresh)) o = 1;", "if (d > P->occ_thresh) o = 1;",
     [METH + "test_final_map_flow_source_and_occlusion_rule_on_hand_built_state"]),
    ("oracle_planes.c", "flow[2 * i] = (float)afx[s];", "flow[2 * i] = (float)afx[i];",
     [METH + "test_edge_aware_fill_evaluates_the_seed_plane_at_the_pixel"]),
    # the pipeline (Algorithm 1): gain, cue directions and order, residual mask, freezing, fill
    ("oracle_pipeline.c", "for (size_t i = 0; i < nf; ++i) f2[i] = f2in[i] * g;", "for (size_t i = 0; i < nf; ++i) f2[i] = f2in[i] / g;",
     [METH + "test_tiny_config_accuracy_against_ground_truth"]),
    ("oracle_pipeline.c", "orc_cue_counts(P, l, 1, T[d].m, T[d].fx, T[d].fy, T[1 - d].m, T[1 - d].fx, T[1 - d].fy, S->mi[d], NULL);",
     "orc_cue_counts(P, l, 1, T[d].m, T[d].fx, T[d].fy, T[d].m, T[d].fx, T[d].fy, S->mi[d], NULL);",
     [METH + "test_translating_layer_scene_occlusion_and_flow", METH + "test_tiny_config_accuracy_against_ground_truth"]),
    ("oracle_pipeline.c", "            for (int d = 0; d < 2; ++d) orc_cue_invalidate(P, l, 1, S->mi[d]);\n", "",
     [METH + "test_pipeline_discards_every_stage_one_plane_that_fails_a_cue"]),
    ("oracle_pipeline.c", "for (int i = 0; i < n; ++i) resid[d][i] = S1[d].m[i] < 0;",
     "for (int i = 0; i < n; ++i) resid[d][i] = S1[d].m[i] >= 0;",
     [METH + "test_pipeline_residual_stage_fits_the_pixels_stage_one_left"]),
    ("oracle_pipeline.c", "                orc_many_to_one(P, C[d].m, C[d].L, C[d].fx, C[d].fy, S->cue[d], NULL);\n", "",
     [METH + "test_translating_layer_scene_occlusion_and_flow", METH + "test_tiny_config_accuracy_against_ground_truth"]),
    ("oracle_pipeline.c", "                orc_nnf_update(P, S->am[d], S->afx[d], S->afy[d], S->vx[d], S->vy[d], frozen[d]);\n", "",
     [METH + "test_pipeline_freezes_assigned_pixels_and_fills_from_neighbours"]),
    ("oracle_pipeline.c", "pm_run(P, src[d], tgt[d], d, l, S->mh[d], S->mi[d], frozen[d], S->vx[d], S->vy[d], S->cost[d]);",
     "pm_run(P, src[d], tgt[d], d, l, S->mh[d], S->mi[d], NULL, S->vx[d], S->vy[d], S->cost[d]);",
     [METH + "test_pipeline_freezes_assigned_pixels_and_fills_from_neighbours"]),
    ("oracle_pipeline.c",
     "        orc_fill(P, src[d], tgt[d], S->mh[d], S->mi[d], S->cue[d], S->am[d], S->aL[d], S->afx[d], S->afy[d], NULL);\n",
     "",
     [METH + "test_pipeline_freezes_assigned_pixels_and_fills_from_neighbours"]),
    # census codes (Sec. 6), HSV equalisation (Sec. 4.2), geodesic fill seeds (R28)
    ("oracle_color.c", "if (grey(rgb, W, nx, ny) < c) code |= 1u << bit;", "if (grey(rgb, W, nx, ny) <= c) code |= 1u << bit;",
     [PRIM + "test_census_closed_forms"]),
    ("oracle_color.c", "lut[b] = (lut[b] - (double)cmin) / (double)(n - cmin);", "lut[b] = lut[b] / (double)n;",
     [PRIM + "test_v_lut_closed_form"]),
    ("oracle_color.c", "hh = 2.0 + (b - r) / c;", "hh = 2.0 + (r - b) / c;",
     [PRIM + "test_hsv_conversion_matches_the_library_routine"]),
    ("oracle_color.c", "(c == dist[i] && seed[j] < seed[i])", "(c == dist[i] && seed[j] > seed[i])",
     [PRIM + "test_fill_seeds_flat_frame_are_manhattan_nearest"]),
    ("oracle_core.c", "int i = (int)floor((double)(x - s / 4) / h);", "int i = (int)floor((double)x / h);",
     [METH + "test_distortion_plane_is_the_home_window_model"]),
    ("oracle_color.c", "case 0: *r = v; *g = t; *b = p; break;", "case 0: *r = v; *g = p; *b = t; break;",
     [PRIM + "test_hsv_conversion_matches_the_library_routine"]),
    ("oracle_core.c", "sum += orc_popcount32(a ^ b);", "sum += orc_popcount32(a & b);",
     [PRIM + "test_census_cost_finds_an_integer_shift_exhaustively"]),
    ("oracle_color.c", "q[i] = (int32_t)floor(1024.0 * ((rgb[3 * i] + rgb[3 * i + 1]) + rgb[3 * i + 2]));",
     "q[i] = (int32_t)floor(1023.0 * ((rgb[3 * i] + rgb[3 * i + 1]) + rgb[3 * i + 2]));",
     [PRIM + "test_fill_seeds_grey_quantisation_decides_a_close_call"]),
    ("oracle_color.c", "for (int x = W - 2; x >= 0; --x) relax(q, dist, seed, y * W + x + 1, y * W + x);", ";",
     [PRIM + "test_fill_seeds_flat_frame_are_manhattan_nearest"]),
    ("oracle_planes.c", "return s2 > 0 ? s1 / s2 : 1.0;", "return s2 > 0 ? s2 / s1 : 1.0;",
     [METH + "test_tiny_config_accuracy_against_ground_truth"]),
    ("oracle_color.c", "const long long c = dist[j] + 256 + llabs((long long)q[i] - q[j]);",
     "const long long c = dist[j] + 256;", [PRIM + "test_fill_seeds_respect_an_edge"]),
]


def _copy_tree(dst):
    """The oracle sources, the tests and the input generator (no built library, no GPU code)."""
    os.makedirs(os.path.join(dst, "oracle"))
    for f in os.listdir(os.path.join(ROOT, "oracle")):
        if f.endswith((".c", ".h", ".py")):
            shutil.copy(os.path.join(ROOT, "oracle", f), os.path.join(dst, "oracle", f))
    shutil.copytree(os.path.join(ROOT, "tests"), os.path.join(dst, "tests"),
                    ignore=shutil.ignore_patterns("__pycache__"))
    os.makedirs(os.path.join(dst, "paper_1804_03787_gb300"))
    for f in ("__init__.py", "scene.py"):
        shutil.copy(os.path.join(ROOT, "paper_1804_03787_gb300", f), os.path.join(dst, "paper_1804_03787_gb300", f))
    shutil.copy(os.path.join(ROOT, "pytest.ini"), dst)


def _run_pins(dst, pins):
    env = dict(os.environ, OMP_NUM_THREADS="1", PYTHONPATH=dst, PYTHONDONTWRITEBYTECODE="1")
    r = subprocess.run([sys.executable, "-m", "pytest", "-q", "-x", "-m", "not gpu", *pins], cwd=dst, env=env,
                       stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True, timeout=600)
    return r.returncode, r.stdout[-2000:]


def _mutant(base, k):
    fname, old, new, pins = MUTANTS[k]
    dst = os.path.join(base, f"m{k:02d}")
    _copy_tree(dst)
    path = os.path.join(dst, "oracle", fname)
    src = open(path).read()
    assert src.count(old) == 1, f"mutant {k}: the original text is not found exactly once in {fname}"
    open(path, "w").write(src.replace(old, new))
    return _run_pins(dst, pins)


def test_every_planted_mistake_fails_its_pins(tmp_path):
    base = str(tmp_path)
    pins = sorted({p for m in MUTANTS for p in m[3]})
    clean = os.path.join(base, "clean")
    _copy_tree(clean)
    rc, out = _run_pins(clean, pins)
    assert rc == 0, "the unchanged oracle copy must pass its pins:\n" + out
    with ThreadPoolExecutor(max_workers=max(1, min(8, os.cpu_count() or 1))) as ex:
        results = list(ex.map(lambda k: _mutant(base, k), range(len(MUTANTS))))
    survivors = [(k, MUTANTS[k][0], MUTANTS[k][2]) for k, (rc, _) in enumerate(results) if rc == 0]
    assert not survivors, f"planted mistakes no pin caught: {survivors}"
    # a pin that fails must fail by an assertion, not by a broken copy
    for k, (rc, out) in enumerate(results):
        assert rc == 1, f"mutant {k}: pytest exited {rc}:\n{out}"
