"""The pins catch plausible mistakes in the oracle (CPU only).

Each case plants one mistake in a copy of oracle/stp_oracle.c: a dropped term, a wrong sign,
a clamp turned round, a queue bound off by one step. It builds the copy with the oracle's own
compile line and runs the pins named beside it against that build (STP_ORACLE_LIB). The case
passes when at least one of them fails. A control build of the unchanged source passes every
pin used here. The committed oracle source is never modified.
"""
import concurrent.futures as cf
import os
import subprocess
import sys

import pytest

from oracle import build as OB

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PINS = "tests/test_oracle_pins.py::"
COMP = "tests/test_oracle_composite.py::"

# (name, passage, original text, planted text, pins expected to catch it)
MUTANTS = [
    ("t_opt_denominator_without_sigma_inv", "Eq. dopt (Sec. 3.2)",
     "    matvec3(sinv, d, sd);\n    double num", "    sd[0] = d[0]; sd[1] = d[1]; sd[2] = d[2];\n    double num",
     [COMP + "test_single_isotropic_gaussian_every_pixel"]),
    ("inverse_scale_clamp_turned_round", "Sec. 3.2 (S^-1 <= 1e3)",
     "double si = fmin(exp(-log_scale[k]), inv_scale_max);", "double si = fmax(exp(-log_scale[k]), inv_scale_max);",
     [PINS + "test_sigma_inverse_and_clamp"]),
    ("covariance_from_scale_not_variance", "Sec. 2.1 (Sigma = R S S^T R^T)",
     "exp(2 * log_scale[k])", "exp(log_scale[k])",
     [PINS + "test_sigma_inverse_and_clamp"]),
    ("algorithm1_edge_parameter_unclamped", "Algorithm 1",
     "ty = den > 0 ? clampd(num / den, 0.0, 1.0) : 0.0;", "ty = den > 0 ? num / den : 0.0;",
     [PINS + "test_alg1_matches_grid_search"]),
    ("sh_degree1_sign", "App. B.4 (SH colour)",
     "y[1] = -k1 * Y;", "y[1] = k1 * Y;",
     [PINS + "test_sh_basis_orthonormal_and_matches_textbook"]),
    ("sh_degree3_sign", "App. B.4 (SH colour)",
     "y[13] = -k3c * x * (4 * z * z - x * x - Y * Y);", "y[13] = k3c * x * (4 * z * z - x * x - Y * Y);",
     [PINS + "test_sh_basis_orthonormal_and_matches_textbook"]),
    ("sh_degree2_normalisation", "App. B.4 (SH colour)",
     "k2b = sqrt(5.0 / (16.0 * PI))", "k2b = sqrt(5.0 / (4.0 * PI))",
     [PINS + "test_sh_basis_orthonormal_and_matches_textbook"]),
    ("composite_without_transmittance", "Eq. volume_desc (Sec. 2.1)",
     "ps->C[k] += col[k] * a * ps->T;", "ps->C[k] += col[k] * a;",
     [COMP + "test_stack_on_one_ray_composites_front_to_back"]),
    ("early_out_tested_before_the_step", "Sec. 2.1 (3DGS early-out)",
     "if (Tn < c->P.t_min) {", "if (ps->T < c->P.t_min) {",
     [COMP + "test_termination_gaussian_is_not_blended"]),
    ("background_without_transmittance", "Eq. volume_desc (Sec. 2.1)",
     "sk->rgb[3 * p + k] = ps->C[k] + ps->T * c->P.bg[k];", "sk->rgb[3 * p + k] = ps->C[k] + c->P.bg[k];",
     [COMP + "test_single_isotropic_gaussian_every_pixel"]),
    ("depth_without_transmittance", "Sec. 4.1 (depth evaluation)",
     "ps->Z += t * a * ps->T;", "ps->Z += t * a;",
     [COMP + "test_stack_on_one_ray_composites_front_to_back"]),
    ("alpha_not_clamped", "Sec. 2.1 (alpha <= 0.99)",
     "return fmin(c->P.alpha_max, g->opacity * gauss2(g, ps->x, ps->y));",
     "return g->opacity * gauss2(g, ps->x, ps->y);",
     [COMP + "test_stack_on_one_ray_composites_front_to_back"]),
    ("conic_off_diagonal_sign", "Sec. 2.1 (conic = Sigma2^-1)",
     "g->conic[1] = -g->cov2[1] / g->det;", "g->conic[1] = g->cov2[1] / g->det;",
     [COMP + "test_conic_is_the_inverse_of_the_projected_covariance"]),
    ("ewa_without_dilation", "Sec. 2.1 (EWA splat)",
     "cov2[0] = S2[0] + prm->dilation;", "cov2[0] = S2[0];",
     [PINS + "test_projection_jacobian_is_finite_difference"]),
    ("jacobian_sign", "Sec. 2.1 (EWA splat)",
     "J[2] = -cam->fx * cx / p[2];", "J[2] = cam->fx * cx / p[2];",
     [PINS + "test_projection_jacobian_is_finite_difference"]),
    ("opacity_bound_without_factor_2", "App. B.2",
     "return sqrt(2.0 * log(opacity / eps_o));", "return sqrt(log(opacity / eps_o));",
     [PINS + "test_t_o_bound_printed_value"]),
    ("tile_cull_at_the_box_corner", "Sec. 3.4 (tile-based culling)",
     "double val = g->opacity * gauss2(g, xh[0], xh[1]);\n                double m = fabs(val / P->eps_o - 1.0);",
     "double val = g->opacity * gauss2(g, box[0], box[2]);\n                double m = fabs(val / P->eps_o - 1.0);",
     [PINS + "test_tile_culling_never_drops_a_contributor"]),
    ("tile_key_through_the_centre", "Sec. 3.4 (tile-depth adjustment)",
     "                else t = depth_at(c, g, xh[0], xh[1]);\n                if (near_decision",
     "                else t = depth_at(c, g, 0.5 * (box[0] + box[1]), 0.5 * (box[2] + box[3]));\n"
     "                if (near_decision",
     [PINS + "test_tile_depth_adjustment_reduces_sort_error"]),
    ("tile_rectangle_half_a_tile_short", "App. B.2 (rectangle)",
     "int tx0 = (int)ceil((g->mean2[0] - r - 15.5) / 16.0)", "int tx0 = (int)ceil((g->mean2[0] - r) / 16.0)",
     [PINS + "test_tile_culling_never_drops_a_contributor"]),
    ("head_queue_one_short", "Sec. 3.3 (k-buffer)",
     "    if (ps->nh > hsize) {", "    if (ps->nh >= hsize) {",
     [PINS + "test_resort_window_k"]),
    ("tail_queue_drained_a_batch_early", "Sec. 3.4 (tail queue 32n+32)",
     "while (s->nt > P->tail - 32) {", "while (s->nt > P->tail - 48) {",
     [PINS + "test_hier_window_is_25_in_the_worst_case"]),
    ("mid_queue_popped_early", "Sec. 3.4 (mid queue 4m+4)",
     "if (s->nm[q] > c->P.mid - 4) {", "if (s->nm[q] > c->P.mid - 8) {",
     [PINS + "test_hier_window_is_25_in_the_worst_case"]),
    ("merge_puts_new_entries_first_on_ties", "Sec. 3.4 (queue merges)",
     "out[k++] = (q[i].t <= nw[j].t) ? q[i++] : nw[j++];", "out[k++] = (q[i].t < nw[j].t) ? q[i++] : nw[j++];",
     [PINS + "test_equal_depths_keep_their_list_order"]),
    ("head_inserts_before_equals", "Sec. 3.3 (insertion)",
     "while (pos < ps->nh && ps->head[pos].t <= e.t) pos++;", "while (pos < ps->nh && ps->head[pos].t < e.t) pos++;",
     [PINS + "test_equal_depths_keep_their_list_order"]),
    ("batch_sort_unstable", "Sec. 3.4 (batch sort)",
     "while (j >= 0 && a[j].t > x.t) { a[j + 1] = a[j]; j--; }",
     "while (j >= 0 && a[j].t >= x.t) { a[j + 1] = a[j]; j--; }",
     [PINS + "test_equal_depths_keep_their_list_order"]),
    ("adjoint_without_background_term", "Sec. 3.5",
     "            da -= gbg * Tf / (1.0 - a);\n", "",
     [PINS + "test_adjoint_suffix_terms_equal_a_back_to_front_pass",
      PINS + "test_adjoint_matches_central_differences"]),
    ("adjoint_conic_off_diagonal_halved", "Sec. 3.5",
     "gcon[3 * id + 1] += dG * G2 * (-dx * dy);", "gcon[3 * id + 1] += dG * G2 * (-0.5 * dx * dy);",
     [PINS + "test_adjoint_matches_central_differences"]),
    ("adjoint_depth_without_suffix", "Sec. 3.5, Sec. 4.1",
     "da += gz * (t * T - (Zf - Za) / (1.0 - a));", "da += gz * t * T;",
     [PINS + "test_adjoint_suffix_terms_equal_a_back_to_front_pass",
      PINS + "test_adjoint_matches_central_differences"]),
    ("adjoint_t_opt_wrong_vector", "Eq. dopt, Sec. 3.5",
     "gmu[3 * id + r] += dt * sd[r] / den;", "gmu[3 * id + r] += dt * sm[r] / den;",
     [PINS + "test_adjoint_matches_central_differences"]),
    ("adjoint_view_direction_unprojected", "App. B.4, Sec. 3.5",
     "dmu[r] += (ddir[r] - dd * G->dir[r]) / G->ulen;", "dmu[r] += ddir[r] / G->ulen;",
     [PINS + "test_adjoint_matches_central_differences"]),
    ("adjoint_quaternion_unprojected", "Sec. 3.5",
     "dq[k] = (gq[k] - dotq * G->qn[k]) / G->qlen;", "dq[k] = gq[k] / G->qlen;",
     [PINS + "test_adjoint_matches_central_differences"]),
    ("adjoint_sigmoid_derivative_short", "Sec. 3.5",
     "dlogit = gop[i] * G->opacity * (1.0 - G->opacity);", "dlogit = gop[i] * G->opacity;",
     [PINS + "test_adjoint_matches_central_differences"]),
    ("adjoint_ignores_the_colour_clamp", "App. B.4, Sec. 3.5",
     "double draw = G->raw[ch] > 0 ? gcol[3 * i + ch] : 0.0;", "double draw = gcol[3 * i + ch];",
     [PINS + "test_adjoint_matches_central_differences"]),
    ("view_direction_reversed", "App. B.4 (SH colour)",
     "for (int k = 0; k < 3; k++) g->u[k] = g->mu[k] - c->o[k];",
     "for (int k = 0; k < 3; k++) g->u[k] = c->o[k] - g->mu[k];",
     [PINS + "test_sh_colour_uses_the_direction_from_the_camera_to_the_mean"]),
    ("colour_not_clamped_at_zero", "App. B.4 (SH colour)",
     "g->color[ch] = s > 0 ? s : 0.0;", "g->color[ch] = s;",
     [PINS + "test_sh_colour_uses_the_direction_from_the_camera_to_the_mean"]),
    ("sh_without_the_half_offset", "App. B.4 (SH colour)",
     "        double s = 0.5;\n", "        double s = 0.0;\n",
     [PINS + "test_sh_degree0_colour_is_view_independent"]),
    ("sigmoid_sign", "Sec. 2.1 (opacity)",
     "g->opacity = 1.0 / (1.0 + exp(-sc->logits[i]));", "g->opacity = 1.0 / (1.0 + exp(sc->logits[i]));",
     [COMP + "test_single_isotropic_gaussian_every_pixel"]),
    ("rotation_from_the_raw_quaternion", "Sec. 2.1 (Sigma = R S S^T R^T)",
     "    normalise_quat(quat, q, &l);\n    quat_to_rot(q, R);\n    for (int i = 0; i < 3; i++)\n"
     "        for (int j = 0; j < 3; j++) {\n            double s = 0;\n"
     "            for (int k = 0; k < 3; k++) s += R[3 * i + k] * exp(2",
     "    normalise_quat(quat, q, &l);\n    quat_to_rot(quat, R);\n    for (int i = 0; i < 3; i++)\n"
     "        for (int j = 0; j < 3; j++) {\n            double s = 0;\n"
     "            for (int k = 0; k < 3; k++) s += R[3 * i + k] * exp(2",
     [PINS + "test_sigma_inverse_and_clamp"]),
    ("jacobian_not_clamped_outside_the_view", "Sec. 2.1 (EWA splat, clamp kept)",
     "double cx = clampd(ux, -limx, limx), cy = clampd(uy, -limy, limy);", "double cx = ux, cy = uy;",
     [PINS + "test_splat_shape_stops_changing_beyond_the_jacobian_clamp"]),
    ("near_plane_at_zero", "preprocess (near plane kept)",
     "g->visible = (g->p[2] > P->znear) && (g->opacity >= P->eps_o);",
     "g->visible = (g->p[2] > 0) && (g->opacity >= P->eps_o);",
     [PINS + "test_near_plane_culls_gaussians_in_front_of_znear"]),
    ("radius_from_the_smaller_eigenvalue", "App. B.2",
     "double lam = mid + sqrt(fmax(0.0, mid * mid - g->det));", "double lam = mid - sqrt(fmax(0.0, mid * mid - g->det));",
     [PINS + "test_tile_culling_never_drops_a_contributor"]),
    ("ray_direction_not_normalised", "Eq. dopt (unit ray)",
     "    d[0] /= l; d[1] /= l; d[2] /= l;", "    (void)l;",
     [COMP + "test_single_isotropic_gaussian_every_pixel"]),
    ("pixel_ray_through_the_corner", "Sec. 3.4 (pixel centres)",
     "    ps->x = X + 0.5;", "    ps->x = X;",
     [COMP + "test_single_isotropic_gaussian_every_pixel"]),
    ("tile_box_through_pixel_corners", "Sec. 3.4 (tile-based culling)",
     "    box[0] = ox + 0.5; box[1] = xe + 0.5;", "    box[0] = ox; box[1] = xe;",
     [PINS + "test_tile_culling_never_drops_a_contributor"]),
    ("full_sort_by_the_tile_key", "Sec. 3.2 (full per-ray sort)",
     "                    buf[k].t = pixel_depth(c, L->e[j].id, ps);", "                    buf[k].t = L->e[j].t;",
     [COMP + "test_single_isotropic_gaussian_every_pixel",
      PINS + "test_sort_error_full_is_zero_and_hier_beats_small_windows"]),
    ("full_sort_skipped", "Sec. 3.2 (full per-ray sort)",
     "qsort(buf, (size_t)k, sizeof(fent), cmp_fent);", "(void)cmp_fent;",
     [PINS + "test_sort_error_full_is_zero_and_hier_beats_small_windows"]),
    ("k_buffer_blends_its_farthest", "Sec. 3.3 (k-buffer)",
     "        hent f = ps->head[0];\n        memmove(&ps->head[0], &ps->head[1], (size_t)(ps->nh - 1) * sizeof(hent));\n"
     "        ps->nh--;\n        blend(c, ps, sk, f.t, f.id, f.a, cnt);\n    }\n}",
     "        hent f = ps->head[ps->nh - 1];\n        ps->nh--;\n        blend(c, ps, sk, f.t, f.id, f.a, cnt);\n    }\n}",
     [PINS + "test_resort_window_k"]),
    ("pixel_alpha_threshold_doubled", "Sec. 3.4 (alpha >= eps_O)",
     "            if (a < c->P.eps_o) continue;\n            hent h", "            if (a <= 2 * c->P.eps_o) continue;\n            hent h",
     [PINS + "test_hier_blends_the_same_set_as_full_sort"]),
    ("adjoint_mean2_wrong_conic_entry", "Sec. 3.5",
     "gm2[2 * id + 0] += dG * G2 * (G->conic[0] * dx + G->conic[1] * dy);",
     "gm2[2 * id + 0] += dG * G2 * (G->conic[0] * dx + G->conic[2] * dy);",
     [PINS + "test_adjoint_matches_central_differences"]),
    ("adjoint_log_scale_without_chain_factor", "Sec. 3.5",
     "dls[k] += mb * G->Rq[3 * r + k] * G->s[k];", "dls[k] += mb * G->Rq[3 * r + k];",
     [PINS + "test_adjoint_matches_central_differences"]),
    ("key_cut_ignored", "depth slices (prefix exactness)",
     "            L->n = m;\n            batch_margins(L, key_cut);", "            (void)m;\n            batch_margins(L, key_cut);",
     [PINS + "test_key_prefix_keeps_pixels_finished_inside_its_complete_batches"]),
    ("global_order_through_a_k_buffer", "Sec. 3.2 (3DGS order)",
     "                    if (P->mode == 2) blend(c, ps, sk, t, L->e[j].id, a, cnt);",
     "                    if (P->mode == 99) blend(c, ps, sk, t, L->e[j].id, a, cnt);",
     [PINS + "test_sort_error_full_is_zero_and_hier_beats_small_windows"]),
    ("k_buffer_never_flushed", "Sec. 3.3 (k-buffer)",
     "                if (P->mode == 3) head_flush(c, ps, sk, cnt);", "                (void)0;",
     [COMP + "test_stack_on_one_ray_composites_front_to_back"]),
    ("sort_error_counts_every_gap", "Sec. 3.3 (sort error)",
     "if (ps->has_last && ps->last_t > t) ps->delta += ps->last_t - t;", "if (ps->has_last) ps->delta += fabs(ps->last_t - t);",
     [PINS + "test_sort_error_full_is_zero_and_hier_beats_small_windows"]),
    ("evict_first_reading_ignored", "Sec. 3.4 (full head queue, other reading)",
     "if ((c->P.flags & 1) && ps->nh == hsize) {", "if ((c->P.flags & 1) && ps->nh == hsize + 1000) {",
     [PINS + "test_evict_first_reading_shrinks_every_window_by_one"]),
    ("level_centre_reading_ignored", "Sec. 3.4 (level rays, other reading)",
     "    if (c->P.flags & 2) *t = depth_at(c, g, 0.5 * (box[0] + box[1]), 0.5 * (box[2] + box[3]));",
     "    if (c->P.flags & 0) *t = depth_at(c, g, 0.5 * (box[0] + box[1]), 0.5 * (box[2] + box[3]));",
     [PINS + "test_readings_change_the_order_never_the_set"]),
    ("view_depth_ablation_ignored", "Tab. performance_ablation B",
     "if (P->flags & 8) t = g->p[2];", "if (P->flags & 0) t = g->p[2];",
     [PINS + "test_tile_depth_adjustment_reduces_sort_error"]),
    ("tile_cull_ablation_ignored", "Tab. performance_ablation D",
     "                if (P->flags & 512) {", "                if (P->flags & 0) {",
     [PINS + "test_without_tile_culling_lists_grow_but_per_pixel_orders_do_not_change"]),
    ("hierarchical_cull_ablation_ignored", "Tab. performance_ablation E",
     "    if (c->P.flags & 1024) *margin = INFINITY;", "    if (c->P.flags & 0) *margin = INFINITY;",
     [PINS + "test_without_hierarchical_culling_every_entry_reaches_the_pixels"]),
    ("tiny_quaternion_accepted", "invalid inputs (reading)",
     "if (!(q2 >= 1e-20) || !isfinite(sc->logits[i])) return 0;", "if (!(q2 > 0) || !isfinite(sc->logits[i])) return 0;",
     [COMP + "test_quaternion_length_threshold"]),
    ("non_finite_mean_accepted", "invalid inputs (reading)",
     "if (!isfinite(sc->means[3 * i + k]) || !isfinite(sc->log_scales[3 * i + k])) return 0;",
     "if (!isfinite(sc->log_scales[3 * i + k])) return 0;",
     [COMP + "test_invalid_gaussians_are_dropped_and_counted"]),
    ("non_finite_sh_accepted", "invalid inputs (reading)",
     "        if (!isfinite(sc->sh[i * 3 * K + j])) return 0;", "        (void)0;",
     [COMP + "test_invalid_gaussians_are_dropped_and_counted"]),
]


def _run(src_text: str, tag: str, pins, tmp) -> subprocess.CompletedProcess:
    d = tmp / tag
    d.mkdir()
    (d / "stp_oracle.c").write_text(src_text)
    with open(os.path.join(os.path.dirname(OB.SRC), "stp_oracle.h")) as f:
        (d / "stp_oracle.h").write_text(f.read())
    so = str(d / "libstp_oracle.so")
    subprocess.run(OB.gcc_command(str(d / "stp_oracle.c"), so), check=True, capture_output=True)
    env = dict(os.environ, STP_ORACLE_LIB=so, OMP_NUM_THREADS="1")
    return subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider", *pins],
                          cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)


@pytest.fixture(scope="module")
def results(tmp_path_factory):
    tmp = tmp_path_factory.mktemp("mutants")
    with open(OB.SRC) as f:
        src = f.read()
    jobs = {"control": (src, sorted({p for m in MUTANTS for p in m[4]}))}
    for name, _, old, new, pins in MUTANTS:
        assert src.count(old) == 1, "%s: the planted text must match the source once" % name
        jobs[name] = (src.replace(old, new), pins)
    with cf.ThreadPoolExecutor(max(2, min(12, os.cpu_count() or 2))) as ex:
        futs = {k: ex.submit(_run, s, k, p, tmp) for k, (s, p) in jobs.items()}
        return {k: f.result() for k, f in futs.items()}


def test_control_build_passes_every_pin_used(results):
    r = results["control"]
    assert r.returncode == 0, r.stdout[-2000:]


@pytest.mark.parametrize("name", [m[0] for m in MUTANTS])
def test_planted_mistake_is_caught(results, name):
    r = results[name]
    # exit code 1: tests ran and one failed (2 or more would be a harness or collection error)
    assert r.returncode == 1, (name, r.returncode, r.stdout[-1500:], r.stderr[-500:])
    assert "FAILED" in r.stdout or " failed" in r.stdout
