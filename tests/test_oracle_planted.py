"""Planted mistakes: the oracle's pins catch each plausible slip.

Each case copies oracle.c, plants one mistake of the kind a restatement of
the method could contain (a dropped term, a wrong sign, index or bound, a
transposed operand, an off-by-one), builds the copy with gcc and runs the pin
modules of the function it touches against that build (PMSP_ORACLE_LIB): at
least one pin must fail. The unplanted oracle passes the same modules in the
rest of the suite. A case whose snippet no longer occurs once in oracle.c
fails, so the list follows the source.

One slip no pin can catch, because it cannot change a result: wrapping
versus clamping the nearest pixel's column in the completeness splat
(rounding a projection, which lies in [-0.5, W - 0.5), never leaves
[0, W - 1]).
"""
import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "oracle.c")

CAMERA = ["tests/test_oracle_camera.py"]
RNG = ["tests/test_oracle_rng.py"]
COST = ["tests/test_oracle_cost.py"]
PM = ["tests/test_oracle_patchmatch.py"]
FILTER = ["tests/test_oracle_filter.py"]
WARP = ["tests/test_oracle_warp.py"]
MEDIAN = ["tests/test_oracle_median.py"]
VIEW = ["tests/test_oracle_view.py", "tests/test_golden_parameters.py"]
FUSION = ["tests/test_oracle_fusion.py"]

# (name, original text, planted text, pin modules)
PLANTED = [
    # camera (Sec. III-C equirectangular model)
    ("bearing_latitude_sign", "r[1] = -sin(lat);", "r[1] = sin(lat);", CAMERA),
    ("projection_half_pixel_dropped", "*uc = W * (lon + ORC_PI) / (2.0 * ORC_PI) - 0.5;",
     "*uc = W * (lon + ORC_PI) / (2.0 * ORC_PI);", CAMERA),
    ("projection_latitude_from_x_only", "double lat = atan2(-Y[1], sqrt(Y[0] * Y[0] + Y[2] * Y[2]));",
     "double lat = atan2(-Y[1], fabs(Y[2]));", CAMERA),
    ("sample_seam_clamped", "x1 = wrap_i(i0 + 1, im->W);", "x1 = clamp_i(i0 + 1, 0, im->W - 1);", CAMERA),
    ("bearing_half_pixel_dropped", "double lon = 2.0 * ORC_PI * (u + 0.5) / W - ORC_PI;",
     "double lon = 2.0 * ORC_PI * u / W - ORC_PI;", CAMERA),
    ("sample_weights_swapped", "return (1.0 - fy) * ((1.0 - fx) * t00 + fx * t10)",
     "return (1.0 - fy) * (fx * t00 + (1.0 - fx) * t10)", CAMERA),
    ("bearing_z_without_cos_lat", "r[2] = cos(lat) * cos(lon);", "r[2] = cos(lon);", CAMERA),
    ("sample_rows_wrapped", "y1 = clamp_i(j0 + 1, 0, im->H - 1);", "y1 = wrap_i(j0 + 1, im->H);", CAMERA),
    ("rel_pose_translation_sign", "out->t[i] = s->t[i] - acc;", "out->t[i] = s->t[i] + acc;", CAMERA),
    ("rel_pose_transposed", "acc += s->R[3 * i + k] * r->R[3 * j + k];",
     "acc += s->R[3 * i + k] * r->R[3 * k + j];", CAMERA),
    # random numbers
    ("philox_key_word", "uint64_t y0 = hi1 ^ x1 ^ k0,", "uint64_t y0 = hi1 ^ x1 ^ k1,", RNG),
    ("philox_weyl_swapped", "k0 += W0; k1 += W1;", "k0 += W1; k1 += W0;", RNG),
    ("u24_shift", "(double)(w >> 40) * (1.0 / 16777216.0)", "(double)(w >> 41) * (1.0 / 16777216.0)", RNG),
    # matching cost (weighted NCC, best-k)
    ("ncc_mean_term_dropped", "double cov = sw[s] * sIJ[s] - sI[s] * sJ[s];", "double cov = sw[s] * sIJ[s];",
     COST),
    ("ncc_variance_uses_wrong_sum", "double varJ = sw[s] * sJJ[s] - sJ[s] * sJ[s];",
     "double varJ = sw[s] * sJJ[s] - sI[s] * sJ[s];", COST),
    ("spatial_weight_dy_dropped", "e += (double)(ox * ox + oy * oy)", "e += (double)(ox * ox)", COST),
    ("colour_weight_not_squared", "e += (Iq - Ip) * (Iq - Ip) / (2.0 * p->sigma_color * p->sigma_color);",
     "e += (Iq - Ip) / (2.0 * p->sigma_color * p->sigma_color);", COST),
    ("weight_sum_unweighted", "sw[s] += w;", "sw[s] += 1.0;", COST),
    ("ncc_scaled", "double ncc = cov / sqrt(varI * varJ);", "double ncc = cov / sqrt(varI * varJ) * 0.999;", COST),
    ("colour_weight_sign", "double w = exp(-e);", "double w = exp(e);", COST),
    ("plane_ray_ratio_inverted", "double tq = d * ndotrp / denom;", "double tq = d * denom / ndotrp;", COST),
    ("best_k_takes_largest", "if (!used[s] && (best < 0 || c[s] < c[best])) best = s;",
     "if (!used[s] && (best < 0 || c[s] > c[best])) best = s;", COST),
    ("best_k_mean_over_all", "return sum / p->best_k;", "return sum / S;", COST),
    ("reference_patch_is_centre_pixel", "double Iq = pb->ref.I[(size_t)qv * W + qu];",
     "double Iq = pb->ref.I[(size_t)v * W + u];", COST),
    ("patch_stride_ignored", "for (int o = -r; o <= r; o += p->patch_stride) offs[n++] = o;",
     "for (int o = -r; o <= r; o += 1) offs[n++] = o;", COST),
    ("flat_source_not_rejected", "if (varI < eps || varJ < eps) { c[s] = 2.0; continue; }",
     "if (varI < eps) { c[s] = 2.0; continue; }", COST),
    ("ncc_clamp_sign", "if (ncc < -1.0) ncc = -1.0;", "if (ncc < -1.0) ncc = 1.0;", COST),
    ("patch_behind_plane_sign", "if (!(denom < -1e-6)) { invalid = 1; break; }",
     "if (!(denom > -1e-6)) { invalid = 1; break; }", COST),
    ("ncc_to_cost_sign", "c[s] = 1.0 - ncc;", "c[s] = 1.0 + ncc;", COST),
    # initialisation and propagation (Sec. III-B, III-C)
    ("init_uniform_in_range", "double inv = 1.0 / p->d_max + r[0] * (1.0 / p->d_min - 1.0 / p->d_max);",
     "double inv = 1.0 / (p->d_min + r[0] * (p->d_max - p->d_min));", PM),
    ("init_normal_y_from_cosine", "n[1] = rho * sin(phi);", "n[1] = rho * cos(phi);", PM),
    ("init_normal_hemisphere", "double z = 1.0 - 2.0 * r[1], phi", "double z = 1.0 - r[1], phi", PM),
    ("face_camera_sign", "} else if (c > 0) {", "} else if (c < 0) {", COST + PM),
    ("neighbours_same_colour", "static const int t0[16] = {0, -3, 0, 3, -3, 0, 3, 0,",
     "static const int t0[16] = {0, -2, 0, 2, -2, 0, 2, 0,", PM),
    ("propagation_no_reintersection", "double dc = depth[j] * dot3(nq, rq) / den;", "double dc = depth[j];", PM),
    ("init_draw_layout_transposed", "draw4(p, (uint64_t)v * pb->ref.W + u, 0, 0, r);",
     "draw4(p, (uint64_t)u * pb->ref.H + v, 0, 0, r);", PM),
    ("propagation_range_check_dropped", "if (!(dc >= p->d_min && dc <= p->d_max)) continue;",
     "if (!(dc > 0)) continue;", PM),
    ("propagation_grazing_sign", "if (!(den < -1e-6)) continue;\n        double dc",
     "if (!(den > 1e-6)) continue;\n        double dc", PM),
    ("refine_normal_not_renormalised", "nc[0] /= len; nc[1] /= len; nc[2] /= len;", "(void)len;", PM),
    ("refine_range_not_clamped", "if (inv < inv_lo) inv = inv_lo;", "", PM),
    ("propagation_rows_clamped", "if (qv < 0 || qv >= H) continue;\n        int qu",
     "if (qv < 0 || qv >= H) qv = clamp_i(qv, 0, H - 1);\n        int qu", PM),
    ("refine_draws_init_stage", "draw4(p, (uint64_t)i, (uint64_t)iter, (uint64_t)(1 + k), r);",
     "draw4(p, (uint64_t)i, (uint64_t)iter, (uint64_t)k, r);", PM),
    ("refine_normal_y_from_x_draw", "bn[1] + s * (2.0 * r[2] - 1.0)", "bn[1] + s * (2.0 * r[1] - 1.0)", PM),
    ("halfsweep_colour_ignores_row", "for (int u = (v + colour) & 1; u < W; u += 2)",
     "for (int u = colour; u < W; u += 2)", PM),
    ("refine_range_not_halved", "double s = ldexp(1.0, -(k + 1));", "double s = 1.0;", PM),
    ("refine_one_sided_depth", "double inv = 1.0 / bd + (2.0 * r[0] - 1.0) * s * (inv_hi - inv_lo);",
     "double inv = 1.0 / bd + r[0] * s * (inv_hi - inv_lo);", PM),
    # caught only by the refinement-schedule pin (tests after the first)
    ("refine_scale_quartered", "double s = ldexp(1.0, -(k + 1));", "double s = ldexp(1.0, -(2 * k + 1));", PM),
    ("refine_range_around_starting_plane", "double inv = 1.0 / bd + (2.0 * r[0] - 1.0)",
     "double inv = 1.0 / depth[i] + (2.0 * r[0] - 1.0)", PM),
    # caught only by the brute-force sweep pin (slower convergence, every step well formed)
    ("refine_normal_around_starting_plane",
     "double nc[3] = {bn[0] + s * (2.0 * r[1] - 1.0), bn[1] + s * (2.0 * r[2] - 1.0),\n"
     "                        bn[2] + s * (2.0 * r[3] - 1.0)};",
     "double nc[3] = {normal[i] + s * (2.0 * r[1] - 1.0), normal[N + i] + s * (2.0 * r[2] - 1.0),\n"
     "                        normal[2 * N + i] + s * (2.0 * r[3] - 1.0)};", PM),
    # consistency filter (Sec. III)
    ("filter_seam_not_wrapped", "du -= W * floor(du / W + 0.5);", "du -= 0.0;", FILTER),
    ("filter_min_views_strict", "out[i] = (d > 0 && cnt >= min_views) ? d : 0.0;",
     "out[i] = (d > 0 && cnt > min_views) ? d : 0.0;", FILTER),
    ("filter_poses_swapped", "orc_rel_pose(pose_r, &pose_j[j], &rel_f[j]);",
     "orc_rel_pose(&pose_j[j], pose_r, &rel_f[j]);", FILTER),
    ("filter_floor_not_nearest", "double fu = floor(uc + 0.5), fv = floor(vc + 0.5);\n                    double m1",
     "double fu = floor(uc), fv = floor(vc);\n                    double m1", FILTER),
    ("filter_zero_neighbour_range_used", "if (!(dj > 0)) continue;", "if (dj < 0) continue;", FILTER),
    ("filter_neighbour_bearing_from_reference_grid", "orc_bearing(Wj[j], Hj[j], ui, vi, rq);",
     "orc_bearing(W, H, ui, vi, rq);", FILTER),
    ("filter_back_projection_forward_pose", "apply_pose(&rel_b[j], Xj, Z);", "apply_pose(&rel_f[j], Xj, Z);",
     FILTER),
    # plane-map warping (Sec. III-B)
    ("warp_farther_wins", "if (rng < best[q] || (rng == best[q] && (int)j < who[q])) {",
     "if (rng > best[q] || best[q] == INFINITY) {", WARP),
    ("warp_normal_transposed",
     "n[a] = rel->R[3 * a] * nj[0] + rel->R[3 * a + 1] * nj[1] + rel->R[3 * a + 2] * nj[2];",
     "n[a] = rel->R[a] * nj[0] + rel->R[3 + a] * nj[1] + rel->R[6 + a] * nj[2];", WARP),
    ("warp_floor_not_nearest", "double fu = floor(uc + 0.5), fv = floor(vc + 0.5);\n            int qu",
     "double fu = floor(uc), fv = floor(vc);\n            int qu", WARP),
    ("warp_plane_ignored", "if (!used) orc_random_plane(pb, u, v, &d, n);", "orc_random_plane(pb, u, v, &d, n);",
     WARP),
    ("warp_normal_not_rotated",
     "n[a] = rel->R[3 * a] * nj[0] + rel->R[3 * a + 1] * nj[1] + rel->R[3 * a + 2] * nj[2];",
     "n[a] = nj[a];", WARP),
    ("warp_plane_offset_from_own_ray", "d = dot3(n, Y) / den;", "d = sqrt(dot3(Y, Y));", WARP),
    # median post-filter (Sec. III-C)
    ("median_upper", "m = win[(n - 1) / 2];", "m = win[n / 2];", MEDIAN),
    ("median_rows_clamped", "if (y < 0 || y >= H) continue;", "if (y < 0 || y >= H) y = clamp_i(y, 0, H - 1);",
     MEDIAN),
    ("median_threshold_inclusive", "out[i] = diff > lim ? 0.0 : d;", "out[i] = diff >= lim ? 0.0 : d;", MEDIAN),
    ("median_seam_clamped", "double x = depth[(size_t)y * W + wrap_i(u + dx, W)];",
     "double x = depth[(size_t)y * W + clamp_i(u + dx, 0, W - 1)];", MEDIAN),
    ("median_window_short", "for (int dy = -r; dy <= r; ++dy) {", "for (int dy = -r; dy < r; ++dy) {", MEDIAN),
    ("median_counts_holes", "if (x > 0) win[n++] = x;", "win[n++] = x;", MEDIAN),
    ("median_threshold_absolute", "lim = tau32 * m32;", "lim = tau32;", MEDIAN),
    # View Filter (Sec. III-A, Eq. 1)
    ("view_share_inclusive", "return f > min_frac;", "return f >= min_frac;", VIEW),
    ("view_centre_not_transposed",
     "ca[k] = -(A->R[k] * A->t[0] + A->R[3 + k] * A->t[1] + A->R[6 + k] * A->t[2]);",
     "ca[k] = -(A->R[3 * k] * A->t[0] + A->R[3 * k + 1] * A->t[1] + A->R[3 * k + 2] * A->t[2]);", VIEW),
    ("view_cosine_wrong_norm", "double c = dot3(a, b) / (la * lb);", "double c = dot3(a, b) / (la * la);", VIEW),
    ("view_lower_bound_dropped", "ok = th >= min_deg && th <= max_deg;", "ok = th <= max_deg;", VIEW),
    ("view_half_angle", "th = acos(c) * (180.0 / ORC_PI);", "th = acos(c) * (90.0 / ORC_PI);", VIEW),
    # fusion and completeness (Sec. III, IV)
    ("fuse_truncates_keys", "double q = X[a] / voxel, f = floor(q);", "double q = X[a] / voxel, f = trunc(q);",
     FUSION),
    ("fuse_rotation_not_transposed",
     "for (int a = 0; a < 3; ++a) X[a] = P->R[a] * Xc[0] + P->R[3 + a] * Xc[1] + P->R[6 + a] * Xc[2];",
     "for (int a = 0; a < 3; ++a) X[a] = P->R[3 * a] * Xc[0] + P->R[3 * a + 1] * Xc[1] + P->R[3 * a + 2] * Xc[2];",
     FUSION),
    ("fuse_duplicates_by_two_keys",
     "if (j > 0 && v[j].k[0] == v[j - 1].k[0] && v[j].k[1] == v[j - 1].k[1] && v[j].k[2] == v[j - 1].k[2])",
     "if (j > 0 && v[j].k[0] == v[j - 1].k[0] && v[j].k[1] == v[j - 1].k[1])", FUSION),
    ("fuse_holes_kept", "            if (!(d > 0)) {\n                if (margin)",
     "            if (d < 0) {\n                if (margin)", FUSION),
    ("fuse_translation_sign",
     "for (int a = 0; a < 3; ++a) Xc[a] = d * r[a] - P->t[a];\n            for (int a = 0; a < 3; ++a) X[a]",
     "for (int a = 0; a < 3; ++a) Xc[a] = d * r[a] + P->t[a];\n            for (int a = 0; a < 3; ++a) X[a]",
     FUSION),
    ("completeness_pose_ignored", "apply_pose(pose, pts + 3 * i, Y);",
     "Y[0] = pts[3 * i]; Y[1] = pts[3 * i + 1]; Y[2] = pts[3 * i + 2];", FUSION),
    ("fuse_keeps_last", "return (x->order > y->order) - (x->order < y->order);",
     "return (x->order < y->order) - (x->order > y->order);", FUSION),
    ("completeness_denominator", "return (double)c / ((double)W * H);", "return (double)c / ((double)W * H + W);",
     FUSION),
    ("completeness_row_rounding", "double fu = floor(uc + 0.5), fv = floor(vc + 0.5);\n        double mg = 0.5",
     "double fu = floor(uc + 0.5), fv = floor(vc + 1.0);\n        double mg = 0.5", FUSION),
]


def _run(base, name, orig, planted, modules, threads):
    """Build oracle.c with one mistake planted; run its pin modules against it."""
    src = open(SRC).read()
    if src.count(orig) != 1:
        return None, f"{name}: snippet must occur once in oracle.c"
    d = base / name
    d.mkdir()
    (d / "oracle.c").write_text(src.replace(orig, planted))
    lib = d / "liboracle.so"
    subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-o", str(lib), str(d / "oracle.c"), "-lm"])
    env = dict(os.environ, PMSP_ORACLE_LIB=str(lib), OMP_NUM_THREADS=str(threads))
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider", "-m", "not gpu",
                        *modules], cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    return r.returncode, r.stdout[-2000:]


@pytest.fixture(scope="module")
def planted_runs(tmp_path_factory):
    """Every case starts at once on a pool of the host's cores; each test waits for its own."""
    base = tmp_path_factory.mktemp("planted")
    cores = os.cpu_count() or 1
    workers = max(1, min(8, cores))
    ex = ThreadPoolExecutor(workers)
    futures = {p[0]: ex.submit(_run, base, *p, max(1, cores // workers)) for p in PLANTED}
    yield futures
    ex.shutdown(wait=True, cancel_futures=True)


@pytest.mark.parametrize("name", [p[0] for p in PLANTED])
def test_pins_catch_planted_mistake(name, planted_runs):
    rc, out = planted_runs[name].result()
    assert rc is not None, out
    # exit code 1: tests ran and at least one failed (not a crash, usage or collection error)
    assert rc == 1, f"{name}: pins did not catch it (exit {rc})\n{out}"
