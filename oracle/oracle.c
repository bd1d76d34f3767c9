/*
 * CPU oracle for PatchMatch-Stereo-Panorama densification (FP64).
 *
 * TEST INFRASTRUCTURE ONLY. This is a plain, slow, obviously-correct
 * restatement of the method used to check the CUDA path; it is linked by
 * nothing but the tests, the smoke check and the benchmark's CPU-baseline
 * leg. It shares no code with the CUDA library.
 *
 * Every function follows the paper (Surmann, Thurow, Slomma: "PatchMatch-
 * Stereo-Panorama, a fast dense reconstruction from 360 degree video images")
 * and the cited PatchMatch works, with the free choices fixed by the project's
 * written conventions:
 *   - equirectangular camera (Sec. III-C: rectangular patch in the reference,
 *     arbitrary shape in the sources);
 *   - random initialisation of the plane map (Sec. III-B);
 *   - red-black propagation over an 8-neighbourhood whose inner neighbours
 *     sit one position further out than in Galliani et al. (Sec. III-C,
 *     Fig. 5);
 *   - six random refinement tests on a shrinking search range (Sec. III-C,
 *     item 1);
 *   - consistency filter over neighbouring depth maps (Sec. III);
 *   - initialisation by plane-map warping (Sec. III-B);
 *   - median post-filter of the depth map (Sec. III-C, item 2);
 *   - View Filter on sparse points (Sec. III-A, Eq. 1);
 *   - dense point-cloud fusion (Sec. III) and keyframe completeness (Sec. IV).
 * Precision: double throughout. Random numbers: Philox4x64-10 (Salmon,
 * Moraes, Dror, Shaw, "Parallel random numbers: as easy as 1, 2, 3", SC'11).
 * The matching cost (bilaterally weighted NCC, best-k view aggregation) is
 * the one the cited PatchMatch stereo works use (Bleyer et al. 2011 for the
 * adaptive weights; Galliani et al. 2015 for the best-k multi-view cost).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_PI 3.14159265358979323846
#define ORC_MAX_SRC 16
#define ORC_MAX_TAPS 64

typedef struct { double R[9]; double t[3]; } orc_pose; /* world->camera, X_c = R X_w + t */

typedef struct {
    double d_min, d_max;
    int32_t patch_w, patch_stride, iterations, best_k;
    double sigma_color, sigma_space;
    int32_t n_refine, neighbor_table;
    uint64_t seed, keyframe_id;
} orc_params;

typedef struct { int32_t W, H; const double* I; } orc_img; /* intensities, row-major */

typedef struct {
    orc_img ref;
    int32_t S;
    orc_img src[ORC_MAX_SRC];
    orc_pose rel[ORC_MAX_SRC]; /* reference camera -> source camera */
    orc_params p;
} orc_problem;

/* ---------------------------------------------------------------- camera */

/* Unit bearing of continuous pixel coordinates (u, v); integer = pixel centre. */
void orc_bearing(int W, int H, double u, double v, double r[3]) {
    double lon = 2.0 * ORC_PI * (u + 0.5) / W - ORC_PI;
    double lat = 0.5 * ORC_PI - ORC_PI * (v + 0.5) / H;
    r[0] = cos(lat) * sin(lon);
    r[1] = -sin(lat);
    r[2] = cos(lat) * cos(lon);
}

/* Continuous pixel coordinates of direction Y (any length > 0). */
void orc_project(int W, int H, const double Y[3], double* uc, double* vc) {
    double lon = atan2(Y[0], Y[2]);
    double lat = atan2(-Y[1], sqrt(Y[0] * Y[0] + Y[2] * Y[2]));
    *uc = W * (lon + ORC_PI) / (2.0 * ORC_PI) - 0.5;
    *vc = H * (0.5 * ORC_PI - lat) / ORC_PI - 0.5;
}

static int wrap_i(int x, int W) { int m = x % W; return m < 0 ? m + W : m; }
static int clamp_i(int x, int lo, int hi) { return x < lo ? lo : (x > hi ? hi : x); }

/* Bilinear sample, longitude wrapped, latitude clamped. */
double orc_sample(const orc_img* im, double uc, double vc) {
    double fi = floor(uc), fj = floor(vc);
    double fx = uc - fi, fy = vc - fj;
    int i0 = (int)fi, j0 = (int)fj;
    int x0 = wrap_i(i0, im->W), x1 = wrap_i(i0 + 1, im->W);
    int y0 = clamp_i(j0, 0, im->H - 1), y1 = clamp_i(j0 + 1, 0, im->H - 1);
    const double* I = im->I;
    double t00 = I[(size_t)y0 * im->W + x0], t10 = I[(size_t)y0 * im->W + x1];
    double t01 = I[(size_t)y1 * im->W + x0], t11 = I[(size_t)y1 * im->W + x1];
    return (1.0 - fy) * ((1.0 - fx) * t00 + fx * t10) + fy * ((1.0 - fx) * t01 + fx * t11);
}

/* Relative pose reference->source: R = R_s R_r^T, t = t_s - R t_r. */
void orc_rel_pose(const orc_pose* r, const orc_pose* s, orc_pose* out) {
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double acc = 0.0;
            for (int k = 0; k < 3; ++k) acc += s->R[3 * i + k] * r->R[3 * j + k];
            out->R[3 * i + j] = acc;
        }
    for (int i = 0; i < 3; ++i) {
        double acc = 0.0;
        for (int k = 0; k < 3; ++k) acc += out->R[3 * i + k] * r->t[k];
        out->t[i] = s->t[i] - acc;
    }
}

static void apply_pose(const orc_pose* P, const double X[3], double Y[3]) {
    for (int i = 0; i < 3; ++i)
        Y[i] = P->R[3 * i] * X[0] + P->R[3 * i + 1] * X[1] + P->R[3 * i + 2] * X[2] + P->t[i];
}

static double dot3(const double a[3], const double b[3]) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }

/* ------------------------------------------------------------------- rng */

static void mulhilo64(uint64_t a, uint64_t b, uint64_t* hi, uint64_t* lo) {
    unsigned __int128 p = (unsigned __int128)a * (unsigned __int128)b;
    *hi = (uint64_t)(p >> 64);
    *lo = (uint64_t)p;
}

/* Philox4x64 with 10 rounds (SC'11 paper, Sec. 4: multipliers and Weyl key
 * increments as published there). */
void orc_philox4x64_10(const uint64_t ctr[4], const uint64_t key[2], uint64_t out[4]) {
    const uint64_t M0 = 0xD2E7470EE14C6C93ULL, M1 = 0xCA5A826395121157ULL;
    const uint64_t W0 = 0x9E3779B97F4A7C15ULL, W1 = 0xBB67AE8584CAA73BULL;
    uint64_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
    uint64_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        uint64_t hi0, lo0, hi1, lo1;
        mulhilo64(M0, x0, &hi0, &lo0);
        mulhilo64(M1, x2, &hi1, &lo1);
        uint64_t y0 = hi1 ^ x1 ^ k0, y1 = lo1, y2 = hi0 ^ x3 ^ k1, y3 = lo0;
        x0 = y0; x1 = y1; x2 = y2; x3 = y3;
        k0 += W0; k1 += W1;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/* Uniform in [0, 1) from the top 24 bits of a word (exact in float and double). */
double orc_u24(uint64_t w) { return (double)(w >> 40) * (1.0 / 16777216.0); }

static void draw4(const orc_params* p, uint64_t pixel, uint64_t iter, uint64_t stage, double u[4]) {
    uint64_t ctr[4] = {pixel, iter, stage, 0}, key[2] = {p->seed, p->keyframe_id}, w[4];
    orc_philox4x64_10(ctr, key, w);
    for (int i = 0; i < 4; ++i) u[i] = orc_u24(w[i]);
}

/* ------------------------------------------------------------------ cost */

/* Patch sample offsets along one axis: -r, -r+s, ..., r = (patch_w-1)/2. */
int orc_patch_offsets(const orc_params* p, int* offs) {
    int r = (p->patch_w - 1) / 2, n = 0;
    for (int o = -r; o <= r; o += p->patch_stride) offs[n++] = o;
    return n;
}

/* Orient a normal towards the camera: n.r_p must be negative. */
static void face_camera(double n[3], const double rp[3]) {
    double c = dot3(n, rp);
    if (fabs(c) < 1e-3) {
        n[0] = -rp[0]; n[1] = -rp[1]; n[2] = -rp[2];
    } else if (c > 0) {
        n[0] = -n[0]; n[1] = -n[1]; n[2] = -n[2];
    }
}

/*
 * Matching cost of plane (range d along r_p, normal n) at reference pixel
 * (u, v). Per view: 1 - weighted Pearson correlation of the reference patch
 * and its reprojection through the plane, 2 for an invalid or flat patch;
 * the result is the mean of the best_k smallest view costs. `view_cost`
 * (nullable) receives the S per-view costs.
 */
double orc_cost(const orc_problem* pb, int u, int v, double d, const double n[3], double* view_cost) {
    const orc_params* p = &pb->p;
    const int W = pb->ref.W, H = pb->ref.H, S = pb->S;
    int offs[ORC_MAX_TAPS];
    int K = orc_patch_offsets(p, offs);
    double rp[3];
    orc_bearing(W, H, u, v, rp);
    double Ip = pb->ref.I[(size_t)v * W + u];
    double ndotrp = dot3(n, rp);

    double sw[ORC_MAX_SRC] = {0}, sI[ORC_MAX_SRC] = {0}, sII[ORC_MAX_SRC] = {0};
    double sJ[ORC_MAX_SRC] = {0}, sJJ[ORC_MAX_SRC] = {0}, sIJ[ORC_MAX_SRC] = {0};
    int invalid = 0;
    for (int a = 0; a < K && !invalid; ++a) {
        for (int b = 0; b < K; ++b) {
            int oy = offs[a], ox = offs[b];
            int qu = wrap_i(u + ox, W), qv = clamp_i(v + oy, 0, H - 1);
            double rq[3];
            orc_bearing(W, H, qu, qv, rq);
            double Iq = pb->ref.I[(size_t)qv * W + qu];
            double e = 0.0;
            if (p->sigma_color > 0) e += (Iq - Ip) * (Iq - Ip) / (2.0 * p->sigma_color * p->sigma_color);
            if (p->sigma_space > 0) e += (double)(ox * ox + oy * oy) / (2.0 * p->sigma_space * p->sigma_space);
            double w = exp(-e);
            double denom = dot3(n, rq);
            if (!(denom < -1e-6)) { invalid = 1; break; }
            double tq = d * ndotrp / denom;
            double X[3] = {tq * rq[0], tq * rq[1], tq * rq[2]};
            for (int s = 0; s < S; ++s) {
                double Y[3], uc, vc;
                apply_pose(&pb->rel[s], X, Y);
                orc_project(pb->src[s].W, pb->src[s].H, Y, &uc, &vc);
                double J = orc_sample(&pb->src[s], uc, vc);
                sw[s] += w;
                sI[s] += w * Iq;
                sII[s] += w * Iq * Iq;
                sJ[s] += w * J;
                sJJ[s] += w * J * J;
                sIJ[s] += w * Iq * J;
            }
        }
    }
    double c[ORC_MAX_SRC];
    for (int s = 0; s < S; ++s) {
        if (invalid) { c[s] = 2.0; continue; }
        double varI = sw[s] * sII[s] - sI[s] * sI[s];
        double varJ = sw[s] * sJJ[s] - sJ[s] * sJ[s];
        double cov = sw[s] * sIJ[s] - sI[s] * sJ[s];
        double eps = 1e-8 * sw[s] * sw[s];
        if (varI < eps || varJ < eps) { c[s] = 2.0; continue; }
        double ncc = cov / sqrt(varI * varJ);
        if (ncc > 1.0) ncc = 1.0;
        if (ncc < -1.0) ncc = -1.0;
        c[s] = 1.0 - ncc;
    }
    if (view_cost)
        for (int s = 0; s < S; ++s) view_cost[s] = c[s];
    /* mean of the k smallest: selection by repeated minimum */
    int used[ORC_MAX_SRC] = {0};
    double sum = 0.0;
    for (int k = 0; k < p->best_k; ++k) {
        int best = -1;
        for (int s = 0; s < S; ++s)
            if (!used[s] && (best < 0 || c[s] < c[best])) best = s;
        used[best] = 1;
        sum += c[best];
    }
    return sum / p->best_k;
}

void orc_cost_map(const orc_problem* pb, const double* depth, const double* normal, double* cost) {
    const int W = pb->ref.W, H = pb->ref.H;
    const size_t N = (size_t)W * H;
#pragma omp parallel for schedule(dynamic, 8)
    for (int v = 0; v < H; ++v)
        for (int u = 0; u < W; ++u) {
            size_t i = (size_t)v * W + u;
            double n[3] = {normal[i], normal[N + i], normal[2 * N + i]};
            cost[i] = orc_cost(pb, u, v, depth[i], n, NULL);
        }
}

/* --------------------------------------------------------- initialisation */

/* Random plane at pixel (u, v) (Sec. III-B): inverse range uniform on
 * [1/d_max, 1/d_min), normal uniform on the sphere turned to face the camera. */
void orc_random_plane(const orc_problem* pb, int u, int v, double* d, double n[3]) {
    const orc_params* p = &pb->p;
    double rp[3], r[4];
    orc_bearing(pb->ref.W, pb->ref.H, u, v, rp);
    draw4(p, (uint64_t)v * pb->ref.W + u, 0, 0, r);
    double inv = 1.0 / p->d_max + r[0] * (1.0 / p->d_min - 1.0 / p->d_max);
    *d = 1.0 / inv;
    double z = 1.0 - 2.0 * r[1], phi = 2.0 * ORC_PI * r[2];
    double rho = sqrt(fmax(0.0, 1.0 - z * z));
    n[0] = rho * cos(phi);
    n[1] = rho * sin(phi);
    n[2] = z;
    face_camera(n, rp);
}

void orc_init(const orc_problem* pb, double* depth, double* normal, double* cost) {
    const int W = pb->ref.W, H = pb->ref.H;
    const size_t N = (size_t)W * H;
#pragma omp parallel for schedule(dynamic, 8)
    for (int v = 0; v < H; ++v)
        for (int u = 0; u < W; ++u) {
            size_t i = (size_t)v * W + u;
            double d, n[3];
            orc_random_plane(pb, u, v, &d, n);
            depth[i] = d;
            normal[i] = n[0]; normal[N + i] = n[1]; normal[2 * N + i] = n[2];
            cost[i] = orc_cost(pb, u, v, d, n, NULL);
        }
}

/* ----------------------------------------------------- propagation tables */

/* Opposite-colour neighbours (dx, dy), in the order they are tried. Table 0:
 * axis neighbours at distance 3 (the inner ring moved one position outward,
 * keeping the opposite colour) and at distance 5; table 1: distances 1 and 5. */
int orc_neighbor_table(int id, int dxdy[16]) {
    static const int t0[16] = {0, -3, 0, 3, -3, 0, 3, 0, 0, -5, 0, 5, -5, 0, 5, 0};
    static const int t1[16] = {0, -1, 0, 1, -1, 0, 1, 0, 0, -5, 0, 5, -5, 0, 5, 0};
    memcpy(dxdy, id == 1 ? t1 : t0, sizeof(t0));
    return 8;
}

/*
 * One pixel's update in a half-sweep (Sec. III-C): try the 8 neighbours'
 * planes re-intersected with this pixel's ray, then `n_refine` random
 * perturbations of the current best on a range that halves each test; a
 * candidate replaces the incumbent only if its cost is strictly lower.
 * Reads the state arrays (this pixel and its opposite-colour neighbours) and
 * returns the new state without writing it.
 */
void orc_update_pixel(const orc_problem* pb, const double* depth, const double* normal,
                      const double* cost, int u, int v, int iter, double* d_out, double n_out[3],
                      double* c_out) {
    const orc_params* p = &pb->p;
    const int W = pb->ref.W, H = pb->ref.H;
    const size_t N = (size_t)W * H;
    size_t i = (size_t)v * W + u;
    double rp[3];
    orc_bearing(W, H, u, v, rp);
    double bd = depth[i], bn[3] = {normal[i], normal[N + i], normal[2 * N + i]}, bc = cost[i];

    int tab[16];
    int nn = orc_neighbor_table(p->neighbor_table, tab);
    for (int k = 0; k < nn; ++k) {
        int qv = v + tab[2 * k + 1];
        if (qv < 0 || qv >= H) continue;
        int qu = wrap_i(u + tab[2 * k], W);
        size_t j = (size_t)qv * W + qu;
        double nq[3] = {normal[j], normal[N + j], normal[2 * N + j]};
        double rq[3];
        orc_bearing(W, H, qu, qv, rq);
        double den = dot3(nq, rp);
        if (!(den < -1e-6)) continue;
        double dc = depth[j] * dot3(nq, rq) / den;
        if (!(dc >= p->d_min && dc <= p->d_max)) continue;
        double c = orc_cost(pb, u, v, dc, nq, NULL);
        if (c < bc) {
            bd = dc; bc = c;
            bn[0] = nq[0]; bn[1] = nq[1]; bn[2] = nq[2];
        }
    }

    const double inv_lo = 1.0 / p->d_max, inv_hi = 1.0 / p->d_min;
    for (int k = 0; k < p->n_refine; ++k) {
        double s = ldexp(1.0, -(k + 1));
        double r[4];
        draw4(p, (uint64_t)i, (uint64_t)iter, (uint64_t)(1 + k), r);
        double inv = 1.0 / bd + (2.0 * r[0] - 1.0) * s * (inv_hi - inv_lo);
        if (inv < inv_lo) inv = inv_lo;
        if (inv > inv_hi) inv = inv_hi;
        double dc = 1.0 / inv;
        double nc[3] = {bn[0] + s * (2.0 * r[1] - 1.0), bn[1] + s * (2.0 * r[2] - 1.0),
                        bn[2] + s * (2.0 * r[3] - 1.0)};
        double len = sqrt(dot3(nc, nc));
        nc[0] /= len; nc[1] /= len; nc[2] /= len;
        face_camera(nc, rp);
        double c = orc_cost(pb, u, v, dc, nc, NULL);
        if (c < bc) {
            bd = dc; bc = c;
            bn[0] = nc[0]; bn[1] = nc[1]; bn[2] = nc[2];
        }
    }
    *d_out = bd;
    n_out[0] = bn[0]; n_out[1] = bn[1]; n_out[2] = bn[2];
    *c_out = bc;
}

/* All pixels with (u + v) % 2 == colour, in place (they read only the other colour). */
void orc_halfsweep(const orc_problem* pb, double* depth, double* normal, double* cost, int colour,
                   int iter) {
    const int W = pb->ref.W, H = pb->ref.H;
    const size_t N = (size_t)W * H;
#pragma omp parallel for schedule(dynamic, 4)
    for (int v = 0; v < H; ++v)
        for (int u = (v + colour) & 1; u < W; u += 2) {
            size_t i = (size_t)v * W + u;
            double d, n[3], c;
            orc_update_pixel(pb, depth, normal, cost, u, v, iter, &d, n, &c);
            depth[i] = d;
            normal[i] = n[0]; normal[N + i] = n[1]; normal[2 * N + i] = n[2];
            cost[i] = c;
        }
}

/* Random init, then `iterations` x (red half-sweep, black half-sweep). */
void orc_densify(const orc_problem* pb, double* depth, double* normal, double* cost) {
    orc_init(pb, depth, normal, cost);
    for (int t = 0; t < pb->p.iterations; ++t) {
        orc_halfsweep(pb, depth, normal, cost, 0, t);
        orc_halfsweep(pb, depth, normal, cost, 1, t);
    }
}

/* Exhaustive search over inverse-range levels x given normals (test pin). */
void orc_plane_sweep(const orc_problem* pb, int n_levels, const double* normals, int n_normals,
                     double* best_cost, double* best_depth) {
    const int W = pb->ref.W, H = pb->ref.H;
    const orc_params* p = &pb->p;
#pragma omp parallel for schedule(dynamic, 1)
    for (int v = 0; v < H; ++v)
        for (int u = 0; u < W; ++u) {
            double rp[3];
            orc_bearing(W, H, u, v, rp);
            double bc = INFINITY, bd = 0.0;
            for (int l = 0; l < n_levels; ++l) {
                double inv = 1.0 / p->d_max + (1.0 / p->d_min - 1.0 / p->d_max) * l / (n_levels - 1);
                for (int m = 0; m < n_normals; ++m) {
                    const double* n = normals + 3 * m;
                    if (!(dot3(n, rp) < -1e-3)) continue;
                    double c = orc_cost(pb, u, v, 1.0 / inv, n, NULL);
                    if (c < bc) { bc = c; bd = 1.0 / inv; }
                }
            }
            best_cost[(size_t)v * W + u] = bc;
            best_depth[(size_t)v * W + u] = bd;
        }
}

/* ------------------------------------------------- consistency filtering */

/*
 * Geometric consistency filter (Sec. III: a depth map is checked against its
 * neighbours' depth maps and outliers are removed). A reference pixel with
 * range d > 0 is lifted to 3-D, projected into neighbour j, the nearest pixel
 * of D_j is lifted back and reprojected into the reference; the view agrees if
 * the reprojection error (longitude difference wrapped to half a panorama) is
 * below max_px. A pixel is kept when at least min_views views agree,
 * otherwise its range becomes 0. `agree` (nullable) receives the count;
 * `margin` (nullable) the smallest distance of any decision of the pixel to
 * its threshold (error vs max_px, nearest-pixel rounding vs the half-pixel).
 */
void orc_consistency_filter(int W, int H, const double* depth, const orc_pose* pose_r, int n,
                            const int* Wj, const int* Hj, const double* const* Dj,
                            const orc_pose* pose_j, double max_px, int min_views, double* out,
                            int* agree, double* margin) {
    orc_pose rel_f[ORC_MAX_SRC], rel_b[ORC_MAX_SRC];
    for (int j = 0; j < n; ++j) {
        orc_rel_pose(pose_r, &pose_j[j], &rel_f[j]); /* reference -> j */
        orc_rel_pose(&pose_j[j], pose_r, &rel_b[j]); /* j -> reference */
    }
#pragma omp parallel for schedule(dynamic, 8)
    for (int v = 0; v < H; ++v)
        for (int u = 0; u < W; ++u) {
            size_t i = (size_t)v * W + u;
            double d = depth[i];
            int cnt = 0;
            double mg = INFINITY;
            if (d > 0) {
                double rp[3];
                orc_bearing(W, H, u, v, rp);
                double X[3] = {d * rp[0], d * rp[1], d * rp[2]};
                for (int j = 0; j < n; ++j) {
                    double Y[3], uc, vc;
                    apply_pose(&rel_f[j], X, Y);
                    orc_project(Wj[j], Hj[j], Y, &uc, &vc);
                    double fu = floor(uc + 0.5), fv = floor(vc + 0.5);
                    double m1 = fabs(uc + 0.5 - fu - 0.5), m2 = fabs(vc + 0.5 - fv - 0.5);
                    mg = fmin(mg, 0.5 - m1);
                    if (fv >= 0 && fv <= Hj[j] - 1) mg = fmin(mg, 0.5 - m2);
                    int ui = wrap_i((int)fu, Wj[j]), vi = clamp_i((int)fv, 0, Hj[j] - 1);
                    double dj = Dj[j][(size_t)vi * Wj[j] + ui];
                    if (!(dj > 0)) continue;
                    double rq[3], Xj[3], Z[3], u2, v2;
                    orc_bearing(Wj[j], Hj[j], ui, vi, rq);
                    Xj[0] = dj * rq[0]; Xj[1] = dj * rq[1]; Xj[2] = dj * rq[2];
                    apply_pose(&rel_b[j], Xj, Z);
                    orc_project(W, H, Z, &u2, &v2);
                    double du = u2 - u, dv = v2 - v;
                    du -= W * floor(du / W + 0.5);
                    double e = sqrt(du * du + dv * dv);
                    mg = fmin(mg, fabs(e - max_px));
                    if (e < max_px) ++cnt;
                }
            }
            out[i] = (d > 0 && cnt >= min_views) ? d : 0.0;
            if (agree) agree[i] = cnt;
            if (margin) margin[i] = mg;
        }
}

/* ------------------------------------------------------ plane-map warping */

/*
 * Initialisation by plane-map warping (Sec. III-B: the optimised plane map of
 * the preceding keyframe is transferred into the current one, after Shen
 * 2013; the algorithm figure is missing, so this follows the project's
 * reading). Every previous pixel j with range d_j > 0 is lifted to 3-D with
 * its plane, moved into the current camera (rel: previous -> current) and
 * splatted onto the nearest current pixel; per pixel the candidate with the
 * smallest range wins (ties: smallest j). A winning plane is re-intersected
 * with the pixel's own ray; if that is invalid (grazing, behind, or outside
 * [d_min, d_max]) or no candidate reached the pixel, the random plane of the
 * ordinary initialisation is used. Costs are those of the chosen planes.
 * `src` (nullable) receives the winning j or -1; `clear` (nullable) is 1
 * where every decision is at least 1e-3 px (rounding) and 1e-5 relative
 * (range order) from its threshold.
 */
void orc_warp_init(const orc_problem* pb, int Wp, int Hp, const double* prev_depth, const double* prev_normal,
                   const orc_pose* rel, double* depth, double* normal, double* cost, int* src, int* clear) {
    const int W = pb->ref.W, H = pb->ref.H;
    const size_t N = (size_t)W * H, Np = (size_t)Wp * Hp;
    double* best = (double*)malloc(N * sizeof(double));
    double* second = (double*)malloc(N * sizeof(double));
    int* who = (int*)malloc(N * sizeof(int));
    int* ok = (int*)malloc(N * sizeof(int));
    for (size_t i = 0; i < N; ++i) { best[i] = INFINITY; second[i] = INFINITY; who[i] = -1; ok[i] = 1; }
    for (int v = 0; v < Hp; ++v)
        for (int u = 0; u < Wp; ++u) {
            size_t j = (size_t)v * Wp + u;
            double d = prev_depth[j];
            if (!(d > 0)) continue;
            double r[3], X[3], Y[3], uc, vc;
            orc_bearing(Wp, Hp, u, v, r);
            X[0] = d * r[0]; X[1] = d * r[1]; X[2] = d * r[2];
            apply_pose(rel, X, Y);
            orc_project(W, H, Y, &uc, &vc);
            double fu = floor(uc + 0.5), fv = floor(vc + 0.5);
            int qu = wrap_i((int)fu, W), qv = clamp_i((int)fv, 0, H - 1);
            size_t q = (size_t)qv * W + qu;
            double rng = sqrt(dot3(Y, Y));
            /* a point within 1e-3 px of a rounding boundary may land on the pixel
               across it in a lower precision: both pixels are marked unclear */
            double eu = uc + 0.5 - fu, ev = vc + 0.5 - fv;
            int au = eu < 1e-3 ? -1 : (eu > 1.0 - 1e-3 ? 1 : 0);
            int av = ev < 1e-3 ? -1 : (ev > 1.0 - 1e-3 ? 1 : 0);
            if (au || av) {
                for (int a = 0; a <= (au != 0); ++a)
                    for (int b = 0; b <= (av != 0); ++b) {
                        int pu = wrap_i((int)fu + a * au, W), pv = clamp_i((int)fv + b * av, 0, H - 1);
                        ok[(size_t)pv * W + pu] = 0;
                    }
            }
            if (rng < best[q] || (rng == best[q] && (int)j < who[q])) {
                second[q] = best[q];
                best[q] = rng;
                who[q] = (int)j;
            } else if (rng < second[q]) {
                second[q] = rng;
            }
        }
    (void)Np;
#pragma omp parallel for schedule(dynamic, 8)
    for (int v = 0; v < H; ++v)
        for (int u = 0; u < W; ++u) {
            size_t i = (size_t)v * W + u;
            double rp[3], d = 0.0, n[3] = {0, 0, 0};
            orc_bearing(W, H, u, v, rp);
            int used = 0, clr = ok[i];
            if (who[i] >= 0) {
                size_t j = (size_t)who[i];
                int ju = (int)(j % Wp), jv = (int)(j / Wp);
                double r[3], X[3], Y[3], nj[3] = {prev_normal[j], prev_normal[Np + j], prev_normal[2 * Np + j]};
                orc_bearing(Wp, Hp, ju, jv, r);
                X[0] = prev_depth[j] * r[0]; X[1] = prev_depth[j] * r[1]; X[2] = prev_depth[j] * r[2];
                apply_pose(rel, X, Y);
                for (int a = 0; a < 3; ++a)
                    n[a] = rel->R[3 * a] * nj[0] + rel->R[3 * a + 1] * nj[1] + rel->R[3 * a + 2] * nj[2];
                double den = dot3(n, rp);
                if (second[i] < INFINITY && (second[i] - best[i]) < 1e-5 * best[i]) clr = 0;
                if (fabs(den) < 1e-4) clr = 0;
                if (den < -1e-6) {
                    d = dot3(n, Y) / den;
                    if (fabs(d - pb->p.d_min) < 1e-6 * d || fabs(d - pb->p.d_max) < 1e-6 * d) clr = 0;
                    used = d >= pb->p.d_min && d <= pb->p.d_max;
                }
            }
            if (!used) orc_random_plane(pb, u, v, &d, n);
            depth[i] = d;
            normal[i] = n[0]; normal[N + i] = n[1]; normal[2 * N + i] = n[2];
            cost[i] = orc_cost(pb, u, v, d, n, NULL);
            if (src) src[i] = used ? who[i] : -1;
            if (clear) clear[i] = clr;
        }
    free(best); free(second); free(who); free(ok);
}

/* ------------------------------------------------------ median post-filter */

static int cmp_double(const void* a, const void* b) {
    double x = *(const double*)a, y = *(const double*)b;
    return (x > y) - (x < y);
}

/*
 * Median post-filter (Sec. III-C, item 2: a median filter runs over a copy of
 * the depth image and depths that deviate from the filtered copy by more than
 * a threshold are removed; window and threshold are not given, so this
 * follows the project's reading). For a pixel with range d > 0, the valid
 * ranges (> 0) of the (2r+1) x (2r+1) window around it (columns wrapped at
 * the seam, rows outside the panorama left out) are sorted and the lower
 * median m, the element of rank floor((n-1)/2), is taken. The range is
 * removed (set to 0) when |d - m| > tau * m, decided in single precision as
 * the depth maps are stored. Every decision reads the unfiltered input.
 * `med` (nullable) receives m (0 where d <= 0).
 */
void orc_median_filter(int W, int H, const double* depth, int r, double tau, double* out, double* med) {
    const float tau32 = (float)tau;
#pragma omp parallel for schedule(dynamic, 8)
    for (int v = 0; v < H; ++v) {
        double win[(2 * 16 + 1) * (2 * 16 + 1)];
        for (int u = 0; u < W; ++u) {
            size_t i = (size_t)v * W + u;
            double d = depth[i], m = 0.0;
            if (d > 0) {
                int n = 0;
                for (int dy = -r; dy <= r; ++dy) {
                    int y = v + dy;
                    if (y < 0 || y >= H) continue;
                    for (int dx = -r; dx <= r; ++dx) {
                        double x = depth[(size_t)y * W + wrap_i(u + dx, W)];
                        if (x > 0) win[n++] = x;
                    }
                }
                qsort(win, (size_t)n, sizeof(double), cmp_double);
                m = win[(n - 1) / 2];
                float d32 = (float)d, m32 = (float)m;
                float diff = fabsf(d32 - m32), lim = tau32 * m32;
                out[i] = diff > lim ? 0.0 : d;
            } else {
                out[i] = 0.0;
            }
            if (med) med[i] = m;
        }
    }
}

/* ------------------------------------------------------------- view filter */

/*
 * View Filter (Sec. III-A, Eq. 1; the equation is garbled in the source and
 * read as the parallax angle at p between the rays to the two camera
 * centres): for every sparse point p seen by keyframes A and B,
 * theta_p = arccos((t_A - p).(t_B - p) / (|t_A - p| |t_B - p|)), with t_K the
 * camera centre -R^T t of pose K. B is accepted when the share of points with
 * theta_p in [min_deg, max_deg] exceeds min_frac (6, 60 degrees and 20 % in
 * the paper). A point at a camera centre has no angle and counts as out of
 * range. `theta_deg` and `in_range` (nullable) receive the per-point values;
 * `frac` (nullable) the share. Returns 1 (accept) or 0.
 */
int orc_view_filter(const orc_pose* A, const orc_pose* B, const double* pts, int n, double min_deg,
                    double max_deg, double min_frac, double* theta_deg, int* in_range, double* frac) {
    double ca[3], cb[3];
    for (int k = 0; k < 3; ++k) {
        ca[k] = -(A->R[k] * A->t[0] + A->R[3 + k] * A->t[1] + A->R[6 + k] * A->t[2]);
        cb[k] = -(B->R[k] * B->t[0] + B->R[3 + k] * B->t[1] + B->R[6 + k] * B->t[2]);
    }
    int cnt = 0;
    for (int i = 0; i < n; ++i) {
        const double* p = pts + 3 * (size_t)i;
        double a[3] = {ca[0] - p[0], ca[1] - p[1], ca[2] - p[2]};
        double b[3] = {cb[0] - p[0], cb[1] - p[1], cb[2] - p[2]};
        double la = sqrt(dot3(a, a)), lb = sqrt(dot3(b, b));
        double th = NAN;
        int ok = 0;
        if (la > 0 && lb > 0) {
            double c = dot3(a, b) / (la * lb);
            c = c > 1 ? 1 : (c < -1 ? -1 : c);
            th = acos(c) * (180.0 / ORC_PI);
            ok = th >= min_deg && th <= max_deg;
        }
        cnt += ok;
        if (theta_deg) theta_deg[i] = th;
        if (in_range) in_range[i] = ok;
    }
    double f = n > 0 ? (double)cnt / n : 0.0;
    if (frac) *frac = f;
    return f > min_frac;
}

/* ------------------------------------------ point-cloud fusion, completeness */

typedef struct { int64_t k[3]; int64_t order; } orc_vox;

static int cmp_vox(const void* a, const void* b) {
    const orc_vox *x = (const orc_vox*)a, *y = (const orc_vox*)b;
    for (int i = 0; i < 3; ++i)
        if (x->k[i] != y->k[i]) return (x->k[i] > y->k[i]) - (x->k[i] < y->k[i]);
    return (x->order > y->order) - (x->order < y->order);
}

/*
 * Dense point-cloud fusion (Sec. III: the point-cloud thread takes the
 * filtered depth maps of consecutive keyframes and erases duplicate points;
 * the duplicate rule is not given, so this follows the project's reading).
 * Every pixel with range d > 0 of keyframe k becomes the world point
 * X = R_k^T (d r_p - t_k). Points are binned into cubic voxels of edge
 * `voxel` (key floor(X / voxel) per axis); of the points in one voxel the
 * first in (keyframe, pixel index) order is kept. Writes the kept points (3
 * doubles each) and their sources (k << 32 | pixel) in increasing key order
 * (x, then y, then z key), at most `cap` of them, and returns how many
 * voxels are occupied. `margin` (nullable, one per input pixel in keyframe
 * order, -1 where d <= 0) receives the smallest distance of the point's
 * coordinates to a voxel face, in voxels.
 */
int64_t orc_fuse(int n, const int* Ws, const int* Hs, const double* const* depth, const orc_pose* poses,
                 double voxel, double* pts, int64_t* src, int64_t cap, double* margin) {
    int64_t total = 0;
    for (int k = 0; k < n; ++k) total += (int64_t)Ws[k] * Hs[k];
    orc_vox* v = (orc_vox*)malloc((size_t)(total > 0 ? total : 1) * sizeof(orc_vox));
    int64_t m = 0, base = 0;
    for (int k = 0; k < n; ++k) {
        const orc_pose* P = &poses[k];
        for (int i = 0; i < Ws[k] * Hs[k]; ++i) {
            double d = depth[k][i];
            if (!(d > 0)) {
                if (margin) margin[base + i] = -1;
                continue;
            }
            double r[3], Xc[3], X[3];
            orc_bearing(Ws[k], Hs[k], i % Ws[k], i / Ws[k], r);
            for (int a = 0; a < 3; ++a) Xc[a] = d * r[a] - P->t[a];
            for (int a = 0; a < 3; ++a) X[a] = P->R[a] * Xc[0] + P->R[3 + a] * Xc[1] + P->R[6 + a] * Xc[2];
            double mg = INFINITY;
            for (int a = 0; a < 3; ++a) {
                double q = X[a] / voxel, f = floor(q);
                v[m].k[a] = (int64_t)f;
                mg = fmin(mg, fmin(q - f, f + 1 - q));
            }
            if (margin) margin[base + i] = mg;
            v[m].order = ((int64_t)k << 32) | i;
            ++m;
        }
        base += (int64_t)Ws[k] * Hs[k];
    }
    qsort(v, (size_t)m, sizeof(orc_vox), cmp_vox);
    int64_t out = 0;
    for (int64_t j = 0; j < m; ++j) {
        if (j > 0 && v[j].k[0] == v[j - 1].k[0] && v[j].k[1] == v[j - 1].k[1] && v[j].k[2] == v[j - 1].k[2])
            continue;
        if (out < cap) {
            int k = (int)(v[j].order >> 32), i = (int)(v[j].order & 0xffffffff);
            const orc_pose* P = &poses[k];
            double r[3], Xc[3], d = depth[k][i];
            orc_bearing(Ws[k], Hs[k], i % Ws[k], i / Ws[k], r);
            for (int a = 0; a < 3; ++a) Xc[a] = d * r[a] - P->t[a];
            for (int a = 0; a < 3; ++a)
                pts[3 * out + a] = P->R[a] * Xc[0] + P->R[3 + a] * Xc[1] + P->R[6 + a] * Xc[2];
            if (src) src[out] = v[j].order;
        }
        ++out;
    }
    free(v);
    return out;
}

/*
 * Keyframe-related completeness (Sec. IV: at each keyframe position a
 * panorama is rendered from the point cloud and the share of its pixels onto
 * which some 3-D point projects is the completeness; 720 x 360 in the paper).
 * Every point is moved into the camera of `pose` and projected onto the
 * nearest pixel of a W x H panorama (u wrapped, v clamped); occlusion plays
 * no part. Returns the share of pixels hit; `hit` (nullable, W*H) receives
 * the per-pixel flags and `margin` (nullable, one per point) the distance of
 * the projection to the nearest pixel boundary, in pixels (a point at the
 * camera centre gets -1 and hits nothing).
 */
double orc_completeness(const double* pts, int64_t n, const orc_pose* pose, int W, int H, int* hit,
                        double* margin) {
    int* h = hit ? hit : (int*)malloc((size_t)W * H * sizeof(int));
    memset(h, 0, (size_t)W * H * sizeof(int));
    for (int64_t i = 0; i < n; ++i) {
        double Y[3], uc, vc;
        apply_pose(pose, pts + 3 * i, Y);
        if (dot3(Y, Y) == 0) {
            if (margin) margin[i] = -1;
            continue;
        }
        orc_project(W, H, Y, &uc, &vc);
        double fu = floor(uc + 0.5), fv = floor(vc + 0.5);
        double mg = 0.5 - fabs(uc - fu);
        if (fv >= 0 && fv <= H - 1) mg = fmin(mg, 0.5 - fabs(vc - fv));
        if (margin) margin[i] = mg;
        h[(size_t)clamp_i((int)fv, 0, H - 1) * W + wrap_i((int)fu, W)] = 1;
    }
    int64_t c = 0;
    for (size_t j = 0; j < (size_t)W * H; ++j) c += h[j];
    if (!hit) free(h);
    return (double)c / ((double)W * H);
}
