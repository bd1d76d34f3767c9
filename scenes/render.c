/*
 * Seeded synthetic equirectangular scene renderer (input generator).
 *
 * This file produces the inputs that both the CUDA path and the CPU oracle
 * consume: grayscale panoramas of a textured box room with optional spheres
 * and boxes, and the ground-truth range of every pixel's centre ray. It
 * holds none of the densification arithmetic (no plane hypotheses, no
 * matching cost, no random search); it only casts rays and evaluates a
 * procedural texture.
 *
 * Conventions (shared with the rest of the project by specification):
 *   - camera frame: x right, y down, z forward; world frame uses the same
 *     handedness, y pointing down;
 *   - pixel (u, v) of a W x H panorama looks along longitude
 *     lon = 2*pi*(u + 0.5)/W - pi and latitude lat = pi/2 - pi*(v + 0.5)/H,
 *     bearing (cos lat sin lon, -sin lat, cos lat cos lon);
 *   - poses are world->camera: X_c = R X_w + t (R row-major).
 *
 * Texture: 4-octave 3-D value noise (lacunarity 2, gain 0.5) evaluated at
 * the world-space hit point, with trilinear interpolation of hashed lattice
 * values under a smoothstep fade (Perlin, "An image synthesizer", 1985).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>

#define OBJ_SPHERE 0
#define OBJ_BOX 1

typedef struct {
    int32_t kind;       /* OBJ_SPHERE or OBJ_BOX */
    int32_t tex_seed;   /* per-object texture seed */
    double c[3];        /* centre (world) */
    double r;           /* sphere radius or box half-extent */
    double gain, bias;  /* albedo = bias + gain * noise */
} scene_object;

typedef struct {
    double lo[3], hi[3];   /* room bounds (world) */
    int32_t tex_seed;      /* wall texture seed */
    double freq;           /* base texture frequency, cycles per metre */
    double gain, bias;     /* wall albedo = bias + gain * noise */
    int32_t n_obj;
    const scene_object* obj;
} scene_desc;

static uint32_t mix32(uint32_t h) {
    /* 32-bit avalanche finaliser (MurmurHash3 fmix32, public domain). */
    h ^= h >> 16; h *= 0x85ebca6bu;
    h ^= h >> 13; h *= 0xc2b2ae35u;
    h ^= h >> 16;
    return h;
}

static double lattice(int32_t x, int32_t y, int32_t z, uint32_t seed) {
    uint32_t h = mix32((uint32_t)x * 0x8da6b343u ^ mix32((uint32_t)y * 0xd8163841u ^
                       mix32((uint32_t)z * 0xcb1ab31fu ^ mix32(seed + 0x9e3779b9u))));
    return (double)(h >> 8) * (1.0 / 16777216.0);
}

static double fade(double t) { return t * t * (3.0 - 2.0 * t); }

static double value_noise(double x, double y, double z, uint32_t seed) {
    double fx = floor(x), fy = floor(y), fz = floor(z);
    int32_t ix = (int32_t)fx, iy = (int32_t)fy, iz = (int32_t)fz;
    double tx = fade(x - fx), ty = fade(y - fy), tz = fade(z - fz);
    double c[2][2][2];
    for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b)
            for (int d = 0; d < 2; ++d) c[a][b][d] = lattice(ix + a, iy + b, iz + d, seed);
    double x00 = c[0][0][0] + tx * (c[1][0][0] - c[0][0][0]);
    double x10 = c[0][1][0] + tx * (c[1][1][0] - c[0][1][0]);
    double x01 = c[0][0][1] + tx * (c[1][0][1] - c[0][0][1]);
    double x11 = c[0][1][1] + tx * (c[1][1][1] - c[0][1][1]);
    double y0 = x00 + ty * (x10 - x00);
    double y1 = x01 + ty * (x11 - x01);
    return y0 + tz * (y1 - y0);
}

static double fbm(const double p[3], double freq, uint32_t seed) {
    double sum = 0.0, amp = 1.0, norm = 0.0, f = freq;
    for (int o = 0; o < 4; ++o) {
        sum += amp * value_noise(p[0] * f, p[1] * f, p[2] * f, seed + 7919u * (uint32_t)o);
        norm += amp;
        amp *= 0.5;
        f *= 2.0;
    }
    return sum / norm;
}

/* Distance along unit direction d from o (inside the room) to the room wall. */
static double hit_room(const scene_desc* s, const double o[3], const double d[3]) {
    double best = INFINITY;
    for (int a = 0; a < 3; ++a) {
        if (d[a] > 0) {
            double t = (s->hi[a] - o[a]) / d[a];
            if (t < best) best = t;
        } else if (d[a] < 0) {
            double t = (s->lo[a] - o[a]) / d[a];
            if (t < best) best = t;
        }
    }
    return best;
}

static double hit_sphere(const scene_object* ob, const double o[3], const double d[3]) {
    double oc[3] = {o[0] - ob->c[0], o[1] - ob->c[1], o[2] - ob->c[2]};
    double b = oc[0] * d[0] + oc[1] * d[1] + oc[2] * d[2];
    double c = oc[0] * oc[0] + oc[1] * oc[1] + oc[2] * oc[2] - ob->r * ob->r;
    double disc = b * b - c;
    if (disc < 0) return INFINITY;
    double sq = sqrt(disc);
    double t0 = -b - sq;
    if (t0 > 1e-9) return t0;
    double t1 = -b + sq;
    if (t1 > 1e-9 && c > 0) return t1;
    return INFINITY;
}

static double hit_box(const scene_object* ob, const double o[3], const double d[3]) {
    double tn = -INFINITY, tf = INFINITY;
    for (int a = 0; a < 3; ++a) {
        double lo = ob->c[a] - ob->r, hi = ob->c[a] + ob->r;
        if (d[a] == 0.0) {
            if (o[a] < lo || o[a] > hi) return INFINITY;
            continue;
        }
        double t1 = (lo - o[a]) / d[a], t2 = (hi - o[a]) / d[a];
        if (t1 > t2) { double tmp = t1; t1 = t2; t2 = tmp; }
        if (t1 > tn) tn = t1;
        if (t2 < tf) tf = t2;
    }
    if (tn > tf || tn <= 1e-9) return INFINITY;
    return tn;
}

/* Nearest hit: returns range and writes the albedo of the surface hit. */
static double trace(const scene_desc* s, const double o[3], const double d[3], double* albedo) {
    double t = hit_room(s, o, d);
    int which = -1;
    for (int i = 0; i < s->n_obj; ++i) {
        double ti = s->obj[i].kind == OBJ_SPHERE ? hit_sphere(&s->obj[i], o, d)
                                                 : hit_box(&s->obj[i], o, d);
        if (ti < t) { t = ti; which = i; }
    }
    double p[3] = {o[0] + t * d[0], o[1] + t * d[1], o[2] + t * d[2]};
    if (albedo) {
        if (which < 0) {
            *albedo = s->bias + s->gain * fbm(p, s->freq, (uint32_t)s->tex_seed);
        } else {
            const scene_object* ob = &s->obj[which];
            *albedo = ob->bias + ob->gain * fbm(p, s->freq, (uint32_t)ob->tex_seed);
        }
    }
    return t;
}

static void pixel_dir(int W, int H, double u, double v, const double R[9], double dw[3]) {
    const double pi = 3.14159265358979323846;
    double lon = 2.0 * pi * (u + 0.5) / W - pi;
    double lat = 0.5 * pi - pi * (v + 0.5) / H;
    double b[3] = {cos(lat) * sin(lon), -sin(lat), cos(lat) * cos(lon)};
    /* camera->world rotation is R^T */
    dw[0] = R[0] * b[0] + R[3] * b[1] + R[6] * b[2];
    dw[1] = R[1] * b[0] + R[4] * b[1] + R[7] * b[2];
    dw[2] = R[2] * b[0] + R[5] * b[1] + R[8] * b[2];
}

/*
 * Render one panorama.
 *   R, t        world->camera pose (row-major R)
 *   ss          supersampling factor per axis (sub-ray grid ss x ss)
 *   img         out, H*W doubles: mean albedo * 255 (DN scale, unquantised)
 *   range       out, H*W doubles: range of the centre ray (may be NULL)
 */
void scene_render(const scene_desc* s, const double R[9], const double t[3], int W, int H,
                  int ss, double* img, double* range) {
    double C[3] = {-(R[0] * t[0] + R[3] * t[1] + R[6] * t[2]),
                   -(R[1] * t[0] + R[4] * t[1] + R[7] * t[2]),
                   -(R[2] * t[0] + R[5] * t[1] + R[8] * t[2])};
#pragma omp parallel for schedule(dynamic, 4)
    for (int v = 0; v < H; ++v) {
        for (int u = 0; u < W; ++u) {
            double acc = 0.0;
            for (int a = 0; a < ss; ++a)
                for (int b = 0; b < ss; ++b) {
                    double du = (b + 0.5) / ss - 0.5, dv = (a + 0.5) / ss - 0.5;
                    double d[3], alb;
                    pixel_dir(W, H, u + du, v + dv, R, d);
                    trace(s, C, d, &alb);
                    acc += alb;
                }
            img[(size_t)v * W + u] = 255.0 * acc / (ss * ss);
            if (range) {
                double d[3];
                pixel_dir(W, H, u, v, R, d);
                range[(size_t)v * W + u] = trace(s, C, d, NULL);
            }
        }
    }
}

/* Range along arbitrary world-space rays (for analytic tests). */
void scene_ray_range(const scene_desc* s, int n, const double* origins, const double* dirs,
                     double* out) {
    for (int i = 0; i < n; ++i) out[i] = trace(s, origins + 3 * i, dirs + 3 * i, NULL);
}

/* Distance from point p to the surface of an object (0 inside). */
double scene_point_object_distance(const scene_object* ob, const double p[3]) {
    if (ob->kind == OBJ_SPHERE) {
        double dx = p[0] - ob->c[0], dy = p[1] - ob->c[1], dz = p[2] - ob->c[2];
        double dist = sqrt(dx * dx + dy * dy + dz * dz) - ob->r;
        return dist > 0 ? dist : 0.0;
    }
    double acc = 0.0;
    for (int a = 0; a < 3; ++a) {
        double q = fabs(p[a] - ob->c[a]) - ob->r;
        if (q > 0) acc += q * q;
    }
    return sqrt(acc);
}
