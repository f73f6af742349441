/*
 * scenegen.c - seeded synthetic hair scenes for the multi-view direction-fusion path.
 *
 * Produces the inputs the fusion step consumes (Sec. 3.1 of the paper: a raw outer point
 * cloud P_raw, calibrated pinhole cameras Pi_v, per-view 2D orientation maps O_v and
 * confidence maps C_v) plus the k-nearest-neighbour patch lists, for scenes of helical,
 * wavy and straight strands grown from a spherical scalp cap.
 *
 * This module is shared input plumbing.  It holds none of the fusion arithmetic: no cost,
 * no hypothesis set, no argmin, no refinement.  Random numbers come from a counter-based
 * generator (SplitMix64, Steele/Lea/Flood 2014) keyed by (seed, stream, counter), so every
 * output is a pure function of the configuration and the seed, independent of thread count.
 *
 * Maps are rendered from the CLEAN poses; when pose noise is requested the cameras handed
 * to the fusion are the NOISY ones (they model calibration error).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define SG_PI 3.14159265358979323846

typedef struct {
    int n_strands;
    int n_segments;        /* segments per strand polyline */
    int points_mode;       /* 0: pts_per_strand evenly spaced in arc length; 1: one per segment midpoint */
    int pts_per_strand;
    int strand_mix;        /* 0: all helices; 1: thirds straight / wavy / curly */
    double helix_r_lo, helix_r_hi;     /* helix radius range */
    double pitch_lo, pitch_hi;         /* helix pitch range (advance per turn) */
    double wave_a_lo, wave_a_hi;       /* wavy amplitude range */
    double wave_len_lo, wave_len_hi;   /* wavy wavelength range */
    double len_lo, len_hi;             /* strand arc length range (head radii) */
    double cap_deg;                    /* scalp cap half-angle about +y */
    int V, width, height;
    double f, cx, cy;
    int cam_mode;          /* 0: ring in y=0 plane; 1: half orbit az [-90,90] + elevation jitter; 2: full orbit */
    double cam_radius;
    double elev_jitter_deg;
    double pose_noise_deg; /* std-dev of per-frame rotation noise applied to the fused cameras */
    double angle_noise_deg;/* std-dev of per-pixel orientation noise */
    double conf_lo, conf_hi;           /* confidence on covered pixels */
    double outlier_frac;   /* fraction of pixels replaced by uniform angle, conf in [0, outlier_conf_hi) */
    double outlier_conf_hi;
    int k;                 /* neighbours per point */
    uint64_t seed;
} sg_config;

/* ---------------------------------------------------------------- random numbers */

static uint64_t sm64(uint64_t x) {
    x += 0x9E3779B97F4A7C15ULL;
    x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ULL;
    x = (x ^ (x >> 27)) * 0x94D049BB133111EBULL;
    return x ^ (x >> 31);
}

typedef struct { uint64_t key; uint64_t ctr; } rng_t;

static rng_t rng_make(uint64_t seed, uint64_t stream_tag, uint64_t stream) {
    rng_t r;
    r.key = sm64(sm64(seed ^ 0x5CE5CE5CE5CE5CE5ULL) ^ sm64(stream_tag) ^ (stream * 0xD1B54A32D192ED03ULL));
    r.ctr = 0;
    return r;
}
static uint64_t rng_u64(rng_t* r) { return sm64(r->key + (r->ctr++) * 0x9E3779B97F4A7C15ULL); }
/* uniform in [0,1) with 53 random bits */
static double rng_uni(rng_t* r) { return (double)(rng_u64(r) >> 11) * (1.0 / 9007199254740992.0); }
static double rng_range(rng_t* r, double lo, double hi) { return lo + (hi - lo) * rng_uni(r); }
static double rng_normal(rng_t* r) {
    double u1 = rng_uni(r), u2 = rng_uni(r);
    if (u1 < 1e-300) u1 = 1e-300;
    return sqrt(-2.0 * log(u1)) * cos(2.0 * SG_PI * u2);
}

/* ---------------------------------------------------------------- small vector helpers */

static void v_cross(const double* a, const double* b, double* o) {
    o[0] = a[1] * b[2] - a[2] * b[1];
    o[1] = a[2] * b[0] - a[0] * b[2];
    o[2] = a[0] * b[1] - a[1] * b[0];
}
static double v_dot(const double* a, const double* b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }
static void v_norm(double* a) {
    double n = sqrt(v_dot(a, a));
    if (n > 0) { a[0] /= n; a[1] /= n; a[2] /= n; }
}

/* float -> IEEE half, round to nearest even (bit manipulation). */
static uint16_t f32_to_f16(float f) {
    uint32_t x; memcpy(&x, &f, 4);
    uint32_t sign = (x >> 16) & 0x8000u;
    uint32_t ax = x & 0x7FFFFFFFu;
    if (ax >= 0x7F800000u) return (uint16_t)(sign | 0x7C00u | (ax > 0x7F800000u ? 0x200u : 0));
    if (ax >= 0x477FF000u) return (uint16_t)(sign | 0x7C00u); /* overflow -> inf */
    if (ax < 0x38800000u) {  /* subnormal half or zero */
        if (ax < 0x33000000u) return (uint16_t)sign;
        /* value = m * 2^(e-150); in units of the half subnormal step 2^-24 that is m >> (126-e) */
        uint32_t e = ax >> 23, m = (ax & 0x7FFFFFu) | 0x800000u;
        uint32_t sh = 126 - e; /* 14..24 */
        uint32_t mant = m >> sh;
        uint32_t rem = m & ((1u << sh) - 1);
        uint32_t half = 1u << (sh - 1);
        if (rem > half || (rem == half && (mant & 1))) mant++;
        return (uint16_t)(sign | mant);
    }
    uint32_t e = (ax >> 23) - 112, m = ax & 0x7FFFFFu;
    uint32_t out = (e << 10) | (m >> 13);
    uint32_t rem = m & 0x1FFFu;
    if (rem > 0x1000u || (rem == 0x1000u && (out & 1))) out++;
    return (uint16_t)(sign | out);
}

/* ---------------------------------------------------------------- strands */

/* Polyline vertices of strand s, (n_segments+1) x 3, in double. */
static void make_strand(const sg_config* c, int s, double* verts) {
    rng_t r = rng_make(c->seed, 1, (uint64_t)s);
    double cos_cap = cos(c->cap_deg * SG_PI / 180.0);
    double cy = rng_range(&r, cos_cap, 1.0);           /* cos(polar), uniform area on the cap */
    double az = rng_range(&r, 0.0, 2.0 * SG_PI);
    double sy = sqrt(fmax(0.0, 1.0 - cy * cy));
    double n[3] = {sy * cos(az), cy, sy * sin(az)};    /* root on unit sphere, outward normal */
    double a[3] = {1, 0, 0};
    if (fabs(n[0]) > 0.9) { a[0] = 0; a[2] = 1; }
    double e1[3], e2[3], d = v_dot(a, n);
    e1[0] = a[0] - d * n[0]; e1[1] = a[1] - d * n[1]; e1[2] = a[2] - d * n[2];
    v_norm(e1);
    v_cross(n, e1, e2);
    double L = rng_range(&r, c->len_lo, c->len_hi);
    int type = 2; /* 0 straight, 1 wavy, 2 helix */
    if (c->strand_mix == 1) type = s % 3;
    double phase = rng_range(&r, 0.0, 2.0 * SG_PI);
    int ns = c->n_segments;
    if (type == 2) {
        double R = rng_range(&r, c->helix_r_lo, c->helix_r_hi);
        double pitch = rng_range(&r, c->pitch_lo, c->pitch_hi);
        double adv = pitch / (2.0 * SG_PI);            /* axial advance per radian */
        double speed = sqrt(adv * adv + R * R);        /* arc length per radian */
        double smax = L / speed;
        for (int i = 0; i <= ns; i++) {
            double t = smax * (double)i / ns;
            double cc = cos(t + phase) - cos(phase), ss = sin(t + phase) - sin(phase);
            for (int q = 0; q < 3; q++)
                verts[3 * i + q] = n[q] + adv * t * n[q] + R * (cc * e1[q] + ss * e2[q]);
        }
    } else if (type == 1) {
        double A = rng_range(&r, c->wave_a_lo, c->wave_a_hi);
        double lam = rng_range(&r, c->wave_len_lo, c->wave_len_hi);
        /* arc length of u -> (u, A sin(2 pi u / lam + phase)) by fine trapezoid stepping */
        const int fine = 64 * ns;
        double umax = L, len = 0.0, du = 2.0 * L / fine, u = 0.0;
        for (int i = 0; i < 4 * fine && len < L; i++) {
            double g0 = 2 * SG_PI * A / lam * cos(2 * SG_PI * u / lam + phase);
            double g1 = 2 * SG_PI * A / lam * cos(2 * SG_PI * (u + du) / lam + phase);
            double dl = 0.5 * du * (sqrt(1 + g0 * g0) + sqrt(1 + g1 * g1));
            if (len + dl >= L) { umax = u + du * (L - len) / dl; len = L; break; }
            len += dl; u += du; umax = u;
        }
        for (int i = 0; i <= ns; i++) {
            double uu = umax * (double)i / ns;
            double w = A * (sin(2 * SG_PI * uu / lam + phase) - sin(phase));
            for (int q = 0; q < 3; q++) verts[3 * i + q] = n[q] + uu * n[q] + w * e1[q];
        }
    } else {
        for (int i = 0; i <= ns; i++) {
            double uu = L * (double)i / ns;
            for (int q = 0; q < 3; q++) verts[3 * i + q] = n[q] + uu * n[q];
        }
    }
}

long long sg_num_points(const sg_config* c) {
    if (c->points_mode == 0) return (long long)c->n_strands * c->pts_per_strand;
    return (long long)c->n_strands * c->n_segments;
}

/* Points (f32) on the polylines, their unit tangents (segment directions, f32), strand ids,
 * and the polyline vertices themselves (f32, n_strands x (n_segments+1) x 3). */
int sg_make_points(const sg_config* c, float* pts, float* tan, int32_t* sid, float* verts_out) {
    int ns = c->n_segments;
#pragma omp parallel
    {
        double* v = (double*)malloc(sizeof(double) * 3 * (ns + 1));
        double* cum = (double*)malloc(sizeof(double) * (ns + 1));
#pragma omp for schedule(static)
        for (int s = 0; s < c->n_strands; s++) {
            make_strand(c, s, v);
            if (verts_out)
                for (int i = 0; i < 3 * (ns + 1); i++) verts_out[(size_t)s * 3 * (ns + 1) + i] = (float)v[i];
            cum[0] = 0;
            for (int i = 0; i < ns; i++) {
                double d[3] = {v[3 * i + 3] - v[3 * i], v[3 * i + 4] - v[3 * i + 1], v[3 * i + 5] - v[3 * i + 2]};
                cum[i + 1] = cum[i] + sqrt(v_dot(d, d));
            }
            int np = c->points_mode == 0 ? c->pts_per_strand : ns;
            for (int j = 0; j < np; j++) {
                int seg;
                double t;
                if (c->points_mode == 0) {
                    double target = cum[ns] * (j + 0.5) / np;
                    seg = 0;
                    while (seg < ns - 1 && cum[seg + 1] < target) seg++;
                    double sl = cum[seg + 1] - cum[seg];
                    t = sl > 0 ? (target - cum[seg]) / sl : 0.5;
                } else {
                    seg = j;
                    t = 0.5;
                }
                double d[3], p[3];
                for (int q = 0; q < 3; q++) {
                    d[q] = v[3 * seg + 3 + q] - v[3 * seg + q];
                    p[q] = v[3 * seg + q] + t * d[q];
                }
                v_norm(d);
                size_t o = (size_t)s * np + j;
                for (int q = 0; q < 3; q++) { pts[3 * o + q] = (float)p[q]; tan[3 * o + q] = (float)d[q]; }
                if (sid) sid[o] = s;
            }
        }
        free(v);
        free(cum);
    }
    return 0;
}

/* ---------------------------------------------------------------- cameras
 * Camera record (16 floats): fx, fy, cx, cy, R (3x3 row-major, world->camera), t (3).
 * Camera frame: x right, y down, z forward (looking at the origin), world up = +y. */

static void look_at(const double* C, double* R, double* t) {
    double f[3] = {-C[0], -C[1], -C[2]};
    v_norm(f);
    double up[3] = {0, 1, 0}, right[3], down[3];
    v_cross(f, up, right);
    v_norm(right);
    v_cross(f, right, down);
    v_norm(down);
    for (int q = 0; q < 3; q++) { R[q] = right[q]; R[3 + q] = down[q]; R[6 + q] = f[q]; }
    for (int r = 0; r < 3; r++) t[r] = -(R[3 * r] * C[0] + R[3 * r + 1] * C[1] + R[3 * r + 2] * C[2]);
}

/* Rodrigues rotation matrix for unit axis a and angle th. */
static void axis_angle(const double* a, double th, double* M) {
    double c = cos(th), s = sin(th), C = 1 - c;
    M[0] = c + a[0] * a[0] * C;        M[1] = a[0] * a[1] * C - a[2] * s; M[2] = a[0] * a[2] * C + a[1] * s;
    M[3] = a[1] * a[0] * C + a[2] * s; M[4] = c + a[1] * a[1] * C;        M[5] = a[1] * a[2] * C - a[0] * s;
    M[6] = a[2] * a[0] * C - a[1] * s; M[7] = a[2] * a[1] * C + a[0] * s; M[8] = c + a[2] * a[2] * C;
}

int sg_make_cameras(const sg_config* c, float* cams_clean, float* cams_noisy) {
    for (int v = 0; v < c->V; v++) {
        rng_t r = rng_make(c->seed, 2, (uint64_t)v);
        double az, el = 0.0;
        if (c->cam_mode == 0) {
            az = 2.0 * SG_PI * v / c->V;
        } else if (c->cam_mode == 1) {
            az = c->V > 1 ? (-0.5 * SG_PI + SG_PI * v / (c->V - 1)) : 0.0;
            el = rng_range(&r, -c->elev_jitter_deg, c->elev_jitter_deg) * SG_PI / 180.0;
        } else {
            az = 2.0 * SG_PI * v / c->V;
            el = rng_range(&r, -c->elev_jitter_deg, c->elev_jitter_deg) * SG_PI / 180.0;
        }
        double C[3] = {c->cam_radius * cos(el) * sin(az), c->cam_radius * sin(el), c->cam_radius * cos(el) * cos(az)};
        double R[9], t[3];
        look_at(C, R, t);
        float* o = cams_clean + 16 * v;
        o[0] = (float)c->f; o[1] = (float)c->f; o[2] = (float)c->cx; o[3] = (float)c->cy;
        for (int q = 0; q < 9; q++) o[4 + q] = (float)R[q];
        for (int q = 0; q < 3; q++) o[13 + q] = (float)t[q];
        /* noisy pose: rotate the camera about a random axis through its centre */
        double Rn[9], tn[3];
        if (c->pose_noise_deg > 0) {
            double ax[3] = {rng_normal(&r), rng_normal(&r), rng_normal(&r)};
            v_norm(ax);
            double th = rng_normal(&r) * c->pose_noise_deg * SG_PI / 180.0, M[9];
            axis_angle(ax, th, M);
            for (int i = 0; i < 3; i++)
                for (int j = 0; j < 3; j++)
                    Rn[3 * i + j] = M[3 * i] * R[j] + M[3 * i + 1] * R[3 + j] + M[3 * i + 2] * R[6 + j];
            for (int i = 0; i < 3; i++) tn[i] = -(Rn[3 * i] * C[0] + Rn[3 * i + 1] * C[1] + Rn[3 * i + 2] * C[2]);
        } else {
            memcpy(Rn, R, sizeof R);
            memcpy(tn, t, sizeof t);
        }
        o = cams_noisy + 16 * v;
        o[0] = (float)c->f; o[1] = (float)c->f; o[2] = (float)c->cx; o[3] = (float)c->cy;
        for (int q = 0; q < 9; q++) o[4 + q] = (float)Rn[q];
        for (int q = 0; q < 3; q++) o[13 + q] = (float)tn[q];
    }
    return 0;
}

/* ---------------------------------------------------------------- map rendering */

static void cam_apply(const float* cam, const double* p, double* X) {
    for (int r = 0; r < 3; r++)
        X[r] = (double)cam[4 + 3 * r] * p[0] + (double)cam[5 + 3 * r] * p[1] + (double)cam[6 + 3 * r] * p[2] + (double)cam[13 + r];
}

/* Strand maps: 1-px-wide DDA rasterisation of every polyline segment, z-buffered, in each view.
 * angle = projected segment direction mod pi plus N(0, angle_noise) noise; conf ~ U[conf_lo, conf_hi]
 * on covered pixels, 0 elsewhere; then a fraction of pixels is replaced by outliers.
 * verts: n_strands x (n_segments+1) x 3 (f32), cams: the CLEAN cameras. */
int sg_render_strand_maps(const sg_config* c, const float* verts, const float* cams,
                          float* angle, void* conf, int conf_f16, float* depth) {
    const int W = c->width, H = c->height, ns = c->n_segments;
    const size_t npx = (size_t)W * H;
#pragma omp parallel
    {
        float* zb = (float*)malloc(sizeof(float) * npx);
        float* cf = (float*)malloc(sizeof(float) * npx);
#pragma omp for schedule(dynamic, 1)
        for (int v = 0; v < c->V; v++) {
            const float* cam = cams + 16 * v;
            float* ang = angle + npx * v;
            for (size_t i = 0; i < npx; i++) { zb[i] = INFINITY; ang[i] = 0.0f; cf[i] = 0.0f; }
            rng_t r = rng_make(c->seed, 3, (uint64_t)v);
            for (int s = 0; s < c->n_strands; s++) {
                const float* sv = verts + (size_t)s * 3 * (ns + 1);
                for (int i = 0; i < ns; i++) {
                    double pa[3] = {sv[3 * i], sv[3 * i + 1], sv[3 * i + 2]};
                    double pb[3] = {sv[3 * i + 3], sv[3 * i + 4], sv[3 * i + 5]};
                    double Xa[3], Xb[3];
                    cam_apply(cam, pa, Xa);
                    cam_apply(cam, pb, Xb);
                    if (Xa[2] < 1e-2 || Xb[2] < 1e-2) continue;
                    double ua = cam[0] * Xa[0] / Xa[2] + cam[2], va = cam[1] * Xa[1] / Xa[2] + cam[3];
                    double ub = cam[0] * Xb[0] / Xb[2] + cam[2], vb = cam[1] * Xb[1] / Xb[2] + cam[3];
                    double du = ub - ua, dv = vb - va;
                    double th = atan2(dv, du);
                    if (th < 0) th += SG_PI;
                    if (th >= SG_PI) th -= SG_PI;
                    int steps = (int)ceil(fmax(fabs(du), fabs(dv))) + 1;
                    if (steps > 4 * (W + H)) continue; /* degenerate, near the camera plane */
                    for (int q = 0; q <= steps; q++) {
                        double tq = (double)q / steps;
                        double u = ua + tq * du, vv = va + tq * dv;
                        if (!(u >= 0 && u < W && vv >= 0 && vv < H)) continue;
                        int x = (int)floor(u), y = (int)floor(vv);
                        double z = Xa[2] + tq * (Xb[2] - Xa[2]);
                        size_t o = (size_t)y * W + x;
                        if (z < zb[o]) {
                            zb[o] = (float)z;
                            double a = th + rng_normal(&r) * c->angle_noise_deg * SG_PI / 180.0;
                            a = fmod(a, SG_PI);
                            if (a < 0) a += SG_PI;
                            float af = (float)a;
                            if (af >= (float)SG_PI) af = 0.0f;
                            ang[o] = af;
                            cf[o] = (float)rng_range(&r, c->conf_lo, c->conf_hi);
                        }
                    }
                }
            }
            if (c->outlier_frac > 0) {
                for (size_t i = 0; i < npx; i++) {
                    if (rng_uni(&r) < c->outlier_frac) {
                        float af = (float)rng_range(&r, 0.0, SG_PI);
                        if (af >= (float)SG_PI) af = 0.0f;
                        ang[i] = af;
                        cf[i] = (float)rng_range(&r, 0.0, c->outlier_conf_hi);
                    }
                }
            }
            if (conf_f16) {
                uint16_t* o = (uint16_t*)conf + npx * v;
                for (size_t i = 0; i < npx; i++) o[i] = f32_to_f16(cf[i]);
            } else {
                memcpy((float*)conf + npx * v, cf, sizeof(float) * npx);
            }
            /* the z-buffer: camera-space depth of the front-most strand, +inf where none */
            if (depth) memcpy(depth + npx * v, zb, sizeof(float) * npx);
        }
        free(zb);
        free(cf);
    }
    return 0;
}

/* "Exact" maps: every point is splatted into the pixel it projects to (z-buffered by depth),
 * writing the direction angle of its projected true tangent with confidence 1; every other
 * pixel has confidence 0.  Used to check that the true tangent is a zero-cost direction.
 * The projection is evaluated in double from the f32 point and camera values.
 * owner (optional, V x N int32): 1 where the point won its pixel in that view. */
int sg_render_exact_maps(const sg_config* c, long long N, const float* pts, const float* tan,
                         const float* cams, float* angle, float* conf, int32_t* owner) {
    const int W = c->width, H = c->height;
    const size_t npx = (size_t)W * H;
#pragma omp parallel
    {
        double* zb = (double*)malloc(sizeof(double) * npx);
        int32_t* who = (int32_t*)malloc(sizeof(int32_t) * npx);
#pragma omp for schedule(dynamic, 1)
        for (int v = 0; v < c->V; v++) {
            const float* cam = cams + 16 * v;
            float* ang = angle + npx * v;
            float* cf = conf + npx * v;
            for (size_t i = 0; i < npx; i++) { zb[i] = INFINITY; who[i] = -1; ang[i] = 0; cf[i] = 0; }
            for (long long i = 0; i < N; i++) {
                double p[3] = {pts[3 * i], pts[3 * i + 1], pts[3 * i + 2]}, X[3];
                cam_apply(cam, p, X);
                if (!(X[2] > 1e-6)) continue;
                double u = (double)cam[0] * (X[0] / X[2]) + (double)cam[2];
                double vv = (double)cam[1] * (X[1] / X[2]) + (double)cam[3];
                if (!(u >= 0 && u < W && vv >= 0 && vv < H)) continue;
                size_t o = (size_t)floor(vv) * W + (size_t)floor(u);
                if (X[2] < zb[o]) {
                    zb[o] = X[2];
                    who[o] = (int32_t)i;
                    /* image-plane direction of the tangent: derivative of the projection */
                    double d[3] = {tan[3 * i], tan[3 * i + 1], tan[3 * i + 2]}, q[3];
                    for (int r = 0; r < 3; r++) q[r] = cam[4 + 3 * r] * d[0] + cam[5 + 3 * r] * d[1] + cam[6 + 3 * r] * d[2];
                    double a = X[0] / X[2], b = X[1] / X[2];
                    double rx = cam[0] * (q[0] - a * q[2]), ry = cam[1] * (q[1] - b * q[2]);
                    double th = atan2(ry, rx);
                    if (th < 0) th += SG_PI;
                    float af = (float)th;
                    if (af >= (float)SG_PI) af = 0.0f;
                    ang[o] = af;
                    cf[o] = 1.0f;
                }
            }
            if (owner) {
                int32_t* ow = owner + (size_t)v * N;
                for (long long i = 0; i < N; i++) ow[i] = 0;
                for (size_t o = 0; o < npx; o++)
                    if (who[o] >= 0) ow[who[o]] = 1;
            }
        }
        free(zb);
        free(who);
    }
    return 0;
}

/* ---------------------------------------------------------------- k nearest neighbours
 * k nearest OTHER points by Euclidean distance (double from the f32 coordinates),
 * ties broken by the lower index; rows sorted nearest first.  Uniform-grid search. */

typedef struct { double d2; int32_t idx; } cand_t;

static int cand_less(const cand_t* a, const cand_t* b) {
    return a->d2 < b->d2 || (a->d2 == b->d2 && a->idx < b->idx);
}

int sg_knn(long long N, const float* pts, int k, int32_t* nbr) {
    if (k <= 0) return 0;
    if (k >= N) return -1;
    double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (long long i = 0; i < N; i++)
        for (int q = 0; q < 3; q++) {
            lo[q] = fmin(lo[q], pts[3 * i + q]);
            hi[q] = fmax(hi[q], pts[3 * i + q]);
        }
    double ext = fmax(fmax(hi[0] - lo[0], hi[1] - lo[1]), hi[2] - lo[2]);
    if (!(ext > 0)) ext = 1.0;
    double vol = fmax((hi[0] - lo[0]) * (hi[1] - lo[1]) * (hi[2] - lo[2]), 1e-12);
    double h = cbrt(vol * (double)(2 * k + 2) / (double)N);  /* ~ (2k+2) points per occupied cell */
    if (!(h > 0) || h > ext) h = ext;
    int g[3];
    for (int q = 0; q < 3; q++) {
        double n = floor((hi[q] - lo[q]) / h) + 1;
        if (n > 1024) n = 1024;
        g[q] = (int)n;
    }
    double hq[3];
    for (int q = 0; q < 3; q++) hq[q] = fmax((hi[q] - lo[q]) / g[q], 1e-30) * (1.0 + 1e-9);
    double hmin = fmin(fmin(hq[0], hq[1]), hq[2]);
    size_t ncell = (size_t)g[0] * g[1] * g[2];
    int32_t* cell_of = (int32_t*)malloc(sizeof(int32_t) * N);
    int64_t* start = (int64_t*)calloc(ncell + 1, sizeof(int64_t));
    int32_t* order = (int32_t*)malloc(sizeof(int32_t) * N);
    for (long long i = 0; i < N; i++) {
        int ci[3];
        for (int q = 0; q < 3; q++) {
            int c = (int)floor((pts[3 * i + q] - lo[q]) / hq[q]);
            ci[q] = c < 0 ? 0 : (c >= g[q] ? g[q] - 1 : c);
        }
        cell_of[i] = (int32_t)(((size_t)ci[2] * g[1] + ci[1]) * g[0] + ci[0]);
        start[cell_of[i] + 1]++;
    }
    for (size_t c = 0; c < ncell; c++) start[c + 1] += start[c];
    {
        int64_t* fill = (int64_t*)malloc(sizeof(int64_t) * ncell);
        memcpy(fill, start, sizeof(int64_t) * ncell);
        for (long long i = 0; i < N; i++) order[fill[cell_of[i]]++] = (int32_t)i;  /* ascending index per cell */
        free(fill);
    }
    int maxr = g[0] > g[1] ? g[0] : g[1];
    if (g[2] > maxr) maxr = g[2];
#pragma omp parallel
    {
        cand_t* best = (cand_t*)malloc(sizeof(cand_t) * (k + 1));
#pragma omp for schedule(dynamic, 1024)
        for (long long i = 0; i < N; i++) {
            int nb = 0;
            int cx = (int)(cell_of[i] % g[0]), cyy = (int)((cell_of[i] / g[0]) % g[1]), cz = (int)(cell_of[i] / ((size_t)g[0] * g[1]));
            double p[3] = {pts[3 * i], pts[3 * i + 1], pts[3 * i + 2]};
            for (int r = 0; r <= maxr; r++) {
                for (int z = cz - r; z <= cz + r; z++) {
                    if (z < 0 || z >= g[2]) continue;
                    for (int y = cyy - r; y <= cyy + r; y++) {
                        if (y < 0 || y >= g[1]) continue;
                        for (int x = cx - r; x <= cx + r; x++) {
                            if (x < 0 || x >= g[0]) continue;
                            if (abs(x - cx) != r && abs(y - cyy) != r && abs(z - cz) != r) continue;
                            size_t c = ((size_t)z * g[1] + y) * g[0] + x;
                            for (int64_t e = start[c]; e < start[c + 1]; e++) {
                                int32_t j = order[e];
                                if (j == i) continue;
                                double dx = pts[3 * j] - p[0], dy = pts[3 * j + 1] - p[1], dz = pts[3 * j + 2] - p[2];
                                cand_t cd = {dx * dx + dy * dy + dz * dz, j};
                                if (nb == k && !cand_less(&cd, &best[k - 1])) continue;
                                int pos = nb < k ? nb : k - 1;
                                while (pos > 0 && cand_less(&cd, &best[pos - 1])) { best[pos] = best[pos - 1]; pos--; }
                                best[pos] = cd;
                                if (nb < k) nb++;
                            }
                        }
                    }
                }
                /* every point in ring r+1 or beyond is at least r*hmin away */
                if (nb == k && best[k - 1].d2 <= (r * hmin) * (r * hmin)) break;
            }
            for (int q = 0; q < k; q++) nbr[(size_t)i * k + q] = best[q].idx;
        }
        free(best);
    }
    free(cell_of);
    free(start);
    free(order);
    return 0;
}
