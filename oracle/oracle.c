/*
 * oracle.c - plain FP64 CPU oracle for the multi-view direction-fusion step.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may call, link or load this file:
 * only the tests, the smoke check and the benchmark's CPU-baseline leg use it.  It shares no
 * code, header, table or constant with the CUDA library.
 *
 * What it computes, for a point p_i, a unit direction d and a set of calibrated views
 * (Sec. 3.1 "Patch-based Consistency Optimization", Eqs. proj_r, sim, patchloss, patch_min,
 * final_dout, applied to an explicit hypothesis set instead of depth-sampled candidates):
 *
 *   u_i^v = Pi_v(p_i)                                   pinhole projection (Sec. 3.1.1)
 *   r_v(d) = dPi_v/dp (p_i) . d                         Eq. proj_r in the limit of a short offset
 *   sim_j  = | < r_v / |r_v| , O_v(u_j^v) > |           Eq. sim, with O = (cos theta, sin theta)
 *   L_j    = sim_j * C_v(u_j^v)                         Eq. patchloss
 *   L_v    = max over the patch members j visible in v  Eq. patch_min (patch = point + k nbrs)
 *   c_i(d) = 1 - mean over the views V_i of L_v         view aggregation, arg-max of Eq. final_dout
 *
 * then the best of the H hypotheses (lowest cost, lowest index on ties) and T rounds of a
 * six-neighbour rotation pattern search with halving step.  All arithmetic is IEEE double,
 * evaluated straight from the definitions (atan2/cos for the angle, no doubled-angle algebra).
 *
 * Readings of the paper taken here (each is listed in the design notes):
 *  - the offset reprojection of Eq. proj_r is taken in its short-offset limit (the Jacobian),
 *  - r is normalised so that sim lies in [0, 1] (Eq. sim dots an unnormalised offset),
 *  - the patch is the point plus its k nearest other points, each sampled at its own pixel,
 *  - nearest-pixel sampling, pixel (floor u, floor v), pixel centres at +0.5,
 *  - visibility is the frustum/bounds test (no depth maps are given),
 *  - views are aggregated by an unweighted mean over the visible (or top-K) views,
 *  - the angle map stores theta in [0, pi) in pixel axes (+u right, +v down).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_PI 3.14159265358979323846

enum { OR_OK = 0, OR_NO_VIEWS = 1, OR_BAD_INPUT = 2 };
/* exemption flags reported per point (not part of the method; used by the parity tests) */
enum { OR_FLAG_IDX_TIE = 1, OR_FLAG_REFINE_TIE = 2, OR_FLAG_BOUNDARY = 4 };

typedef struct {
    long long N;
    int V, W, H, k;
    const double* pts;     /* N x 3 (the f32 inputs widened exactly) */
    const double* cams;    /* V x 16: fx, fy, cx, cy, R row-major (world->cam), t */
    const float* angle;    /* V x H x W, radians in [0, pi) */
    const void* conf;      /* V x H x W, f32 or IEEE half */
    int conf_f16;
    const int32_t* nbr;    /* N x k */
} or_scene;

/* IEEE binary16 -> double, from the bit fields. */
static double half_to_double(uint16_t h) {
    int s = (h >> 15) & 1, e = (h >> 10) & 31, m = h & 1023;
    double v;
    if (e == 0) v = ldexp((double)m, -24);
    else if (e == 31) v = m ? NAN : INFINITY;
    else v = ldexp(1.0 + m / 1024.0, e - 15);
    return s ? -v : v;
}

static double conf_at(const or_scene* s, int v, long long px) {
    size_t o = (size_t)v * s->W * s->H + (size_t)px;
    if (s->conf_f16) return half_to_double(((const uint16_t*)s->conf)[o]);
    return (double)((const float*)s->conf)[o];
}

/* Projection u = Pi_v(p) of a point into view v (Sec. 3.1.1).  Returns 1 when the point is in
 * front of the camera (X_z > 1e-6) and inside the image (0 <= u < W, 0 <= v < H); fills the
 * pixel coordinates and the ratios a = X_x/X_z, b = X_y/X_z. */
int or_project(const double* cam, const double* p, int W, int H, double* u, double* v, double* a, double* b) {
    double X[3];
    for (int r = 0; r < 3; r++)
        X[r] = cam[4 + 3 * r] * p[0] + cam[5 + 3 * r] * p[1] + cam[6 + 3 * r] * p[2] + cam[13 + r];
    if (!(X[2] > 1e-6)) return 0;
    *a = X[0] / X[2];
    *b = X[1] / X[2];
    *u = cam[0] * *a + cam[2];
    *v = cam[1] * *b + cam[3];
    return (*u >= 0.0 && *u < (double)W && *v >= 0.0 && *v < (double)H) ? 1 : 0;
}

/* Image-plane offset of direction d at point p: r = dPi/dp . d, i.e. Eq. proj_r for an
 * offset point p + eps d, divided by eps, eps -> 0.  With X = R p + t, q = R d:
 * r = (fx (q_x - a q_z) / X_z, fy (q_y - b q_z) / X_z), a = X_x/X_z, b = X_y/X_z.
 * Returns X_z (the depth). */
double or_reproject_dir(const double* cam, const double* p, const double* d, double* r) {
    double X[3], q[3];
    for (int i = 0; i < 3; i++) {
        X[i] = cam[4 + 3 * i] * p[0] + cam[5 + 3 * i] * p[1] + cam[6 + 3 * i] * p[2] + cam[13 + i];
        q[i] = cam[4 + 3 * i] * d[0] + cam[5 + 3 * i] * d[1] + cam[6 + 3 * i] * d[2];
    }
    double a = X[0] / X[2], b = X[1] / X[2];
    r[0] = cam[0] * (q[0] - a * q[2]) / X[2];
    r[1] = cam[1] * (q[1] - b * q[2]) / X[2];
    return X[2];
}

/* Patch term of one view, Eqs. sim, patchloss, patch_min: the largest confidence-weighted
 * bidirectional similarity between the reprojected direction and the orientation map over
 * the patch members visible in view v.  Returns 0 when no member is visible or |r| ~ 0. */
double or_view_term(const or_scene* s, long long i, int v, const double* d) {
    const double* cam = s->cams + 16 * v;
    double u, vv, a, b;
    if (!or_project(cam, s->pts + 3 * i, s->W, s->H, &u, &vv, &a, &b)) return 0.0;
    double r[2];
    double Z = or_reproject_dir(cam, s->pts + 3 * i, d, r);
    /* degenerate view: d (nearly) along the viewing ray, |r| below 1e-10 of the image
     * offset sqrt(fx^2 + fy^2) |d| / Z of a direction across the ray */
    double dn2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
    double rn2 = r[0] * r[0] + r[1] * r[1];
    double f2 = cam[0] * cam[0] + cam[1] * cam[1];
    if (!(rn2 * Z * Z >= 1e-20 * f2 * dn2)) return 0.0;
    double rn = sqrt(rn2);
    double best = 0.0;
    for (int m = -1; m < s->k; m++) {
        long long j = m < 0 ? i : (long long)s->nbr[i * s->k + m];
        double uj, vj, aj, bj;
        if (!or_project(cam, s->pts + 3 * j, s->W, s->H, &uj, &vj, &aj, &bj)) continue;
        long long px = (long long)floor(vj) * s->W + (long long)floor(uj);
        double th = (double)s->angle[(size_t)v * s->W * s->H + (size_t)px];
        double C = conf_at(s, v, px);
        double sim = fabs((r[0] / rn) * cos(th) + (r[1] / rn) * sin(th));
        double L = sim * C;
        if (L > best) best = L;
    }
    return best;
}

/* The point's view set V_i: views in which it is visible; with top_k > 0 only the top_k of
 * them by the confidence at the point's own pixel, ties to the lower view index (Sec. 3.1.2).
 * Writes a 0/1 mask of V entries and returns |V_i|. */
int or_view_set(const or_scene* s, long long i, int top_k, unsigned char* mask) {
    int n = 0;
    double* cv = (double*)malloc(sizeof(double) * s->V);
    for (int v = 0; v < s->V; v++) {
        double u, vv, a, b;
        mask[v] = (unsigned char)or_project(s->cams + 16 * v, s->pts + 3 * i, s->W, s->H, &u, &vv, &a, &b);
        cv[v] = mask[v] ? conf_at(s, v, (long long)floor(vv) * s->W + (long long)floor(u)) : -1.0;
        n += mask[v];
    }
    if (top_k > 0 && n > top_k) {
        unsigned char* keep = (unsigned char*)calloc(s->V, 1);
        for (int t = 0; t < top_k; t++) {
            int bestv = -1;
            for (int v = 0; v < s->V; v++)
                if (mask[v] && !keep[v] && (bestv < 0 || cv[v] > cv[bestv])) bestv = v;
            keep[bestv] = 1;
        }
        memcpy(mask, keep, s->V);
        free(keep);
        n = top_k;
    }
    free(cv);
    return n;
}

/* Cost c_i(d) = 1 - (1/|V_i|) sum_{v in V_i} L_v(d); 1 when V_i is empty. */
double or_cost_masked(const or_scene* s, long long i, const double* d, const unsigned char* mask) {
    double sum = 0.0;
    int n = 0;
    for (int v = 0; v < s->V; v++) {
        if (!mask[v]) continue;
        sum += or_view_term(s, i, v, d);
        n++;
    }
    return n ? 1.0 - sum / n : 1.0;
}

double or_cost(const or_scene* s, long long i, const double* d, int top_k) {
    unsigned char* mask = (unsigned char*)malloc(s->V);
    or_view_set(s, i, top_k, mask);
    double c = or_cost_masked(s, i, d, mask);
    free(mask);
    return c;
}

/* Costs of M given directions per listed point: dirs is n_idx x M x 3, out n_idx x M. */
int or_eval_costs(const or_scene* s, long long n_idx, const long long* idx, int M, const double* dirs,
                  int top_k, double* out, int n_threads) {
#ifdef _OPENMP
    if (n_threads > 0) omp_set_num_threads(n_threads);
#endif
#pragma omp parallel for schedule(dynamic, 16)
    for (long long q = 0; q < n_idx; q++) {
        unsigned char* mask = (unsigned char*)malloc(s->V);
        or_view_set(s, idx[q], top_k, mask);
        for (int m = 0; m < M; m++) {
            out[q * M + m] = or_cost_masked(s, idx[q], dirs + ((size_t)q * M + m) * 3, mask);
        }
        free(mask);
    }
    return 0;
}

/* Hypothesis set: H directions of a Fibonacci lattice on the upper hemisphere,
 * z_m = 1 - (m + 1/2)/H, azimuth m * pi * (3 - sqrt 5).  The cost is sign-invariant
 * (Eq. sim), so one hemisphere covers all directions. */
void or_fibonacci_hemisphere(int H, double* out) {
    double ga = OR_PI * (3.0 - sqrt(5.0));
    for (int m = 0; m < H; m++) {
        double z = 1.0 - (m + 0.5) / H;
        double rho = sqrt(fmax(0.0, 1.0 - z * z));
        out[3 * m] = rho * cos(m * ga);
        out[3 * m + 1] = rho * sin(m * ga);
        out[3 * m + 2] = z;
    }
}

/* Exemption thresholds for the parity tests (bookkeeping, not part of the method).
 * Hypothesis index: the two best costs within 1e-5 relative (plus a 1e-6 floor for costs near 0).
 * Refinement: two best of the seven costs of a round within 2e-6, about twice the worst-case
 * error of an FP32 evaluation of the cost, below which the order of two candidates is not fixed
 * by FP32 arithmetic. */
static int near_tie(double c1, double c2) {
    double m = fmax(fabs(c1), fabs(c2));
    return fabs(c1 - c2) <= 1e-5 * m + 1e-6;
}
static int near_tie_refine(double c1, double c2) { return fabs(c1 - c2) <= 2e-6; }

/* rotation of d about world axis ax (0 x, 1 y, 2 z) by angle th (right-handed) */
static void rotate_axis(int ax, double th, const double* d, double* o) {
    double c = cos(th), sn = sin(th);
    if (ax == 0) { o[0] = d[0]; o[1] = c * d[1] - sn * d[2]; o[2] = sn * d[1] + c * d[2]; }
    else if (ax == 1) { o[0] = c * d[0] + sn * d[2]; o[1] = d[1]; o[2] = -sn * d[0] + c * d[2]; }
    else { o[0] = c * d[0] - sn * d[1]; o[1] = sn * d[0] + c * d[1]; o[2] = d[2]; }
}

/* does any sample the point's cost could read (any view, any patch member) lie within
 * 1e-6 px of a pixel edge, where a last-bit difference in the projection may pick another pixel? */
static int boundary_ambiguous(const or_scene* s, long long i) {
    for (int v = 0; v < s->V; v++) {
        for (int m = -1; m < s->k; m++) {
            long long j = m < 0 ? i : (long long)s->nbr[i * s->k + m];
            double u, vv, a, b, X[3];
            const double* cam = s->cams + 16 * v;
            const double* p = s->pts + 3 * j;
            for (int r = 0; r < 3; r++)
                X[r] = cam[4 + 3 * r] * p[0] + cam[5 + 3 * r] * p[1] + cam[6 + 3 * r] * p[2] + cam[13 + r];
            if (fabs(X[2] - 1e-6) < 1e-12) return 1;
            if (!or_project(cam, p, s->W, s->H, &u, &vv, &a, &b)) {
                if (!(X[2] > 1e-6)) continue;
                u = cam[0] * (X[0] / X[2]) + cam[2];
                vv = cam[1] * (X[1] / X[2]) + cam[3];
            }
            if (fabs(u - floor(u + 0.5)) < 1e-6 || fabs(vv - floor(vv + 0.5)) < 1e-6) return 1;
        }
    }
    return 0;
}

/* T rounds of the refinement from direction d0 with cost c0: rotations by +alpha and -alpha about
 * world x, then y, then z, move to the first strictly lowest cost, halve alpha.  Writes the
 * normalised direction with canonical sign and its cost; records near-ties for the tests. */
static void refine_from(const or_scene* s, long long i, const unsigned char* mask, const double* d0, double c0, int T,
                        double alpha, double* dir, double* cost, uint8_t* flags, int8_t* tie_step) {
    double d[3] = {d0[0], d0[1], d0[2]}, bc = c0;
    for (int t = 0; t < T; t++) {
        double cs[7], cand[6][3];
        cs[0] = bc;
        int choice = -1;
        double best = bc;
        for (int c = 0; c < 6; c++) {
            rotate_axis(c / 2, (c % 2 == 0) ? alpha : -alpha, d, cand[c]);
            cs[c + 1] = or_cost_masked(s, i, cand[c], mask);
            if (cs[c + 1] < best) { best = cs[c + 1]; choice = c; }
        }
        /* exemption bookkeeping: the two lowest of the seven costs */
        double l1 = INFINITY, l2 = INFINITY;
        for (int c = 0; c < 7; c++) {
            if (cs[c] < l1) { l2 = l1; l1 = cs[c]; }
            else if (cs[c] < l2) l2 = cs[c];
        }
        if (near_tie_refine(l1, l2)) {
            *flags |= OR_FLAG_REFINE_TIE;
            if (*tie_step < 0) *tie_step = (int8_t)t;
        }
        if (choice >= 0) { d[0] = cand[choice][0]; d[1] = cand[choice][1]; d[2] = cand[choice][2]; bc = best; }
        alpha *= 0.5;
    }
    double n = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    for (int q = 0; q < 3; q++) d[q] /= n;
    double sg = 1.0;
    if (fabs(d[2]) > 1e-12) sg = d[2] < 0 ? -1.0 : 1.0;
    else if (fabs(d[1]) > 1e-12) sg = d[1] < 0 ? -1.0 : 1.0;
    else sg = d[0] < 0 ? -1.0 : 1.0;
    for (int q = 0; q < 3; q++) dir[q] = sg * d[q];
    *cost = bc;
}

/* Fusion of one point: best hypothesis, then T refinement rounds.
 * Refinement: step alpha_0 = sqrt(2 pi / H) / 2; each round tries d rotated by +alpha, -alpha
 * about world x, then y, then z (in that order), moves to the first strictly lowest cost,
 * then halves alpha.  The result is normalised and its sign made canonical: the first of
 * z, y, x with magnitude above 1e-12 is positive. */
void or_fuse_point(const or_scene* s, long long i, const double* hyps, int H, int T, int top_k,
                   double* dir, double* cost, int32_t* idx, uint8_t* status, uint8_t* flags, int8_t* tie_step) {
    const double* p = s->pts + 3 * i;
    *flags = 0;
    *tie_step = -1;
    if (!(isfinite(p[0]) && isfinite(p[1]) && isfinite(p[2]))) {
        dir[0] = dir[1] = dir[2] = 0.0;
        *cost = NAN;
        *idx = -1;
        *status = OR_BAD_INPUT;
        return;
    }
    unsigned char* mask = (unsigned char*)malloc(s->V);
    int nv = or_view_set(s, i, top_k, mask);
    *status = nv ? OR_OK : OR_NO_VIEWS;
    if (boundary_ambiguous(s, i)) *flags |= OR_FLAG_BOUNDARY;
    int bm = 0;
    double bc = INFINITY, second = INFINITY;
    for (int m = 0; m < H; m++) {
        double c = or_cost_masked(s, i, hyps + 3 * m, mask);
        if (c < bc) { second = bc; bc = c; bm = m; }
        else if (c < second) second = c;
    }
    if (H > 1 && near_tie(bc, second)) *flags |= OR_FLAG_IDX_TIE;
    *idx = bm;
    refine_from(s, i, mask, hyps + 3 * bm, bc, T, 0.5 * sqrt(2.0 * OR_PI / H), dir, cost, flags, tie_step);
    free(mask);
}

/* Learned path, from a given start direction (the proposal): its cost, then T rounds of the same
 * refinement with first step alpha0; same outputs as or_fuse_point except the index (-1). */
void or_refine_point(const or_scene* s, long long i, const double* d0, int T, double alpha0, int top_k, double* dir,
                     double* cost, uint8_t* status, uint8_t* flags, int8_t* tie_step) {
    const double* p = s->pts + 3 * i;
    *flags = 0;
    *tie_step = -1;
    if (!(isfinite(p[0]) && isfinite(p[1]) && isfinite(p[2]))) {
        dir[0] = dir[1] = dir[2] = 0.0;
        *cost = NAN;
        *status = OR_BAD_INPUT;
        return;
    }
    unsigned char* mask = (unsigned char*)malloc(s->V);
    int nv = or_view_set(s, i, top_k, mask);
    *status = nv ? OR_OK : OR_NO_VIEWS;
    if (boundary_ambiguous(s, i)) *flags |= OR_FLAG_BOUNDARY;
    refine_from(s, i, mask, d0, or_cost_masked(s, i, d0, mask), T, alpha0, dir, cost, flags, tie_step);
    free(mask);
}

int or_refine(const or_scene* s, long long n_idx, const long long* idx, const double* d0, int T, double alpha0,
              int top_k, double* dir, double* cost, uint8_t* status, uint8_t* flags, int8_t* tie_step, int n_threads) {
#ifdef _OPENMP
    if (n_threads > 0) omp_set_num_threads(n_threads);
#endif
#pragma omp parallel for schedule(dynamic, 16)
    for (long long q = 0; q < n_idx; q++) {
        long long i = idx ? idx[q] : q;
        or_refine_point(s, i, d0 + 3 * q, T, alpha0, top_k, dir + 3 * q, cost + q, status + q, flags + q, tie_step + q);
    }
    return 0;
}

/* Features of the proposal network for point i: for the 16 views v_m = floor(m V / 16),
 * (sin 2 theta, cos 2 theta, C) at the point's pixel, zeros when it projects outside; then the
 * position (p - centre) / half of the bounding box box = (lo[3], hi[3]), half = largest half side. */
void or_features(const or_scene* s, long long i, const double* box, double* f) {
    for (int q = 0; q < 64; q++) f[q] = 0.0;
    const double* p = s->pts + 3 * i;
    for (int m = 0; m < 16; m++) {
        int v = (m * s->V) / 16;
        double u, vv, a, b;
        if (!or_project(s->cams + 16 * v, p, s->W, s->H, &u, &vv, &a, &b)) continue;
        long long px = (long long)floor(vv) * s->W + (long long)floor(u);
        double th = (double)s->angle[(size_t)v * s->W * s->H + (size_t)px];
        f[3 * m] = sin(2.0 * th);
        f[3 * m + 1] = cos(2.0 * th);
        f[3 * m + 2] = conf_at(s, v, px);
    }
    double half = 0.5 * fmax(fmax(box[3] - box[0], box[4] - box[1]), box[5] - box[2]);
    if (!(half > 0.0)) half = 1.0;
    for (int q = 0; q < 3; q++) f[48 + q] = isfinite(p[q]) ? (p[q] - 0.5 * (box[q] + box[3 + q])) / half : 0.0;
}

int or_features_all(const or_scene* s, const double* box, double* out) {
#pragma omp parallel for schedule(static)
    for (long long i = 0; i < s->N; i++) or_features(s, i, box, out + 64 * i);
    return 0;
}

/* Fusion of the listed points (idx = NULL: all N); hyps H x 3. */
int or_fuse(const or_scene* s, long long n_idx, const long long* idx, const double* hyps, int H, int T,
            int top_k, double* dir, double* cost, int32_t* out_idx, uint8_t* status, uint8_t* flags,
            int8_t* tie_step, int n_threads) {
#ifdef _OPENMP
    if (n_threads > 0) omp_set_num_threads(n_threads);
#endif
#pragma omp parallel for schedule(dynamic, 16)
    for (long long q = 0; q < n_idx; q++) {
        long long i = idx ? idx[q] : q;
        or_fuse_point(s, i, hyps, H, T, top_k, dir + 3 * q, cost + q, out_idx + q, status + q, flags + q,
                      tie_step + q);
    }
    return 0;
}

/* Number of threads OpenMP will use for the parallel loops above. */
int or_max_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ==============================================================================================
 * FPMVO as the paper states it (Sec. 3.1.1-3.1.3): candidate directions from depth samples
 * around pixel-offset points, medoid fusion per depth layer over the top-K views, and the
 * patch-based consistency over a P x P pixel patch.  Readings (listed in the design notes):
 *  - depth maps hold the camera-space depth Z of the front-most hair, +inf where none; a view
 *    sees point i when it projects inside the image and X_z <= D_v(pixel) + eps_vis;
 *  - the offset pixel is u_i^v + lambda (cos theta, sin theta) with theta the map's angle at u_i^v
 *    (Eq. 1); its depth is read at its nearest pixel; S samples z + delta_s, delta_s spread evenly
 *    over [-Delta, Delta] including both ends (Eq. 2); back-projection through the continuous
 *    offset pixel (Eq. 3); a view whose offset pixel leaves the image or has no depth gives none;
 *  - candidate directions are unit vectors (the squared norm in Dir(p) read as the norm);
 *  - top-K views by the confidence at the point's pixel, ties to the lower view; the weight of a
 *    view's candidates is that confidence; the medoid sum includes the candidate itself; if the
 *    weights sum to 0 every candidate scores 0 and the first is taken;
 *  - Eq. proj_r with the finite fused offset point; r normalised; the patch is the P x P pixels
 *    centred on the point's pixel (pixels outside the image skipped); the per-view maxima are
 *    averaged over the top-K views; the highest average wins, lowest s on ties; the output
 *    direction is normalised with the canonical sign and its cost is 1 - that average.
 * ============================================================================================== */
typedef struct {
    int K, S, P;
    double lambda_px, delta, eps_vis;
} or_fpmvo_cfg;

enum { OR_FLAG_MEDOID_TIE = 8, OR_FLAG_SEL_TIE = 16, OR_FLAG_DEPTH_EDGE = 32 };

/* Inverse projection (Eq. 3): the world point at camera depth z on the ray through pixel (u, v),
 * p = R^-1 (X - t).  The inverse is the true 3 x 3 inverse (adjugate over determinant), not R^T:
 * a rotation stored in single precision is orthonormal only to ~1e-7, and R^T would move the
 * point off the ray by that much times |p|, which is not small beside a pixel-sized offset. */
void or_backproject(const double* cam, double u, double v, double z, double* p) {
    const double* R = cam + 4;
    const double X[3] = {(u - cam[2]) * z / cam[0], (v - cam[3]) * z / cam[1], z};
    const double Y[3] = {X[0] - cam[13], X[1] - cam[14], X[2] - cam[15]};
    const double a[9] = {R[4] * R[8] - R[5] * R[7], R[2] * R[7] - R[1] * R[8], R[1] * R[5] - R[2] * R[4],
                         R[5] * R[6] - R[3] * R[8], R[0] * R[8] - R[2] * R[6], R[2] * R[3] - R[0] * R[5],
                         R[3] * R[7] - R[4] * R[6], R[1] * R[6] - R[0] * R[7], R[0] * R[4] - R[1] * R[3]};
    const double det = R[0] * a[0] + R[1] * a[3] + R[2] * a[6];
    for (int c = 0; c < 3; c++) p[c] = (a[3 * c] * Y[0] + a[3 * c + 1] * Y[1] + a[3 * c + 2] * Y[2]) / det;
}

/* Medoid of n unit directions with weights w (Eq. G, sigma, argmax): index of the largest
 * sum_j w_j |<d_i, d_j>| / sum_j w_j, first on ties; *second receives the runner-up score. */
int or_medoid(int n, const double* d, const double* w, double* best_score, double* second) {
    double wsum = 0.0;
    for (int j = 0; j < n; j++) wsum += w[j];
    int bi = -1;
    double bs = -1.0, sc2 = -1.0;
    for (int i = 0; i < n; i++) {
        double acc = 0.0;
        for (int j = 0; j < n; j++)
            acc += w[j] * fabs(d[3 * i] * d[3 * j] + d[3 * i + 1] * d[3 * j + 1] + d[3 * i + 2] * d[3 * j + 2]);
        const double sig = wsum > 0.0 ? acc / wsum : 0.0;
        if (sig > bs) {
            sc2 = bs;
            bs = sig;
            bi = i;
        } else if (sig > sc2) {
            sc2 = sig;
        }
    }
    if (best_score) *best_score = bs;
    if (second) *second = sc2;
    return bi;
}

/* The output sign convention: positive z, else positive y, else non-negative x. */
static void canonical_sign(const double* d, double* out) {
    const double sg = fabs(d[2]) > 1e-12 ? (d[2] > 0 ? 1.0 : -1.0)
                      : fabs(d[1]) > 1e-12 ? (d[1] > 0 ? 1.0 : -1.0)
                                           : (d[0] >= 0 ? 1.0 : -1.0);
    for (int r = 0; r < 3; r++) out[r] = sg * d[r];
}

static double map_depth(const float* depth, const or_scene* s, int v, long long px) {
    return (double)depth[(size_t)v * s->W * s->H + (size_t)px];
}

/* One point.  layer_L (S values) and layer_dir (S x 3), when not NULL, receive every depth layer's
 * mean consistency (-1 where the layer has no candidate) and its fused direction with the canonical
 * sign, so that a caller can check a result taken among near-tied layers. */
void or_fpmvo_point(const or_scene* s, const float* depth, const or_fpmvo_cfg* c, long long i, double* dir,
                    double* cost, int32_t* sel, uint8_t* status, uint8_t* flags, double* layer_L, double* layer_dir) {
    const double* p = s->pts + 3 * i;
    if (layer_L)
        for (int k = 0; k < c->S; k++) {
            layer_L[k] = -1.0;
            layer_dir[3 * k] = layer_dir[3 * k + 1] = layer_dir[3 * k + 2] = 0.0;
        }
    *flags = 0;
    *sel = -1;
    *cost = 1.0;
    dir[0] = dir[1] = dir[2] = 0.0;
    if (!(isfinite(p[0]) && isfinite(p[1]) && isfinite(p[2]))) {
        *status = OR_BAD_INPUT;
        *cost = NAN;
        return;
    }
    const int V = s->V, K = c->K, S = c->S;
    /* visible views: bounds and depth test */
    int* vv_ = (int*)malloc(sizeof(int) * V);
    double* vc = (double*)malloc(sizeof(double) * V);
    double* vu = (double*)malloc(sizeof(double) * 2 * V);
    int nvis = 0;
    for (int v = 0; v < V; v++) {
        const double* cam = s->cams + 16 * v;
        double u, w, a, b;
        if (!or_project(cam, p, s->W, s->H, &u, &w, &a, &b)) continue;
        if (fabs(u - floor(u + 0.5)) < 1e-6 || fabs(w - floor(w + 0.5)) < 1e-6) *flags |= OR_FLAG_BOUNDARY;
        const double Z = cam[10] * p[0] + cam[11] * p[1] + cam[12] * p[2] + cam[15];
        const long long px = (long long)floor(w) * s->W + (long long)floor(u);
        const double D = map_depth(depth, s, v, px);
        if (fabs(Z - (D + c->eps_vis)) < 1e-5) *flags |= OR_FLAG_DEPTH_EDGE;
        if (!(Z <= D + c->eps_vis)) continue;
        vv_[nvis] = v;
        vc[nvis] = conf_at(s, v, px);
        vu[2 * nvis] = u;
        vu[2 * nvis + 1] = w;
        ++nvis;
    }
    /* top-K by confidence, ties to the lower view (selection keeps the view order on ties) */
    int tk[16], nk = 0;
    unsigned char* used = (unsigned char*)calloc(nvis > 0 ? nvis : 1, 1);
    for (; nk < K && nk < nvis; nk++) {
        int bj = -1;
        for (int j = 0; j < nvis; j++)
            if (!used[j] && (bj < 0 || vc[j] > vc[bj])) bj = j;
        used[bj] = 1;
        tk[nk] = bj;
    }
    free(used);
    if (nk == 0) {
        *status = OR_NO_VIEWS;
        free(vv_), free(vc), free(vu);
        return;
    }
    /* candidates: cand[j][s] offset points and unit directions */
    double* off = (double*)malloc(sizeof(double) * 3 * nk * S);
    double* dd = (double*)malloc(sizeof(double) * 3 * nk * S);
    unsigned char* ok = (unsigned char*)calloc(nk * S, 1);
    for (int j = 0; j < nk; j++) {
        const int q = tk[j], v = vv_[q];
        const double* cam = s->cams + 16 * v;
        const long long px = (long long)floor(vu[2 * q + 1]) * s->W + (long long)floor(vu[2 * q]);
        const double th = (double)s->angle[(size_t)v * s->W * s->H + (size_t)px];
        const double ux = vu[2 * q] + c->lambda_px * cos(th), uy = vu[2 * q + 1] + c->lambda_px * sin(th);
        if (fabs(ux - floor(ux + 0.5)) < 1e-5 || fabs(uy - floor(uy + 0.5)) < 1e-5) *flags |= OR_FLAG_BOUNDARY;
        if (!(ux >= 0.0 && ux < (double)s->W && uy >= 0.0 && uy < (double)s->H)) continue;
        const double z = map_depth(depth, s, v, (long long)floor(uy) * s->W + (long long)floor(ux));
        if (!isfinite(z)) continue;
        for (int k = 0; k < S; k++) {
            const double zs = z + (S > 1 ? -c->delta + 2.0 * c->delta * k / (S - 1) : 0.0);
            double* o = off + 3 * (j * S + k);
            or_backproject(cam, ux, uy, zs, o);
            const double e[3] = {o[0] - p[0], o[1] - p[1], o[2] - p[2]};
            const double n = sqrt(e[0] * e[0] + e[1] * e[1] + e[2] * e[2]);
            if (!(n > 1e-12)) continue;
            for (int r = 0; r < 3; r++) dd[3 * (j * S + k) + r] = e[r] / n;
            ok[j * S + k] = 1;
        }
    }
    /* per depth layer: medoid, then the patch consistency of its offset point */
    double best = -1.0, second = -1.0;
    int bs = -1;
    double bdir[3] = {0.0, 0.0, 0.0};
    const int h = c->P / 2;
    for (int k = 0; k < S; k++) {
        double cd[3 * 16], cw[16], co[3 * 16];
        int n = 0;
        for (int j = 0; j < nk; j++) {
            if (!ok[j * S + k]) continue;
            for (int r = 0; r < 3; r++) {
                cd[3 * n + r] = dd[3 * (j * S + k) + r];
                co[3 * n + r] = off[3 * (j * S + k) + r];
            }
            cw[n] = vc[tk[j]];
            ++n;
        }
        if (n == 0) continue;
        double m1, m2;
        const int mi = or_medoid(n, cd, cw, &m1, &m2);
        if (n > 1 && m1 - m2 < 1e-5) *flags |= OR_FLAG_MEDOID_TIE;
        const double* pf = co + 3 * mi;
        double Lsum = 0.0;
        for (int j = 0; j < nk; j++) {
            const int q = tk[j], v = vv_[q];
            const double* cam = s->cams + 16 * v;
            double uf, wf, a, b;
            or_project(cam, pf, s->W, s->H, &uf, &wf, &a, &b);
            const double Zf = cam[10] * pf[0] + cam[11] * pf[1] + cam[12] * pf[2] + cam[15];
            if (!(Zf > 1e-6)) continue;
            const double r[2] = {uf - vu[2 * q], wf - vu[2 * q + 1]};
            const double rn2 = r[0] * r[0] + r[1] * r[1];
            const double Z = cam[10] * p[0] + cam[11] * p[1] + cam[12] * p[2] + cam[15];
            const double e[3] = {pf[0] - p[0], pf[1] - p[1], pf[2] - p[2]};
            const double en2 = e[0] * e[0] + e[1] * e[1] + e[2] * e[2];
            if (!(rn2 * Z * Z >= 1e-20 * (cam[0] * cam[0] + cam[1] * cam[1]) * en2)) continue;
            const double rn = sqrt(rn2);
            const long long x0 = (long long)floor(vu[2 * q]), y0 = (long long)floor(vu[2 * q + 1]);
            double Lv = 0.0;
            for (int dy = -h; dy <= h; dy++)
                for (int dx = -h; dx <= h; dx++) {
                    const long long x = x0 + dx, y = y0 + dy;
                    if (x < 0 || y < 0 || x >= s->W || y >= s->H) continue;
                    const long long px = y * s->W + x;
                    const double th = (double)s->angle[(size_t)v * s->W * s->H + (size_t)px];
                    const double L = conf_at(s, v, px) * fabs((r[0] / rn) * cos(th) + (r[1] / rn) * sin(th));
                    if (L > Lv) Lv = L;
                }
            Lsum += Lv;
        }
        const double Lbar = Lsum / nk;
        if (layer_L) {
            const double e[3] = {pf[0] - p[0], pf[1] - p[1], pf[2] - p[2]};
            const double en = sqrt(e[0] * e[0] + e[1] * e[1] + e[2] * e[2]);
            const double u[3] = {e[0] / en, e[1] / en, e[2] / en};
            layer_L[k] = Lbar;
            canonical_sign(u, layer_dir + 3 * k);
        }
        if (Lbar > best) {
            second = best;
            best = Lbar;
            bs = k;
            const double e[3] = {pf[0] - p[0], pf[1] - p[1], pf[2] - p[2]};
            const double en = sqrt(e[0] * e[0] + e[1] * e[1] + e[2] * e[2]);
            for (int r = 0; r < 3; r++) bdir[r] = e[r] / en;
        } else if (Lbar > second) {
            second = Lbar;
        }
    }
    if (bs < 0) {
        *status = OR_NO_VIEWS;
    } else {
        if (second >= 0.0 && best - second < 2e-6) *flags |= OR_FLAG_SEL_TIE;
        canonical_sign(bdir, dir);
        *cost = 1.0 - best;
        *sel = bs;
        *status = OR_OK;
    }
    free(off), free(dd), free(ok);
    free(vv_), free(vc), free(vu);
}

int or_fpmvo(const or_scene* s, const float* depth, const or_fpmvo_cfg* c, long long n_idx, const long long* idx,
             double* dir, double* cost, int32_t* sel, uint8_t* status, uint8_t* flags, double* layer_L,
             double* layer_dir, int n_threads) {
    if (c->K < 1 || c->K > 16 || c->S < 1 || c->S > 16 || c->P < 1 || !(c->P & 1)) return -1;
#ifdef _OPENMP
    if (n_threads > 0) omp_set_num_threads(n_threads);
#endif
#pragma omp parallel for schedule(dynamic, 16)
    for (long long q = 0; q < n_idx; q++) {
        long long i = idx ? idx[q] : q;
        or_fpmvo_point(s, depth, c, i, dir + 3 * q, cost + q, sel + q, status + q, flags + q,
                       layer_L ? layer_L + (size_t)q * c->S : NULL, layer_L ? layer_dir + (size_t)3 * q * c->S : NULL);
    }
    return 0;
}
