/*
 * phg.c - CPU oracle of the paper's Parallel Hair Growing consumer (Sec. 3.2): the volumetric
 * occupancy / orientation representation, guide strands traced from scalp seeds in batches with
 * deferred occupancy, segments grown from the occupied voxels no strand reached, and the linking of
 * segments by Eq. segment_connection.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may call, link or load this file: only
 * the tests, the smoke check and the benchmark's CPU-baseline leg use it.  It shares no code,
 * header, table or constant with the CUDA library.
 *
 * Precision.  Tracing turns positions into voxel indices (floor), so an FP64 trace would leave the
 * FP32 one at the first voxel boundary it meets within rounding.  Every quantity that feeds such a
 * decision is therefore computed here in IEEE single precision with one rounding per written
 * operation (fmaf where a fused multiply-add is written, the file compiled without contraction),
 * the same sequence the CUDA path takes; integer results (counts, fixed-point sums, indices,
 * labels) are exact.  What is computed, step by step (readings in the design notes):
 *
 *  A  splat: voxel c(p) = floor((p - o) / h) per axis; occ[c] += 1 and, in fixed point,
 *     T[c] += rint(2^30 fl(d_a d_b)) for the six entries of d d^T;
 *  B  orientation: the dominant eigenvector of T[c] by 12 rounds of power iteration from the
 *     column with the largest diagonal entry, sign made canonical (z > 0, else y > 0, else x > 0);
 *  C  guide strands: seed h with normal n, direction d = n; per step: stop outside the grid; in an
 *     empty voxel walk on along d while no occupied voxel was met and fewer than root_steps steps
 *     were taken, else stop; stop where earlier batches left occ_cap strands; o = ori[c] turned to
 *     <o, d> >= 0; stop when <o, d> < cos_turn; d = o; p = p + step d; at most max_steps steps;
 *     after each batch of seeds, every voxel a strand of the batch entered counts one more strand;
 *  D  segments: every occupied voxel no strand has entered seeds one at its centre, in voxel order
 *     and in batches (a seed whose voxel earlier batches entered is skipped); it is traced along
 *     +ori and along -ori with the rules of C (no empty-voxel walk), and counts like C;
 *  E  linking (Eq. segment_connection): every strand end (the tip of a guide strand, both ends of
 *     a segment; outward tangent t = the last step's direction) takes the nearest end q of another
 *     segment with |p - p_q| < delta_d and <t, -t_q> > cos(delta_theta) (squared distances,
 *     ties to the lower end); the strands so joined form the connected components, each labelled
 *     by its lowest strand index (guide strands first, then segments).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
    float origin[3];
    float voxel;
    int nx, ny, nz;
    float step;
    int max_steps, root_steps;
    float cos_turn;
    int occ_cap, batch;
    float link_dist, link_cos;
} or_phg_cfg;

enum { OR_PHG_MAXLEN = 1, OR_PHG_OUTSIDE = 2, OR_PHG_EMPTY = 3, OR_PHG_CROWDED = 4, OR_PHG_TURN = 5,
       OR_PHG_NO_ROOT = 6 };

/* Voxel of p: index >= 0, or -1 outside the grid. */
long long or_phg_voxel(const or_phg_cfg* g, const float* p) {
    int c[3];
    const int n[3] = {g->nx, g->ny, g->nz};
    for (int a = 0; a < 3; a++) {
        const float q = (p[a] - g->origin[a]) / g->voxel;
        if (!(q >= 0.0f && q < (float)n[a])) return -1;
        c[a] = (int)floorf(q);
    }
    return ((long long)c[2] * g->ny + c[1]) * g->nx + c[0];
}

/* A: occupancy counts and fixed-point structure tensors (xx, xy, xz, yy, yz, zz). */
void or_phg_splat(const or_phg_cfg* g, long long n, const float* pts, const float* dirs, const uint8_t* valid,
                  int32_t* occ, int64_t* T) {
    const long long nv = (long long)g->nx * g->ny * g->nz;
    memset(occ, 0, sizeof(int32_t) * nv);
    memset(T, 0, sizeof(int64_t) * 6 * nv);
    for (long long i = 0; i < n; i++) {
        if (valid && !valid[i]) continue;
        const float* p = pts + 3 * i;
        const float* d = dirs + 3 * i;
        if (!(isfinite(p[0]) && isfinite(p[1]) && isfinite(p[2]) && isfinite(d[0]) && isfinite(d[1]) &&
              isfinite(d[2])))
            continue;
        const long long c = or_phg_voxel(g, p);
        if (c < 0) continue;
        occ[c] += 1;
        const int ia[6] = {0, 0, 0, 1, 1, 2}, ib[6] = {0, 1, 2, 1, 2, 2};
        for (int e = 0; e < 6; e++) {
            const float prod = d[ia[e]] * d[ib[e]];
            T[6 * c + e] += (int64_t)rintf(prod * 1073741824.0f);
        }
    }
}

/* B: the voxel's orientation (0 for an empty voxel). */
void or_phg_orient_one(const int64_t* t6, int32_t count, float* out) {
    out[0] = out[1] = out[2] = 0.0f;
    if (count <= 0) return;
    const float m[3][3] = {{(float)t6[0], (float)t6[1], (float)t6[2]},
                           {(float)t6[1], (float)t6[3], (float)t6[4]},
                           {(float)t6[2], (float)t6[4], (float)t6[5]}};
    int a = 0;
    if (m[1][1] > m[a][a]) a = 1;
    if (m[2][2] > m[a][a]) a = 2;
    float x[3] = {m[0][a], m[1][a], m[2][a]};
    float nn = sqrtf(fmaf(x[0], x[0], fmaf(x[1], x[1], x[2] * x[2])));
    if (!(nn > 0.0f)) return;
    float r = 1.0f / nn;
    for (int q = 0; q < 3; q++) x[q] = x[q] * r;
    for (int it = 0; it < 12; it++) {
        float y[3];
        for (int q = 0; q < 3; q++) y[q] = fmaf(m[q][0], x[0], fmaf(m[q][1], x[1], m[q][2] * x[2]));
        nn = sqrtf(fmaf(y[0], y[0], fmaf(y[1], y[1], y[2] * y[2])));
        if (!(nn > 0.0f)) break;
        r = 1.0f / nn;
        for (int q = 0; q < 3; q++) x[q] = y[q] * r;
    }
    const int neg = x[2] < 0.0f || (x[2] == 0.0f && (x[1] < 0.0f || (x[1] == 0.0f && x[0] < 0.0f)));
    for (int q = 0; q < 3; q++) out[q] = neg ? -x[q] : x[q];
}

void or_phg_orient(const or_phg_cfg* g, const int32_t* occ, const int64_t* T, float* ori) {
    const long long nv = (long long)g->nx * g->ny * g->nz;
    for (long long c = 0; c < nv; c++) or_phg_orient_one(T + 6 * c, occ[c], ori + 3 * c);
}

static void step_to(float* p, float step, const float* d) {
    for (int a = 0; a < 3; a++) p[a] = fmaf(step, d[a], p[a]);
}

/* One trace by the rules of C (walk = root_steps for a guide strand, 0 for a segment half): up to
 * max_steps + 1 vertices, the start included; *dlast the direction of the last step (d0 when none
 * was taken); returns the vertex count, 0 for a guide that met no occupied voxel. */
static int trace(const or_phg_cfg* g, const int32_t* occ, const float* ori, const int32_t* crowd, const float* p0,
                 const float* d0, int walk, float* verts, float* dlast, int* stop) {
    float p[3] = {p0[0], p0[1], p0[2]}, d[3] = {d0[0], d0[1], d0[2]};
    int nv = 1, met = walk == 0;
    memcpy(verts, p, sizeof(p));
    *stop = OR_PHG_MAXLEN;
    for (int t = 0; t < g->max_steps; t++) {
        const long long c = or_phg_voxel(g, p);
        if (c < 0) {
            *stop = met ? OR_PHG_OUTSIDE : OR_PHG_NO_ROOT;
            break;
        }
        if (occ[c] == 0) {
            if (!met && t < walk) {
                step_to(p, g->step, d);
                memcpy(verts + 3 * nv++, p, sizeof(p));
                continue;
            }
            *stop = met ? OR_PHG_EMPTY : OR_PHG_NO_ROOT;
            break;
        }
        met = 1;
        if (crowd[c] >= g->occ_cap) {
            *stop = OR_PHG_CROWDED;
            break;
        }
        float o[3] = {ori[3 * c], ori[3 * c + 1], ori[3 * c + 2]};
        float sd = fmaf(o[0], d[0], fmaf(o[1], d[1], o[2] * d[2]));
        if (sd < 0.0f) {
            for (int a = 0; a < 3; a++) o[a] = -o[a];
            sd = -sd;
        }
        if (sd < g->cos_turn) {
            *stop = OR_PHG_TURN;
            break;
        }
        memcpy(d, o, sizeof(d));
        step_to(p, g->step, d);
        memcpy(verts + 3 * nv++, p, sizeof(p));
    }
    if (!met) nv = 0;
    memcpy(dlast, d, sizeof(d));
    return nv;
}

/* Deferred occupancy: one more strand in every voxel a polyline enters (consecutive vertices in
 * the same voxel count once; empty and outside voxels are not counted). */
static void count_visits(const or_phg_cfg* g, const int32_t* occ, const float* verts, int nv, int32_t* crowd) {
    long long last = -1;
    for (int k = 0; k < nv; k++) {
        const long long c = or_phg_voxel(g, verts + 3 * k);
        if (c >= 0 && occ[c] > 0 && c != last) crowd[c] += 1;
        last = c;
    }
}

static long long find_root(long long* par, long long x) {
    while (par[x] != x) {
        par[x] = par[par[x]];
        x = par[x];
    }
    return x;
}

/* The whole consumer, A to E.  Sizes: nvox = nx ny nz; guides: S x (max_steps + 1) x 3 vertices,
 * S counts, S stop codes, S x 3 tip tangents; segments: at most seg_cap, each 2 max_steps + 1
 * vertices (the backward half reversed, the seed, the forward half), counts, the seed voxel, the
 * two end tangents (start outward, end outward); labels: S + segments.  Returns the number of
 * segment seeds, or -1 when they exceed seg_cap. */
long long or_phg_run(const or_phg_cfg* g, long long n, const float* pts, const float* dirs, const uint8_t* valid,
                     long long S, const float* seeds, const float* normals, int32_t* occ, float* ori, int32_t* crowd,
                     float* gverts, int32_t* glen, int32_t* gstop, float* gtan, long long seg_cap, float* sverts,
                     int32_t* slen, int64_t* svox, float* stan, int32_t* label) {
    const long long nvox = (long long)g->nx * g->ny * g->nz;
    const int L = g->max_steps, GV = L + 1, SV = 2 * L + 1;
    int64_t* T = (int64_t*)malloc(sizeof(int64_t) * 6 * (size_t)nvox);
    or_phg_splat(g, n, pts, dirs, valid, occ, T);
    or_phg_orient(g, occ, T, ori);
    free(T);
    memset(crowd, 0, sizeof(int32_t) * nvox);
    /* C: guide strands, batch by batch */
    for (long long b0 = 0; b0 < S; b0 += g->batch) {
        const long long b1 = b0 + g->batch < S ? b0 + g->batch : S;
        for (long long i = b0; i < b1; i++) {
            int stop;
            glen[i] = trace(g, occ, ori, crowd, seeds + 3 * i, normals + 3 * i, g->root_steps,
                            gverts + (size_t)3 * GV * i, gtan + 3 * i, &stop);
            gstop[i] = stop;
        }
        for (long long i = b0; i < b1; i++) count_visits(g, occ, gverts + (size_t)3 * GV * i, glen[i], crowd);
    }
    /* D: segment seeds = occupied voxels no strand entered, in voxel order */
    long long K = 0;
    for (long long c = 0; c < nvox; c++)
        if (occ[c] > 0 && crowd[c] == 0) {
            if (K >= seg_cap) return -1;
            svox[K++] = c;
        }
    float* half = (float*)malloc(sizeof(float) * 3 * GV);
    for (long long b0 = 0; b0 < K; b0 += g->batch) {
        const long long b1 = b0 + g->batch < K ? b0 + g->batch : K;
        for (long long k = b0; k < b1; k++) {
            float* sv = sverts + (size_t)3 * SV * k;
            const long long c = svox[k];
            slen[k] = 0;
            if (crowd[c] > 0) continue;   /* an earlier batch reached this voxel */
            const long long cx = c % g->nx, cy = (c / g->nx) % g->ny, cz = c / ((long long)g->nx * g->ny);
            const float p0[3] = {fmaf((float)cx + 0.5f, g->voxel, g->origin[0]),
                                 fmaf((float)cy + 0.5f, g->voxel, g->origin[1]),
                                 fmaf((float)cz + 0.5f, g->voxel, g->origin[2])};
            const float fwd[3] = {ori[3 * c], ori[3 * c + 1], ori[3 * c + 2]};
            const float bwd[3] = {-fwd[0], -fwd[1], -fwd[2]};
            int stop;
            const int nb = trace(g, occ, ori, crowd, p0, bwd, 0, half, stan + 6 * k, &stop);
            for (int q = 0; q < nb; q++) memcpy(sv + 3 * q, half + 3 * (nb - 1 - q), sizeof(float) * 3);
            const int nf = trace(g, occ, ori, crowd, p0, fwd, 0, half, stan + 6 * k + 3, &stop);
            memcpy(sv + 3 * (nb - 1), half, sizeof(float) * 3 * nf);   /* the seed once */
            slen[k] = nb + nf - 1;
        }
        for (long long k = b0; k < b1; k++) count_visits(g, occ, sverts + (size_t)3 * SV * k, slen[k], crowd);
    }
    free(half);
    /* E: every end takes its nearest compatible segment end; the joined strands' components */
    const long long NS = S + K;
    long long* par = (long long*)malloc(sizeof(long long) * (size_t)NS);
    for (long long x = 0; x < NS; x++) par[x] = x;
    const float L2 = g->link_dist * g->link_dist;
    const long long NE = S + 2 * K;
    for (long long e = 0; e < NE; e++) {
        const float *pe, *te;
        long long se;
        if (e < S) {
            if (glen[e] <= 0) continue;
            se = e;
            pe = gverts + (size_t)3 * GV * e + 3 * (glen[e] - 1);
            te = gtan + 3 * e;
        } else {
            const long long k = (e - S) >> 1, side = (e - S) & 1;
            if (slen[k] <= 0) continue;
            se = S + k;
            pe = sverts + (size_t)3 * SV * k + (side ? 3 * (slen[k] - 1) : 0);
            te = stan + 6 * k + 3 * side;
        }
        long long best = -1;
        float bd = 0.0f;
        for (long long q = 0; q < 2 * K; q++) {
            const long long k = q >> 1, side = q & 1;
            if (slen[k] <= 0 || S + k == se) continue;
            const float* pq = sverts + (size_t)3 * SV * k + (side ? 3 * (slen[k] - 1) : 0);
            const float* tq = stan + 6 * k + 3 * side;
            const float dx = pe[0] - pq[0], dy = pe[1] - pq[1], dz = pe[2] - pq[2];
            const float d2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
            if (!(d2 < L2)) continue;
            const float dt = fmaf(te[0], tq[0], fmaf(te[1], tq[1], te[2] * tq[2]));
            if (!(-dt > g->link_cos)) continue;
            if (best < 0 || d2 < bd) {
                best = q;
                bd = d2;
            }
        }
        if (best >= 0) {
            const long long a = find_root(par, se), b = find_root(par, S + (best >> 1));
            if (a != b) par[a > b ? a : b] = a < b ? a : b;
        }
    }
    for (long long x = 0; x < NS; x++) label[x] = (int32_t)find_root(par, x);
    free(par);
    return K;
}
