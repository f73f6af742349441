// hf_fpmvo.cu - the paper's FPMVO step on the GPU (Sec. 3.1.1-3.1.3), warp per point:
//
//   lanes over views   visibility (frustum, bounds, depth test against the depth map) and the
//                      confidence at the point's pixel; then the top-K views (K warp argmaxes);
//   lane j < K         pixel offset u + lambda O(u) of view j (Eq. 1) and the depth there;
//   lane s K + j       candidate of view j at depth sample s (Eqs. 2-3), a unit direction;
//   group s            medoid of its K candidates (similarity |<d_i, d_j>|, confidence weights);
//   lane s K + j       patch consistency of layer s's fused offset point in view j: Eq. proj_r
//                      with the finite offset, Eqs. sim and patchloss over the P x P patch around
//                      the point's pixel (staged once per view in shared memory), Eq. patch_min;
//   lane 0             mean over the views per layer, the best layer (Eq. final_dout), outputs.
//
// Pixel decisions (the point's pixel and the offset pixel) use float-float arithmetic, as in the
// projection kernel, so they agree with an exact evaluation except within ~1e-10 px of an edge.
#include <math.h>
#include <stdint.h>

#include "hf_ff.cuh"
#include "hf_internal.cuh"

using namespace hf_ff;

namespace {

constexpr int kFpWarps = 4;   // points per CTA
constexpr float kU = 5.9604645e-8f;   // 2^-24, the unit roundoff of FP32

// FP32 projection of p into a view together with a bound on its rounding error, so that a pixel or
// depth decision is taken in FP32 when it lies farther from its edge than the bound and repeated in
// float-float otherwise (the decisions are then those of the float-float path exactly).
//  - X_r = R_r p + t_r by three FMAs: |fl(X_r) - X_r| <= 3u (sum_c |R_rc p_c| + |t_r|) to first
//    order; e_r = 4u M_r (M_r that sum, itself rounded) covers the rest;
//  - x = X0 / X2 with a 2-ulp reciprocal and a rounded product, u_f = fx x + cx by one FMA:
//    |u_f - u| <= fx (e0 + |x| e2) / X2 + fx |x| (2^-22 + u) + u |u_f|, taken with a factor 1.25.
struct FastProj {
    float uf, wf;   // pixel coordinates
    float Z, eZ;    // depth and its error bound
    float mu, mw;   // error bounds of uf, wf
};
__device__ __forceinline__ FastProj fast_project(const float* cam, float p0, float p1, float p2, float a0, float a1,
                                                 float a2) {
    FastProj f;
    const float X0 = fmaf(cam[4], p0, fmaf(cam[5], p1, fmaf(cam[6], p2, cam[13])));
    const float X1 = fmaf(cam[7], p0, fmaf(cam[8], p1, fmaf(cam[9], p2, cam[14])));
    f.Z = fmaf(cam[10], p0, fmaf(cam[11], p1, fmaf(cam[12], p2, cam[15])));
    const float M0 = fmaf(fabsf(cam[4]), a0, fmaf(fabsf(cam[5]), a1, fmaf(fabsf(cam[6]), a2, fabsf(cam[13]))));
    const float M1 = fmaf(fabsf(cam[7]), a0, fmaf(fabsf(cam[8]), a1, fmaf(fabsf(cam[9]), a2, fabsf(cam[14]))));
    const float M2 = fmaf(fabsf(cam[10]), a0, fmaf(fabsf(cam[11]), a1, fmaf(fabsf(cam[12]), a2, fabsf(cam[15]))));
    f.eZ = 4.0f * kU * M2;
    const float rz = __fdividef(1.0f, f.Z);
    const float x = X0 * rz, y = X1 * rz;
    f.uf = fmaf(cam[0], x, cam[2]);
    f.wf = fmaf(cam[1], y, cam[3]);
    const float ax = fabsf(x), ay = fabsf(y);
    f.mu = 1.25f * fmaf(cam[0] * rz, fmaf(ax, f.eZ, 4.0f * kU * M0), fmaf(cam[0], ax, fabsf(f.uf)) * 3.0e-7f);
    f.mw = 1.25f * fmaf(cam[1] * rz, fmaf(ay, f.eZ, 4.0f * kU * M1), fmaf(cam[1], ay, fabsf(f.wf)) * 3.0e-7f);
    return f;
}
// floor(x) when x is farther than m from both integers around it, else -1 (undecided in FP32)
__device__ __forceinline__ bool sure_floor(float x, float m, float& fl) {
    fl = floorf(x);
    return fminf(x - fl, (fl + 1.0f) - x) > m;
}
// The depth test X_z <= D + eps on the float-float depth (the difference of two nearby depths is
// exact, then the low part); +inf depth (no hair) passes.
__device__ __forceinline__ bool depth_test_ff(ff Z, float D, float eps) {
    return __fadd_rn(__fsub_rn(Z.hi, D), Z.lo) <= eps;
}
// The same test from the FP32 depth with its error bound: 1 pass, 0 fail, -1 undecided.
__device__ __forceinline__ int depth_test_fast(float Z, float eZ, float D, float eps) {
    if (!(fabsf(D) < INFINITY)) return D > 0.0f ? 1 : 0;   // +inf passes, -inf and NaN fail
    const float d = Z - D;
    const float md = fmaf(fabsf(d) + eps, 2.4e-7f, eZ);    // |fl(Z - D) - (Z - D)| and the rounding below
    return d <= eps - md ? 1 : (d > eps + md ? 0 : -1);
}
// Selection key of a view: confidence bits + 1 for a view that sees the point (non-negative floats
// order as their bits), 0 otherwise.
__device__ __forceinline__ uint32_t conf_key(float c) { return __float_as_uint(c + 0.0f) + 1u; }

// The pixel of p in view cam (index y W + x within the view), -1 when p is behind the camera or
// outside the image; decided in FP32 where the error bound allows, else in float-float, in which
// case zff receives the float-float depth and have_ff is set.
__device__ __forceinline__ int view_pixel(const float* cam, float p0, float p1, float p2, float a0, float a1, float a2,
                                          int W, int H, FastProj& f, ff& zff, bool& have_ff) {
    f = fast_project(cam, p0, p1, p2, a0, a1, a2);
    have_ff = false;
    float fu, fv;
    if (f.Z - f.eZ > 1.0001e-6f) {   // in front for certain (the exact test is X_z > 1e-6)
        // outside the image for certain (twice the bound covers the rounding of these sums)
        if (f.uf + 2.0f * f.mu < 0.0f || f.uf - 2.0f * f.mu >= (float)W || f.wf + 2.0f * f.mw < 0.0f ||
            f.wf - 2.0f * f.mw >= (float)H)
            return -1;
        const bool su = sure_floor(f.uf, f.mu, fu);
        if (!(sure_floor(f.wf, f.mw, fv) && su)) have_ff = true;
    } else if (f.Z + f.eZ < 0.9999e-6f) {   // behind for certain
        return -1;
    } else {
        have_ff = true;
    }
    if (have_ff) {   // float-float projection: the decisions of the exact projection
        const ff X0 = ff_dot3_plus(cam[4], cam[5], cam[6], p0, p1, p2, cam[13]);
        const ff X1 = ff_dot3_plus(cam[7], cam[8], cam[9], p0, p1, p2, cam[14]);
        zff = ff_dot3_plus(cam[10], cam[11], cam[12], p0, p1, p2, cam[15]);
        if (!(zff.hi > 1e-6f)) return -1;
        fu = ff_floor(ff_affine(cam[0], ff_div(X0, zff), cam[2]));
        fv = ff_floor(ff_affine(cam[1], ff_div(X1, zff), cam[3]));
    }
    if (!(fu >= 0.0f && fu < (float)W && fv >= 0.0f && fv < (float)H)) return -1;
    return (int)fv * W + (int)fu;
}

// Phase 2 of k_fpmvo for one point, by one warp: the candidates from its top views, medoid fusion per
// depth layer, patch consistency and the outputs.  tkv / tkc: its nk top views and their
// confidences; patch: K x P x P float2 of shared memory; px: K pixel slots of shared memory.
template <int P>
__device__ __forceinline__ void fpmvo_point(const FpmvoArgs& a, int i, int nk, const int* tkv, const float* tkc,
                                            float2* patch, int (*px)[2], int lane) {
    constexpr int P2 = P * P, h = P / 2;
    const int S = a.S;
    const size_t npx = (size_t)a.W * a.H;
    if (nk <= 0) {   // -1: non-finite point; 0: no view sees it
        if (lane == 0) {
            a.dir_out[3 * i] = a.dir_out[3 * i + 1] = a.dir_out[3 * i + 2] = 0.0f;
            if (a.cost_out) a.cost_out[i] = nk < 0 ? __int_as_float(0x7fc00000) : 1.0f;
            if (a.sel_out) a.sel_out[i] = -1;
            if (a.status_out) a.status_out[i] = nk < 0 ? HF_STATUS_BAD_INPUT : HF_STATUS_NO_VIEWS;
        }
        return;
    }
    const float p0 = a.pts[3 * i], p1 = a.pts[3 * i + 1], p2 = a.pts[3 * i + 2];
    const float a0 = fabsf(p0), a1 = fabsf(p1), a2 = fabsf(p2);
    // ---- per top view: the point's pixel and the offset pixel's depth (Eq. 1)
    // lane j keeps: the point's pixel position (u, w), its camera depth Zp (float-float), the offset
    // lambda (cos theta, sin theta) and the depth z at the offset pixel.  The angle read at the
    // point's pixel and the patch reads below are issued together; then the offset pixel's depth.
    float pu = 0.0f, pw = 0.0f, zph = 0.0f, zpl = 0.0f, lc = 0.0f, ls = 0.0f, zc = 0.0f;
    bool vok = false;
    FastProj ft;
    ff u = {0.0f, 0.0f}, w = {0.0f, 0.0f}, X2 = {0.0f, 0.0f};
    bool sure = true;
    float th = 0.0f;
    const float* tcam = a.cams + 16 * tkv[lane < nk ? lane : 0];
    const size_t tbase = (size_t)tkv[lane < nk ? lane : 0] * npx;
    if (lane < nk) {
        const float* cam = tcam;
        ft = fast_project(cam, p0, p1, p2, a0, a1, a2);
        X2 = ff_dot3_plus(cam[10], cam[11], cam[12], p0, p1, p2, cam[15]);   // for the offsets
        float fu, fv;
        const bool su = sure_floor(ft.uf, ft.mu, fu);
        sure = sure_floor(ft.wf, ft.mw, fv) && su;
        u = ff{ft.uf, 0.0f};
        w = ff{ft.wf, 0.0f};
        if (!sure) {
            const ff X0 = ff_dot3_plus(cam[4], cam[5], cam[6], p0, p1, p2, cam[13]);
            const ff X1 = ff_dot3_plus(cam[7], cam[8], cam[9], p0, p1, p2, cam[14]);
            u = ff_affine(cam[0], ff_div(X0, X2), cam[2]);
            w = ff_affine(cam[1], ff_div(X1, X2), cam[3]);
            fu = ff_floor(u);
            fv = ff_floor(w);
        }
        px[lane][0] = (int)fu;
        px[lane][1] = (int)fv;
        th = __ldg(&a.amap[tbase + (size_t)((int)fv * a.W + (int)fu)].x);
    }
    __syncwarp();
    // the P x P patch of every top view: C (cos theta, sin theta), 0 outside the image; up to 128
    // elements per pass, four loads per lane in flight
    constexpr int kPatchRegs = 4;
    const int npatch = nk * P2;
    float2 pv[kPatchRegs];
#pragma unroll
    for (int r = 0; r < kPatchRegs; ++r) {
        const int e = lane + 32 * r;
        pv[r] = make_float2(0.0f, 0.0f);
        if (e < npatch) {
            const int j = e / P2, q = e - j * P2;
            const int x = px[j][0] + (q % P) - h, y = px[j][1] + (q / P) - h;
            if (x >= 0 && y >= 0 && x < a.W && y < a.H)
                pv[r] = __ldg(a.vmap + (size_t)tkv[j] * npx + (size_t)(y * a.W + x));
        }
    }
    if (lane < nk) {
        float sn, cs;
        sincosf(th, &sn, &cs);
        lc = a.lambda * cs;
        ls = a.lambda * sn;
        // the offset pixel floor(u + lambda cos theta), floor(w + lambda sin theta)
        float gx, gy;
        bool osure = false;
        if (sure) {
            const float ux = ft.uf + lc, uy = ft.wf + ls;
            const bool sx = sure_floor(ux, fmaf(fabsf(ux), 1.2e-7f, ft.mu), gx);
            osure = sure_floor(uy, fmaf(fabsf(uy), 1.2e-7f, ft.mw), gy) && sx;
        }
        if (!osure) {
            if (sure) {   // the point's pixel was decided in FP32: its float-float position now
                const float* cam = tcam;
                const ff X0 = ff_dot3_plus(cam[4], cam[5], cam[6], p0, p1, p2, cam[13]);
                const ff X1 = ff_dot3_plus(cam[7], cam[8], cam[9], p0, p1, p2, cam[14]);
                u = ff_affine(cam[0], ff_div(X0, X2), cam[2]);
                w = ff_affine(cam[1], ff_div(X1, X2), cam[3]);
            }
            gx = ff_floor(ff_add(u, ff{lc, 0.0f}));
            gy = ff_floor(ff_add(w, ff{ls, 0.0f}));
        }
        pu = u.hi + u.lo;
        pw = w.hi + w.lo;
        zph = X2.hi;
        zpl = X2.lo;
        if (gx >= 0.0f && gx < (float)a.W && gy >= 0.0f && gy < (float)a.H)
            zc = __ldg(&a.dmap[tbase + (size_t)((int)gy * a.W + (int)gx)].x);
        else
            zc = __int_as_float(0x7f800000);   // no depth outside the image
    }
#pragma unroll
    for (int r = 0; r < kPatchRegs; ++r)
        if (lane + 32 * r < npatch) patch[lane + 32 * r] = pv[r];
    for (int e = lane + 32 * kPatchRegs; e < npatch; e += 32) {   // larger K x P x P
        const int j = e / P2, q = e - j * P2;
        const int x = px[j][0] + (q % P) - h, y = px[j][1] + (q / P) - h;
        float2 sv = make_float2(0.0f, 0.0f);
        if (x >= 0 && y >= 0 && x < a.W && y < a.H)
            sv = __ldg(a.vmap + (size_t)tkv[j] * npx + (size_t)(y * a.W + x));
        patch[e] = sv;
    }
    vok = lane < nk && isfinite(zc);
    __syncwarp();
    // ---- candidates (Eqs. 2-3): lane c = s K + j
    const int nc = nk * S;
    const int s = lane / nk, j = lane - s * nk;   // meaningful for lane < nc
    const int srcj = lane < nc ? j : 0;
    const float bu = __shfl_sync(0xffffffffu, pu, srcj), bw = __shfl_sync(0xffffffffu, pw, srcj);
    const float bzh = __shfl_sync(0xffffffffu, zph, srcj), bzl = __shfl_sync(0xffffffffu, zpl, srcj);
    const float blc = __shfl_sync(0xffffffffu, lc, srcj), bls = __shfl_sync(0xffffffffu, ls, srcj);
    const float bz = __shfl_sync(0xffffffffu, zc, srcj);
    const bool bok = __shfl_sync(0xffffffffu, (int)vok, srcj) != 0;
    float e0 = 0.0f, e1 = 0.0f, e2 = 0.0f, d0 = 0.0f, d1 = 0.0f, d2 = 0.0f, wj = 0.0f;
    bool cok = false;
    if (lane < nc && bok) {
        const float* cam = a.cams + 16 * tkv[j];
        const float ds = S > 1 ? -a.delta + 2.0f * a.delta * (float)s / (float)(S - 1) : 0.0f;
        const float zs = bz + ds;
        // the offset in camera coordinates without cancellation: with Zp the point's depth,
        // X_cand - X_p = ((lambda c zs + (u - cx)(zs - Zp)) / fx, (lambda s zs + (w - cy)(zs - Zp)) / fy,
        // zs - Zp), and zs - Zp = (z - Zp.hi) - Zp.lo + delta_s (the first difference is exact)
        const float dz = __fadd_rn(__fsub_rn(__fsub_rn(bz, bzh), bzl), ds);
        const float Y0 = fmaf(blc, zs, (bu - cam[2]) * dz) / cam[0];
        const float Y1 = fmaf(bls, zs, (bw - cam[3]) * dz) / cam[1];
        // world offset e = R^T Y
        e0 = fmaf(cam[4], Y0, fmaf(cam[7], Y1, cam[10] * dz));
        e1 = fmaf(cam[5], Y0, fmaf(cam[8], Y1, cam[11] * dz));
        e2 = fmaf(cam[6], Y0, fmaf(cam[9], Y1, cam[12] * dz));
        const float n = sqrtf(e0 * e0 + e1 * e1 + e2 * e2);
        if (n > 1e-12f) {
            const float rn = 1.0f / n;
            d0 = e0 * rn;
            d1 = e1 * rn;
            d2 = e2 * rn;
            cok = true;
        }
        wj = tkc[j];
    }
    // ---- medoid of group s: sigma = sum_k w_k |<d, d_k>| / sum_k w_k over the group's valid candidates
    const int g0 = lane < nc ? s * nk : 0;
    float num = 0.0f, den = 0.0f;
    for (int k = 0; k < nk; ++k) {
        const float q0 = __shfl_sync(0xffffffffu, d0, g0 + k), q1 = __shfl_sync(0xffffffffu, d1, g0 + k);
        const float q2 = __shfl_sync(0xffffffffu, d2, g0 + k), qw = __shfl_sync(0xffffffffu, wj, g0 + k);
        const bool qk = __shfl_sync(0xffffffffu, (int)cok, g0 + k) != 0;
        if (qk) {
            num += qw * fabsf(fmaf(d0, q0, fmaf(d1, q1, d2 * q2)));
            den += qw;
        }
    }
    const float sigma = cok ? (den > 0.0f ? num / den : 0.0f) : -1.0f;
    int med = -1;   // lane of the group's medoid
    float msig = -1.0f;
    for (int k = 0; k < nk; ++k) {
        const float sk = __shfl_sync(0xffffffffu, sigma, g0 + k);
        if (sk > msig) {
            msig = sk;
            med = g0 + k;
        }
    }
    const bool layer_ok = lane < nc && msig >= 0.0f;
    // the fused offset point of layer s, as an offset from p
    const int msrc = med >= 0 ? med : 0;
    const float f0 = __shfl_sync(0xffffffffu, e0, msrc), f1 = __shfl_sync(0xffffffffu, e1, msrc);
    const float f2 = __shfl_sync(0xffffffffu, e2, msrc);
    // ---- patch consistency of layer s in view j (Eqs. proj_r, sim, patchloss, patch_min)
    float Lv = 0.0f;
    if (layer_ok) {
        const float* cam = a.cams + 16 * tkv[j];
        const float X0 = fmaf(cam[4], p0, fmaf(cam[5], p1, fmaf(cam[6], p2, cam[13])));
        const float X1 = fmaf(cam[7], p0, fmaf(cam[8], p1, fmaf(cam[9], p2, cam[14])));
        const float Z = fmaf(cam[10], p0, fmaf(cam[11], p1, fmaf(cam[12], p2, cam[15])));
        const float q0 = fmaf(cam[4], f0, fmaf(cam[5], f1, cam[6] * f2));
        const float q1 = fmaf(cam[7], f0, fmaf(cam[8], f1, cam[9] * f2));
        const float q2 = fmaf(cam[10], f0, fmaf(cam[11], f1, cam[12] * f2));
        const float Zf = Z + q2;
        if (Zf > 1e-6f) {
            // Pi(p + f) - Pi(p) without cancellation: fx (Z q_x - X_x q_z) / (Z Z_f)
            const float rden = 1.0f / (Z * Zf);
            const float rx = cam[0] * fmaf(Z, q0, -X0 * q2) * rden, ry = cam[1] * fmaf(Z, q1, -X1 * q2) * rden;
            const float rn2 = fmaf(rx, rx, ry * ry);
            const float en2 = fmaf(f0, f0, fmaf(f1, f1, f2 * f2));
            if (rn2 * Z * Z >= 1e-20f * fmaf(cam[0], cam[0], cam[1] * cam[1]) * en2) {
                const float inv = rsqrtf(rn2);
                const float ux = rx * inv, uy = ry * inv;
                const float2* pt = patch + j * P2;
#pragma unroll
                for (int q = 0; q < P2; ++q) {
                    const float2 sq = pt[q];
                    Lv = fmaxf(Lv, fabsf(fmaf(ux, sq.x, uy * sq.y)));
                }
            }
        }
    }
    // mean over the views of layer s, in view order
    float lsum = 0.0f;
    for (int k = 0; k < nk; ++k) lsum += __shfl_sync(0xffffffffu, Lv, g0 + k);
    const float lbar = layer_ok ? lsum / (float)nk : -1.0f;
    // ---- the best layer (lowest s on ties) and the outputs
    float best = -1.0f;
    int bs = -1;
    for (int q = 0; q < S; ++q) {
        const float lq = __shfl_sync(0xffffffffu, lbar, q * nk < nc ? q * nk : 0);
        if (lq > best) {
            best = lq;
            bs = q;
        }
    }
    const int osrc = bs >= 0 ? bs * nk : 0;
    const float o0 = __shfl_sync(0xffffffffu, f0, osrc), o1 = __shfl_sync(0xffffffffu, f1, osrc);
    const float o2 = __shfl_sync(0xffffffffu, f2, osrc);
    if (lane == 0) {
        if (bs < 0) {
            a.dir_out[3 * i] = a.dir_out[3 * i + 1] = a.dir_out[3 * i + 2] = 0.0f;
            if (a.cost_out) a.cost_out[i] = 1.0f;
            if (a.sel_out) a.sel_out[i] = -1;
            if (a.status_out) a.status_out[i] = HF_STATUS_NO_VIEWS;
        } else {
            const float n = sqrtf(o0 * o0 + o1 * o1 + o2 * o2);
            const float x0 = o0 / n, x1 = o1 / n, x2 = o2 / n;
            const float sgn = fabsf(x2) > 1e-12f ? copysignf(1.0f, x2)
                              : fabsf(x1) > 1e-12f ? copysignf(1.0f, x1) : copysignf(1.0f, x0);
            a.dir_out[3 * i] = sgn * x0;
            a.dir_out[3 * i + 1] = sgn * x1;
            a.dir_out[3 * i + 2] = sgn * x2;
            if (a.cost_out) a.cost_out[i] = 1.0f - best;
            if (a.sel_out) a.sel_out[i] = bs;
            if (a.status_out) a.status_out[i] = HF_STATUS_OK;
        }
    }
}


// Top-K insertion: (key descending, view ascending) over kTopSlots slots, the last slot dropping
// out.  The order is total, so an entry pushed down by the new one keeps its place among equal keys.
constexpr int kTopSlots = HF_FPMVO_MAX_K;
__device__ __forceinline__ void top_insert(uint32_t (&tk)[kTopSlots], int (&tv)[kTopSlots], uint32_t key, int v) {
#pragma unroll
    for (int q = 0; q < kTopSlots; ++q) {
        if (key > tk[q] || (key == tk[q] && v < tv[q])) {
            const uint32_t k2 = tk[q];
            const int v2 = tv[q];
            tk[q] = key;
            tv[q] = v;
            key = k2;
            v = v2;
        }
    }
}

// Phase 1, a thread per point: every view's pixel decision and (depth, confidence) gather, the
// depth test and the top-K views.  The threads of a warp hold consecutive points, which lie along
// the same strands, so each of their gathers goes to nearby pixels of the same view.  Two views
// per step keep two gathers in flight.  Phase 2, a warp per point: fpmvo_point.
constexpr int kFpThreads = kFpWarps * 32;
template <int P>
__global__ void __launch_bounds__(kFpThreads, 8) k_fpmvo(FpmvoArgs a) {
    constexpr int P2 = P * P;
    extern __shared__ __align__(16) float2 fp_patch[];   // [kFpWarps][K * P2]
    __shared__ int s_tv[kFpThreads][HF_FPMVO_MAX_K];
    __shared__ float s_tc[kFpThreads][HF_FPMVO_MAX_K];
    __shared__ int s_nk[kFpThreads];
    __shared__ int s_px[kFpWarps][HF_FPMVO_MAX_K][2];
    const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
    const int i0 = blockIdx.x * kFpThreads;
    {
        const int i = i0 + t;
        int nk = 0;
        if (i < a.N) {
            const float p0 = a.pts[3 * i], p1 = a.pts[3 * i + 1], p2 = a.pts[3 * i + 2];
            if (!(isfinite(p0) && isfinite(p1) && isfinite(p2))) {
                nk = -1;
            } else {
                const float a0 = fabsf(p0), a1 = fabsf(p1), a2 = fabsf(p2);
                const size_t npx = (size_t)a.W * a.H;
                uint32_t tk[kTopSlots];
                int tv[kTopSlots];
#pragma unroll
                for (int q = 0; q < kTopSlots; ++q) {
                    tk[q] = 0u;
                    tv[q] = 0;
                }
                constexpr int G = 2;
                for (int v0 = 0; v0 < a.V; v0 += G) {
                    int pix[G];
                    FastProj f[G];
                    ff zff[G];
                    bool hf[G];
#pragma unroll
                    for (int r = 0; r < G; ++r)
                        pix[r] = v0 + r < a.V ? view_pixel(a.cams + 16 * (v0 + r), p0, p1, p2, a0, a1, a2, a.W, a.H,
                                                           f[r], zff[r], hf[r])
                                              : -1;
                    float2 dc[G];
#pragma unroll
                    for (int r = 0; r < G; ++r)
                        dc[r] = pix[r] >= 0 ? __ldg(a.dmap + (size_t)(v0 + r) * npx + pix[r]) : make_float2(0.0f, 0.0f);
#pragma unroll
                    for (int r = 0; r < G; ++r) {
                        if (pix[r] < 0) continue;
                        int vis = hf[r] ? -1 : depth_test_fast(f[r].Z, f[r].eZ, dc[r].x, a.eps);
                        if (vis < 0) {
                            const float* cam = a.cams + 16 * (v0 + r);
                            if (!hf[r]) zff[r] = ff_dot3_plus(cam[10], cam[11], cam[12], p0, p1, p2, cam[15]);
                            vis = depth_test_ff(zff[r], dc[r].x, a.eps);
                        }
                        if (vis) top_insert(tk, tv, conf_key(dc[r].y), v0 + r);
                    }
                }
#pragma unroll
                for (int q = 0; q < kTopSlots; ++q) {
                    if (q < a.K && tk[q] != 0u) {
                        s_tv[t][q] = tv[q];
                        s_tc[t][q] = __uint_as_float(tk[q] - 1u);
                        nk = q + 1;
                    }
                }
            }
        }
        s_nk[t] = nk;
    }
    __syncthreads();
    float2* patch = fp_patch + (size_t)warp * a.K * P2;
    for (int q = 0; q < 32; ++q) {
        const int tt = warp * 32 + q, i = i0 + tt;
        if (i >= a.N) break;
        fpmvo_point<P>(a, i, s_nk[tt], s_tv[tt], s_tc[tt], patch, s_px[warp], lane);
        __syncwarp();
    }
}

template <int P>
cudaError_t launch_fpmvo(const FpmvoArgs& a, cudaStream_t s) {
    const size_t smem = (size_t)kFpWarps * a.K * P * P * sizeof(float2);
    k_fpmvo<P><<<(a.N + kFpThreads - 1) / kFpThreads, kFpThreads, smem, s>>>(a);
    return cudaGetLastError();
}

// The maps FPMVO gathers from, built once per depth upload: (depth, confidence) for the depth test
// and the top-view selection (one 8-byte read), and C (cos theta, sin theta) for the patches.
__global__ void k_fpmvo_maps(const float* __restrict__ depth, const float2* __restrict__ amap, size_t npx,
                             float2* __restrict__ dmap, float2* __restrict__ vmap) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < npx; i += (size_t)gridDim.x * blockDim.x) {
        const float2 t = amap[i];
        float sn, cs;
        sincosf(t.x, &sn, &cs);
        dmap[i] = make_float2(depth[i], t.y);
        vmap[i] = make_float2(t.y * cs, t.y * sn);
    }
}

}  // namespace

cudaError_t hf_launch_fpmvo(const FpmvoArgs& a, cudaStream_t s) {
    switch (a.P) {
        case 1: return launch_fpmvo<1>(a, s);
        case 3: return launch_fpmvo<3>(a, s);
        case 5: return launch_fpmvo<5>(a, s);
        case 7: return launch_fpmvo<7>(a, s);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t hf_launch_fpmvo_maps(const float* depth, const float2* amap, size_t npx, float2* dmap, float2* vmap,
                                 cudaStream_t s) {
    if (!npx) return cudaSuccess;
    const size_t blocks = (npx + 255) / 256;
    k_fpmvo_maps<<<(unsigned)(blocks < 148 * 16 ? blocks : 148 * 16), 256, 0, s>>>(depth, amap, npx, dmap, vmap);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ C ABI
extern "C" int hair_fuse_upload_depth(hf_ctx* c, const float* depth, int mem_kind) {
    if (!c) return HF_ERR_INVALID_ARG;
    if (c->V <= 0) return hf_set_err(c, HF_ERR_NOT_UPLOADED, "upload the views first (the depth maps have their size)");
    if (!depth) return hf_set_err(c, HF_ERR_INVALID_ARG, "null depth pointer");
    if (mem_kind != HF_HOST && mem_kind != HF_DEVICE) return hf_set_err(c, HF_ERR_INVALID_ARG, "bad mem_kind");
    const size_t npx = (size_t)c->V * c->W * c->Hh;
    int rc;
    if ((rc = hf_ensure(c, c->dmap, npx * sizeof(float2)))) return rc;
    if ((rc = hf_ensure(c, c->vmap, npx * sizeof(float2)))) return rc;
    const float* src = depth;
    cudaError_t e = cudaSuccess;
    if (mem_kind == HF_HOST) {   // staged through the context's buffer
        if ((rc = hf_ensure(c, c->depth, npx * sizeof(float)))) return rc;
        e = cudaMemcpyAsync(c->depth.p, depth, npx * sizeof(float), cudaMemcpyHostToDevice, c->stream);
        if (e != cudaSuccess) return hf_cuda_err(c, e, "upload depth");
        src = (const float*)c->depth.p;
    }
    if ((rc = run_launch(c, "k_fpmvo_maps", [&] {
             return hf_launch_fpmvo_maps(src, (const float2*)c->amap.p, npx, (float2*)c->dmap.p, (float2*)c->vmap.p,
                                         c->stream);
         })))
        return rc;
    if (mem_kind == HF_HOST && (e = cudaStreamSynchronize(c->stream)) != cudaSuccess)
        return hf_cuda_err(c, e, "upload depth");
    c->depth_gen = c->views_gen;
    return HF_OK;
}

extern "C" int hair_fuse_fpmvo(hf_ctx* c, const hf_fpmvo_cfg* cfg, float* dir_out, float* cost_out, int32_t* sel_out,
                               uint8_t* status_out, int mem_kind) {
    if (!c || !cfg || !dir_out) return HF_ERR_INVALID_ARG;
    if (c->V <= 0 || c->N <= 0) return hf_set_err(c, HF_ERR_NOT_UPLOADED, "views or points not uploaded");
    if (!c->dmap.p || c->depth_gen != c->views_gen)
        return hf_set_err(c, HF_ERR_NOT_UPLOADED, "depth maps not uploaded for the current views");
    if (mem_kind != HF_HOST && mem_kind != HF_DEVICE) return hf_set_err(c, HF_ERR_INVALID_ARG, "bad mem_kind");
    const hf_fpmvo_cfg g = *cfg;
    if (g.K < 1 || g.K > HF_FPMVO_MAX_K || g.S < 1 || g.K * g.S > 32 || g.P < 1 || g.P > 7 || !(g.P & 1) ||
        !(isfinite(g.lambda_px) && g.lambda_px >= 0.0f) || !(isfinite(g.delta) && g.delta >= 0.0f) ||
        !(isfinite(g.eps_vis) && g.eps_vis >= 0.0f))
        return hf_set_err(c, HF_ERR_INVALID_ARG,
                          "fpmvo: K in [1, 8], K * S <= 32, P odd in [1, 7], lambda, delta, eps finite and >= 0");
    const int N = c->N;
    float *d_dir = dir_out, *d_cost = cost_out;
    int32_t* d_sel = sel_out;
    uint8_t* d_st = status_out;
    int rc;
    if (mem_kind == HF_HOST) {
        if ((rc = hf_ensure(c, c->outs, (size_t)N * 21))) return rc;
        char* base = (char*)c->outs.p;
        d_dir = (float*)base;
        d_cost = cost_out ? (float*)(base + (size_t)N * 12) : nullptr;
        d_sel = sel_out ? (int32_t*)(base + (size_t)N * 16) : nullptr;
        d_st = status_out ? (uint8_t*)(base + (size_t)N * 20) : nullptr;
    }
    FpmvoArgs a{(const float*)c->pts.p, N, (const float*)c->cams.p, c->V, c->W, c->Hh, (const float2*)c->amap.p,
                (const float2*)c->dmap.p, (const float2*)c->vmap.p, g.K, g.S, g.P, g.lambda_px, g.delta, g.eps_vis,
                d_dir, d_cost, d_sel, d_st};
    if ((rc = run_launch(c, "k_fpmvo", [&] { return hf_launch_fpmvo(a, c->stream); }))) return rc;
    if (mem_kind == HF_HOST) {
        cudaError_t e = cudaMemcpyAsync(dir_out, d_dir, (size_t)N * 12, cudaMemcpyDeviceToHost, c->stream);
        if (e == cudaSuccess && cost_out) e = cudaMemcpyAsync(cost_out, d_cost, (size_t)N * 4, cudaMemcpyDeviceToHost, c->stream);
        if (e == cudaSuccess && sel_out) e = cudaMemcpyAsync(sel_out, d_sel, (size_t)N * 4, cudaMemcpyDeviceToHost, c->stream);
        if (e == cudaSuccess && status_out) e = cudaMemcpyAsync(status_out, d_st, (size_t)N, cudaMemcpyDeviceToHost, c->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
        if (e != cudaSuccess) return hf_cuda_err(c, e, "copy outputs");
    }
    return HF_OK;
}
