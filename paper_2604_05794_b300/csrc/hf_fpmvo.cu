// hf_fpmvo.cu - the paper's FPMVO step on the GPU (Sec. 3.1.1-3.1.3) in two kernels.
//
// k_fpmvo_views, a thread per point (the lanes of a warp hold consecutive points along the strands,
// so their gathers meet nearby pixels of one view at a time):
//   every view         pixel decision, (depth, confidence) gather, depth test; the top-K views;
//   every top view     the pixel offset u + lambda O(u) (Eq. 1) and the depth there, written as a
//                      record for the second kernel.
// k_fpmvo_fuse, a warp per point:
//   lane e             element e of the P x P patches of C (cos theta, sin theta) around the pixel;
//   lane s nk + j      candidate of top view j at depth sample s (Eqs. 2-3), a unit direction;
//   group s            medoid of its candidates (similarity |<d_i, d_j>|, confidence weights);
//   lane s nk + j      patch consistency of layer s's fused offset point in view j: Eq. proj_r
//                      with the finite offset, Eqs. sim and patchloss over the patch, Eq. patch_min;
//   lane 0             mean over the views per layer, the best layer (Eq. final_dout), outputs.
//
// Pixel and depth-test decisions are taken in FP32 where a proven bound on its rounding error
// leaves them unambiguous and in float-float otherwise, so they agree with an exact evaluation
// except within ~1e-10 px (or depth units) of an edge.
#include <math.h>
#include <stdint.h>
#include <string.h>

#include "hf_ff.cuh"
#include "hf_internal.cuh"

using namespace hf_ff;

namespace {

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

// Top-K insertion: (key descending, view ascending) over K slots, the last slot dropping out.  The
// order is total, so an entry pushed down by the new one keeps its place among equal keys.
template <int K>
__device__ __forceinline__ void top_insert(uint32_t (&tk)[K], int (&tv)[K], uint32_t key, int v) {
#pragma unroll
    for (int q = 0; q < K; ++q) {
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

// Zero records q0 .. K-1 of point i (the fusion kernel loads all K); record 0 carries nk in its
// last word either way.
__device__ __forceinline__ void write_empty_records(const FpmvoArgs& a, int i, int q0, int nk) {
    for (int q = q0; q < a.K; ++q) {
        float4* r = a.rec + ((size_t)i * a.K + q) * 3;
        r[0] = r[1] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        r[2] = make_float4(0.0f, 0.0f, 0.0f, q == 0 ? __int_as_float(nk) : 0.0f);
    }
}

// ------------------------------------------------------------------ k_fpmvo_views: a thread per point
// Every view's pixel decision and (depth, confidence) gather, the depth test, the top-K views, and
// per top view the pixel offset and the depth there (Eq. 1).  The threads of a warp hold
// consecutive points, which lie along the same strands, so each of their gathers goes to nearby
// pixels of the same view; two views per step keep two gathers in flight.  Output per point: K
// records of three 16-byte words, one per top view and zeros past the last (see FpmvoArgs).
constexpr int kViewsThreads = 128;
template <int K>
__global__ void __launch_bounds__(kViewsThreads, 9) k_fpmvo_views(FpmvoArgs a) {
    __shared__ int s_tv[kViewsThreads][HF_FPMVO_MAX_K];
    __shared__ float s_tc[kViewsThreads][HF_FPMVO_MAX_K];
    const int t = threadIdx.x;
    const int i = blockIdx.x * kViewsThreads + t;
    if (i >= a.N) return;
    const float p0 = a.pts[3 * i], p1 = a.pts[3 * i + 1], p2 = a.pts[3 * i + 2];
    if (!(isfinite(p0) && isfinite(p1) && isfinite(p2))) {
        write_empty_records(a, i, 0, -1);
        return;
    }
    const float a0 = fabsf(p0), a1 = fabsf(p1), a2 = fabsf(p2);
    const size_t npx = (size_t)a.W * a.H;
    uint32_t tk[K];
    int tv[K];
#pragma unroll
    for (int q = 0; q < K; ++q) {
        tk[q] = 0u;
        tv[q] = 0;
    }
    constexpr int G = 2;
    for (int v0 = 0; v0 < a.V; v0 += G) {
        int pix[G];
        FastProj f[G];
        bool hf[G];
#pragma unroll
        for (int r = 0; r < G; ++r) {
            ff zff;
            pix[r] = v0 + r < a.V ? view_pixel(a.cams + 16 * (v0 + r), p0, p1, p2, a0, a1, a2, a.W, a.H, f[r], zff,
                                               hf[r])
                                  : -1;
        }
        float2 dc[G];
#pragma unroll
        for (int r = 0; r < G; ++r)
            dc[r] = pix[r] >= 0 ? __ldg(a.dmap + (size_t)(v0 + r) * npx + pix[r]) : make_float2(0.0f, 0.0f);
#pragma unroll
        for (int r = 0; r < G; ++r) {
            if (pix[r] < 0) continue;
            int vis = hf[r] ? -1 : depth_test_fast(f[r].Z, f[r].eZ, dc[r].x, a.eps);
            if (vis < 0) {   // float-float depth (recomputed: rare, and cheaper than keeping it live)
                const float* cam = a.cams + 16 * (v0 + r);
                vis = depth_test_ff(ff_dot3_plus(cam[10], cam[11], cam[12], p0, p1, p2, cam[15]), dc[r].x, a.eps);
            }
            if (vis) top_insert(tk, tv, conf_key(dc[r].y), v0 + r);
        }
    }
    int nk = 0;
#pragma unroll
    for (int q = 0; q < K; ++q) {
        if (tk[q] != 0u) {
            s_tv[t][q] = tv[q];
            s_tc[t][q] = __uint_as_float(tk[q] - 1u);
            nk = q + 1;
        }
    }
    // per top view: the point's pixel position, its float-float depth, the offset pixel and its depth
    for (int q = 0; q < nk; ++q) {
        const int v = s_tv[t][q];
        const float* cam = a.cams + 16 * v;
        const FastProj f = fast_project(cam, p0, p1, p2, a0, a1, a2);
        const ff X2 = ff_dot3_plus(cam[10], cam[11], cam[12], p0, p1, p2, cam[15]);
        float fu, fv;
        const bool su = sure_floor(f.uf, f.mu, fu);
        const bool sure = sure_floor(f.wf, f.mw, fv) && su;
        ff u = {f.uf, 0.0f}, w = {f.wf, 0.0f};
        bool have_uw = false;
        if (!sure) {
            const ff X0 = ff_dot3_plus(cam[4], cam[5], cam[6], p0, p1, p2, cam[13]);
            const ff X1 = ff_dot3_plus(cam[7], cam[8], cam[9], p0, p1, p2, cam[14]);
            u = ff_affine(cam[0], ff_div(X0, X2), cam[2]);
            w = ff_affine(cam[1], ff_div(X1, X2), cam[3]);
            fu = ff_floor(u);
            fv = ff_floor(w);
            have_uw = true;
        }
        const float th = __ldg(&a.amap[(size_t)v * npx + (size_t)((int)fv * a.W + (int)fu)].x);
        float sn, cs;
        sincosf(th, &sn, &cs);
        const float lc = a.lambda * cs, ls = a.lambda * sn;
        // the offset pixel floor(u + lambda cos theta), floor(w + lambda sin theta)
        float gx, gy;
        bool osure = false;
        if (!have_uw) {
            const float ux = f.uf + lc, uy = f.wf + ls;
            const bool sx = sure_floor(ux, fmaf(fabsf(ux), 1.2e-7f, f.mu), gx);
            osure = sure_floor(uy, fmaf(fabsf(uy), 1.2e-7f, f.mw), gy) && sx;
        }
        if (!osure) {
            if (!have_uw) {
                const ff X0 = ff_dot3_plus(cam[4], cam[5], cam[6], p0, p1, p2, cam[13]);
                const ff X1 = ff_dot3_plus(cam[7], cam[8], cam[9], p0, p1, p2, cam[14]);
                u = ff_affine(cam[0], ff_div(X0, X2), cam[2]);
                w = ff_affine(cam[1], ff_div(X1, X2), cam[3]);
            }
            gx = ff_floor(ff_add(u, ff{lc, 0.0f}));
            gy = ff_floor(ff_add(w, ff{ls, 0.0f}));
        }
        float zc = __int_as_float(0x7f800000);   // no depth outside the image
        if (gx >= 0.0f && gx < (float)a.W && gy >= 0.0f && gy < (float)a.H)
            zc = __ldg(&a.dmap[(size_t)v * npx + (size_t)((int)gy * a.W + (int)gx)].x);
        float4* r = a.rec + ((size_t)i * a.K + q) * 3;
        r[0] = make_float4(__int_as_float(v), s_tc[t][q], fu, fv);
        r[1] = make_float4(u.hi + u.lo, w.hi + w.lo, lc, ls);
        r[2] = make_float4(X2.hi, X2.lo, zc, __int_as_float(nk));
    }
    write_empty_records(a, i, nk, nk);
}

// ------------------------------------------------------------------ k_fpmvo_fuse: a warp per point
// From the records of the point's top views: the P x P patches (each lane loads a patch row), the
// candidates of Eqs. 2-3 (lane c = s K + j: top view j, depth sample s), the medoid of each depth layer
// (Eqs. G, sigma), the patch consistency of each layer's fused offset point in each top view (Eqs.
// proj_r, sim, patchloss, patch_min), the mean over the views, the best layer and the outputs.
constexpr int kFuseWarps = 4;
__constant__ int c_div256[HF_FPMVO_MAX_K + 1] = {0, 256, 128, 86, 64, 52, 43, 37, 32};   // ceil(256 / n)
// One point of k_fpmvo_fuse, by one warp.  nk: its number of top views; R0, R1, R2: lane j < K
// holds the record of top view j (zeros for j >= nk); cand, offs, slot0, patch: the warp's shared
// memory.  KT, ST: K and S when fixed at compile time (the paper's configuration), 0 to read them.
// Lane groups are K wide whatever nk is: a lane j >= nk has no candidate (weight 0, so it adds
// nothing to the weighted sums) and a patch term of 0 (so the view sums are those over nk views).
template <int P, int KT, int ST>
__device__ __forceinline__ void fuse_point(const FpmvoArgs& a, int i, int nk, const float4& R0, const float4& R1,
                                           const float4& R2, float4* cand, float4* offs, float4* slot0, float2* patch,
                                           int lane) {
    constexpr int P2 = P * P, h = P / 2;
    const int K = KT ? KT : a.K, S = ST ? ST : a.S;
    if (nk <= 0) {   // -1: non-finite point; 0: no view sees it
        if (lane == 0) {
            a.dir_out[3 * i] = a.dir_out[3 * i + 1] = a.dir_out[3 * i + 2] = 0.0f;
            if (a.cost_out) a.cost_out[i] = nk < 0 ? __int_as_float(0x7fc00000) : 1.0f;
            if (a.sel_out) a.sel_out[i] = -1;
            if (a.status_out) a.status_out[i] = nk < 0 ? HF_STATUS_BAD_INPUT : HF_STATUS_NO_VIEWS;
        }
        return;
    }
    const size_t npx = (size_t)a.W * a.H;
    const float p0 = __ldg(a.pts + 3 * i), p1 = __ldg(a.pts + 3 * i + 1), p2 = __ldg(a.pts + 3 * i + 2);
    if (lane < nk) slot0[lane] = R0;
    __syncwarp();
    // the P x P patches of C (cos theta, sin theta) around the point's pixel in every top view, 0
    // outside the image: consecutive lanes take consecutive pixels of a row, four loads in flight
    const int npatch = nk * P2;
    for (int e0 = 0; e0 < npatch; e0 += 128) {
        float2 pv[4];
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const int e = e0 + lane + 32 * r;
            pv[r] = make_float2(0.0f, 0.0f);
            if (e < npatch) {
                const int j = e / P2, q = e - j * P2;
                const int dy = q / P, dx = q - dy * P;
                const float4 r0 = slot0[j];
                const int x = (int)r0.z + dx - h, y = (int)r0.w + dy - h;
                if (x >= 0 && y >= 0 && x < a.W && y < a.H)
                    pv[r] = __ldg(a.vmap + (size_t)__float_as_int(r0.x) * npx + (size_t)(y * a.W + x));
            }
        }
#pragma unroll
        for (int r = 0; r < 4; ++r)
            if (e0 + lane + 32 * r < npatch) patch[e0 + lane + 32 * r] = pv[r];
    }
    // ---- candidates (Eqs. 2-3)
    const int nc = K * S;
    // s = lane / K (as (lane ceil(256 / K)) >> 8 when K is not fixed: exact for lane < 32, K <= 8)
    const int s = KT ? lane / KT : (lane * c_div256[K]) >> 8, j = lane - s * K;   // meaningful for lane < nc
    const bool cand_lane = lane < nc && j < nk;
    const int srcj = lane < nc ? j : 0;
    const int vj = __float_as_int(__shfl_sync(0xffffffffu, R0.x, srcj));
    // the camera of view j: (fx, fy, cx, cy), R rows, t
    const float4* cq = reinterpret_cast<const float4*>(a.cams) + 4 * vj;
    const float4 c0 = __ldg(cq), c1 = __ldg(cq + 1), c2 = __ldg(cq + 2), c3 = __ldg(cq + 3);
    const float fx = c0.x, fy = c0.y, cx = c0.z, cy = c0.w;
    const float r00 = c1.x, r01 = c1.y, r02 = c1.z, r10 = c1.w, r11 = c2.x, r12 = c2.y, r20 = c2.z, r21 = c2.w,
                r22 = c3.x, t0 = c3.y, t1 = c3.z;
    const float wj = __shfl_sync(0xffffffffu, R0.y, srcj);
    const float bu = __shfl_sync(0xffffffffu, R1.x, srcj), bw = __shfl_sync(0xffffffffu, R1.y, srcj);
    const float blc = __shfl_sync(0xffffffffu, R1.z, srcj), bls = __shfl_sync(0xffffffffu, R1.w, srcj);
    const float bzh = __shfl_sync(0xffffffffu, R2.x, srcj), bzl = __shfl_sync(0xffffffffu, R2.y, srcj);
    const float bz = __shfl_sync(0xffffffffu, R2.z, srcj);
    float e0 = 0.0f, e1 = 0.0f, e2 = 0.0f;
    bool cok = false;
    float4 cd = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    if (cand_lane && isfinite(bz)) {
        const float ds = a.ds[s];
        const float zs = bz + ds;
        // the offset in camera coordinates without cancellation: with Zp the point's depth,
        // X_cand - X_p = ((lambda c zs + (u - cx)(zs - Zp)) / fx, (lambda s zs + (w - cy)(zs - Zp)) / fy,
        // zs - Zp), and zs - Zp = (z - Zp.hi) - Zp.lo + delta_s (the first difference is exact)
        const float dz = __fadd_rn(__fsub_rn(__fsub_rn(bz, bzh), bzl), ds);
        const float Y0 = __fdividef(fmaf(blc, zs, (bu - cx) * dz), fx);
        const float Y1 = __fdividef(fmaf(bls, zs, (bw - cy) * dz), fy);
        // world offset e = R^T Y
        e0 = fmaf(r00, Y0, fmaf(r10, Y1, r20 * dz));
        e1 = fmaf(r01, Y0, fmaf(r11, Y1, r21 * dz));
        e2 = fmaf(r02, Y0, fmaf(r12, Y1, r22 * dz));
        const float n2 = fmaf(e0, e0, fmaf(e1, e1, e2 * e2));
        if (n2 > 1e-24f) {
            const float rn = rsqrtf(n2);
            cd = make_float4(e0 * rn, e1 * rn, e2 * rn, wj);
            cok = true;
        }
    }
    cand[lane] = cd;   // an invalid candidate has weight 0 and adds nothing below
    offs[lane] = make_float4(e0, e1, e2, 0.0f);
    __syncwarp();
    // ---- medoid of group s: sigma = sum_k w_k |<d, d_k>| / sum_k w_k over the group's candidates
    // (the members of a group share the denominator, so the numerators decide; a zero weight sum
    // makes every numerator 0 and the first candidate wins, as sigma = 0 would)
    const int g0 = lane < nc ? s * K : 0;
    float num = 0.0f;
#pragma unroll
    for (int k = 0; k < K; ++k) {
        const float4 q = cand[g0 + k];
        num = fmaf(q.w, fabsf(fmaf(cd.x, q.x, fmaf(cd.y, q.y, cd.z * q.z))), num);
    }
    const float sigma = cok ? num : -1.0f;
    int med = -1;   // lane of the group's medoid
    float msig = -1.0f;
#pragma unroll
    for (int k = 0; k < K; ++k) {
        const float sk = __shfl_sync(0xffffffffu, sigma, g0 + k);
        if (sk > msig) {
            msig = sk;
            med = g0 + k;
        }
    }
    const bool layer_ok = lane < nc && msig >= 0.0f;   // the layer has a candidate
    // the fused offset point of layer s, as an offset from p
    const float4 fo = offs[med >= 0 ? med : 0];
    // ---- patch consistency of layer s in view j
    float Lv = 0.0f;
    if (layer_ok && j < nk) {
        const float X0 = fmaf(r00, p0, fmaf(r01, p1, fmaf(r02, p2, t0)));
        const float X1 = fmaf(r10, p0, fmaf(r11, p1, fmaf(r12, p2, t1)));
        const float Z = bzh;
        const float q0 = fmaf(r00, fo.x, fmaf(r01, fo.y, r02 * fo.z));
        const float q1 = fmaf(r10, fo.x, fmaf(r11, fo.y, r12 * fo.z));
        const float q2 = fmaf(r20, fo.x, fmaf(r21, fo.y, r22 * fo.z));
        const float Zf = Z + q2;
        if (Zf > 1e-6f) {
            // Pi(p + f) - Pi(p) = fx (Z q_x - X_x q_z) / (Z Z_f), ...: the positive factor 1 / (Z Z_f)
            // drops out of the normalised direction and moves to the other side of the degeneracy test
            const float rx = fx * fmaf(Z, q0, -X0 * q2), ry = fy * fmaf(Z, q1, -X1 * q2);
            const float rn2 = fmaf(rx, rx, ry * ry);
            const float en2 = fmaf(fo.x, fo.x, fmaf(fo.y, fo.y, fo.z * fo.z));
            if (rn2 >= 1e-20f * fmaf(fx, fx, fy * fy) * en2 * (Zf * Zf)) {
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
    // (every layer divides by the same nk, so the sums decide; lane 0 divides the best one)
    float lsum = 0.0f;
#pragma unroll
    for (int k = 0; k < K; ++k) lsum += __shfl_sync(0xffffffffu, Lv, g0 + k);
    const float lbar = layer_ok ? lsum : -1.0f;
    // ---- the best layer (lowest s on ties) and the outputs
    float best = -1.0f;
    int bs = -1;
#pragma unroll
    for (int q = 0; q < S; ++q) {
        const float lq = __shfl_sync(0xffffffffu, lbar, q * K);
        if (lq > best) {
            best = lq;
            bs = q;
        }
    }
    // the best layer's fused offset: that of the medoid lane of group bs
    const int osrc = __shfl_sync(0xffffffffu, med, bs >= 0 ? bs * K : 0);
    if (lane == 0) {
        if (bs < 0) {
            a.dir_out[3 * i] = a.dir_out[3 * i + 1] = a.dir_out[3 * i + 2] = 0.0f;
            if (a.cost_out) a.cost_out[i] = 1.0f;
            if (a.sel_out) a.sel_out[i] = -1;
            if (a.status_out) a.status_out[i] = HF_STATUS_NO_VIEWS;
        } else {
            const float4 o = offs[osrc >= 0 ? osrc : 0];
            const float rn = rsqrtf(fmaf(o.x, o.x, fmaf(o.y, o.y, o.z * o.z)));
            const float x0 = o.x * rn, x1 = o.y * rn, x2 = o.z * rn;
            const float sgn = fabsf(x2) > 1e-12f ? copysignf(1.0f, x2)
                              : fabsf(x1) > 1e-12f ? copysignf(1.0f, x1) : copysignf(1.0f, x0);
            a.dir_out[3 * i] = sgn * x0;
            a.dir_out[3 * i + 1] = sgn * x1;
            a.dir_out[3 * i + 2] = sgn * x2;
            if (a.cost_out) a.cost_out[i] = 1.0f - best / (float)nk;
            if (a.sel_out) a.sel_out[i] = bs;
            if (a.status_out) a.status_out[i] = HF_STATUS_OK;
        }
    }
}

template <int P, int KT, int ST>
__global__ void __launch_bounds__(kFuseWarps * 32) k_fpmvo_fuse(FpmvoArgs a) {
    constexpr int P2 = P * P;
    extern __shared__ __align__(16) float4 fu_smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int i = blockIdx.x * kFuseWarps + warp;
    if (i >= a.N) return;   // whole warp
    const int K = a.K;
    // per warp: 32 candidates (unit direction, weight), 32 offsets e, the first record word of each
    // top view, K x P2 patch float2
    float4* cand = fu_smem + (size_t)warp * (64 + HF_FPMVO_MAX_K + (K * P2 + 1) / 2);
    float4* offs = cand + 32;
    float4* slot0 = offs + 32;
    float2* patch = reinterpret_cast<float2*>(slot0 + HF_FPMVO_MAX_K);
    // every point has K records, so they load without waiting for the count (in record 0)
    float4 R0 = make_float4(0.0f, 0.0f, 0.0f, 0.0f), R1 = R0, R2 = R0;
    if (lane < K) {
        const float4* r = a.rec + ((size_t)i * K + lane) * 3;
        R0 = __ldg(r);
        R1 = __ldg(r + 1);
        R2 = __ldg(r + 2);
    }
    const int nk = __float_as_int(__shfl_sync(0xffffffffu, R2.w, 0));
    fuse_point<P, KT, ST>(a, i, nk, R0, R1, R2, cand, offs, slot0, patch, lane);
}

template <int P, int KT = 0, int ST = 0>
cudaError_t launch_fpmvo_fuse(const FpmvoArgs& a, cudaStream_t s) {
    const size_t smem = (size_t)kFuseWarps * (64 + HF_FPMVO_MAX_K + (a.K * P * P + 1) / 2) * sizeof(float4);
    k_fpmvo_fuse<P, KT, ST><<<(a.N + kFuseWarps - 1) / kFuseWarps, kFuseWarps * 32, smem, s>>>(a);
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

cudaError_t hf_launch_fpmvo_views(const FpmvoArgs& a, cudaStream_t s) {
    const unsigned vb = (unsigned)((a.N + kViewsThreads - 1) / kViewsThreads);
    switch (a.K) {
        case 1: k_fpmvo_views<1><<<vb, kViewsThreads, 0, s>>>(a); break;
        case 2: k_fpmvo_views<2><<<vb, kViewsThreads, 0, s>>>(a); break;
        case 3: k_fpmvo_views<3><<<vb, kViewsThreads, 0, s>>>(a); break;
        case 4: k_fpmvo_views<4><<<vb, kViewsThreads, 0, s>>>(a); break;
        case 5: k_fpmvo_views<5><<<vb, kViewsThreads, 0, s>>>(a); break;
        case 6: k_fpmvo_views<6><<<vb, kViewsThreads, 0, s>>>(a); break;
        case 7: k_fpmvo_views<7><<<vb, kViewsThreads, 0, s>>>(a); break;
        case 8: k_fpmvo_views<8><<<vb, kViewsThreads, 0, s>>>(a); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t hf_launch_fpmvo_fuse(const FpmvoArgs& a, cudaStream_t s) {
    switch (a.P) {
        case 1: return launch_fpmvo_fuse<1>(a, s);
        case 3: return launch_fpmvo_fuse<3>(a, s);
        case 5: return a.K == 5 && a.S == 5 ? launch_fpmvo_fuse<5, 5, 5>(a, s) : launch_fpmvo_fuse<5>(a, s);
        case 7: return launch_fpmvo_fuse<7>(a, s);
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
    // depth samples delta_s = -Delta + 2 Delta s / (S - 1), s = 0 .. S-1 (0 for S = 1), in double
    float ds[32];
    for (int q = 0; q < 32; ++q)
        ds[q] = q < g.S && g.S > 1 ? (float)(-(double)g.delta + 2.0 * (double)g.delta * q / (g.S - 1)) : 0.0f;
    if ((rc = hf_ensure(c, c->fprec, (size_t)N * g.K * 3 * sizeof(float4)))) return rc;
    FpmvoArgs a{(const float*)c->pts.p, N, (const float*)c->cams.p, c->V, c->W, c->Hh, (const float2*)c->amap.p,
                (const float2*)c->dmap.p, (const float2*)c->vmap.p, (float4*)c->fprec.p, g.K, g.S, g.P, g.lambda_px, g.delta, g.eps_vis,
                d_dir, d_cost, d_sel, d_st};
    memcpy(a.ds, ds, sizeof(ds));
    if ((rc = run_launch(c, "k_fpmvo_views", [&] { return hf_launch_fpmvo_views(a, c->stream); }))) return rc;
    if ((rc = run_launch(c, "k_fpmvo_fuse", [&] { return hf_launch_fpmvo_fuse(a, c->stream); }))) return rc;
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
