// hf_cost.cuh - device code of the cost kernels (K2 + K3, the learned path's proposal cost and
// short refinement, the cost of given directions), shared by the single-scene kernels
// (hf_kernels.cu) and the batched persistent kernels (hf_batch_kernels.cu).
#pragma once

#include "hf_internal.cuh"

namespace hf_cost {

// ------------------------------------------------------------------ K2 + K3: the cost kernels
//
// A point is served by a group of L lanes (L in {4, 8, 16, 32}; 32 / L points per warp).  The views
// of the point's view set V_i, in view order, are dealt to the lanes in pairs: member n of V_i goes
// to lane n mod L; a lane holds NP pairs (a, b) of views.  Per chunk of 2 NP L views a lane gathers,
// for each of its views, the projection Jacobian at the point (single precision, scaled by Z, which
// cancels), the view's degenerate threshold and the samples C (cos theta, sin theta) of the k + 1
// patch members at their own pixels, and packs the two views of a pair into the two halves of
// f32x2 registers.  With one chunk (the usual case) these stay in registers while every direction
// is evaluated: the H hypotheses, then the T rounds of six rotations.  Each packed instruction
// (fma.rn.f32x2 / mul.rn.f32x2, each half rounded exactly like the scalar instruction) serves both
// views of a pair; the patch maxima fold two or three absolute values per three-input max.f32.
// A direction's terms are summed over the lane's views, then over the group: for a batch of L
// directions a reduce-scatter of shuffles leaves lane l with the group total of direction l, the
// same bits in every lane that holds it.  Larger view sets are processed chunk by chunk (the chunk
// gathered again for every batch of directions).
//
// The patch term of a direction d in view v (Eqs. proj_r, sim, patchloss, patch_min):
//   r = J d (Z times the image offset), L_v = max_j |<r, s_j>| / |r|, 0 when |r|^2 < threshold.
// The cost is c = 1 - (sum_v L_v) / |V_i| (Eq. final_dout with the view mean); minimising c is
// maximising the sum, which the kernels compare.
typedef unsigned long long f32x2;
__device__ __forceinline__ f32x2 pk(float a, float b) {
    f32x2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ void upk(f32x2 r, float& a, float& b) { asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(r)); }
__device__ __forceinline__ f32x2 fma2(f32x2 a, f32x2 b, f32x2 c) {
    f32x2 d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
__device__ __forceinline__ f32x2 mul2(f32x2 a, f32x2 b) {
    f32x2 d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
// max(m, |a|, |b|), max(|a|, |b|, |c|), max(m, |a|)
__device__ __forceinline__ float max3abs(float m, float a, float b) {
    float r;
    asm("{ .reg .f32 t, u; abs.f32 t, %1; abs.f32 u, %2; max.f32 %0, %3, t, u; }" : "=f"(r) : "f"(a), "f"(b), "f"(m));
    return r;
}
__device__ __forceinline__ float max3abs3(float a, float b, float c) {
    float r;
    asm("{ .reg .f32 t, u, v; abs.f32 t, %1; abs.f32 u, %2; abs.f32 v, %3; max.f32 %0, t, u, v; }"
        : "=f"(r) : "f"(a), "f"(b), "f"(c));
    return r;
}
__device__ __forceinline__ float max2abs(float m, float a) {
    float r;
    asm("{ .reg .f32 t; abs.f32 t, %1; max.f32 %0, %2, t; }" : "=f"(r) : "f"(a), "f"(m));
    return r;
}

// 1/sqrt(x) by the special-function unit: rsqrt.approx with subnormal inputs flushed to zero.  The
// patch term uses it only for |r|^2 at or above the degenerate threshold 1e-20 (fx^2 + fy^2), far
// above the subnormal range, where the flush changes nothing.
__device__ __forceinline__ float rsqrt_ftz(float x) {
    float r;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// Two views of the point held by a lane, view a in the low and view b in the high half.
template <int KP>
struct VPair {
    f32x2 j0, j1, j2, j3, j4, j5;   // rows of Z x the projection Jacobian: fx (R_0 - a R_2), fy (R_1 - b R_2)
    f32x2 thr;                      // degenerate thresholds of the views; +inf for an empty view
    f32x2 sx[KP], sy[KP];           // member samples C cos theta, C sin theta
};

// A direction broadcast to both halves.
struct Dir2 {
    f32x2 x, y, z;
};
__device__ __forceinline__ Dir2 dir2(float a, float b, float c) { return Dir2{pk(a, a), pk(b, b), pk(c, c)}; }

// max_j |u_j| of one half, u from the members' products
template <int KP>
__device__ __forceinline__ float patch_max(const float (&u)[KP]) {
    if (KP == 1) return fabsf(u[0]);
    if (KP == 2) return max2abs(fabsf(u[0]), u[1]);
    float m = max3abs3(u[0], u[1], u[2]);
#pragma unroll
    for (int j = 3; j + 1 < KP; j += 2) m = max3abs(m, u[j], u[j + 1]);
    if (KP > 3 && ((KP - 3) & 1)) m = max2abs(m, u[KP - 1]);
    return m;
}

// L_a + L_b of direction d in the lane's two views.  TS: thresholds scaled by tscale (directions of
// any length).
template <int KP, bool TS>
__device__ __forceinline__ float pair_term(const VPair<KP>& p, const Dir2& d, float tscale) {
    const f32x2 RX = fma2(p.j0, d.x, fma2(p.j1, d.y, mul2(p.j2, d.z)));
    const f32x2 RY = fma2(p.j3, d.x, fma2(p.j4, d.y, mul2(p.j5, d.z)));
    const f32x2 R2 = fma2(RX, RX, mul2(RY, RY));
    float ua[KP], ub[KP];
#pragma unroll
    for (int j = 0; j < KP; ++j) upk(fma2(RX, p.sx[j], mul2(RY, p.sy[j])), ua[j], ub[j]);
    const float ma = patch_max<KP>(ua), mb = patch_max<KP>(ub);
    float ra, rb, ta, tb;
    upk(R2, ra, rb);
    upk(p.thr, ta, tb);
    if (TS) {
        ta = __fmul_rn(ta, tscale);
        tb = __fmul_rn(tb, tscale);
    }
    const float La = ra >= ta ? __fmul_rn(ma, rsqrt_ftz(ra)) : 0.0f;
    const float Lb = rb >= tb ? __fmul_rn(mb, rsqrt_ftz(rb)) : 0.0f;
    return __fadd_rn(La, Lb);
}

// the n-th (from 0) set bit of a mask word
__device__ __forceinline__ int nth_bit(unsigned long long x, int n) {
    const unsigned lo = (unsigned)x, hi = (unsigned)(x >> 32);
    const int cl = __popc(lo);
    return n < cl ? (int)__fns(lo, 0, n + 1) : 32 + (int)__fns(hi, 0, n - cl + 1);
}

// the view of member n of a point's view set, or -1
__device__ __forceinline__ int nth_view(const CostArgs& a, int i, unsigned long long w0, int n) {
    if (a.Vw == 1) return n < __popcll(w0) ? nth_bit(w0, n) : -1;
    const unsigned long long* m = a.vmask + (size_t)i * a.Vw;
    for (int w = 0; w < a.Vw; ++w) {
        const unsigned long long x = w ? m[w] : w0;
        const int c = __popcll(x);
        if (n < c) return 64 * w + nth_bit(x, n);
        n -= c;
    }
    return -1;
}

// Per-point state of a lane's group.
template <int KP>
struct PointCtx {
    int i;           // point index (0 for a group without a point)
    bool in;         // the group has a point
    bool finite;     // its coordinates are finite
    int nv;          // |V_i|
    unsigned long long w0;   // first mask word
    float p0, p1, p2;
    int nb[KP];      // patch members: the point, its neighbours, -1 past k
};

template <int KP>
__device__ __forceinline__ void point_ctx(const CostArgs& a, int q, int cnt, PointCtx<KP>& pc) {
    pc.in = q < cnt;
    pc.i = pc.in ? (a.list ? a.list[q] : q) : 0;
    const int i = pc.i;
    pc.p0 = a.pts[3 * i];
    pc.p1 = a.pts[3 * i + 1];
    pc.p2 = a.pts[3 * i + 2];
    pc.finite = pc.in && isfinite(pc.p0) && isfinite(pc.p1) && isfinite(pc.p2);
    pc.w0 = pc.finite ? a.vmask[(size_t)i * a.Vw] : 0ull;
    int nv = __popcll(pc.w0);
    if (pc.finite)
        for (int w = 1; w < a.Vw; ++w) nv += __popcll(a.vmask[(size_t)i * a.Vw + w]);
    pc.nv = nv;
    pc.nb[0] = pc.finite ? i : -1;
#pragma unroll
    for (int j = 1; j < KP; ++j) pc.nb[j] = (pc.finite && (j - 1) < a.k) ? a.nbr[(size_t)i * a.k + (j - 1)] : -1;
}

// One view of the point: Jacobian rows, threshold and member samples (zeros and +inf when v < 0).
template <int KP>
__device__ __forceinline__ void view_data(const CostArgs& a, const PointCtx<KP>& pc, int v, float (&j)[6], float& thr,
                                          float2 (&sm)[KP]) {
    if (v < 0) {
#pragma unroll
        for (int q = 0; q < 6; ++q) j[q] = 0.0f;
        thr = INFINITY;
#pragma unroll
        for (int m = 0; m < KP; ++m) sm[m] = make_float2(0.0f, 0.0f);
        return;
    }
    const float* cam = a.cams + 16 * v;
    const float fx = __ldg(cam), fy = __ldg(cam + 1);
    const float r00 = __ldg(cam + 4), r01 = __ldg(cam + 5), r02 = __ldg(cam + 6);
    const float r10 = __ldg(cam + 7), r11 = __ldg(cam + 8), r12 = __ldg(cam + 9);
    const float r20 = __ldg(cam + 10), r21 = __ldg(cam + 11), r22 = __ldg(cam + 12);
    const float2 r = __ldg(a.ab + hf_pv(v, pc.i, a.N));
    const float ra = r.x, rb = r.y;
    j[0] = __fmul_rn(fx, fmaf(-ra, r20, r00));
    j[1] = __fmul_rn(fx, fmaf(-ra, r21, r01));
    j[2] = __fmul_rn(fx, fmaf(-ra, r22, r02));
    j[3] = __fmul_rn(fy, fmaf(-rb, r20, r10));
    j[4] = __fmul_rn(fy, fmaf(-rb, r21, r11));
    j[5] = __fmul_rn(fy, fmaf(-rb, r22, r12));
    thr = __ldg(a.vthr + v);
#pragma unroll
    for (int m = 0; m < KP; ++m)
        sm[m] = pc.nb[m] >= 0 ? __ldg(a.samp + hf_pv(v, pc.nb[m], a.N)) : make_float2(0.0f, 0.0f);
}

// Gather chunk `chunk` of the point's view set into the lane's NP view pairs (pairs >= np stay
// empty): view n = ((chunk NP + p) 2 + h) L + lg of V_i for pair p, half h.
template <int KP, int L, int NP>
__device__ __forceinline__ void gather(const CostArgs& a, const PointCtx<KP>& pc, int lg, int chunk, int np,
                                       VPair<KP> (&P)[NP]) {
#pragma unroll
    for (int p = 0; p < NP; ++p) {
        float ja[6], jb[6], ta, tb;
        float2 sa[KP], sb[KP];
        const int n0 = ((chunk * NP + p) * 2) * L + lg;
        const int va = (p < np && n0 < pc.nv) ? nth_view(a, pc.i, pc.w0, n0) : -1;
        const int vb = (p < np && n0 + L < pc.nv) ? nth_view(a, pc.i, pc.w0, n0 + L) : -1;
        view_data<KP>(a, pc, va, ja, ta, sa);
        view_data<KP>(a, pc, vb, jb, tb, sb);
        VPair<KP>& q = P[p];
        q.j0 = pk(ja[0], jb[0]);
        q.j1 = pk(ja[1], jb[1]);
        q.j2 = pk(ja[2], jb[2]);
        q.j3 = pk(ja[3], jb[3]);
        q.j4 = pk(ja[4], jb[4]);
        q.j5 = pk(ja[5], jb[5]);
        q.thr = pk(ta, tb);
#pragma unroll
        for (int m = 0; m < KP; ++m) {
            q.sx[m] = pk(sa[m].x, sb[m].x);
            q.sy[m] = pk(sa[m].y, sb[m].y);
        }
    }
}

// Reduce-scatter of N values over the L lanes of a group (N, L powers of two): afterwards the
// lane lg of the group holds, in v[0 .. max(N / L, 1)), the group totals of the values with index
// lg (N / L) + q when N >= L, or the total of value lg / (L / N) when N < L.  The order of the
// additions depends on the lane position only, so every lane holding a total has the same bits.
template <int N, int L>
__device__ __forceinline__ void reduce_scatter(float (&v)[N], int lg) {
#pragma unroll
    for (int t = 0; (1 << t) < L; ++t) {
        const int o = L >> (t + 1);
        const int c = N >> t;   // values held before this level
        if (c >= 2) {
            const bool up = (lg & o) != 0;
#pragma unroll
            for (int q = 0; q < c / 2; ++q) {
                const float send = up ? v[q] : v[q + c / 2];
                const float keep = up ? v[q + c / 2] : v[q];
                v[q] = __fadd_rn(keep, __shfl_xor_sync(0xffffffffu, send, o));
            }
        } else {
            v[0] = __fadd_rn(v[0], __shfl_xor_sync(0xffffffffu, v[0], o));
        }
    }
}

// The same reduction when lane lg has put the value of index q ^ perm(lg) into slot q, with
// perm(lg) = (lg / (L / N)) mod N for N <= L: every level keeps the lower half and sends the upper,
// so no selects are needed; afterwards v[0] is the total of index perm(lg).
template <int N, int L>
__device__ __forceinline__ int rs_perm(int lg) {
    return N <= L ? (lg / (L / N)) & (N - 1) : 0;
}
template <int N, int L>
__device__ __forceinline__ void reduce_scatter_perm(float (&v)[N]) {
    static_assert(N <= L, "one value per lane at most");
#pragma unroll
    for (int t = 0; (1 << t) < L; ++t) {
        const int o = L >> (t + 1);
        const int c = N >> t;
        if (c >= 2) {
#pragma unroll
            for (int q = 0; q < c / 2; ++q) v[q] = __fadd_rn(v[q], __shfl_xor_sync(0xffffffffu, v[q + c / 2], o));
        } else {
            v[0] = __fadd_rn(v[0], __shfl_xor_sync(0xffffffffu, v[0], o));
        }
    }
}

// Full group sum of one value.
template <int L>
__device__ __forceinline__ float group_sum(float x) {
#pragma unroll
    for (int o = 1; o < L; o <<= 1) x = __fadd_rn(x, __shfl_xor_sync(0xffffffffu, x, o));
    return x;
}

// Lane partial sums of ND directions get(0 .. ND) over the lane's views (with several chunks, each
// gathered here again).
template <int KP, int L, int NP, int ND, bool TS, typename Get>
__device__ __forceinline__ void lane_sums(const CostArgs& a, const PointCtx<KP>& pc, int lg, int nch, int np,
                                          VPair<KP> (&P)[NP], Get get, float tscale, float (&out)[ND]) {
#pragma unroll
    for (int q = 0; q < ND; ++q) out[q] = 0.0f;
    for (int c = 0; c < nch; ++c) {
        if (nch > 1) gather<KP, L, NP>(a, pc, lg, c, NP, P);
#pragma unroll
        for (int q = 0; q < ND; ++q) {
            const Dir2 dq = get(q);
#pragma unroll
            for (int p = 0; p < NP; ++p)
                if (p < np || nch > 1) out[q] = __fadd_rn(out[q], pair_term<KP, TS>(P[p], dq, tscale));
        }
    }
}

// Group geometry of the calling lane for tile `tile`: returns false when the whole warp is past
// the end of the work list (a warp-uniform exit).
struct Lanes {
    int lane, lg, g, q;   // lane, lane in group, group in warp, work-list position of the group
};
template <int L>
__device__ __forceinline__ bool lanes_of(int tile, int cnt, Lanes& ln) {
    ln.lane = threadIdx.x & 31;
    ln.lg = ln.lane & (L - 1);
    ln.g = ln.lane / L;
    constexpr int ppw = 32 / L;
    const int w = tile * (blockDim.x >> 5) + (threadIdx.x >> 5);
    ln.q = w * ppw + ln.g;
    return w * ppw < cnt;
}

// chunks and view pairs in use, uniform over the warp
template <int L, int NP>
__device__ __forceinline__ void chunking(int nv, int& nch, int& np) {
    constexpr int per = 2 * L * NP;
    nch = (int)__reduce_max_sync(0xffffffffu, (unsigned)((nv + per - 1) / per));
    np = (int)__reduce_max_sync(0xffffffffu, (unsigned)min(NP, (nv + 2 * L - 1) / (2 * L)));
    if (nch < 1) nch = 1;
}

__device__ __forceinline__ void write_bad(const CostArgs& a, int i) {
    const int o = i - a.out_first;   // output row
    a.dir_out[3 * o] = a.dir_out[3 * o + 1] = a.dir_out[3 * o + 2] = 0.0f;
    if (a.cost_out) a.cost_out[o] = __int_as_float(0x7fc00000);
    if (a.idx_out) a.idx_out[o] = -1;
    if (a.status_out) a.status_out[o] = HF_STATUS_BAD_INPUT;
}

// T rounds of six rotations of d by +-alpha about world x, y, z (in that order): move to the first
// strictly larger sum (the first strictly lower cost).  d is kept broadcast in both halves.
template <int KP, int L, int NP>
__device__ __forceinline__ void refine_rounds(const CostArgs& a, const PointCtx<KP>& pc, int lane, int lg, int nch,
                                              int np, VPair<KP> (&P)[NP], Dir2& d, float& best) {
    for (int t = 0; t < a.T; ++t) {
        const float2 cr = a.rot[t];
        const f32x2 C = pk(cr.x, cr.x), S = pk(cr.y, cr.y), nS = pk(-cr.y, -cr.y);
        // every product rounded once and added with an explicit fused multiply-add
        Dir2 cd[6];
        cd[0] = Dir2{d.x, fma2(C, d.y, mul2(nS, d.z)), fma2(S, d.y, mul2(C, d.z))};
        cd[1] = Dir2{d.x, fma2(C, d.y, mul2(S, d.z)), fma2(nS, d.y, mul2(C, d.z))};
        cd[2] = Dir2{fma2(C, d.x, mul2(S, d.z)), d.y, fma2(nS, d.x, mul2(C, d.z))};
        cd[3] = Dir2{fma2(C, d.x, mul2(nS, d.z)), d.y, fma2(S, d.x, mul2(C, d.z))};
        cd[4] = Dir2{fma2(C, d.x, mul2(nS, d.y)), fma2(S, d.x, mul2(C, d.y)), d.z};
        cd[5] = Dir2{fma2(C, d.x, mul2(S, d.y)), fma2(nS, d.x, mul2(C, d.y)), d.z};
        float s6[6], v[8];
        lane_sums<KP, L, NP, 6, false>(a, pc, lg, nch, np, P, [&](int q) { return cd[q]; }, 1.0f, s6);
#pragma unroll
        for (int q = 0; q < 6; ++q) v[q] = s6[q];
        v[6] = v[7] = 0.0f;
        reduce_scatter<8, L>(v, lg);
        // every lane fetches the six totals (candidate q sits at group lane q (L / 8), or for L = 4 at
        // lane q / 2, slot q % 2) and takes the same decision
        const int base = lane & ~(L - 1);
        float tot[6];
#pragma unroll
        for (int q = 0; q < 6; ++q) {
            if (L >= 8) tot[q] = __shfl_sync(0xffffffffu, v[0], base + q * (L / 8));
            else tot[q] = __shfl_sync(0xffffffffu, v[q & 1], base + (q >> 1));
        }
        int choice = -1;
#pragma unroll
        for (int q = 0; q < 6; ++q)
            if (tot[q] > best) {
                best = tot[q];
                choice = q;
            }
        if (choice >= 0) {
            // the chosen rotation again, rounded exactly as its candidate above: the rotated pair
            // (u, w) of components becomes (c u + sg w, -sg u + c w), the products rounded once
            const int ax = choice >> 1;
            const bool neg = choice & 1;
            const float sg = (neg != (ax == 1)) ? cr.y : -cr.y;
            float d0, d1, d2, x_;
            upk(d.x, d0, x_);
            upk(d.y, d1, x_);
            upk(d.z, d2, x_);
            const float u = ax == 0 ? d1 : d0, w = ax == 2 ? d1 : d2;
            const float u2 = fmaf(cr.x, u, __fmul_rn(sg, w)), w2 = fmaf(-sg, u, __fmul_rn(cr.x, w));
            if (ax == 0) {
                d1 = u2;
                d2 = w2;
            } else if (ax == 1) {
                d0 = u2;
                d2 = w2;
            } else {
                d0 = u2;
                d1 = w2;
            }
            d = dir2(d0, d1, d2);
        }
    }
}

// Normalised direction with the canonical sign, the cost, index and status of a point.
__device__ __forceinline__ void write_out(const CostArgs& a, int i, int nv, const Dir2& dd, float best, int idx) {
    float d0, d1, d2, x;
    upk(dd.x, d0, x);
    upk(dd.y, d1, x);
    upk(dd.z, d2, x);
    const float n = sqrtf(fmaf(d0, d0, fmaf(d1, d1, __fmul_rn(d2, d2))));
    d0 /= n;
    d1 /= n;
    d2 /= n;
    const float sgn = fabsf(d2) > 1e-12f ? copysignf(1.0f, d2) : fabsf(d1) > 1e-12f ? copysignf(1.0f, d1) : copysignf(1.0f, d0);
    const int o = i - a.out_first;   // output row
    a.dir_out[3 * o] = sgn * d0;
    a.dir_out[3 * o + 1] = sgn * d1;
    a.dir_out[3 * o + 2] = sgn * d2;
    if (a.cost_out) a.cost_out[o] = nv ? 1.0f - best / (float)nv : 1.0f;
    if (a.idx_out) a.idx_out[o] = idx;
    if (a.status_out) a.status_out[o] = a.fell_back ? HF_STATUS_FELL_BACK : (nv ? HF_STATUS_OK : HF_STATUS_NO_VIEWS);
}

// K3: T rounds of the refinement for the points of one tile, lanes over views.  The start is the
// argmin hypothesis hyps[best_idx[i]] (index output) or a given direction start_dir[i] (index -1);
// its sum is taken first, in the same summation order as the candidates.
template <int KP, int L, int NP>
__device__ __forceinline__ void refine_tile_l(const CostArgs& a, int tile) {
    const int cnt = a.list ? *a.list_count : a.N;
    Lanes ln;
    if (!lanes_of<L>(tile, cnt, ln)) return;
    PointCtx<KP> pc;
    point_ctx<KP>(a, ln.q, cnt, pc);
    int nch, np;
    chunking<L, NP>(pc.nv, nch, np);
    VPair<KP> P[NP];
    if (nch == 1) gather<KP, L, NP>(a, pc, ln.lg, 0, np, P);
    int idx = -1;
    float d0 = 1.0f, d1 = 0.0f, d2 = 0.0f;
    if (a.start_dir) {
        if (pc.finite) {
            d0 = a.start_dir[3 * pc.i];
            d1 = a.start_dir[3 * pc.i + 1];
            d2 = a.start_dir[3 * pc.i + 2];
        }
    } else {
        idx = pc.finite ? a.best_idx[pc.i] : 0;
        d0 = a.hyps[3 * idx];
        d1 = a.hyps[3 * idx + 1];
        d2 = a.hyps[3 * idx + 2];
    }
    Dir2 d = dir2(d0, d1, d2);
    float l0[1];
    lane_sums<KP, L, NP, 1, false>(a, pc, ln.lg, nch, np, P, [&](int) { return d; }, 1.0f, l0);
    float best = group_sum<L>(l0[0]);
    refine_rounds<KP, L, NP>(a, pc, ln.lane, ln.lg, nch, np, P, d, best);
    if (ln.lg != 0 || !pc.in) return;
    if (!pc.finite) {
        write_bad(a, pc.i);
        return;
    }
    write_out(a, pc.i, pc.nv, d, best, idx);
}

// view pairs per lane for a patch width
template <int KP>
struct PairsFor {
    static constexpr int value = 1;
};

// ---- shared-memory staging for the point-per-thread kernels (argmin, refinement)
__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void cp_async8(void* sdst, const void* gsrc) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(smem_addr(sdst)), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// Per-thread ring of S views of patch data: item 0 = the point's (a, b), items 1..KP = the patch
// samples; laid out [stage][item][thread] so a warp reads consecutive 8-byte words.  View v lives
// in stage v % S and is copied in S - 1 views ahead of its use.
constexpr int kRefineStages = 2;
constexpr int kCamStageViews = 64;    // camera rows staged per view block (a multiple of 2)
template <int KP, int NT>
struct PatchStage {
    float2 v[kRefineStages][KP + 1][NT];
};
// The refinement's ring holds view pairs: one 16-byte element per item for views 2q and 2q + 1.
template <int KP, int NT>
struct PairStage {
    float4 v[kRefineStages][KP + 1][NT];
};
template <int KP, int NT>
__host__ __device__ constexpr size_t refine_smem_bytes() {
    return sizeof(PairStage<KP, NT>) + (size_t)kCamStageViews * 3 * sizeof(float4);
}

__device__ __forceinline__ void cp_async16(void* sdst, const void* gsrc) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_addr(sdst)), "l"(gsrc) : "memory");
}

// Queue the copies of view pair q's patch data into stage st (16 bytes an item, L2 only; one commit
// group per call, also when the thread has nothing to copy).
template <int KP, int NT>
__device__ __forceinline__ void issue_pair(PairStage<KP, NT>& sg, int st, const float2* __restrict__ ab,
                                           const float2* __restrict__ samp, int q, int N, int i, const int (&nb)[KP],
                                           bool active) {
    const int t = threadIdx.x;
    if (active) {
        const float4* ab4 = reinterpret_cast<const float4*>(ab) + (size_t)q * N;
        const float4* sp4 = reinterpret_cast<const float4*>(samp) + (size_t)q * N;
        cp_async16(&sg.v[st][0][t], ab4 + i);
        cp_async16(&sg.v[st][1][t], sp4 + i);
#pragma unroll
        for (int j = 1; j < KP; ++j)
            if (nb[j] >= 0) cp_async16(&sg.v[st][1 + j][t], sp4 + nb[j]);
    }
    cp_async_commit();
}

// Queue the copies of one view's patch data into stage st (one commit group per call, also when
// the thread has nothing to copy, so that group counting stays uniform).
template <int KP, int NT>
__device__ __forceinline__ void issue_patch(PatchStage<KP, NT>& sg, int st, const float2* __restrict__ ab,
                                            const float2* __restrict__ samp, int v, int N, int i, const int (&nb)[KP],
                                            bool active) {
    const int t = threadIdx.x;
    if (active) {
        cp_async8(&sg.v[st][0][t], ab + hf_pv(v, i, N));
        cp_async8(&sg.v[st][1][t], samp + hf_pv(v, i, N));
#pragma unroll
        for (int j = 1; j < KP; ++j)
            if (nb[j] >= 0) cp_async8(&sg.v[st][1 + j][t], samp + hf_pv(v, nb[j], N));
    }
    cp_async_commit();
}

// ------------------------------------------------------------------ K2: thread per point
// The cost of every hypothesis and the argmin (largest sum, lowest index on ties), a point per
// thread.  Hypotheses are evaluated in pairs: the packed instructions carry hypotheses m and m + 1
// of one view, with the view's patch samples broadcast to both halves.  The hypothesis table of a
// chunk of HC hypotheses x a block of views and the views' camera rows sit in shared memory
// (read by all threads at the same address); the next view's ratios (a, b) and k + 1 samples are
// copied into shared memory (cp.async) while the current view is evaluated.
//   qtab[v][2p]     = (fx q_x(2p), fx q_x(2p+1), fx q_z(2p), fx q_z(2p+1)),  q = R_v h
//   qtab[v][2p + 1] = (fy q_y(2p), fy q_y(2p+1), fy q_z(2p), fy q_z(2p+1))
//   r = (fx q_x - a fx q_z, fy q_y - b fy q_z) = Z times the image offset of h
constexpr int kArgminHC = 32;   // hypotheses per chunk
constexpr int kArgminVB = 32;   // views per staged block
template <int KP, int NT>
__host__ __device__ constexpr size_t argmin_smem_bytes() {
    return sizeof(PatchStage<KP, NT>) + (size_t)kArgminVB * kArgminHC * sizeof(float4) + (size_t)kArgminVB * sizeof(float);
}

template <int KP, int NT>
__device__ __forceinline__ void argmin_tile(const CostArgs& a, int blk, unsigned char* smem) {
    constexpr int HC = kArgminHC, VB = kArgminVB, S = kRefineStages;
    PatchStage<KP, NT>& sg = *reinterpret_cast<PatchStage<KP, NT>*>(smem);
    float4* qs = reinterpret_cast<float4*>(smem + sizeof(PatchStage<KP, NT>));                        // [VB][HC]
    float* ts = reinterpret_cast<float*>(smem + sizeof(PatchStage<KP, NT>) + (size_t)VB * HC * sizeof(float4));   // [VB]
    const int tid = threadIdx.x;
    const int cnt = a.list ? *a.list_count : a.N;
    if (blk * NT >= cnt) return;   // whole block past the list: uniform exit
    const int q = blk * NT + tid;
    const bool in = q < cnt;
    const int i = in ? (a.list ? a.list[q] : q) : 0;
    const float p0 = a.pts[3 * i], p1 = a.pts[3 * i + 1], p2 = a.pts[3 * i + 2];
    const bool active = in && isfinite(p0) && isfinite(p1) && isfinite(p2);
    int nb[KP];
    nb[0] = active ? i : -1;
#pragma unroll
    for (int j = 1; j < KP; ++j) nb[j] = (active && (j - 1) < a.k) ? a.nbr[(size_t)i * a.k + (j - 1)] : -1;
    // padded / inactive members read as zero samples in every stage, never overwritten
#pragma unroll
    for (int j = 1; j < KP; ++j)
        if (nb[j] < 0)
#pragma unroll
            for (int st = 0; st < S; ++st) sg.v[st][1 + j][tid] = make_float2(0.0f, 0.0f);
    float best = -1.0f;
    int bm = 0;
    for (int c0 = 0; c0 < a.Hq; c0 += HC) {
        float acc[HC];
#pragma unroll
        for (int m = 0; m < HC; ++m) acc[m] = 0.0f;
        for (int p = 0; p < S - 1; ++p)
            if (p < a.V) issue_patch<KP, NT>(sg, p, a.ab, a.samp, p, a.N, i, nb, active);
            else cp_async_commit();
        for (int vb = 0; vb < a.V; vb += VB) {
            const int nvb = min(VB, a.V - vb);
            __syncthreads();
            for (int e = tid; e < nvb * HC; e += NT) qs[e] = a.qtab[(size_t)(vb + e / HC) * a.Hq + c0 + e % HC];
            for (int e = tid; e < nvb; e += NT) ts[e] = a.vthr[vb + e];
            __syncthreads();
            for (int v = vb; v < vb + nvb; ++v) {
                const int vn = v + S - 1;
                if (vn < a.V) issue_patch<KP, NT>(sg, vn % S, a.ab, a.samp, vn, a.N, i, nb, active);
                else cp_async_commit();
                cp_async_wait<S - 1>();
                if (!active) continue;
                const int st = v % S;
                const float2 r = sg.v[st][0][tid];
                if (r.x != r.x) continue;   // v is not in the point's view set
                const float thr = ts[v - vb];
                f32x2 SX[KP], SY[KP];
#pragma unroll
                for (int j = 0; j < KP; ++j) {
                    const float2 sj = sg.v[st][1 + j][tid];
                    SX[j] = pk(sj.x, sj.x);
                    SY[j] = pk(sj.y, sj.y);
                }
                const f32x2 NA = pk(-r.x, -r.x), NB = pk(-r.y, -r.y);
                const f32x2* qv = reinterpret_cast<const f32x2*>(qs + (v - vb) * HC);
#pragma unroll
                for (int m = 0; m < HC; m += 2) {
                    const f32x2 RX = fma2(NA, qv[2 * m + 1], qv[2 * m]);
                    const f32x2 RY = fma2(NB, qv[2 * m + 3], qv[2 * m + 2]);
                    const f32x2 R2 = fma2(RX, RX, mul2(RY, RY));
                    float u0[KP], u1[KP];
#pragma unroll
                    for (int j = 0; j < KP; ++j) upk(fma2(RX, SX[j], mul2(RY, SY[j])), u0[j], u1[j]);
                    const float m0 = patch_max<KP>(u0), m1 = patch_max<KP>(u1);
                    float r0, r1;
                    upk(R2, r0, r1);
                    acc[m] = __fadd_rn(acc[m], r0 >= thr ? __fmul_rn(m0, rsqrt_ftz(r0)) : 0.0f);
                    acc[m + 1] = __fadd_rn(acc[m + 1], r1 >= thr ? __fmul_rn(m1, rsqrt_ftz(r1)) : 0.0f);
                }
            }
        }
        cp_async_wait<0>();
#pragma unroll
        for (int m = 0; m < HC; ++m)
            if (c0 + m < a.H && acc[m] > best) {
                best = acc[m];
                bm = c0 + m;
            }
    }
    if (in) a.best_idx[i] = bm;
}

// Patch terms of two directions (the packed halves of rx, ry) in one view, samples broadcast.
template <int KP>
__device__ __forceinline__ void view_term2(f32x2 rx, f32x2 ry, const f32x2 (&SX)[KP], const f32x2 (&SY)[KP], float thr,
                                           float& L0, float& L1) {
    const f32x2 r2 = fma2(rx, rx, mul2(ry, ry));
    float u0[KP], u1[KP];
#pragma unroll
    for (int j = 0; j < KP; ++j) upk(fma2(rx, SX[j], mul2(ry, SY[j])), u0[j], u1[j]);
    const float m0 = patch_max<KP>(u0), m1 = patch_max<KP>(u1);
    float a0, a1;
    upk(r2, a0, a1);
    L0 = a0 >= thr ? __fmul_rn(m0, rsqrt_ftz(a0)) : 0.0f;
    L1 = a1 >= thr ? __fmul_rn(m1, rsqrt_ftz(a1)) : 0.0f;
}

// K3, a point per thread: T rounds of the refinement from hyps[best_idx[i]] (index output) or
// start_dir[i] (index -1).  Per round every view of the point's set is visited once, in view order:
// the patch data of the next view pair is copied into shared memory (cp.async, 16 bytes an item
// for the two views) while the current pair's two views are evaluated; the Jacobian rows come from
// the staged camera rows and the point's ratios (a, b); the two candidates of one axis (+alpha,
// -alpha) are evaluated as a packed pair with the samples broadcast to both halves.  Round 0 also
// evaluates the start (paired with itself), so that every compared sum is taken in the same order.
template <int KP, int NT>
__device__ __forceinline__ void refine_stage_tile(const CostArgs& a, int blk, unsigned char* smem_raw) {
    constexpr int S = kRefineStages;
    PairStage<KP, NT>& sg = *reinterpret_cast<PairStage<KP, NT>*>(smem_raw);
    float4* cs4 = reinterpret_cast<float4*>(smem_raw + sizeof(PairStage<KP, NT>));   // [view in block][3]
    const int tid = threadIdx.x;
    const int cnt = a.list ? *a.list_count : a.N;
    if (blk * NT >= cnt) return;   // whole block past the list: uniform exit
    const int q = blk * NT + tid;
    const bool in = q < cnt;
    const int i = in ? (a.list ? a.list[q] : q) : 0;
    const float p0 = a.pts[3 * i], p1 = a.pts[3 * i + 1], p2 = a.pts[3 * i + 2];
    const bool active = in && isfinite(p0) && isfinite(p1) && isfinite(p2);
    int nb[KP];
    nb[0] = active ? i : -1;
#pragma unroll
    for (int j = 1; j < KP; ++j) nb[j] = (active && (j - 1) < a.k) ? a.nbr[(size_t)i * a.k + (j - 1)] : -1;
    // padded / inactive members read as zero samples in every stage, never overwritten
#pragma unroll
    for (int j = 1; j < KP; ++j)
        if (nb[j] < 0)
#pragma unroll
            for (int st = 0; st < S; ++st) sg.v[st][1 + j][tid] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    int idx = -1;
    float d0 = 1.0f, d1 = 0.0f, d2 = 0.0f;
    if (a.start_dir) {
        if (active) {
            d0 = a.start_dir[3 * i];
            d1 = a.start_dir[3 * i + 1];
            d2 = a.start_dir[3 * i + 2];
        }
    } else {
        idx = active ? a.best_idx[i] : 0;
        d0 = a.hyps[3 * idx];
        d1 = a.hyps[3 * idx + 1];
        d2 = a.hyps[3 * idx + 2];
    }
    float best = 0.0f;
    int nv = 0;
    const int nblk = (a.V + kCamStageViews - 1) / kCamStageViews;
    const int npair = hf_view_pairs(a.V);
    const int rounds = a.T > 0 ? a.T : 1;   // with T = 0 round 0 takes the start's sum and stops
    for (int t = 0; t < rounds; ++t) {
        const float2 cr = t < a.T ? a.rot[t] : make_float2(1.0f, 0.0f);
        const float c = cr.x, sn = cr.y;
        // every product rounded once and added with an explicit fused multiply-add
        const float cd[6][3] = {{d0, fmaf(c, d1, __fmul_rn(-sn, d2)), fmaf(sn, d1, __fmul_rn(c, d2))},
                                {d0, fmaf(c, d1, __fmul_rn(sn, d2)), fmaf(-sn, d1, __fmul_rn(c, d2))},
                                {fmaf(c, d0, __fmul_rn(sn, d2)), d1, fmaf(-sn, d0, __fmul_rn(c, d2))},
                                {fmaf(c, d0, __fmul_rn(-sn, d2)), d1, fmaf(sn, d0, __fmul_rn(c, d2))},
                                {fmaf(c, d0, __fmul_rn(-sn, d1)), fmaf(sn, d0, __fmul_rn(c, d1)), d2},
                                {fmaf(c, d0, __fmul_rn(sn, d1)), fmaf(-sn, d0, __fmul_rn(c, d1)), d2}};
        f32x2 CX[3], CY[3], CZ[3];
#pragma unroll
        for (int p = 0; p < 3; ++p) {
            CX[p] = pk(cd[2 * p][0], cd[2 * p + 1][0]);
            CY[p] = pk(cd[2 * p][1], cd[2 * p + 1][1]);
            CZ[p] = pk(cd[2 * p][2], cd[2 * p + 1][2]);
        }
        const bool centre = t == 0;
        const f32x2 D0 = pk(d0, d0), D1 = pk(d1, d1), D2 = pk(d2, d2);
        float acc[6] = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f}, acc_c = 0.0f;
        int n = 0;
        for (int p = 0; p < S - 1; ++p)
            if (p < npair) issue_pair<KP, NT>(sg, p, a.ab, a.samp, p, a.N, i, nb, active);
            else cp_async_commit();
        for (int vb = 0; vb < a.V; vb += kCamStageViews) {
            const int nvb = min(kCamStageViews, a.V - vb);
            if (nblk > 1 || t == 0) {
                __syncthreads();
                for (int e = tid; e < nvb; e += NT) {
                    const float* cam = a.cams + 16 * (vb + e);
                    cs4[3 * e] = make_float4(cam[0], cam[1], cam[4], cam[5]);
                    cs4[3 * e + 1] = make_float4(cam[6], cam[7], cam[8], cam[9]);
                    cs4[3 * e + 2] = make_float4(cam[10], cam[11], cam[12], a.vthr[vb + e]);
                }
                __syncthreads();
            }
            // the pairs of this block (kCamStageViews is even, so a pair never straddles two blocks)
            for (int q = vb >> 1; q < (vb + nvb + 1) >> 1; ++q) {
                const int qn = q + S - 1;
                if (qn < npair) issue_pair<KP, NT>(sg, qn % S, a.ab, a.samp, qn, a.N, i, nb, active);
                else cp_async_commit();
                cp_async_wait<S - 1>();
                if (!active) continue;
                const int st = q % S;
#pragma unroll 1
                for (int h = 0; h < 2; ++h) {   // view h of the pair: the h-th 8-byte half of each item
                    const int v = 2 * q + h;
                    if (v >= vb + nvb) break;   // the missing second view of an odd V
                    const float2 r = reinterpret_cast<const float2*>(&sg.v[st][0][tid])[h];
                    if (r.x != r.x) continue;   // v is not in the point's view set
                    ++n;
                    f32x2 SX[KP], SY[KP];
#pragma unroll
                    for (int j = 0; j < KP; ++j) {
                        const float2 sj = reinterpret_cast<const float2*>(&sg.v[st][1 + j][tid])[h];
                        SX[j] = pk(sj.x, sj.x);
                        SY[j] = pk(sj.y, sj.y);
                    }
                    // staged rows: k0 = (fx, fy, R00, R01), k1 = (R02, R10, R11, R12), k2 = (R20, R21, R22, thr)
                    const float4 k0 = cs4[3 * (v - vb)], k1 = cs4[3 * (v - vb) + 1], k2 = cs4[3 * (v - vb) + 2];
                    // Z times the projection Jacobian: rows fx (R_0 - a R_2), fy (R_1 - b R_2)
                    const float j0 = __fmul_rn(k0.x, fmaf(-r.x, k2.x, k0.z)), j1 = __fmul_rn(k0.x, fmaf(-r.x, k2.y, k0.w)),
                                j2 = __fmul_rn(k0.x, fmaf(-r.x, k2.z, k1.x));
                    const float j3 = __fmul_rn(k0.y, fmaf(-r.y, k2.x, k1.y)), j4 = __fmul_rn(k0.y, fmaf(-r.y, k2.y, k1.z)),
                                j5 = __fmul_rn(k0.y, fmaf(-r.y, k2.z, k1.w));
                    const f32x2 J0 = pk(j0, j0), J1 = pk(j1, j1), J2 = pk(j2, j2);
                    const f32x2 J3 = pk(j3, j3), J4 = pk(j4, j4), J5 = pk(j5, j5);
#pragma unroll
                    for (int p = 0; p < 3; ++p) {   // the +alpha / -alpha pair of axis p
                        float L0, L1;
                        view_term2<KP>(fma2(J0, CX[p], fma2(J1, CY[p], mul2(J2, CZ[p]))),
                                       fma2(J3, CX[p], fma2(J4, CY[p], mul2(J5, CZ[p]))), SX, SY, k2.w, L0, L1);
                        acc[2 * p] = __fadd_rn(acc[2 * p], L0);
                        acc[2 * p + 1] = __fadd_rn(acc[2 * p + 1], L1);
                    }
                    if (centre) {
                        float L0, L1;
                        view_term2<KP>(fma2(J0, D0, fma2(J1, D1, mul2(J2, D2))), fma2(J3, D0, fma2(J4, D1, mul2(J5, D2))),
                                       SX, SY, k2.w, L0, L1);
                        acc_c = __fadd_rn(acc_c, L0);
                    }
                }
            }
        }
        cp_async_wait<0>();
        if (centre) {
            nv = n;
            best = acc_c;
        }
        if (t >= a.T) break;
        int choice = -1;
#pragma unroll
        for (int e = 0; e < 6; ++e)
            if (acc[e] > best) {
                best = acc[e];
                choice = e;
            }
#pragma unroll
        for (int e = 0; e < 6; ++e)
            if (e == choice) {
                d0 = cd[e][0];
                d1 = cd[e][1];
                d2 = cd[e][2];
            }
    }
    if (!in) return;
    if (!active) {
        write_bad(a, i);
        return;
    }
    write_out(a, i, nv, dir2(d0, d1, d2), best, idx);
}

// The learned path's selection, a point per thread: the cost c_i of the proposal; points with a view
// and c_i > tau are appended to the fallback list, the other finite points to the accepted list
// (warp-aggregated appends, in the order warps reach them), |V_i| to the matching work count;
// non-finite points get their BAD_INPUT outputs here and no list.  The views' camera rows are staged
// in shared memory per block of views; the next view pair's ratios and patch samples (one 16-byte
// element an item) are loaded into registers while the current pair's two views are evaluated.
constexpr int kSelectViews = 128;   // camera rows staged per view block
template <int KP>
__device__ __forceinline__ void select_tile(const LearnArgs& la, int blk) {
    __shared__ float4 cs4[kSelectViews * 3];
    const CostArgs& a = la.f;
    const int i = blk * blockDim.x + threadIdx.x;
    const bool in = i < a.N;
    const int ic = in ? i : 0;
    const float p0 = a.pts[3 * ic], p1 = a.pts[3 * ic + 1], p2 = a.pts[3 * ic + 2];
    const bool active = in && isfinite(p0) && isfinite(p1) && isfinite(p2);
    int nb[KP];
    nb[0] = active ? ic : -1;
#pragma unroll
    for (int j = 1; j < KP; ++j) nb[j] = (active && (j - 1) < a.k) ? a.nbr[(size_t)ic * a.k + (j - 1)] : -1;
    float d0 = 1.0f, d1 = 0.0f, d2 = 0.0f;
    if (active) {
        d0 = la.start_dir[3 * ic];
        d1 = la.start_dir[3 * ic + 1];
        d2 = la.start_dir[3 * ic + 2];
    }
    float acc = 0.0f;
    int nv = 0;
    for (int vb = 0; vb < a.V; vb += kSelectViews) {
        const int nvb = min(kSelectViews, a.V - vb);
        __syncthreads();   // the previous block's rows are no longer read
        for (int e = threadIdx.x; e < nvb; e += blockDim.x) {
            const float* cam = a.cams + 16 * (vb + e);
            cs4[3 * e] = make_float4(cam[0], cam[1], cam[4], cam[5]);
            cs4[3 * e + 1] = make_float4(cam[6], cam[7], cam[8], cam[9]);
            cs4[3 * e + 2] = make_float4(cam[10], cam[11], cam[12], a.vthr[vb + e]);
        }
        __syncthreads();
        if (!active) continue;
        // view pairs: one 16-byte load per item brings both views; the next pair is loaded while
        // the current pair's two views are evaluated
        const float4* ab4 = reinterpret_cast<const float4*>(a.ab);
        const float4* sp4 = reinterpret_cast<const float4*>(a.samp);
        const int q0 = vb >> 1, q1 = (vb + nvb + 1) >> 1;   // kSelectViews is even: pairs stay in the block
        float4 rn = __ldg(ab4 + (size_t)q0 * a.N + ic), sn[KP];
#pragma unroll
        for (int j = 0; j < KP; ++j) sn[j] = nb[j] >= 0 ? __ldg(sp4 + (size_t)q0 * a.N + nb[j]) : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        for (int q = q0; q < q1; ++q) {
            const float4 r4 = rn;
            float4 s4[KP];
#pragma unroll
            for (int j = 0; j < KP; ++j) s4[j] = sn[j];
            if (q + 1 < q1) {
                rn = __ldg(ab4 + (size_t)(q + 1) * a.N + ic);
#pragma unroll
                for (int j = 0; j < KP; ++j)
                    sn[j] = nb[j] >= 0 ? __ldg(sp4 + (size_t)(q + 1) * a.N + nb[j]) : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
            }
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int v = 2 * q + h;
                if (v >= vb + nvb) break;   // the missing second view of an odd V
                const float2 r = h ? make_float2(r4.z, r4.w) : make_float2(r4.x, r4.y);
                if (r.x != r.x) continue;
                ++nv;
                // staged rows: k0 = (fx, fy, R00, R01), k1 = (R02, R10, R11, R12), k2 = (R20, R21, R22, thr)
                const float4 k0 = cs4[3 * (v - vb)], k1 = cs4[3 * (v - vb) + 1], k2 = cs4[3 * (v - vb) + 2];
                // q = R d, then Z times the image offset (fx (q_x - a q_z), fy (q_y - b q_z))
                const float qx = fmaf(k0.z, d0, fmaf(k0.w, d1, __fmul_rn(k1.x, d2)));
                const float qy = fmaf(k1.y, d0, fmaf(k1.z, d1, __fmul_rn(k1.w, d2)));
                const float qz = fmaf(k2.x, d0, fmaf(k2.y, d1, __fmul_rn(k2.z, d2)));
                const float rx = __fmul_rn(k0.x, fmaf(-r.x, qz, qx)), ry = __fmul_rn(k0.y, fmaf(-r.y, qz, qy));
                const float r2 = fmaf(rx, rx, __fmul_rn(ry, ry));
                float u[KP];
#pragma unroll
                for (int j = 0; j < KP; ++j) {
                    const float sx = h ? s4[j].z : s4[j].x, sy = h ? s4[j].w : s4[j].y;
                    u[j] = fmaf(rx, sx, __fmul_rn(ry, sy));
                }
                const float mx = patch_max<KP>(u);
                acc = __fadd_rn(acc, r2 >= k2.w ? __fmul_rn(mx, rsqrt_ftz(r2)) : 0.0f);
            }
        }
    }
    const float c0 = nv ? 1.0f - acc / (float)nv : 1.0f;
    if (in && !active) write_bad(a, i);
    const bool fb = active && nv > 0 && c0 > la.tau;
    const bool ok = active && !fb;
    const int lane = threadIdx.x & 31;
    const unsigned below = (1u << lane) - 1u;
#pragma unroll
    for (int q = 0; q < 2; ++q) {   // warp-aggregated appends: fallback, then accepted
        const bool want = q == 0 ? fb : ok;
        const unsigned m = __ballot_sync(0xffffffffu, want);
        if (!m) continue;
        const int leader = __ffs(m) - 1;
        int base = 0;
        if (lane == leader) base = atomicAdd(q == 0 ? la.fb_count : la.acc_count, __popc(m));
        base = __shfl_sync(0xffffffffu, base, leader);
        if (want) (q == 0 ? la.fb_list : la.acc_list)[base + __popc(m & below)] = i;
    }
    const unsigned wfb = __reduce_add_sync(0xffffffffu, fb ? (unsigned)nv : 0u);
    const unsigned wok = __reduce_add_sync(0xffffffffu, ok ? (unsigned)nv : 0u);
    if (lane == 0) {
        if (la.fb_work && wfb) atomicAdd(la.fb_work, (unsigned long long)wfb);
        if (la.acc_work && wok) atomicAdd(la.acc_work, (unsigned long long)wok);
    }
}

// ------------------------------------------------------------------ cost of given directions
template <int KP, int L, int NP>
__device__ __forceinline__ void eval_tile_l(const EvalArgs& e, int tile) {
    const CostArgs& a = e.f;
    Lanes ln;
    if (!lanes_of<L>(tile, a.N, ln)) return;
    PointCtx<KP> pc;
    point_ctx<KP>(a, ln.q, a.N, pc);
    int nch, np;
    chunking<L, NP>(pc.nv, nch, np);
    VPair<KP> P[NP];
    if (nch == 1) gather<KP, L, NP>(a, pc, ln.lg, 0, np, P);
    for (int m = 0; m < e.M; ++m) {
        const float* d = e.dirs + ((size_t)pc.i * e.M + m) * 3;
        const Dir2 dd = dir2(d[0], d[1], d[2]);
        const float dn2 = fmaf(d[0], d[0], fmaf(d[1], d[1], __fmul_rn(d[2], d[2])));
        float l[1];
        lane_sums<KP, L, NP, 1, true>(a, pc, ln.lg, nch, np, P, [&](int) { return dd; }, dn2, l);
        const float s = group_sum<L>(l[0]);
        if (ln.lg == 0 && pc.in) e.cost[(size_t)pc.i * e.M + m] = pc.nv ? 1.0f - s / (float)pc.nv : 1.0f;
    }
}


}  // namespace hf_cost
