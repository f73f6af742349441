// hf_kernels.cu - the fusion path's device code for sm_103a.
//
//   k_prep          per-scene constants: hypotheses (padded to an even count), degenerate
//                   thresholds, refinement rotation steps.
//   k_project       K1, thread per point: projection of the point into every view with the pixel
//                   index decided in float-float arithmetic, nearest-pixel gather of the orientation
//                   and confidence maps, view set (visible or top-K) of the point.
//   k_fuse<KP>      K2 + K3, a group of lanes per point: the cost of every hypothesis (Eqs. proj_r ..
//                   patch_min and the view mean), their argmin, then the T rounds of the six-rotation
//                   refinement, from one gather of the point's patch held in registers.
//   k_learn<KP>     the learned path after the network: cost of the proposal, fallback selection,
//                   short refinement of the accepted proposals.
//   k_eval<KP>      cost of caller-given directions (no argmin).
#include <math.h>

#include <cuda_bf16.h>

#include "hf_ff.cuh"
#include "hf_internal.cuh"

namespace {

using namespace hf_ff;

__device__ __forceinline__ float load_conf(const void* conf, int f16, size_t o) {
    if (f16) return __half2float(reinterpret_cast<const __half*>(conf)[o]);
    return reinterpret_cast<const float*>(conf)[o];
}

// Order-preserving integer encoding of floats (exact, order-independent min / max by atomics).
__device__ __forceinline__ unsigned fkey(float x) {
    const unsigned u = __float_as_uint(x);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float fval(unsigned k) { return __uint_as_float((k & 0x80000000u) ? (k & 0x7fffffffu) : ~k); }

// ------------------------------------------------------------------ K1: project + gather
// One thread per point, views in groups of four.  For view v it writes
//   samp[i][v] = C (cos theta, sin theta) at the point's pixel (0 when outside the view),
// four views (one 32-byte sector of the row) at a time, and the point's view-set mask: every view
// the point projects into, or with top_k > 0 the top_k of them by the confidence at the point's own
// pixel, ties to the lower view index.
constexpr int kProjectThreads = 128;

// With a.box_keys set, the tile also folds its finite coordinates into the point cloud's bounding
// box (keys lo[3] from 0xffffffff, hi[3] from 0, per coordinate).
template <bool TOPK>
__device__ __forceinline__ void project_tile(const ProjectArgs& a, int blk) {
    const int i = blk * kProjectThreads + threadIdx.x;
    if (a.box_keys) {
        const bool in = i < a.N;
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            const float x = in ? a.pts[3 * i + q] : 0.0f;
            const bool f = in && isfinite(x);
            const unsigned lo = __reduce_min_sync(0xffffffffu, f ? fkey(x) : 0xffffffffu);
            const unsigned hi = __reduce_max_sync(0xffffffffu, f ? fkey(x) : 0u);
            if ((threadIdx.x & 31) == 0 && hi != 0u) {
                atomicMin(a.box_keys + q, lo);
                atomicMax(a.box_keys + 3 + q, hi);
            }
        }
    }
    if (i >= a.N) return;
    const float p0 = a.pts[3 * i], p1 = a.pts[3 * i + 1], p2 = a.pts[3 * i + 2];
    const size_t npx = (size_t)a.W * a.H;
    const int Vs = hf_samp_stride(a.V), Vw = hf_mask_words(a.V);
    float4* row = reinterpret_cast<float4*>(a.samp + (size_t)i * Vs);
    unsigned long long* mrow = a.vmask + (size_t)i * Vw;
    float topc[HF_MAX_TOPK];
    int topv[HF_MAX_TOPK];
    int ntop = 0, nset = 0;
    unsigned long long word = 0ull;
    // views in groups of four: the pixel decisions first, then the four gathers in flight together
    constexpr int G = 4;
    for (int v0 = 0; v0 < a.V; v0 += G) {
        long long off[G];
#pragma unroll
        for (int q = 0; q < G; ++q) {
            off[q] = -1;
            const int v = v0 + q;
            if (v >= a.V) continue;
            const float* cam = a.cams + 16 * v;
            const float fx = __ldg(cam), fy = __ldg(cam + 1), cx = __ldg(cam + 2), cy = __ldg(cam + 3);
            const ff X0 = ff_dot3_plus(__ldg(cam + 4), __ldg(cam + 5), __ldg(cam + 6), p0, p1, p2, __ldg(cam + 13));
            const ff X1 = ff_dot3_plus(__ldg(cam + 7), __ldg(cam + 8), __ldg(cam + 9), p0, p1, p2, __ldg(cam + 14));
            const ff X2 = ff_dot3_plus(__ldg(cam + 10), __ldg(cam + 11), __ldg(cam + 12), p0, p1, p2, __ldg(cam + 15));
            if (!(X2.hi > 1e-6f)) continue;
            const float fu = ff_floor(ff_affine(fx, ff_div(X0, X2), cx));
            const float fv = ff_floor(ff_affine(fy, ff_div(X1, X2), cy));
            if (!(fu >= 0.0f && fu < (float)a.W && fv >= 0.0f && fv < (float)a.H)) continue;
            off[q] = (long long)((size_t)v * npx + (size_t)fv * a.W + (size_t)fu);
        }
        float th[G], C[G];
#pragma unroll
        for (int q = 0; q < G; ++q) {
            th[q] = C[q] = 0.0f;
            if (off[q] < 0) continue;
            if (a.amap) {
                const float2 t = __ldg(a.amap + off[q]);
                th[q] = t.x;
                C[q] = t.y;
            } else {
                th[q] = __ldg(a.angle + off[q]);
                C[q] = load_conf(a.conf, a.conf_f16, (size_t)off[q]);
            }
        }
        float sv[2 * G];
#pragma unroll
        for (int q = 0; q < G; ++q) {
            sv[2 * q] = sv[2 * q + 1] = 0.0f;
            if (off[q] < 0) continue;
            float sn, cs;
            sincosf(th[q], &sn, &cs);
            sv[2 * q] = C[q] * cs;
            sv[2 * q + 1] = C[q] * sn;
            const int v = v0 + q;
            word |= 1ull << (v & 63);
            if (TOPK) {
                // keep the top_k (conf desc, view asc); later views need a strictly larger conf
                const float c = C[q];
                if (ntop < a.top_k || c > topc[ntop - 1]) {
                    int pos = ntop < a.top_k ? ntop++ : ntop - 1;
                    while (pos > 0 && c > topc[pos - 1]) {
                        topc[pos] = topc[pos - 1];
                        topv[pos] = topv[pos - 1];
                        --pos;
                    }
                    topc[pos] = c;
                    topv[pos] = v;
                }
            }
        }
        row[v0 / 2] = make_float4(sv[0], sv[1], sv[2], sv[3]);
        row[v0 / 2 + 1] = make_float4(sv[4], sv[5], sv[6], sv[7]);
        if (((v0 + G) & 63) == 0 || v0 + G >= a.V) {   // a mask word is complete
            if (!TOPK) mrow[v0 >> 6] = word;
            nset += __popcll(word);
            word = 0ull;
        }
    }
    if (TOPK) {
        for (int w = 0; w < Vw; ++w) {
            unsigned long long m = 0ull;
            for (int q = 0; q < ntop; ++q)
                if ((topv[q] >> 6) == w) m |= 1ull << (topv[q] & 63);
            mrow[w] = m;
        }
        nset = ntop;
    }
    // warp-aggregated count of the (point, view) pairs in the view sets
    const unsigned am = __activemask();
    const unsigned tot = __reduce_add_sync(am, (unsigned)nset);
    if ((threadIdx.x & 31) == __ffs(am) - 1) atomicAdd(a.work, (unsigned long long)tot);
}

template <bool TOPK>
__global__ void __launch_bounds__(kProjectThreads) k_project(ProjectArgs a) {
    project_tile<TOPK>(a, blockIdx.x);
}

__global__ void k_iota(int32_t* list, int* count, int first, int n) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q < n) list[q] = first + q;
    if (q == 0) *count = n;
}

__global__ void k_interleave(const float* __restrict__ angle, const void* __restrict__ conf, int f16, size_t npx,
                             float2* __restrict__ out) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < npx; i += (size_t)gridDim.x * blockDim.x)
        out[i] = make_float2(angle[i], load_conf(conf, f16, i));
}

// ------------------------------------------------------------------ per-scene constants
// Built-in hypothesis m of H: Fibonacci lattice on the upper hemisphere (the cost is
// sign-invariant, Eq. sim), z_m = 1 - (m + 1/2)/H, azimuth m * pi * (3 - sqrt 5).
__device__ void fib_dir(int m, int H, double* h) {
    const double kPi = 3.14159265358979323846;
    const double z = 1.0 - (m + 0.5) / H;
    const double rho = sqrt(fmax(0.0, 1.0 - z * z));
    const double ph = m * kPi * (3.0 - sqrt(5.0));
    h[0] = rho * cos(ph);
    h[1] = rho * sin(ph);
    h[2] = z;
}

__global__ void k_fib(int H, float* out) {
    for (int m = blockIdx.x * blockDim.x + threadIdx.x; m < H; m += gridDim.x * blockDim.x) {
        double h[3];
        fib_dir(m, H, h);
        for (int q = 0; q < 3; ++q) out[3 * m + q] = (float)h[q];
    }
}

__device__ __forceinline__ void prep_body(const PrepArgs& a) {
    const double kPi = 3.14159265358979323846;
    for (int m = threadIdx.x; m < a.Hpad; m += blockDim.x) {
        const int src = m < a.H ? m : 0;
        double h[3];
        if (a.hyps_in == nullptr) {
            fib_dir(src, a.H, h);
        } else {
            for (int q = 0; q < 3; ++q) h[q] = a.hyps_in[3 * src + q];
            const double n = sqrt(h[0] * h[0] + h[1] * h[1] + h[2] * h[2]);
            if (!(fabs(n - 1.0) <= 1e-3)) atomicOr(a.errw, HF_DEV_ERR_BAD_HYP);
        }
        for (int q = 0; q < 3; ++q) a.hyps[3 * m + q] = (float)h[q];
    }
    for (int v = threadIdx.x; v < a.V; v += blockDim.x) {
        const double fx = a.cams[16 * v], fy = a.cams[16 * v + 1];
        a.vthr[v] = (float)(1e-20 * (fx * fx + fy * fy));
    }
    for (int t = threadIdx.x; t < a.T; t += blockDim.x) {
        const double al = 0.5 * sqrt(2.0 * kPi / a.H) / (double)(1u << t);
        a.rot[t] = make_float2((float)cos(al), (float)sin(al));
    }
}

__global__ void k_prep(PrepArgs a) { prep_body(a); }

// ------------------------------------------------------------------ K2 + K3: the cost kernels
//
// A point is served by a group of L lanes (L in {4, 8, 16, 32}; 32 / L points per warp).  The views
// of the point's view set V_i, in view order, are dealt to the lanes: member n of V_i goes to lane
// n mod L, slot (n / L) mod SM, chunk n / (L SM).  Per chunk a lane gathers, for each of its slots,
// the projection Jacobian of its view at the point (single precision, scaled by Z, which cancels),
// the view's degenerate threshold and the samples C (cos theta, sin theta) of the k + 1 patch
// members at their own pixels.  With one chunk (|V_i| <= L SM, the usual case) these stay in
// registers while every direction is evaluated: the H hypotheses, then the T rounds of six
// rotations.  A direction's patch terms are summed over the lane's slots and then over the group
// by a butterfly of shuffles, which leaves the bitwise-same sum in every lane of the group; every
// lane therefore takes the same decisions.  Larger view sets are processed chunk by chunk (the
// chunk gathered again for every direction).
//
// The patch term of a direction d in view v (Eqs. proj_r, sim, patchloss, patch_min):
//   r = J d (Z times the image offset), L_v = max_j |<r, s_j>| / |r|, 0 when |r|^2 < threshold;
// the members are evaluated in pairs with packed FP32 instructions (fma.rn.f32x2 / mul.rn.f32x2,
// each lane rounded exactly like the scalar instruction) and folded into the running maximum with
// the three-input max.f32 of two absolute values.  The cost is c = 1 - (sum_v L_v) / |V_i| (Eq.
// final_dout with the view mean); minimising c is maximising the sum, which the kernels compare.
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
// max(m, |a|, |b|)
__device__ __forceinline__ float max3abs(float m, float a, float b) {
    float r;
    asm("{ .reg .f32 t, u; abs.f32 t, %1; abs.f32 u, %2; max.f32 %0, %3, t, u; }" : "=f"(r) : "f"(a), "f"(b), "f"(m));
    return r;
}

// slots per lane for a patch width: the patch data of a slot is 2 KP + 7 registers
template <int KP>
struct SlotsFor {
    static constexpr int value = KP <= 9 ? 4 : 2;
};

// One view of the point held by a lane.
template <int KP>
struct Slot {
    static constexpr int NP = KP / 2 > 0 ? KP / 2 : 1;
    float j0, j1, j2, j3, j4, j5;   // rows of Z x the projection Jacobian: fx (R_0 - a R_2), fy (R_1 - b R_2)
    float thr;                      // degenerate threshold of the view; +inf for an empty slot
    f32x2 sx[NP], sy[NP];           // members 2q, 2q+1 (q < KP / 2): (x_2q, x_2q+1), (y_2q, y_2q+1)
    float ox, oy;                   // member KP - 1 when KP is odd
};

template <int KP>
__device__ __forceinline__ float patch_term(const Slot<KP>& s, float d0, float d1, float d2, float thr) {
    const float rx = fmaf(s.j0, d0, fmaf(s.j1, d1, __fmul_rn(s.j2, d2)));
    const float ry = fmaf(s.j3, d0, fmaf(s.j4, d1, __fmul_rn(s.j5, d2)));
    const float r2 = fmaf(rx, rx, __fmul_rn(ry, ry));
    float m = 0.0f;
    if (KP & 1) m = fabsf(fmaf(rx, s.ox, __fmul_rn(ry, s.oy)));
    if (KP >= 2) {
        const f32x2 RX = pk(rx, rx), RY = pk(ry, ry);
#pragma unroll
        for (int q = 0; q < KP / 2; ++q) {
            float u0, u1;
            upk(fma2(RX, s.sx[q], mul2(RY, s.sy[q])), u0, u1);
            m = max3abs(m, u0, u1);
        }
    }
    return r2 >= thr ? __fmul_rn(m, rsqrtf(r2)) : 0.0f;
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

// Gather chunk `chunk` of the point's view set into the lane's slots (slots >= ns stay empty).
template <int KP, int SM>
__device__ __forceinline__ void gather(const CostArgs& a, const PointCtx<KP>& pc, int lg, int chunk, int ns,
                                       Slot<KP> (&S)[SM]) {
#pragma unroll
    for (int s = 0; s < SM; ++s) {
        Slot<KP>& q = S[s];
        const int n = (chunk * SM + s) * a.L + lg;
        const int v = (s < ns && n < pc.nv) ? nth_view(a, pc.i, pc.w0, n) : -1;
        float2 sm[KP];
        if (v < 0) {
            q.j0 = q.j1 = q.j2 = q.j3 = q.j4 = q.j5 = 0.0f;
            q.thr = INFINITY;
#pragma unroll
            for (int j = 0; j < KP; ++j) sm[j] = make_float2(0.0f, 0.0f);
        } else {
            const float* cam = a.cams + 16 * v;
            const float fx = __ldg(cam), fy = __ldg(cam + 1);
            const float r00 = __ldg(cam + 4), r01 = __ldg(cam + 5), r02 = __ldg(cam + 6);
            const float r10 = __ldg(cam + 7), r11 = __ldg(cam + 8), r12 = __ldg(cam + 9);
            const float r20 = __ldg(cam + 10), r21 = __ldg(cam + 11), r22 = __ldg(cam + 12);
            const float X = fmaf(r00, pc.p0, fmaf(r01, pc.p1, fmaf(r02, pc.p2, __ldg(cam + 13))));
            const float Y = fmaf(r10, pc.p0, fmaf(r11, pc.p1, fmaf(r12, pc.p2, __ldg(cam + 14))));
            const float Z = fmaf(r20, pc.p0, fmaf(r21, pc.p1, fmaf(r22, pc.p2, __ldg(cam + 15))));
            const float iz = 1.0f / Z;
            const float ra = __fmul_rn(X, iz), rb = __fmul_rn(Y, iz);
            q.j0 = __fmul_rn(fx, fmaf(-ra, r20, r00));
            q.j1 = __fmul_rn(fx, fmaf(-ra, r21, r01));
            q.j2 = __fmul_rn(fx, fmaf(-ra, r22, r02));
            q.j3 = __fmul_rn(fy, fmaf(-rb, r20, r10));
            q.j4 = __fmul_rn(fy, fmaf(-rb, r21, r11));
            q.j5 = __fmul_rn(fy, fmaf(-rb, r22, r12));
            q.thr = __ldg(a.vthr + v);
#pragma unroll
            for (int j = 0; j < KP; ++j)
                sm[j] = pc.nb[j] >= 0 ? __ldg(a.samp + (size_t)pc.nb[j] * a.Vs + v) : make_float2(0.0f, 0.0f);
        }
#pragma unroll
        for (int p = 0; p < KP / 2; ++p) {
            q.sx[p] = pk(sm[2 * p].x, sm[2 * p + 1].x);
            q.sy[p] = pk(sm[2 * p].y, sm[2 * p + 1].y);
        }
        if (KP & 1) {
            q.ox = sm[KP - 1].x;
            q.oy = sm[KP - 1].y;
        }
    }
}

__device__ __forceinline__ float group_sum(float x, int L) {
#pragma unroll
    for (int o = 1; o < 32; o <<= 1)
        if (o < L) x = __fadd_rn(x, __shfl_xor_sync(0xffffffffu, x, o));
    return x;
}

// Group sums of the patch terms of ND directions (all lanes of the warp take part).  With one chunk
// the slots hold the data (ns of them in use); otherwise each chunk is gathered again here.
template <int KP, int SM, int ND>
__device__ __forceinline__ void dir_sums(const CostArgs& a, const PointCtx<KP>& pc, int lg, int nch, int ns,
                                         Slot<KP> (&S)[SM], const float (&d)[ND][3], float tscale, float (&out)[ND]) {
#pragma unroll
    for (int q = 0; q < ND; ++q) out[q] = 0.0f;
    for (int c = 0; c < nch; ++c) {
        if (nch > 1) gather<KP, SM>(a, pc, lg, c, SM, S);
#pragma unroll
        for (int s = 0; s < SM; ++s) {
            if (s < ns || nch > 1) {
#pragma unroll
                for (int q = 0; q < ND; ++q)
                    out[q] = __fadd_rn(out[q], patch_term<KP>(S[s], d[q][0], d[q][1], d[q][2], __fmul_rn(S[s].thr, tscale)));
            }
        }
    }
#pragma unroll
    for (int q = 0; q < ND; ++q) out[q] = group_sum(out[q], a.L);
}

// Group geometry of the calling lane for tile `tile`: returns false when the whole warp is past
// the end of the work list (a warp-uniform exit).
struct Lanes {
    int lane, lg, g, q;   // lane, lane in group, group in warp, work-list position of the group
};
__device__ __forceinline__ bool lanes_of(int L, int tile, int cnt, Lanes& ln) {
    ln.lane = threadIdx.x & 31;
    ln.lg = ln.lane & (L - 1);
    ln.g = ln.lane / L;
    const int ppw = 32 / L;
    const int w = tile * (blockDim.x >> 5) + (threadIdx.x >> 5);
    ln.q = w * ppw + ln.g;
    return w * ppw < cnt;
}

// chunks and slots in use, uniform over the warp
template <int SM>
__device__ __forceinline__ void chunking(int nv, int L, int& nch, int& ns) {
    const int per = L * SM;
    nch = (int)__reduce_max_sync(0xffffffffu, (unsigned)((nv + per - 1) / per));
    ns = (int)__reduce_max_sync(0xffffffffu, (unsigned)min(SM, (nv + L - 1) / L));
    if (nch < 1) nch = 1;
}

__device__ __forceinline__ void write_bad(const CostArgs& a, int i) {
    const int o = i - a.out_first;   // output row
    a.dir_out[3 * o] = a.dir_out[3 * o + 1] = a.dir_out[3 * o + 2] = 0.0f;
    if (a.cost_out) a.cost_out[o] = __int_as_float(0x7fc00000);
    if (a.idx_out) a.idx_out[o] = -1;
    if (a.status_out) a.status_out[o] = HF_STATUS_BAD_INPUT;
}

// Six rotations of d by +-alpha about world x, y, z (in that order) and their sums; move to the first
// strictly larger sum (the first strictly lower cost).
template <int KP, int SM>
__device__ __forceinline__ void refine_rounds(const CostArgs& a, const PointCtx<KP>& pc, int lg, int nch, int ns,
                                              Slot<KP> (&S)[SM], float& d0, float& d1, float& d2, float& best) {
    for (int t = 0; t < a.T; ++t) {
        const float2 cr = a.rot[t];
        const float c = cr.x, sn = cr.y;
        // every product rounded once and added with an explicit fused multiply-add, so that all
        // instances of this code round alike
        const float cd[6][3] = {{d0, fmaf(c, d1, __fmul_rn(-sn, d2)), fmaf(sn, d1, __fmul_rn(c, d2))},
                                {d0, fmaf(c, d1, __fmul_rn(sn, d2)), fmaf(-sn, d1, __fmul_rn(c, d2))},
                                {fmaf(c, d0, __fmul_rn(sn, d2)), d1, fmaf(-sn, d0, __fmul_rn(c, d2))},
                                {fmaf(c, d0, __fmul_rn(-sn, d2)), d1, fmaf(sn, d0, __fmul_rn(c, d2))},
                                {fmaf(c, d0, __fmul_rn(-sn, d1)), fmaf(sn, d0, __fmul_rn(c, d1)), d2},
                                {fmaf(c, d0, __fmul_rn(sn, d1)), fmaf(-sn, d0, __fmul_rn(c, d1)), d2}};
        float acc[6];
        dir_sums<KP, SM, 6>(a, pc, lg, nch, ns, S, cd, 1.0f, acc);
        int choice = -1;
#pragma unroll
        for (int q = 0; q < 6; ++q)
            if (acc[q] > best) {
                best = acc[q];
                choice = q;
            }
#pragma unroll
        for (int q = 0; q < 6; ++q)
            if (q == choice) {
                d0 = cd[q][0];
                d1 = cd[q][1];
                d2 = cd[q][2];
            }
    }
}

// Normalised direction with the canonical sign, the cost, index and status of a point.
__device__ __forceinline__ void write_out(const CostArgs& a, int i, int nv, float d0, float d1, float d2, float best,
                                          int idx) {
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

// The hypotheses of the scene into shared memory (a CTA-wide barrier follows).
__device__ __forceinline__ void stage_hyps(const CostArgs& a, float* sh) {
    for (int e = threadIdx.x; e < 3 * a.Hpad; e += blockDim.x) sh[e] = a.hyps[e];
    __syncthreads();
}

// K2 + K3 for the points of one tile.
template <int KP>
__device__ __forceinline__ void fuse_tile(const CostArgs& a, int tile, float* sh) {
    constexpr int SM = SlotsFor<KP>::value;
    stage_hyps(a, sh);
    const int cnt = a.list ? *a.list_count : a.N;
    Lanes ln;
    if (!lanes_of(a.L, tile, cnt, ln)) return;
    PointCtx<KP> pc;
    point_ctx<KP>(a, ln.q, cnt, pc);
    int nch, ns;
    chunking<SM>(pc.nv, a.L, nch, ns);
    Slot<KP> S[SM];
    if (nch == 1) gather<KP, SM>(a, pc, ln.lg, 0, ns, S);
    // argmin over the hypotheses, two at a time (largest sum, lowest index on ties)
    float best = -1.0f;
    int bm = 0;
    for (int m = 0; m < a.Hpad; m += 2) {
        const float hd[2][3] = {{sh[3 * m], sh[3 * m + 1], sh[3 * m + 2]}, {sh[3 * m + 3], sh[3 * m + 4], sh[3 * m + 5]}};
        float l[2];
        dir_sums<KP, SM, 2>(a, pc, ln.lg, nch, ns, S, hd, 1.0f, l);
        if (l[0] > best) {
            best = l[0];
            bm = m;
        }
        if (m + 1 < a.H && l[1] > best) {
            best = l[1];
            bm = m + 1;
        }
    }
    float d0 = sh[3 * bm], d1 = sh[3 * bm + 1], d2 = sh[3 * bm + 2];
    refine_rounds<KP, SM>(a, pc, ln.lg, nch, ns, S, d0, d1, d2, best);
    if (ln.lg != 0 || !pc.in) return;
    if (!pc.finite) {
        write_bad(a, pc.i);
        if (a.nvs) a.nvs[pc.i] = -1;
        return;
    }
    write_out(a, pc.i, pc.nv, d0, d1, d2, best, bm);
}

constexpr int kCostThreads = 128;

template <int KP>
__global__ void __launch_bounds__(kCostThreads) k_fuse(CostArgs a) {
    extern __shared__ __align__(16) float smem_f[];
    fuse_tile<KP>(a, blockIdx.x, smem_f);
}

// The learned path after the network, for the points of one tile.
template <int KP>
__device__ __forceinline__ void learn_tile(const LearnArgs& la, int tile) {
    constexpr int SM = SlotsFor<KP>::value;
    const CostArgs& a = la.f;
    const int cnt = a.N;
    Lanes ln;
    if (!lanes_of(a.L, tile, cnt, ln)) return;
    PointCtx<KP> pc;
    point_ctx<KP>(a, ln.q, cnt, pc);
    int nch, ns;
    chunking<SM>(pc.nv, a.L, nch, ns);
    Slot<KP> S[SM];
    if (nch == 1) gather<KP, SM>(a, pc, ln.lg, 0, ns, S);
    float d0 = 1.0f, d1 = 0.0f, d2 = 0.0f;
    if (pc.finite) {
        d0 = la.start_dir[3 * pc.i];
        d1 = la.start_dir[3 * pc.i + 1];
        d2 = la.start_dir[3 * pc.i + 2];
    }
    const float dd[1][3] = {{d0, d1, d2}};
    float l0[1];
    dir_sums<KP, SM, 1>(a, pc, ln.lg, nch, ns, S, dd, 1.0f, l0);
    const float c0 = pc.nv ? 1.0f - l0[0] / (float)pc.nv : 1.0f;
    const bool lead = ln.lg == 0 && pc.in;
    const bool fb = lead && pc.finite && pc.nv > 0 && c0 > la.tau;
    const bool ok = lead && pc.finite && !fb;
    if (lead && a.nvs) a.nvs[pc.i] = pc.finite ? pc.nv : -1;
    // warp-aggregated appends to the fallback list and work counts
    const unsigned mfb = __ballot_sync(0xffffffffu, fb);
    if (mfb) {
        const int leader = __ffs(mfb) - 1;
        int base = 0;
        if (ln.lane == leader) base = atomicAdd(la.fb_count, __popc(mfb));
        base = __shfl_sync(0xffffffffu, base, leader);
        if (fb) la.fb_list[base + __popc(mfb & ((1u << ln.lane) - 1u))] = pc.i;
    }
    const unsigned wfb = __reduce_add_sync(0xffffffffu, fb ? (unsigned)pc.nv : 0u);
    const unsigned wok = __reduce_add_sync(0xffffffffu, ok ? (unsigned)pc.nv : 0u);
    if (ln.lane == 0) {
        if (la.fb_work && wfb) atomicAdd(la.fb_work, (unsigned long long)wfb);
        if (la.acc_work && wok) atomicAdd(la.acc_work, (unsigned long long)wok);
    }
    // short refinement from the proposal (every group takes part in the shuffles; the fallback
    // points' results are dropped)
    float best = l0[0];
    refine_rounds<KP, SM>(a, pc, ln.lg, nch, ns, S, d0, d1, d2, best);
    if (!lead) return;
    if (!pc.finite) {
        write_bad(a, pc.i);
        return;
    }
    if (ok) write_out(a, pc.i, pc.nv, d0, d1, d2, best, -1);
}

template <int KP>
__global__ void __launch_bounds__(kCostThreads) k_learn(LearnArgs la) {
    learn_tile<KP>(la, blockIdx.x);
}

// ------------------------------------------------------------------ cost of given directions
template <int KP>
__global__ void __launch_bounds__(kCostThreads) k_eval(EvalArgs e) {
    constexpr int SM = SlotsFor<KP>::value;
    const CostArgs& a = e.f;
    Lanes ln;
    if (!lanes_of(a.L, blockIdx.x, a.N, ln)) return;
    PointCtx<KP> pc;
    point_ctx<KP>(a, ln.q, a.N, pc);
    int nch, ns;
    chunking<SM>(pc.nv, a.L, nch, ns);
    Slot<KP> S[SM];
    if (nch == 1) gather<KP, SM>(a, pc, ln.lg, 0, ns, S);
    for (int m = 0; m < e.M; ++m) {
        const float* d = e.dirs + ((size_t)pc.i * e.M + m) * 3;
        const float dd[1][3] = {{d[0], d[1], d[2]}};
        const float dn2 = fmaf(dd[0][0], dd[0][0], fmaf(dd[0][1], dd[0][1], __fmul_rn(dd[0][2], dd[0][2])));
        float l[1];
        dir_sums<KP, SM, 1>(a, pc, ln.lg, nch, ns, S, dd, dn2, l);
        if (ln.lg == 0 && pc.in) e.cost[(size_t)pc.i * e.M + m] = pc.nv ? 1.0f - l[0] / (float)pc.nv : 1.0f;
    }
}

// ------------------------------------------------------------------ learned proposal path
// Features of one point for the proposal network: for the 16 views v_m = floor(m V / 16),
// (sin 2 theta, cos 2 theta, C) at the point's pixel (zeros when it projects outside), then the
// position (p - centre) / half_extent of the point cloud's bounding box; bf16, zero-padded to 64.
constexpr int kFeatThreads = 128;

__device__ __forceinline__ void features_tile(const FeatArgs& a, int blk) {
    const int i = blk * kFeatThreads + threadIdx.x;
    if (i >= a.N) return;
    const float p0 = a.pts[3 * i], p1 = a.pts[3 * i + 1], p2 = a.pts[3 * i + 2];
    const size_t npx = (size_t)a.W * a.H;
    uint16_t f[64];
#pragma unroll
    for (int q = 0; q < 64; ++q) f[q] = 0;
    // all 16 pixel decisions first, then the 16 gathers in flight together, then the features
    long long off[16];
#pragma unroll
    for (int m = 0; m < 16; ++m) {
        const int v = (m * a.V) / 16;
        const float* cam = a.cams + 16 * v;
        off[m] = -1;
        const ff X0 = ff_dot3_plus(cam[4], cam[5], cam[6], p0, p1, p2, cam[13]);
        const ff X1 = ff_dot3_plus(cam[7], cam[8], cam[9], p0, p1, p2, cam[14]);
        const ff X2 = ff_dot3_plus(cam[10], cam[11], cam[12], p0, p1, p2, cam[15]);
        if (!(X2.hi > 1e-6f)) continue;
        const float fu = ff_floor(ff_affine(cam[0], ff_div(X0, X2), cam[2]));
        const float fv = ff_floor(ff_affine(cam[1], ff_div(X1, X2), cam[3]));
        if (!(fu >= 0.0f && fu < (float)a.W && fv >= 0.0f && fv < (float)a.H)) continue;
        off[m] = (long long)((size_t)v * npx + (size_t)fv * a.W + (size_t)fu);
    }
    float th[16], C[16];
#pragma unroll
    for (int m = 0; m < 16; ++m) {
        th[m] = 0.0f;
        C[m] = 0.0f;
        if (off[m] < 0) continue;
        if (a.amap) {
            const float2 t = __ldg(a.amap + off[m]);
            th[m] = t.x;
            C[m] = t.y;
        } else {
            th[m] = a.angle[off[m]];
            C[m] = load_conf(a.conf, a.conf_f16, (size_t)off[m]);
        }
    }
#pragma unroll
    for (int m = 0; m < 16; ++m) {
        if (off[m] < 0) continue;
        float s2, c2;
        sincosf(2.0f * th[m], &s2, &c2);
        f[3 * m] = __bfloat16_as_ushort(__float2bfloat16_rn(s2));
        f[3 * m + 1] = __bfloat16_as_ushort(__float2bfloat16_rn(c2));
        f[3 * m + 2] = __bfloat16_as_ushort(__float2bfloat16_rn(C[m]));
    }
    float b[6];
#pragma unroll
    for (int q = 0; q < 6; ++q) b[q] = a.box_keys ? fval(a.box_keys[q]) : a.box[q];
    float half = 0.5f * fmaxf(fmaxf(b[3] - b[0], b[4] - b[1]), b[5] - b[2]);
    if (!(half > 0.0f)) half = 1.0f;
    const float pc[3] = {p0, p1, p2};
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        const float c = 0.5f * (b[q] + b[3 + q]);
        const float x = isfinite(pc[q]) ? (pc[q] - c) / half : 0.0f;
        f[48 + q] = __bfloat16_as_ushort(__float2bfloat16_rn(x));
    }
    uint4* dst = reinterpret_cast<uint4*>(a.x + (size_t)i * 64);
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        uint4 w;
        w.x = f[8 * q] | ((uint32_t)f[8 * q + 1] << 16);
        w.y = f[8 * q + 2] | ((uint32_t)f[8 * q + 3] << 16);
        w.z = f[8 * q + 4] | ((uint32_t)f[8 * q + 5] << 16);
        w.w = f[8 * q + 6] | ((uint32_t)f[8 * q + 7] << 16);
        dst[q] = w;
    }
}

__global__ void __launch_bounds__(kFeatThreads) k_features(FeatArgs a) { features_tile(a, blockIdx.x); }

__global__ void k_rot(float2* rot, int T, double alpha0) {
    const int t = threadIdx.x;
    if (t < T) {
        const double al = alpha0 / (double)(1u << t);
        rot[t] = make_float2((float)cos(al), (float)sin(al));
    }
}

__global__ void k_check_nbr(const int32_t* __restrict__ nbr, long long n, int N, uint32_t* errw) {
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        const int j = nbr[e];
        if (j < 0 || j >= N) {
            atomicOr(errw, HF_DEV_ERR_BAD_NBR);
            return;
        }
    }
}

// ------------------------------------------------------------------ batched scenes
// One persistent grid per stage walks the (scene, tile) items of every scene of a batch, scenes in
// the order of the argument array: a CTA takes the next item from a global counter, copies that
// scene's arguments to shared memory when the scene changes, and runs the single-scene tile body,
// so a batched result is bit-identical to the scene run alone.  With c.done set, the CTA that
// finishes a scene's last tile stamps the global timer (per-scene completion time).
__device__ __forceinline__ unsigned long long gtimer() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// tiles(args) gives a scene's tile count (evaluated on the device: list lengths are device counts)
template <typename Args, typename Tiles, typename Body>
__device__ __forceinline__ void batch_tiles(const Args* __restrict__ args, const BatchCtl& c, Tiles tiles, Body body) {
    __shared__ Args sa;
    __shared__ int pref[HF_MAX_BATCH + 1];
    __shared__ int s_item, s_pos, s_cur;
    if (threadIdx.x == 0) {
        pref[0] = 0;
        for (int p = 0; p < c.ns; ++p) pref[p + 1] = pref[p] + tiles(args[p]);
        s_cur = -1;
    }
    for (;;) {
        __syncthreads();   // the previous item is done with shared memory
        if (threadIdx.x == 0) {
            const int t = (int)atomicAdd(c.next, 1u);
            int p = 0;
            while (p < c.ns - 1 && t >= pref[p + 1]) ++p;
            s_item = t;
            s_pos = p;
            if (t < pref[c.ns] && p != s_cur) {
                sa = args[p];
                s_cur = p;
            }
        }
        __syncthreads();
        const int t = s_item, p = s_pos;
        if (t >= pref[c.ns]) break;
        body(sa, t - pref[p]);
        if (c.done) {
            __syncthreads();   // every thread's outputs of the tile are written
            if (threadIdx.x == 0) {
                __threadfence();
                if ((int)atomicAdd(c.done + p, 1u) + 1 == pref[p + 1] - pref[p]) c.stamp[p] = gtimer();
            }
        }
    }
}

// points per CTA of the cost kernels: 32 / L points per warp
__device__ __forceinline__ int cost_tiles(const CostArgs& a, int cnt) {
    const int ppc = (int)(blockDim.x >> 5) * (32 / a.L);
    return (cnt + ppc - 1) / ppc;
}

template <int KP, int NT>
__global__ void __launch_bounds__(NT) k_fuse_batch(const CostArgs* __restrict__ fa, BatchCtl c) {
    extern __shared__ __align__(16) float smem_f[];
    batch_tiles(fa, c, [](const CostArgs& a) { return cost_tiles(a, a.list ? *a.list_count : a.N); },
                [&](const CostArgs& a, int t) { fuse_tile<KP>(a, t, smem_f); });
}

template <int KP, int NT>
__global__ void __launch_bounds__(NT) k_learn_batch(const LearnArgs* __restrict__ la, BatchCtl c) {
    batch_tiles(la, c, [](const LearnArgs& a) { return cost_tiles(a.f, a.f.N); },
                [](const LearnArgs& a, int t) { learn_tile<KP>(a, t); });
}

__global__ void __launch_bounds__(kProjectThreads) k_project_batch(const ProjectArgs* __restrict__ pa, BatchCtl c) {
    batch_tiles(pa, c, [](const ProjectArgs& a) { return (a.N + kProjectThreads - 1) / kProjectThreads; },
                [](const ProjectArgs& a, int blk) {
                    if (a.top_k > 0) project_tile<true>(a, blk);
                    else project_tile<false>(a, blk);
                });
}

__global__ void __launch_bounds__(kFeatThreads) k_features_batch(const FeatArgs* __restrict__ fe, BatchCtl c) {
    batch_tiles(fe, c, [](const FeatArgs& a) { return (a.N + kFeatThreads - 1) / kFeatThreads; },
                [](const FeatArgs& a, int blk) { features_tile(a, blk); });
}

// Per-scene constants of every scene (block = scene), the batch's counters cleared, empty bounding
// boxes, the short-refinement rotation steps, and the batch start time.
__global__ void k_prep_batch(const PrepArgs* __restrict__ pr, BatchReset r) {
    if (blockIdx.x == 0 && threadIdx.x == 0 && r.t0) *r.t0 = gtimer();
    prep_body(pr[blockIdx.x]);
    if (r.box_keys && threadIdx.x < 6) r.box_keys[6 * blockIdx.x + threadIdx.x] = threadIdx.x < 3 ? 0xffffffffu : 0u;
    if (blockIdx.x == 0) {
        for (int w = threadIdx.x; w < r.nzero; w += blockDim.x) r.zero[w] = 0u;
        if (r.rot_s && (int)threadIdx.x < r.T_short) {
            const double al = r.alpha_short / (double)(1u << threadIdx.x);
            r.rot_s[threadIdx.x] = make_float2((float)cos(al), (float)sin(al));
        }
    }
}

// persistent grid: resident CTAs per SM x SMs
template <typename K>
int persistent_grid(K kernel, int threads, size_t smem) {
    static int sms = 0;
    if (!sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (sms <= 0) sms = 1;
    }
    int per = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kernel, threads, smem) != cudaSuccess || per < 1) per = 1;
    return per * sms;
}

template <typename K>
cudaError_t set_smem(K kernel, size_t smem, cudaStream_t s) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaStreamIsCapturing(s, &cs);
    if (cs != cudaStreamCaptureStatusNone) return cudaSuccess;   // set by the eager launch before capture
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

// patch width (k + 1) rounded up to an instantiated size
int kp_for(int k) {
    const int need = k + 1;
    if (need <= 1) return 1;
    if (need <= 4) return 4;
    if (need <= 6) return 6;
    if (need <= 9) return 9;
    if (need <= 12) return 12;
    return 17;
}

int slots_for_kp(int kp) {
    switch (kp) {
        case 1: return SlotsFor<1>::value;
        case 4: return SlotsFor<4>::value;
        case 6: return SlotsFor<6>::value;
        case 9: return SlotsFor<9>::value;
        case 12: return SlotsFor<12>::value;
        default: return SlotsFor<17>::value;
    }
}

template <int KP, int NT>
cudaError_t launch_fuse_batch(const CostArgs* fa, const BatchCtl& c, int hpad_max, cudaStream_t s) {
    const size_t sm = (size_t)3 * hpad_max * sizeof(float);
    cudaError_t e = set_smem(k_fuse_batch<KP, NT>, sm, s);
    if (e != cudaSuccess) return e;
    const int grid = persistent_grid(k_fuse_batch<KP, NT>, NT, sm);
    k_fuse_batch<KP, NT><<<grid, NT, sm, s>>>(fa, c);
    return cudaGetLastError();
}

template <int KP, int NT>
cudaError_t launch_learn_batch(const LearnArgs* la, const BatchCtl& c, cudaStream_t s) {
    static int grid = 0;
    if (!grid) grid = persistent_grid(k_learn_batch<KP, NT>, NT, 0);
    k_learn_batch<KP, NT><<<grid, NT, 0, s>>>(la, c);
    return cudaGetLastError();
}

template <int KP>
cudaError_t launch_fuse_batch_nt(const CostArgs* fa, const BatchCtl& c, int nt, int hpad_max, cudaStream_t s) {
    switch (nt) {
        case 64: return launch_fuse_batch<KP, 64>(fa, c, hpad_max, s);
        case 256: return launch_fuse_batch<KP, 256>(fa, c, hpad_max, s);
        default: return launch_fuse_batch<KP, 128>(fa, c, hpad_max, s);
    }
}

template <int KP>
cudaError_t launch_learn_batch_nt(const LearnArgs* la, const BatchCtl& c, int nt, cudaStream_t s) {
    switch (nt) {
        case 64: return launch_learn_batch<KP, 64>(la, c, s);
        case 256: return launch_learn_batch<KP, 256>(la, c, s);
        default: return launch_learn_batch<KP, 128>(la, c, s);
    }
}

template <int KP>
cudaError_t launch_fuse_kp(const CostArgs& a, cudaStream_t s) {
    const int cnt_max = a.N;   // with a list, its length is at most N (tiles past the list exit at once)
    const int ppc = kCostThreads / a.L;
    const dim3 grid((cnt_max + ppc - 1) / ppc), block(kCostThreads);
    const size_t sm = (size_t)3 * a.Hpad * sizeof(float);
    cudaError_t e = set_smem(k_fuse<KP>, sm, s);
    if (e != cudaSuccess) return e;
    k_fuse<KP><<<grid, block, sm, s>>>(a);
    return cudaGetLastError();
}

template <int KP>
cudaError_t launch_learn_kp(const LearnArgs& a, cudaStream_t s) {
    const int ppc = kCostThreads / a.f.L;
    k_learn<KP><<<(a.f.N + ppc - 1) / ppc, kCostThreads, 0, s>>>(a);
    return cudaGetLastError();
}

template <int KP>
cudaError_t launch_eval_kp(const EvalArgs& a, cudaStream_t s) {
    const int ppc = kCostThreads / a.f.L;
    k_eval<KP><<<(a.f.N + ppc - 1) / ppc, kCostThreads, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace

int hf_cost_lanes(int veff, int k) {
    const int sm = slots_for_kp(kp_for(k));
    int L = 4;
    while (L < 32 && L * sm < veff) L *= 2;
    return L;
}

cudaError_t hf_launch_project(const ProjectArgs& a, cudaStream_t s) {
    const dim3 grid((a.N + kProjectThreads - 1) / kProjectThreads), block(kProjectThreads);
    if (a.top_k > 0) k_project<true><<<grid, block, 0, s>>>(a);
    else k_project<false><<<grid, block, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t hf_launch_iota(int32_t* list, int* count, int first, int n, cudaStream_t s) {
    k_iota<<<(n + 255) / 256 > 0 ? (n + 255) / 256 : 1, 256, 0, s>>>(list, count, first, n);
    return cudaGetLastError();
}

cudaError_t hf_launch_interleave(const float* angle, const void* conf, int conf_f16, size_t npx, float2* out,
                                 cudaStream_t s) {
    if (!npx) return cudaSuccess;
    const size_t blocks = (npx + 255) / 256;
    k_interleave<<<(unsigned)(blocks < 148 * 16 ? blocks : 148 * 16), 256, 0, s>>>(angle, conf, conf_f16, npx, out);
    return cudaGetLastError();
}

cudaError_t hf_launch_prep(const PrepArgs& a, cudaStream_t s) {
    k_prep<<<1, 256, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t hf_launch_fuse(const CostArgs& a, cudaStream_t s) {
    switch (kp_for(a.k)) {
        case 1: return launch_fuse_kp<1>(a, s);
        case 4: return launch_fuse_kp<4>(a, s);
        case 6: return launch_fuse_kp<6>(a, s);
        case 9: return launch_fuse_kp<9>(a, s);
        case 12: return launch_fuse_kp<12>(a, s);
        default: return launch_fuse_kp<17>(a, s);
    }
}

cudaError_t hf_launch_learn(const LearnArgs& a, cudaStream_t s) {
    switch (kp_for(a.f.k)) {
        case 1: return launch_learn_kp<1>(a, s);
        case 4: return launch_learn_kp<4>(a, s);
        case 6: return launch_learn_kp<6>(a, s);
        case 9: return launch_learn_kp<9>(a, s);
        case 12: return launch_learn_kp<12>(a, s);
        default: return launch_learn_kp<17>(a, s);
    }
}

cudaError_t hf_launch_eval(const EvalArgs& a, cudaStream_t s) {
    switch (kp_for(a.f.k)) {
        case 1: return launch_eval_kp<1>(a, s);
        case 4: return launch_eval_kp<4>(a, s);
        case 6: return launch_eval_kp<6>(a, s);
        case 9: return launch_eval_kp<9>(a, s);
        case 12: return launch_eval_kp<12>(a, s);
        default: return launch_eval_kp<17>(a, s);
    }
}

cudaError_t hf_launch_fib(int H, float* out, cudaStream_t s) {
    k_fib<<<(H + 127) / 128, 128, 0, s>>>(H, out);
    return cudaGetLastError();
}

cudaError_t hf_launch_features(const FeatArgs& a, cudaStream_t s) {
    k_features<<<(a.N + kFeatThreads - 1) / kFeatThreads, kFeatThreads, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t hf_launch_rot(float2* rot, int T, double alpha0, cudaStream_t s) {
    if (T <= 0) return cudaSuccess;
    k_rot<<<1, 32, 0, s>>>(rot, T, alpha0);
    return cudaGetLastError();
}

cudaError_t hf_launch_check_nbr(const int32_t* nbr, long long n, int N, uint32_t* errw, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    const long long blocks = (n + 255) / 256;
    k_check_nbr<<<(unsigned)(blocks < 1184 ? blocks : 1184), 256, 0, s>>>(nbr, n, N, errw);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ batched launchers
int hf_batch_kp_for(int k) { return k + 1 <= 4 ? 4 : (k + 1 <= 9 ? 9 : 17); }

cudaError_t hf_launch_prep_batch(const PrepArgs* pr, int ns, const BatchReset& r, cudaStream_t s) {
    k_prep_batch<<<ns, 256, 0, s>>>(pr, r);
    return cudaGetLastError();
}

cudaError_t hf_launch_project_batch(const ProjectArgs* pa, const BatchCtl& c, cudaStream_t s) {
    static int grid = 0;
    if (!grid) grid = persistent_grid(k_project_batch, kProjectThreads, 0);
    k_project_batch<<<grid, kProjectThreads, 0, s>>>(pa, c);
    return cudaGetLastError();
}

cudaError_t hf_launch_features_batch(const FeatArgs* fe, const BatchCtl& c, cudaStream_t s) {
    static int grid = 0;
    if (!grid) grid = persistent_grid(k_features_batch, kFeatThreads, 0);
    k_features_batch<<<grid, kFeatThreads, 0, s>>>(fe, c);
    return cudaGetLastError();
}

cudaError_t hf_launch_fuse_batch(const CostArgs* fa, const BatchCtl& c, int kp, int nt, int hpad_max, cudaStream_t s) {
    switch (kp) {
        case 4: return launch_fuse_batch_nt<4>(fa, c, nt, hpad_max, s);
        case 9: return launch_fuse_batch_nt<9>(fa, c, nt, hpad_max, s);
        default: return launch_fuse_batch_nt<17>(fa, c, nt, hpad_max, s);
    }
}

cudaError_t hf_launch_learn_batch(const LearnArgs* la, const BatchCtl& c, int kp, int nt, cudaStream_t s) {
    switch (kp) {
        case 4: return launch_learn_batch_nt<4>(la, c, nt, s);
        case 9: return launch_learn_batch_nt<9>(la, c, nt, s);
        default: return launch_learn_batch_nt<17>(la, c, nt, s);
    }
}
