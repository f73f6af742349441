// hf_kernels.cu - the fusion path's device code for sm_103a.
//
//   k_prep          per-scene constants: hypotheses (padded to an even count), degenerate
//                   thresholds, refinement rotation steps.
//   k_project       K1, thread per point: projection of the point into every view with the pixel
//                   index decided in float-float arithmetic, nearest-pixel gather of the orientation
//                   and confidence maps, view set (visible or top-K) of the point.
//   k_argmin<KP>    K2, thread per point: the cost of every hypothesis (Eqs. proj_r .. patch_min and
//                   the view mean) and their argmin, hypotheses in packed pairs.
//   k_refine<KP,L>  K3, a group of L lanes per point: T rounds of the six-rotation refinement from
//                   the argmin hypothesis (or a given start), the point's patch gathered once and held
//                   in registers across the rounds.
//   k_select<KP>    the learned path after the network: cost of the proposal and fallback selection.
//   k_eval<KP,L>    cost of caller-given directions (no argmin).
#include <math.h>

#include <cuda_bf16.h>

#include "hf_batchtiles.cuh"
#include "hf_cost.cuh"
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
// One thread per point, views in order.  For view v it writes
//   samp[v][i] = C (cos theta, sin theta) at the point's pixel (0 when outside the view),
//   ab[v][i]   = (X/Z, Y/Z) when v is in the point's view set, NaN otherwise,
// and the point's view-set mask vmask[i][v / 64] (bit v % 64).  The view set is every view the
// point projects into, or with top_k > 0 the top_k of them by the confidence at the point's own
// pixel, ties to the lower view index.
constexpr int kProjectThreads = 128;

// With a.box_keys set, the tile also folds its finite coordinates into the point cloud's bounding
// box (keys lo[3] from 0xffffffff, hi[3] from 0, per coordinate).
// The pixel of point p in the camera record cam (fx, fy, cx, cy, R row-major, t) and its projection
// ratios (X/Z, Y/Z); false when the depth is not above 1e-6 or the pixel is outside W x H.  FP32
// first, with a bound on its error: X = R p + t by nested FMAs is within 3 u S of exact (u = 2^-24,
// S the sum of the absolute terms; 8 u S is used), the ratio's error is then at most
// (e_X + |ra| e_Z) / (Z - e_Z) + u |ra| (a correctly rounded division), and the pixel coordinate
// f ra + c adds one FMA rounding.  When the interval coordinate +- bound (rounded outward) holds no
// integer, floor() of the coordinate is the exact pixel; otherwise, and when the depth test is that
// close to its threshold, the float-float evaluation decides as before.
__device__ __forceinline__ bool pixel_of(const float* __restrict__ cam, float p0, float p1, float p2, int W, int H,
                                         float& fu, float& fv, float& ra_out, float& rb_out) {
    float4 c0, c1, c2, c3;   // the record: four 16-byte loads when aligned, else sixteen scalar ones
    if ((reinterpret_cast<uintptr_t>(cam) & 15) == 0) {
        const float4* c4 = reinterpret_cast<const float4*>(cam);
        c0 = __ldg(c4);
        c1 = __ldg(c4 + 1);
        c2 = __ldg(c4 + 2);
        c3 = __ldg(c4 + 3);
    } else {
        c0 = make_float4(__ldg(cam), __ldg(cam + 1), __ldg(cam + 2), __ldg(cam + 3));
        c1 = make_float4(__ldg(cam + 4), __ldg(cam + 5), __ldg(cam + 6), __ldg(cam + 7));
        c2 = make_float4(__ldg(cam + 8), __ldg(cam + 9), __ldg(cam + 10), __ldg(cam + 11));
        c3 = make_float4(__ldg(cam + 12), __ldg(cam + 13), __ldg(cam + 14), __ldg(cam + 15));
    }
    const float fx = c0.x, fy = c0.y, cx = c0.z, cy = c0.w;
    const float r00 = c1.x, r01 = c1.y, r02 = c1.z;
    const float r10 = c1.w, r11 = c2.x, r12 = c2.y;
    const float r20 = c2.z, r21 = c2.w, r22 = c3.x;
    const float t0 = c3.y, t1 = c3.z, t2 = c3.w;
    const float x0 = fmaf(r00, p0, fmaf(r01, p1, fmaf(r02, p2, t0)));
    const float x1 = fmaf(r10, p0, fmaf(r11, p1, fmaf(r12, p2, t1)));
    const float x2 = fmaf(r20, p0, fmaf(r21, p1, fmaf(r22, p2, t2)));
    const float e0 = 0x1p-21f * (fabsf(r00 * p0) + fabsf(r01 * p1) + fabsf(r02 * p2) + fabsf(t0));
    const float e1 = 0x1p-21f * (fabsf(r10 * p0) + fabsf(r11 * p1) + fabsf(r12 * p2) + fabsf(t1));
    const float e2 = 0x1p-21f * (fabsf(r20 * p0) + fabsf(r21 * p1) + fabsf(r22 * p2) + fabsf(t2));
    const float zlo = __fsub_rd(x2, e2);
    bool decided = false;
    if (zlo > 2e-6f) {
        const float ra = __fdiv_rn(x0, x2), rb = __fdiv_rn(x1, x2);
        // 1 / zlo rounded up: the bounds take a product instead of two divisions
        const float rz = __frcp_ru(zlo);
        const float dra = 1.01f * ((e0 + fabsf(ra) * e2) * rz + 0x1p-23f * fabsf(ra));
        const float drb = 1.01f * ((e1 + fabsf(rb) * e2) * rz + 0x1p-23f * fabsf(rb));
        const float u = fmaf(fx, ra, cx), v = fmaf(fy, rb, cy);
        const float eu = 1.01f * (fabsf(fx) * dra + 0x1p-23f * fabsf(u)) + 1e-30f;
        const float ev = 1.01f * (fabsf(fy) * drb + 0x1p-23f * fabsf(v)) + 1e-30f;
        const float ulo = floorf(__fsub_rd(u, eu)), uhi = floorf(__fadd_ru(u, eu));
        const float vlo = floorf(__fsub_rd(v, ev)), vhi = floorf(__fadd_ru(v, ev));
        if (ulo == uhi && vlo == vhi && isfinite(u) && isfinite(v)) {
            fu = ulo;
            fv = vlo;
            ra_out = ra;
            rb_out = rb;
            decided = true;
        }
    } else if (__fadd_ru(x2, e2) < 0.5e-6f) {
        return false;   // behind (or at) the camera
    }
    if (!decided) {
        const ff X0 = ff_dot3_plus(r00, r01, r02, p0, p1, p2, t0);
        const ff X1 = ff_dot3_plus(r10, r11, r12, p0, p1, p2, t1);
        const ff X2 = ff_dot3_plus(r20, r21, r22, p0, p1, p2, t2);
        if (!(X2.hi > 1e-6f)) return false;
        const ff ra = ff_div(X0, X2), rb = ff_div(X1, X2);
        fu = ff_floor(ff_affine(fx, ra, cx));
        fv = ff_floor(ff_affine(fy, rb, cy));
        ra_out = ra.hi;
        rb_out = rb.hi;
    }
    return fu >= 0.0f && fu < (float)W && fv >= 0.0f && fv < (float)H;
}

template <bool TOPK, bool FEAT>
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
    const int Vw = hf_mask_words(a.V);
    unsigned long long* mrow = a.vmask + (size_t)i * Vw;
    const float qnan = __int_as_float(0x7fc00000);
    float topc[HF_MAX_TOPK];
    int topv[HF_MAX_TOPK];
    int ntop = 0, nset = 0;
    unsigned long long word = 0ull;
    // the network's view features: slot m (< 16) samples view floor(m V / 16); fm is the next slot
    // and fvw its view (warp-uniform).  Four slots (12 bf16, 24 bytes) are collected in a 192-bit
    // shift register fa : fb : fc and written as three 8-byte stores.
    int fm = 0, fvw = 0;
    uint16_t* frow = FEAT && a.featx ? a.featx + (size_t)i * 64 : nullptr;
    unsigned long long fa = 0ull, fb = 0ull, fc = 0ull;
    // views in groups of four: the pixel decisions first, then the four gathers in flight together
    constexpr int G = 4;
    for (int v0 = 0; v0 < a.V; v0 += G) {
        long long off[G];
        float ra_[G], rb_[G];
#pragma unroll
        for (int q = 0; q < G; ++q) {
            off[q] = -1;
            ra_[q] = rb_[q] = qnan;
            const int v = v0 + q;
            if (v >= a.V) continue;
            float fu, fv, ra, rb;
            if (!pixel_of(a.cams + 16 * v, p0, p1, p2, a.W, a.H, fu, fv, ra, rb)) continue;
            // fu, fv are whole numbers below 2^22: the integer is the low mantissa bits of
            // f + 1.5 * 2^23 (exact; no conversion instruction, none on the FP64 pipe)
            const int iu = __float_as_int(fu + 12582912.0f) - 0x4B400000;
            const int iv = __float_as_int(fv + 12582912.0f) - 0x4B400000;
            off[q] = (long long)v * (long long)npx + (long long)(iv * a.W + iu);
            ra_[q] = ra;
            rb_[q] = rb;
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
        if (FEAT && frow) {
            // (sin 2 theta, cos 2 theta, C) of each feature slot whose view is in this group, zeros
            // when the point projects outside it
#pragma unroll
            for (int q = 0; q < G; ++q) {
                while (fm < 16 && fvw == v0 + q) {
                    uint16_t h0 = 0, h1 = 0, h2 = 0;
                    if (off[q] >= 0) {
                        float s2, c2;
                        sincosf(2.0f * th[q], &s2, &c2);
                        h0 = __bfloat16_as_ushort(__float2bfloat16_rn(s2));
                        h1 = __bfloat16_as_ushort(__float2bfloat16_rn(c2));
                        h2 = __bfloat16_as_ushort(__float2bfloat16_rn(C[q]));
                    }
                    const unsigned long long t = (unsigned long long)h0 | ((unsigned long long)h1 << 16) |
                                                 ((unsigned long long)h2 << 32);
                    fa = (fa >> 48) | (fb << 16);
                    fb = (fb >> 48) | (fc << 16);
                    fc = (fc >> 48) | (t << 16);
                    if ((fm & 3) == 3) {   // slots fm - 3 .. fm: columns 3 (fm - 3) .. 3 fm + 2
                        unsigned long long* dst = reinterpret_cast<unsigned long long*>(frow + 3 * (fm - 3));
                        dst[0] = fa;
                        dst[1] = fb;
                        dst[2] = fc;
                    }
                    ++fm;
                    fvw = (fm * a.V) >> 4;
                }
            }
        }
        float2 svq[G], rq[G];   // this group's samples and ratios (a view past V: 0 and NaN)
#pragma unroll
        for (int q = 0; q < G; ++q) {
            const int v = v0 + q;
            float2 sv = make_float2(0.0f, 0.0f), r = make_float2(qnan, qnan);
            if (v < a.V && off[q] >= 0) {
                float sn, cn;
                __sincosf(th[q], &sn, &cn);   // theta in [0, pi): absolute error below 1e-6
                sv = make_float2(C[q] * cn, C[q] * sn);
                r = make_float2(ra_[q], rb_[q]);
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
            svq[q] = sv;
            rq[q] = r;
        }
        // one 16-byte store per view pair (G is even and v0 a multiple of G: pairs never straddle)
#pragma unroll
        for (int q = 0; q < G; q += 2)
            if (v0 + q < a.V) {
                const size_t e = hf_pv(v0 + q, i, a.N) >> 1;   // float4 element of the pair
                reinterpret_cast<float4*>(a.samp)[e] = make_float4(svq[q].x, svq[q].y, svq[q + 1].x, svq[q + 1].y);
                reinterpret_cast<float4*>(a.ab)[e] = make_float4(rq[q].x, rq[q].y, rq[q + 1].x, rq[q + 1].y);
            }
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
        for (int v = 0; v < a.V; ++v) {
            bool keep = false;
            for (int q = 0; q < ntop; ++q) keep |= (topv[q] == v);
            if (!keep) a.ab[hf_pv(v, i, a.N)] = make_float2(qnan, qnan);
        }
        nset = ntop;
    }
    // warp-aggregated count of the (point, view) pairs in the view sets
    const unsigned am = __activemask();
    const unsigned tot = __reduce_add_sync(am, (unsigned)nset);
    if ((threadIdx.x & 31) == __ffs(am) - 1) atomicAdd(a.work, (unsigned long long)tot);
}

template <bool TOPK, bool FEAT>
__global__ void __launch_bounds__(kProjectThreads) k_project(ProjectArgs a) {
    project_tile<TOPK, FEAT>(a, blockIdx.x);
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
    if (a.qtab) {
        __syncthreads();   // the hypotheses are written
        // hypothesis pairs (m, m+1), q = R_v h in double, folded with fx / fy (past Hpad: h_0)
        for (int e = threadIdx.x; e < a.V * (a.Hq / 2); e += blockDim.x) {
            const int v = e / (a.Hq / 2), m = 2 * (e % (a.Hq / 2));
            const float* cam = a.cams + 16 * v;
            double q[2][3];
            for (int h = 0; h < 2; ++h) {
                const int src = m + h < a.Hpad ? m + h : 0;
                for (int r = 0; r < 3; ++r)
                    q[h][r] = (double)cam[4 + 3 * r] * a.hyps[3 * src] + (double)cam[5 + 3 * r] * a.hyps[3 * src + 1] +
                              (double)cam[6 + 3 * r] * a.hyps[3 * src + 2];
            }
            const double fx = cam[0], fy = cam[1];
            a.qtab[(size_t)v * a.Hq + m] =
                make_float4((float)(fx * q[0][0]), (float)(fx * q[1][0]), (float)(fx * q[0][2]), (float)(fx * q[1][2]));
            a.qtab[(size_t)v * a.Hq + m + 1] =
                make_float4((float)(fy * q[0][1]), (float)(fy * q[1][1]), (float)(fy * q[0][2]), (float)(fy * q[1][2]));
        }
    }
    for (int t = threadIdx.x; t < a.T; t += blockDim.x) {
        const double al = 0.5 * sqrt(2.0 * kPi / a.H) / (double)(1u << t);
        a.rot[t] = make_float2((float)cos(al), (float)sin(al));
    }
}

__global__ void k_prep(PrepArgs a) { prep_body(a); }

// ------------------------------------------------------------------ K2 + K3 (device code in hf_cost.cuh)
using namespace hf_cost;

constexpr int kCostThreads = 128;
// resident CTAs per SM the register budget is sized for: 16 warps per SM (12 for the widest patch)
template <int KP>
struct MinCtas {
    static constexpr int value = KP <= 9 ? 4 : 3;
};

template <int KP>
__global__ void __launch_bounds__(kCostThreads, 4) k_argmin(CostArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    argmin_tile<KP, kCostThreads>(a, blockIdx.x, smem_raw);
}

template <int KP, int L>
__global__ void __launch_bounds__(kCostThreads, MinCtas<KP>::value) k_refine(CostArgs a) {
    refine_tile_l<KP, L, PairsFor<KP>::value>(a, blockIdx.x);
}

template <int KP>
__global__ void __launch_bounds__(kCostThreads) k_refine_t(CostArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    refine_stage_tile<KP, kCostThreads>(a, blockIdx.x, smem_raw);
}

template <int KP>
__global__ void __launch_bounds__(kCostThreads) k_select(LearnArgs la) {
    select_tile<KP>(la, blockIdx.x);
}

template <int KP, int L>
__global__ void __launch_bounds__(kCostThreads) k_eval(EvalArgs e) {
    eval_tile_l<KP, L, PairsFor<KP>::value>(e, blockIdx.x);
}

// ------------------------------------------------------------------ learned proposal path
// Features of one point for the proposal network: for the 16 views v_m = floor(m V / 16),
// (sin 2 theta, cos 2 theta, C) at the point's pixel (zeros when it projects outside), then the
// position (p - centre) / half_extent of the point cloud's bounding box; bf16, zero-padded to 64.
// The view part comes from the projection (project_tile with featx set), which has the samples in
// registers; the position part needs the complete bounding box, which the projection folds, so it
// is written here, one 32-byte row tail per point.
constexpr int kFeatThreads = 128;

__device__ __forceinline__ void featpos_tile(const FeatArgs& a, int blk) {
    const int i = blk * kFeatThreads + threadIdx.x;
    if (i >= a.N) return;
    const float pc[3] = {a.pts[3 * i], a.pts[3 * i + 1], a.pts[3 * i + 2]};
    float b[6];
#pragma unroll
    for (int q = 0; q < 6; ++q) b[q] = a.box_keys ? fval(a.box_keys[q]) : a.box[q];
    float half = 0.5f * fmaxf(fmaxf(b[3] - b[0], b[4] - b[1]), b[5] - b[2]);
    if (!(half > 0.0f)) half = 1.0f;
    uint32_t f[3];
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        const float c = 0.5f * (b[q] + b[3 + q]);
        const float x = isfinite(pc[q]) ? (pc[q] - c) / half : 0.0f;
        f[q] = __bfloat16_as_ushort(__float2bfloat16_rn(x));
    }
    uint4* dst = reinterpret_cast<uint4*>(a.x + (size_t)i * 64 + 48);
    dst[0] = make_uint4(f[0] | (f[1] << 16), f[2], 0u, 0u);
    dst[1] = make_uint4(0u, 0u, 0u, 0u);
}

__global__ void __launch_bounds__(kFeatThreads) k_featpos(FeatArgs a) { featpos_tile(a, blockIdx.x); }

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

// Each point's neighbour list reordered by index distance |j - i|, the later of two equally distant
// indices first (a point per thread, once per upload).  The patch maximum (Eq. patch_min) does not
// depend on the order of the members, so the costs do not change; with this order member slot j of
// consecutive points tends to address nearby samples (points along a strand are consecutive), and
// the cost kernels' gathers of one slot across a warp touch fewer cache lines.
__global__ void k_order_nbr(int32_t* __restrict__ nbr, int N, int k) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N || k < 2 || k > HF_MAX_K) return;
    int32_t* row = nbr + (size_t)i * k;
    int v[HF_MAX_K];
    unsigned long long key[HF_MAX_K];
    for (int q = 0; q < k; ++q) {
        v[q] = row[q];
        const long long d = (long long)v[q] - i;
        key[q] = (unsigned long long)(d < 0 ? -d : d) * 2u + (d < 0 ? 1u : 0u);
    }
    for (int q = 1; q < k; ++q) {   // insertion sort, stable
        const int vq = v[q];
        const unsigned long long kq = key[q];
        int p = q - 1;
        for (; p >= 0 && key[p] > kq; --p) {
            key[p + 1] = key[p];
            v[p + 1] = v[p];
        }
        key[p + 1] = kq;
        v[p + 1] = vq;
    }
    for (int q = 0; q < k; ++q) row[q] = v[q];
}

// ------------------------------------------------------------------ batched scenes (work loop in hf_batchtiles.cuh)
using namespace hf_bt;

template <bool FEAT>
__global__ void __launch_bounds__(kProjectThreads, 7) k_project_batch(const ProjectArgs* __restrict__ pa, BatchCtl c) {
    batch_tiles(pa, c, [](const ProjectArgs& a) { return (a.N + kProjectThreads - 1) / kProjectThreads; },
                [](const ProjectArgs& sa, int blk) {
                    // a register copy: the tile's stores could alias the shared-memory arguments,
                    // which would make every field access a reload from shared memory
                    const ProjectArgs a = sa;
                    if (a.top_k > 0) project_tile<true, FEAT>(a, blk);
                    else project_tile<false, FEAT>(a, blk);
                });
}

__global__ void __launch_bounds__(kFeatThreads) k_featpos_batch(const FeatArgs* __restrict__ fe, BatchCtl c) {
    batch_tiles(fe, c, [](const FeatArgs& a) { return (a.N + kFeatThreads - 1) / kFeatThreads; },
                [](const FeatArgs& a, int blk) { featpos_tile(a, blk); });
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

// views a lane holds at once for a patch width: two per view pair
int slots_for_kp(int kp) {
    switch (kp) {
        case 1: return 2 * PairsFor<1>::value;
        case 4: return 2 * PairsFor<4>::value;
        case 6: return 2 * PairsFor<6>::value;
        case 9: return 2 * PairsFor<9>::value;
        case 12: return 2 * PairsFor<12>::value;
        default: return 2 * PairsFor<17>::value;
    }
}

template <int KP>
cudaError_t launch_argmin_kp(const CostArgs& a, cudaStream_t s) {
    const int cnt_max = a.N;   // with a list, its length is at most N (blocks past the list exit at once)
    const size_t sm = argmin_smem_bytes<KP, kCostThreads>();
    cudaError_t e = set_smem(k_argmin<KP>, sm, s);
    if (e != cudaSuccess) return e;
    k_argmin<KP><<<(cnt_max + kCostThreads - 1) / kCostThreads, kCostThreads, sm, s>>>(a);
    return cudaGetLastError();
}

template <int KP, int L>
cudaError_t launch_refine_l(const CostArgs& a, cudaStream_t s) {
    constexpr int ppc = kCostThreads / L;
    k_refine<KP, L><<<(a.N + ppc - 1) / ppc, kCostThreads, 0, s>>>(a);
    return cudaGetLastError();
}

template <int KP, int L>
cudaError_t launch_eval_l(const EvalArgs& a, cudaStream_t s) {
    constexpr int ppc = kCostThreads / L;
    k_eval<KP, L><<<(a.f.N + ppc - 1) / ppc, kCostThreads, 0, s>>>(a);
    return cudaGetLastError();
}

template <int KP>
cudaError_t launch_refine_kp(const CostArgs& a, cudaStream_t s) {
    if (a.L == 0) {   // a point per thread
        const size_t sm = refine_smem_bytes<KP, kCostThreads>();
        cudaError_t e = set_smem(k_refine_t<KP>, sm, s);
        if (e != cudaSuccess) return e;
        k_refine_t<KP><<<(a.N + kCostThreads - 1) / kCostThreads, kCostThreads, sm, s>>>(a);
        return cudaGetLastError();
    }
    switch (a.L) {
        case 4: return launch_refine_l<KP, 4>(a, s);
        case 8: return launch_refine_l<KP, 8>(a, s);
        case 16: return launch_refine_l<KP, 16>(a, s);
        default: return launch_refine_l<KP, 32>(a, s);
    }
}

template <int KP>
cudaError_t launch_eval_kp(const EvalArgs& a, cudaStream_t s) {
    switch (a.f.L) {
        case 4: return launch_eval_l<KP, 4>(a, s);
        case 8: return launch_eval_l<KP, 8>(a, s);
        case 16: return launch_eval_l<KP, 16>(a, s);
        default: return launch_eval_l<KP, 32>(a, s);
    }
}

template <int KP>
cudaError_t launch_select_kp(const LearnArgs& a, cudaStream_t s) {
    k_select<KP><<<(a.f.N + kCostThreads - 1) / kCostThreads, kCostThreads, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace

// The refinement's layout for view sets of up to veff views: lanes over views when the view set
// fills at least 7/8 of a group's view slots and, for patches of up to 9 members, a group is at
// most 16 lanes (the patch then stays in registers for all rounds at little idle-lane cost), else
// a point per thread (no idle lanes, the patch staged per round).  Measured at k = 8: 32 lanes lose
// to a point per thread (64 views, 1M points: 6.23 against 5.69 ms), 16 lanes tie (32 views:
// 0.59 ms both), and 4 lanes win on a few thousand points, where a thread per point leaves the
// GPU idle.  Larger patches keep 32 lanes (a point per thread stages 18 members per view there).
int hf_cost_lanes(int veff, int k) {
    const int kp = kp_for(k), sm = slots_for_kp(kp);
    int L = 4;
    while (L < 32 && L * sm < veff) L *= 2;
    if (L >= 32 && kp <= 9) return 0;
    return 8 * veff >= 7 * L * sm ? L : 0;
}

cudaError_t hf_launch_project(const ProjectArgs& a, cudaStream_t s) {
    const dim3 grid((a.N + kProjectThreads - 1) / kProjectThreads), block(kProjectThreads);
    // the plain path's instance has no feature code (its registers stay at the plain count)
    if (a.featx) {
        if (a.top_k > 0) k_project<true, true><<<grid, block, 0, s>>>(a);
        else k_project<false, true><<<grid, block, 0, s>>>(a);
    } else {
        if (a.top_k > 0) k_project<true, false><<<grid, block, 0, s>>>(a);
        else k_project<false, false><<<grid, block, 0, s>>>(a);
    }
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

cudaError_t hf_launch_argmin(const CostArgs& a, cudaStream_t s) {
    switch (kp_for(a.k)) {
        case 1: return launch_argmin_kp<1>(a, s);
        case 4: return launch_argmin_kp<4>(a, s);
        case 6: return launch_argmin_kp<6>(a, s);
        case 9: return launch_argmin_kp<9>(a, s);
        case 12: return launch_argmin_kp<12>(a, s);
        default: return launch_argmin_kp<17>(a, s);
    }
}

cudaError_t hf_launch_refine(const CostArgs& a, cudaStream_t s) {
    switch (kp_for(a.k)) {
        case 1: return launch_refine_kp<1>(a, s);
        case 4: return launch_refine_kp<4>(a, s);
        case 6: return launch_refine_kp<6>(a, s);
        case 9: return launch_refine_kp<9>(a, s);
        case 12: return launch_refine_kp<12>(a, s);
        default: return launch_refine_kp<17>(a, s);
    }
}

cudaError_t hf_launch_fuse(const CostArgs& a, cudaStream_t s) {
    cudaError_t e = hf_launch_argmin(a, s);
    return e != cudaSuccess ? e : hf_launch_refine(a, s);
}

cudaError_t hf_launch_select(const LearnArgs& a, cudaStream_t s) {
    switch (kp_for(a.f.k)) {
        case 1: return launch_select_kp<1>(a, s);
        case 4: return launch_select_kp<4>(a, s);
        case 6: return launch_select_kp<6>(a, s);
        case 9: return launch_select_kp<9>(a, s);
        case 12: return launch_select_kp<12>(a, s);
        default: return launch_select_kp<17>(a, s);
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

cudaError_t hf_launch_featpos(const FeatArgs& a, cudaStream_t s) {
    k_featpos<<<(a.N + kFeatThreads - 1) / kFeatThreads, kFeatThreads, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t hf_launch_rot(float2* rot, int T, double alpha0, cudaStream_t s) {
    if (T <= 0) return cudaSuccess;
    k_rot<<<1, 32, 0, s>>>(rot, T, alpha0);
    return cudaGetLastError();
}

cudaError_t hf_launch_order_nbr(int32_t* nbr, int N, int k, cudaStream_t s) {
    k_order_nbr<<<(N + 255) / 256, 256, 0, s>>>(nbr, N, k);
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

cudaError_t hf_launch_project_batch(const ProjectArgs* pa, const BatchCtl& c, bool feat, cudaStream_t s) {
    static int grid[2] = {0, 0};
    if (!grid[feat]) grid[feat] = persistent_grid(feat ? k_project_batch<true> : k_project_batch<false>, kProjectThreads, 0);
    if (feat) k_project_batch<true><<<grid[1], kProjectThreads, 0, s>>>(pa, c);
    else k_project_batch<false><<<grid[0], kProjectThreads, 0, s>>>(pa, c);
    return cudaGetLastError();
}

cudaError_t hf_launch_featpos_batch(const FeatArgs* fe, const BatchCtl& c, cudaStream_t s) {
    static int grid = 0;
    if (!grid) grid = persistent_grid(k_featpos_batch, kFeatThreads, 0);
    k_featpos_batch<<<grid, kFeatThreads, 0, s>>>(fe, c);
    return cudaGetLastError();
}
