// hf_kernels.cu - the fusion path's device code for sm_103a.
//
//   k_prep          per-scene constants: hypothesis table q = R_v h_m (folded with fx, fy),
//                   degenerate thresholds, refinement rotation steps.
//   k_project       K1, thread per point: projection of the point into every view with the pixel
//                   index decided in float-float arithmetic, nearest-pixel gather of the orientation
//                   and confidence maps, view set (visible or top-K) of the point.
//   k_argmin<HC,KP> K2, thread per point: cost of all hypotheses (Eqs. proj_r .. patch_min and the
//                   view mean) and their argmin.
//   k_refine<KP>    K3, thread per point: T rounds of the six-rotation refinement, final outputs.
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

// ------------------------------------------------------------------ K1: project + gather
// One thread per point, views in order.  For view v it writes
//   samp[v][i] = C (cos theta, sin theta) at the point's pixel (0 when outside the view),
//   ab[v][i]   = (X/Z, Y/Z) when v is in the point's view set, NaN otherwise.
// The view set is every view the point projects into, or with top_k > 0 the top_k of them by the
// confidence at the point's own pixel, ties to the lower view index.
// Order-preserving integer encoding of floats (exact, order-independent min / max by atomics).
__device__ __forceinline__ unsigned fkey(float x) {
    const unsigned u = __float_as_uint(x);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float fval(unsigned k) { return __uint_as_float((k & 0x80000000u) ? (k & 0x7fffffffu) : ~k); }

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
    const float qnan = __int_as_float(0x7fc00000);
    float topc[HF_MAX_TOPK];
    int topv[HF_MAX_TOPK];
    int ntop = 0, nset = 0;
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
            const float* cam = a.cams + 16 * v;
            const float fx = __ldg(cam), fy = __ldg(cam + 1), cx = __ldg(cam + 2), cy = __ldg(cam + 3);
            const ff X0 = ff_dot3_plus(__ldg(cam + 4), __ldg(cam + 5), __ldg(cam + 6), p0, p1, p2, __ldg(cam + 13));
            const ff X1 = ff_dot3_plus(__ldg(cam + 7), __ldg(cam + 8), __ldg(cam + 9), p0, p1, p2, __ldg(cam + 14));
            const ff X2 = ff_dot3_plus(__ldg(cam + 10), __ldg(cam + 11), __ldg(cam + 12), p0, p1, p2, __ldg(cam + 15));
            if (!(X2.hi > 1e-6f)) continue;
            const ff ra = ff_div(X0, X2), rb = ff_div(X1, X2);
            const float fu = ff_floor(ff_affine(fx, ra, cx));
            const float fv = ff_floor(ff_affine(fy, rb, cy));
            if (!(fu >= 0.0f && fu < (float)a.W && fv >= 0.0f && fv < (float)a.H)) continue;
            off[q] = (long long)((size_t)v * npx + (size_t)fv * a.W + (size_t)fu);
            ra_[q] = ra.hi;
            rb_[q] = rb.hi;
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
#pragma unroll
        for (int q = 0; q < G; ++q) {
            const int v = v0 + q;
            if (v >= a.V) break;
            float2 sv = make_float2(0.0f, 0.0f), r = make_float2(qnan, qnan);
            if (off[q] >= 0) {
                float sn, cs;
                sincosf(th[q], &sn, &cs);
                sv = make_float2(C[q] * cs, C[q] * sn);
                r = make_float2(ra_[q], rb_[q]);
                ++nset;
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
            a.samp[(size_t)v * a.N + i] = sv;
            a.ab[(size_t)v * a.N + i] = r;
        }
    }
    if (TOPK) {
        for (int v = 0; v < a.V; ++v) {
            bool keep = false;
            for (int q = 0; q < ntop; ++q) keep |= (topv[q] == v);
            if (!keep) a.ab[(size_t)v * a.N + i] = make_float2(qnan, qnan);
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
    __syncthreads();
    // hypothesis pairs (m, m+1) interleaved for packed evaluation, q = R_v h:
    //   qtab[v][m]   = (fx q_x(m), fx q_x(m+1), fx q_z(m), fx q_z(m+1))
    //   qtab[v][m+1] = (fy q_y(m), fy q_y(m+1), fy q_z(m), fy q_z(m+1))
    for (int e = threadIdx.x; e < a.V * (a.Hpad / 2); e += blockDim.x) {
        const int v = e / (a.Hpad / 2), m = 2 * (e % (a.Hpad / 2));
        const float* cam = a.cams + 16 * v;
        double q[2][3];
        for (int h = 0; h < 2; ++h)
            for (int r = 0; r < 3; ++r)
                q[h][r] = (double)cam[4 + 3 * r] * a.hyps[3 * (m + h)] + (double)cam[5 + 3 * r] * a.hyps[3 * (m + h) + 1] +
                          (double)cam[6 + 3 * r] * a.hyps[3 * (m + h) + 2];
        const double fx = cam[0], fy = cam[1];
        a.qtab[(size_t)v * a.Hpad + m] =
            make_float4((float)(fx * q[0][0]), (float)(fx * q[1][0]), (float)(fx * q[0][2]), (float)(fx * q[1][2]));
        a.qtab[(size_t)v * a.Hpad + m + 1] =
            make_float4((float)(fy * q[0][1]), (float)(fy * q[1][1]), (float)(fy * q[0][2]), (float)(fy * q[1][2]));
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

// ------------------------------------------------------------------ K2 + K3
// Patch term of one direction in one view: r = (rx, ry) is Z times the image offset (the scale
// cancels), s[] the patch samples C (cos theta, sin theta).  Returns max_j |<r, s_j>| / |r|, or 0
// when |r|^2 is below the degenerate threshold.
template <int KP>
__device__ __forceinline__ float view_term(float rx, float ry, const float2 (&s)[KP], float thr) {
    const float r2 = fmaf(rx, rx, ry * ry);
    float mx = 0.0f;
#pragma unroll
    for (int j = 0; j < KP; ++j) mx = fmaxf(mx, fabsf(fmaf(rx, s[j].x, ry * s[j].y)));
    return r2 >= thr ? mx * rsqrtf(r2) : 0.0f;
}

template <int KP>
__device__ __forceinline__ void load_patch(const float2* __restrict__ samp, size_t base, int i, const int (&nb)[KP],
                                           float2 (&s)[KP]) {
    s[0] = samp[base + i];
#pragma unroll
    for (int j = 1; j < KP; ++j) s[j] = nb[j] >= 0 ? samp[base + nb[j]] : make_float2(0.0f, 0.0f);
}

// ---- packed FP32 pairs (sm_100+ fma/mul .f32x2): each lane is rounded exactly like the scalar
// instruction, so the packed evaluation gives the same bits as view_term() lane by lane.
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

// Patch terms of two directions in one view: (rx, ry) hold the pair's offsets, SX/SY the patch
// samples broadcast to both lanes.
template <int KP>
__device__ __forceinline__ void view_term2(f32x2 rx, f32x2 ry, const f32x2 (&SX)[KP], const f32x2 (&SY)[KP],
                                           float thr0, float thr1, float& L0, float& L1) {
    const f32x2 r2 = fma2(rx, rx, mul2(ry, ry));
    float mx0 = 0.0f, mx1 = 0.0f;
#pragma unroll
    for (int j = 0; j < KP; ++j) {
        float u0, u1;
        upk(fma2(rx, SX[j], mul2(ry, SY[j])), u0, u1);
        mx0 = fmaxf(mx0, fabsf(u0));
        mx1 = fmaxf(mx1, fabsf(u1));
    }
    float a0, a1;
    upk(r2, a0, a1);
    L0 = a0 >= thr0 ? mx0 * rsqrtf(a0) : 0.0f;
    L1 = a1 >= thr1 ? mx1 * rsqrtf(a1) : 0.0f;
}

// ---- shared-memory staging
__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void cp_async8(void* sdst, const void* gsrc) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(smem_addr(sdst)), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

constexpr int kFuseThreads = 128;
constexpr size_t kQStageBytes = 16384;   // hypothesis-table slice staged per view block
constexpr int kCamStageViews = 256;      // camera rows staged per view block

// Per-thread ring of S views of patch data: item 0 = the point's (a, b), items 1..KP = the patch
// samples; laid out [stage][item][thread] so a warp reads consecutive 8-byte words.  View v lives
// in stage v % S and is copied in S - 1 views ahead of its use.
template <int KP, int S, int NT>
struct PatchStage {
    float2 v[S][KP + 1][NT];
};
constexpr int kArgminStages = 2;
constexpr int kRefineStages = 2;

// Queue the copies of one view's patch data into stage st (one commit group per call, also when
// the thread has nothing to copy, so that group counting stays uniform).
template <int KP, int S, int NT>
__device__ __forceinline__ void issue_patch(PatchStage<KP, S, NT>& sg, int st, const float2* __restrict__ ab,
                                            const float2* __restrict__ samp, size_t base, int i, const int (&nb)[KP],
                                            bool active) {
    const int t = threadIdx.x;
    if (active) {
        cp_async8(&sg.v[st][0][t], ab + base + i);
        cp_async8(&sg.v[st][1][t], samp + base + i);
#pragma unroll
        for (int j = 1; j < KP; ++j)
            if (nb[j] >= 0) cp_async8(&sg.v[st][1 + j][t], samp + base + nb[j]);
    }
    cp_async_commit();
}

template <int KP, int S, int NT>
__device__ __forceinline__ void load_nbrs(const FuseArgs& a, int i, bool active, int (&nb)[KP], PatchStage<KP, S, NT>& sg) {
    nb[0] = active ? i : -1;
#pragma unroll
    for (int j = 1; j < KP; ++j) nb[j] = (active && (j - 1) < a.k) ? a.nbr[(size_t)i * a.k + (j - 1)] : -1;
    // padded / inactive members read as zero samples in every stage, never overwritten
#pragma unroll
    for (int j = 1; j < KP; ++j)
        if (nb[j] < 0)
#pragma unroll
            for (int st = 0; st < S; ++st) sg.v[st][1 + j][threadIdx.x] = make_float2(0.0f, 0.0f);
}

template <int KP, int S, int NT>
__device__ __forceinline__ void stage_samples(const PatchStage<KP, S, NT>& sg, int st, f32x2 (&SX)[KP], f32x2 (&SY)[KP]) {
#pragma unroll
    for (int j = 0; j < KP; ++j) {
        const float2 sj = sg.v[st][1 + j][threadIdx.x];
        SX[j] = pk(sj.x, sj.x);
        SY[j] = pk(sj.y, sj.y);
    }
}

// K2: cost of every hypothesis and the argmin (lowest index on ties), thread per point.  The
// hypothesis table of HC hypotheses x a block of views sits in shared memory; the next view's
// patch data is copied in (cp.async) while the current view is evaluated, two hypotheses at a time.
template <int HC, int KP, int NT>
__device__ __forceinline__ void argmin_tile(const FuseArgs& a, int blk, unsigned char* smem_raw) {
    constexpr int S = kArgminStages;
    PatchStage<KP, S, NT>& sg = *reinterpret_cast<PatchStage<KP, S, NT>*>(smem_raw);
    float4* qs = reinterpret_cast<float4*>(smem_raw + sizeof(PatchStage<KP, S, NT>));   // [view in block][HC]
    const int tid = threadIdx.x;
    const int cnt = a.list ? *a.list_count : a.N;
    if (blk * NT >= cnt) return;   // whole block past the list: uniform exit
    const int t_ = blk * NT + tid;
    const int i = t_ < cnt ? (a.list ? a.list[t_] : t_) : -1;
    bool active = i >= 0;
    if (active) {
        const float p0 = a.pts[3 * i], p1 = a.pts[3 * i + 1], p2 = a.pts[3 * i + 2];
        if (!(isfinite(p0) && isfinite(p1) && isfinite(p2))) {
            a.nvs[i] = -1;
            active = false;
        }
    }
    int nb[KP];
    load_nbrs<KP, S, NT>(a, i, active, nb, sg);
    float best = INFINITY;
    int bestm = 0, nv = 0;
    for (int c0 = 0; c0 < a.Hpad; c0 += HC) {
        float acc[HC];
#pragma unroll
        for (int m = 0; m < HC; ++m) acc[m] = 0.0f;
        nv = 0;
        for (int p = 0; p < S - 1; ++p)
            if (p < a.V) issue_patch<KP, S, NT>(sg, p, a.ab, a.samp, (size_t)p * a.N, i, nb, active);
            else cp_async_commit();
        for (int vb = 0; vb < a.V; vb += a.vblock_q) {
            const int nvb = min(a.vblock_q, a.V - vb);
            __syncthreads();
            for (int e = tid; e < nvb * HC; e += NT)
                qs[e] = a.qtab[(size_t)(vb + e / HC) * a.Hpad + c0 + e % HC];
            __syncthreads();
            for (int v = vb; v < vb + nvb; ++v) {
                const int vn = v + S - 1;
                if (vn < a.V) issue_patch<KP, S, NT>(sg, vn % S, a.ab, a.samp, (size_t)vn * a.N, i, nb, active);
                else cp_async_commit();
                cp_async_wait<S - 1>();
                if (!active) continue;
                const int st = v % S;
                const float2 r = sg.v[st][0][tid];
                if (r.x != r.x) continue;
                ++nv;
                f32x2 SX[KP], SY[KP];
                stage_samples<KP, S, NT>(sg, st, SX, SY);
                const f32x2 na = pk(-r.x, -r.x), nb2 = pk(-r.y, -r.y);
                const float thr = __ldg(a.vthr + v);
                const float4* q = qs + (v - vb) * HC;
#pragma unroll
                for (int m = 0; m < HC; m += 2) {
                    // hypotheses m, m+1: rx = fx q_x - a fx q_z, ry = fy q_y - b fy q_z
                    const float4 QA = q[m], QB = q[m + 1];
                    float L0, L1;
                    view_term2<KP>(fma2(na, pk(QA.z, QA.w), pk(QA.x, QA.y)), fma2(nb2, pk(QB.z, QB.w), pk(QB.x, QB.y)),
                                   SX, SY, thr, thr, L0, L1);
                    acc[m] += L0;
                    acc[m + 1] += L1;
                }
            }
        }
        cp_async_wait<0>();
#pragma unroll
        for (int m = 0; m < HC; ++m) {
            const float c = nv ? 1.0f - acc[m] / (float)nv : 1.0f;
            if (c0 + m < a.H && c < best) {
                best = c;
                bestm = c0 + m;
            }
        }
    }
    if (active) {
        a.best_idx[i] = bestm;
        a.best_cost[i] = best;
        a.nvs[i] = nv;
    }
}

template <int HC, int KP>
__global__ void __launch_bounds__(kFuseThreads) k_argmin(FuseArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    argmin_tile<HC, KP, kFuseThreads>(a, blockIdx.x, smem_raw);
}

// K3: T rounds of +-alpha rotations about world x, y, z from the argmin; move to the first strictly
// lowest cost; halve alpha.  The two candidates of one axis are evaluated as a packed pair.
template <int KP, int NT>
__device__ __forceinline__ void refine_tile(const FuseArgs& a, int blk, unsigned char* smem_raw) {
    constexpr int S = kRefineStages;
    PatchStage<KP, S, NT>& sg = *reinterpret_cast<PatchStage<KP, S, NT>*>(smem_raw);
    float4* cs4 = reinterpret_cast<float4*>(smem_raw + sizeof(PatchStage<KP, S, NT>));   // [view in block][3]
    const int tid = threadIdx.x;
    const int cnt = a.list ? *a.list_count : a.N;
    if (blk * NT >= cnt) return;   // whole block past the list: uniform exit
    const int t_ = blk * NT + tid;
    const int i = t_ < cnt ? (a.list ? a.list[t_] : t_) : -1;
    const bool inb = i >= 0;
    // From a given start direction (the learned proposal) the view count and the start cost are
    // taken in round 0, next to the six candidates; otherwise they come from k_argmin.
    const bool from_start = a.start_dir != nullptr;
    int nv = 0;
    if (inb) {
        if (from_start && a.T > 0) {
            const float p0 = a.pts[3 * i], p1 = a.pts[3 * i + 1], p2 = a.pts[3 * i + 2];
            nv = (isfinite(p0) && isfinite(p1) && isfinite(p2)) ? 0 : -1;
        } else {   // from k_argmin, or (no rounds) from k_start_select
            nv = a.nvs[i];
        }
    }
    if (inb && nv < 0) {
        const int o = i - a.out_first;   // output row
        a.dir_out[3 * o] = a.dir_out[3 * o + 1] = a.dir_out[3 * o + 2] = 0.0f;
        if (a.cost_out) a.cost_out[o] = __int_as_float(0x7fc00000);
        if (a.idx_out) a.idx_out[o] = -1;
        if (a.status_out) a.status_out[o] = HF_STATUS_BAD_INPUT;
        if (from_start) a.nvs[i] = -1;
    }
    // points with no view keep their start (all costs are 1)
    const bool active = inb && ((from_start && a.T > 0) ? nv == 0 : nv > 0);
    int nb[KP];
    load_nbrs<KP, S, NT>(a, i, active, nb, sg);
    // start: the argmin hypothesis, or a given direction (the learned proposal; index -1)
    const int bestm = from_start ? -1 : ((inb && nv >= 0) ? a.best_idx[i] : 0);
    float best = ((!from_start || a.T == 0) && inb && nv >= 0) ? a.best_cost[i] : 0.0f;
    float acc_c = 0.0f;   // round 0 from a start: the start direction's patch terms
    float d0, d1, d2;
    if (a.start_dir) {
        d0 = inb ? a.start_dir[3 * i] : 1.0f;
        d1 = inb ? a.start_dir[3 * i + 1] : 0.0f;
        d2 = inb ? a.start_dir[3 * i + 2] : 0.0f;
    } else {
        d0 = a.hyps[3 * bestm];
        d1 = a.hyps[3 * bestm + 1];
        d2 = a.hyps[3 * bestm + 2];
    }
    const int nblk = (a.V + a.vblock_c - 1) / a.vblock_c;
    for (int t = 0; t < a.T; ++t) {
        const float2 cr = a.rot[t];
        const float c = cr.x, sn = cr.y;
        const float cd[6][3] = {{d0, c * d1 - sn * d2, sn * d1 + c * d2}, {d0, c * d1 + sn * d2, -sn * d1 + c * d2},
                                {c * d0 + sn * d2, d1, -sn * d0 + c * d2}, {c * d0 - sn * d2, d1, sn * d0 + c * d2},
                                {c * d0 - sn * d1, sn * d0 + c * d1, d2}, {c * d0 + sn * d1, -sn * d0 + c * d1, d2}};
        f32x2 CX[3], CY[3], CZ[3];
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            CX[q] = pk(cd[2 * q][0], cd[2 * q + 1][0]);
            CY[q] = pk(cd[2 * q][1], cd[2 * q + 1][1]);
            CZ[q] = pk(cd[2 * q][2], cd[2 * q + 1][2]);
        }
        float acc[6] = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f};
        for (int p = 0; p < S - 1; ++p)
            if (p < a.V) issue_patch<KP, S, NT>(sg, p, a.ab, a.samp, (size_t)p * a.N, i, nb, active);
            else cp_async_commit();
        for (int vb = 0; vb < a.V; vb += a.vblock_c) {
            const int nvb = min(a.vblock_c, a.V - vb);
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
            for (int v = vb; v < vb + nvb; ++v) {
                const int vn = v + S - 1;
                if (vn < a.V) issue_patch<KP, S, NT>(sg, vn % S, a.ab, a.samp, (size_t)vn * a.N, i, nb, active);
                else cp_async_commit();
                cp_async_wait<S - 1>();
                if (!active) continue;
                const int st = v % S;
                const float2 r = sg.v[st][0][tid];
                if (r.x != r.x) continue;
                f32x2 SX[KP], SY[KP];
                stage_samples<KP, S, NT>(sg, st, SX, SY);
                // staged rows: k0 = (fx, fy, R00, R01), k1 = (R02, R10, R11, R12), k2 = (R20, R21, R22, thr)
                const bool centre = from_start && t == 0;
                const float4 k0 = cs4[3 * (v - vb)], k1 = cs4[3 * (v - vb) + 1], k2 = cs4[3 * (v - vb) + 2];
                // Z times the projection Jacobian: rows fx (R_0 - a R_2), fy (R_1 - b R_2)
                const float j0 = k0.x * fmaf(-r.x, k2.x, k0.z), j1 = k0.x * fmaf(-r.x, k2.y, k0.w),
                            j2 = k0.x * fmaf(-r.x, k2.z, k1.x);
                const float j3 = k0.y * fmaf(-r.y, k2.x, k1.y), j4 = k0.y * fmaf(-r.y, k2.y, k1.z),
                            j5 = k0.y * fmaf(-r.y, k2.z, k1.w);
                const f32x2 J0 = pk(j0, j0), J1 = pk(j1, j1), J2 = pk(j2, j2);
                const f32x2 J3 = pk(j3, j3), J4 = pk(j4, j4), J5 = pk(j5, j5);
#pragma unroll
                for (int q = 0; q < 3; ++q) {   // the +alpha / -alpha pair of axis q
                    float L0, L1;
                    view_term2<KP>(fma2(J0, CX[q], fma2(J1, CY[q], mul2(J2, CZ[q]))),
                                   fma2(J3, CX[q], fma2(J4, CY[q], mul2(J5, CZ[q]))), SX, SY, k2.w, k2.w, L0, L1);
                    acc[2 * q] += L0;
                    acc[2 * q + 1] += L1;
                }
                if (centre) {
                    const f32x2 D0 = pk(d0, d0), D1 = pk(d1, d1), D2 = pk(d2, d2);
                    float L0, L1;
                    view_term2<KP>(fma2(J0, D0, fma2(J1, D1, mul2(J2, D2))), fma2(J3, D0, fma2(J4, D1, mul2(J5, D2))), SX,
                                   SY, k2.w, k2.w, L0, L1);
                    acc_c += L0;
                    ++nv;
                }
            }
        }
        cp_async_wait<0>();
        if (from_start && t == 0) best = nv > 0 ? 1.0f - acc_c / (float)nv : 1.0f;
        int choice = -1;
#pragma unroll
        for (int q = 0; q < 6; ++q) {
            const float cq = nv > 0 ? 1.0f - acc[q] / (float)nv : 1.0f;
            if (cq < best) {
                best = cq;
                choice = q;
            }
        }
#pragma unroll
        for (int q = 0; q < 6; ++q)
            if (q == choice) {
                d0 = cd[q][0];
                d1 = cd[q][1];
                d2 = cd[q][2];
            }
    }
    if (!inb || nv < 0) return;
    if (from_start && a.T > 0) a.nvs[i] = nv;
    const float n = sqrtf(d0 * d0 + d1 * d1 + d2 * d2);
    d0 /= n;
    d1 /= n;
    d2 /= n;
    const float sgn = fabsf(d2) > 1e-12f ? copysignf(1.0f, d2) : fabsf(d1) > 1e-12f ? copysignf(1.0f, d1) : copysignf(1.0f, d0);
    const int o = i - a.out_first;   // output row
    a.dir_out[3 * o] = sgn * d0;
    a.dir_out[3 * o + 1] = sgn * d1;
    a.dir_out[3 * o + 2] = sgn * d2;
    if (a.cost_out) a.cost_out[o] = best;
    if (a.idx_out) a.idx_out[o] = bestm;
    if (a.status_out) a.status_out[o] = a.fell_back ? HF_STATUS_FELL_BACK : (nv ? HF_STATUS_OK : HF_STATUS_NO_VIEWS);
}

template <int KP>
__global__ void __launch_bounds__(kFuseThreads) k_refine(FuseArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    refine_tile<KP, kFuseThreads>(a, blockIdx.x, smem_raw);
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

// Cost c_i of the proposal (a.start_dir) and the fallback decision: points with a view and
// c_i > tau go to the fallback list (a.list), the others to the accepted list (s.acc_list), in
// the order warps append them; non-finite points get their BAD_INPUT outputs here and no list.
// best_cost / nvs receive c_i and |V_i| (the refinement's zero-round outputs).
constexpr int kStartThreads = 128;

// One direction per view: the next view's (a, b) and patch samples are loaded while the current
// view is evaluated (register double buffering; loads of views outside V_i are harmless reads).
template <int KP>
__device__ __forceinline__ void start_select_tile(const StartSelectArgs& s, int blk) {
    const FuseArgs& a = s.f;
    const int tid = threadIdx.x;
    const int i = blk * kStartThreads + tid;
    const bool in = i < a.N;
    bool bad = false;
    if (in) {
        const float p0 = a.pts[3 * i], p1 = a.pts[3 * i + 1], p2 = a.pts[3 * i + 2];
        bad = !(isfinite(p0) && isfinite(p1) && isfinite(p2));
    }
    const bool active = in && !bad;
    float acc = 0.0f;
    int nv = 0;
    if (active) {
        int nb[KP];
        nb[0] = i;
#pragma unroll
        for (int j = 1; j < KP; ++j) nb[j] = (j - 1) < a.k ? a.nbr[(size_t)i * a.k + (j - 1)] : -1;
        const float d0 = a.start_dir[3 * i], d1 = a.start_dir[3 * i + 1], d2 = a.start_dir[3 * i + 2];
        float2 rn = a.ab[i];
        float2 sn[KP];
        load_patch<KP>(a.samp, 0, i, nb, sn);
        for (int v = 0; v < a.V; ++v) {
            const float2 r = rn;
            float2 sm[KP];
#pragma unroll
            for (int j = 0; j < KP; ++j) sm[j] = sn[j];
            if (v + 1 < a.V) {
                const size_t nxt = (size_t)(v + 1) * a.N;
                rn = a.ab[nxt + i];
                load_patch<KP>(a.samp, nxt, i, nb, sn);
            }
            if (r.x != r.x) continue;
            ++nv;
            const float* cam = a.cams + 16 * v;
            // Z times the projection Jacobian, rounded as in the refinement's round 0
            const float j0 = cam[0] * fmaf(-r.x, cam[10], cam[4]), j1 = cam[0] * fmaf(-r.x, cam[11], cam[5]),
                        j2 = cam[0] * fmaf(-r.x, cam[12], cam[6]);
            const float j3 = cam[1] * fmaf(-r.y, cam[10], cam[7]), j4 = cam[1] * fmaf(-r.y, cam[11], cam[8]),
                        j5 = cam[1] * fmaf(-r.y, cam[12], cam[9]);
            acc += view_term<KP>(fmaf(j0, d0, fmaf(j1, d1, j2 * d2)), fmaf(j3, d0, fmaf(j4, d1, j5 * d2)), sm,
                                 a.vthr[v]);
        }
    }
    const float c0 = nv ? 1.0f - acc / (float)nv : 1.0f;
    if (active) {
        a.best_cost[i] = c0;
        a.nvs[i] = nv;
    } else if (in) {
        const int o = i - a.out_first;   // output row
        a.nvs[i] = -1;
        a.dir_out[3 * o] = a.dir_out[3 * o + 1] = a.dir_out[3 * o + 2] = 0.0f;
        if (a.cost_out) a.cost_out[o] = __int_as_float(0x7fc00000);
        if (a.idx_out) a.idx_out[o] = -1;
        if (a.status_out) a.status_out[o] = HF_STATUS_BAD_INPUT;
    }
    const bool fb = active && nv > 0 && c0 > s.tau;
    const bool ok = active && !fb;
    const int lane = tid & 31;
    const unsigned below = (1u << lane) - 1u;
#pragma unroll
    for (int q = 0; q < 2; ++q) {   // warp-aggregated appends: fallback, then accepted
        const bool want = q == 0 ? fb : ok;
        const unsigned m = __ballot_sync(0xffffffffu, want);
        if (!m) continue;
        const int leader = __ffs(m) - 1;
        int base = 0;
        if (lane == leader) base = atomicAdd(q == 0 ? const_cast<int*>(a.list_count) : s.acc_count, __popc(m));
        base = __shfl_sync(0xffffffffu, base, leader);
        if (want) (q == 0 ? const_cast<int32_t*>(a.list) : s.acc_list)[base + __popc(m & below)] = i;
    }
}

template <int KP>
__global__ void __launch_bounds__(kStartThreads) k_start_select(StartSelectArgs s) {
    start_select_tile<KP>(s, blockIdx.x);
}


__global__ void k_rot(float2* rot, int T, double alpha0) {
    const int t = threadIdx.x;
    if (t < T) {
        const double al = alpha0 / (double)(1u << t);
        rot[t] = make_float2((float)cos(al), (float)sin(al));
    }
}

// ------------------------------------------------------------------ cost of given directions
template <int KP>
__global__ void __launch_bounds__(128) k_eval(EvalArgs a) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.N) return;
    int nb[KP];
    nb[0] = i;
#pragma unroll
    for (int j = 1; j < KP; ++j) nb[j] = (j - 1) < a.k ? a.nbr[(size_t)i * a.k + (j - 1)] : -1;
    for (int m = 0; m < a.M; ++m) {
        const float* d = a.dirs + ((size_t)i * a.M + m) * 3;
        const float d0 = d[0], d1 = d[1], d2 = d[2];
        const float dn2 = d0 * d0 + d1 * d1 + d2 * d2;
        float acc = 0.0f;
        int nv = 0;
        for (int v = 0; v < a.V; ++v) {
            const size_t base = (size_t)v * a.N;
            const float2 r = a.ab[base + i];
            if (r.x != r.x) continue;
            ++nv;
            float2 s[KP];
            load_patch<KP>(a.samp, base, i, nb, s);
            const float* cam = a.cams + 16 * v;
            const float fx = cam[0], fy = cam[1];
            float q[3];
            for (int rr = 0; rr < 3; ++rr) q[rr] = fmaf(cam[4 + 3 * rr], d0, fmaf(cam[5 + 3 * rr], d1, cam[6 + 3 * rr] * d2));
            const float rx = fx * fmaf(-r.x, q[2], q[0]);
            const float ry = fy * fmaf(-r.y, q[2], q[1]);
            acc += view_term<KP>(rx, ry, s, a.vthr[v] * dn2);
        }
        a.cost_out[(size_t)i * a.M + m] = nv ? 1.0f - acc / (float)nv : 1.0f;
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

template <int NT, typename Args, typename Count, typename Body>
__device__ __forceinline__ void batch_tiles(const Args* __restrict__ args, const BatchCtl& c, Count count, Body body) {
    __shared__ Args sa;
    __shared__ int pref[HF_MAX_BATCH + 1];
    __shared__ int s_item, s_pos, s_cur;
    if (threadIdx.x == 0) {
        pref[0] = 0;
        for (int p = 0; p < c.ns; ++p) pref[p + 1] = pref[p] + (count(args[p]) + NT - 1) / NT;
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

__device__ __forceinline__ int fuse_count(const FuseArgs& a) { return a.list ? *a.list_count : a.N; }

template <int HC, int KP, int NT>
__global__ void __launch_bounds__(NT) k_argmin_batch(const FuseArgs* __restrict__ fa, BatchCtl c) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    batch_tiles<NT>(fa, c, [](const FuseArgs& a) { return fuse_count(a); }, [&](const FuseArgs& a, int blk) { argmin_tile<HC, KP, NT>(a, blk, smem_raw); });
}

template <int KP, int NT>
__global__ void __launch_bounds__(NT) k_refine_batch(const FuseArgs* __restrict__ fa, BatchCtl c) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    batch_tiles<NT>(fa, c, [](const FuseArgs& a) { return fuse_count(a); }, [&](const FuseArgs& a, int blk) { refine_tile<KP, NT>(a, blk, smem_raw); });
}

__global__ void __launch_bounds__(kProjectThreads) k_project_batch(const ProjectArgs* __restrict__ pa, BatchCtl c) {
    batch_tiles<kProjectThreads>(pa, c, [](const ProjectArgs& a) { return a.N; }, [](const ProjectArgs& a, int blk) {
        if (a.top_k > 0) project_tile<true>(a, blk);
        else project_tile<false>(a, blk);
    });
}

__global__ void __launch_bounds__(kFeatThreads) k_features_batch(const FeatArgs* __restrict__ fe, BatchCtl c) {
    batch_tiles<kFeatThreads>(fe, c, [](const FeatArgs& a) { return a.N; },
                              [](const FeatArgs& a, int blk) { features_tile(a, blk); });
}

template <int KP>
__global__ void __launch_bounds__(kStartThreads) k_start_select_batch(const StartSelectArgs* __restrict__ sa,
                                                                      BatchCtl c) {
    batch_tiles<kStartThreads>(sa, c, [](const StartSelectArgs& a) { return a.f.N; },
                               [](const StartSelectArgs& a, int blk) { start_select_tile<KP>(a, blk); });
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

// persistent grid: resident CTAs per SM x SMs (cached per kernel and shared-memory size)
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

template <int HC, int KP, int NT>
cudaError_t launch_argmin_batch(const FuseArgs* fa, const BatchCtl& c, cudaStream_t s) {
    const size_t sm = sizeof(PatchStage<KP, kArgminStages, NT>) + kQStageBytes;
    cudaError_t e = set_smem(k_argmin_batch<HC, KP, NT>, sm, s);
    if (e != cudaSuccess) return e;
    static int grid = 0;
    if (!grid) grid = persistent_grid(k_argmin_batch<HC, KP, NT>, NT, sm);
    k_argmin_batch<HC, KP, NT><<<grid, NT, sm, s>>>(fa, c);
    return cudaGetLastError();
}

template <int KP, int NT>
cudaError_t launch_refine_batch(const FuseArgs* fa, const BatchCtl& c, cudaStream_t s) {
    const size_t sm = sizeof(PatchStage<KP, kRefineStages, NT>) + (size_t)kCamStageViews * 3 * sizeof(float4);
    cudaError_t e = set_smem(k_refine_batch<KP, NT>, sm, s);
    if (e != cudaSuccess) return e;
    static int grid = 0;
    if (!grid) grid = persistent_grid(k_refine_batch<KP, NT>, NT, sm);
    k_refine_batch<KP, NT><<<grid, NT, sm, s>>>(fa, c);
    return cudaGetLastError();
}

template <int HC, int KP>
cudaError_t launch_argmin_batch_nt(const FuseArgs* fa, const BatchCtl& c, int nt, cudaStream_t s) {
    switch (nt) {
        case 64: return launch_argmin_batch<HC, KP, 64>(fa, c, s);
        case 256: return launch_argmin_batch<HC, KP, 256>(fa, c, s);
        default: return launch_argmin_batch<HC, KP, 128>(fa, c, s);
    }
}

template <int HC>
cudaError_t launch_argmin_batch_kp(const FuseArgs* fa, const BatchCtl& c, int kp, int nt, cudaStream_t s) {
    switch (kp) {
        case 4: return launch_argmin_batch_nt<HC, 4>(fa, c, nt, s);
        case 9: return launch_argmin_batch_nt<HC, 9>(fa, c, nt, s);
        default: return launch_argmin_batch_nt<HC, 17>(fa, c, nt, s);
    }
}

template <int KP>
cudaError_t launch_refine_batch_nt(const FuseArgs* fa, const BatchCtl& c, int nt, cudaStream_t s) {
    switch (nt) {
        case 64: return launch_refine_batch<KP, 64>(fa, c, s);
        case 256: return launch_refine_batch<KP, 256>(fa, c, s);
        default: return launch_refine_batch<KP, 128>(fa, c, s);
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

// stage 1: k_argmin, stage 2: k_refine.  Dynamic shared memory above 48 KB needs the function
// attribute, which is cheap and set on every launch (it is per function and per device).
template <int HC, int KP>
cudaError_t launch_fuse_kp(const FuseArgs& a, int stage, cudaStream_t s) {
    const dim3 grid((a.N + kFuseThreads - 1) / kFuseThreads), block(kFuseThreads);
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaStreamIsCapturing(s, &cs);
    const bool set_attr = cs == cudaStreamCaptureStatusNone;   // set outside capture only
    if (stage == 1) {
        const size_t sm = sizeof(PatchStage<KP, kArgminStages, kFuseThreads>) + (size_t)a.vblock_q * HC * sizeof(float4);
        cudaError_t e = set_attr ? cudaFuncSetAttribute(k_argmin<HC, KP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm)
                                 : cudaSuccess;
        if (e != cudaSuccess) return e;
        k_argmin<HC, KP><<<grid, block, sm, s>>>(a);
    } else {
        const size_t sm = sizeof(PatchStage<KP, kRefineStages, kFuseThreads>) + (size_t)a.vblock_c * 3 * sizeof(float4);
        cudaError_t e = set_attr ? cudaFuncSetAttribute(k_refine<KP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm)
                                 : cudaSuccess;
        if (e != cudaSuccess) return e;
        k_refine<KP><<<grid, block, sm, s>>>(a);
    }
    return cudaGetLastError();
}

template <int HC>
cudaError_t launch_fuse_hc(const FuseArgs& a, int stage, cudaStream_t s) {
    switch (kp_for(a.k)) {
        case 1: return launch_fuse_kp<HC, 1>(a, stage, s);
        case 4: return launch_fuse_kp<HC, 4>(a, stage, s);
        case 6: return launch_fuse_kp<HC, 6>(a, stage, s);
        case 9: return launch_fuse_kp<HC, 9>(a, stage, s);
        case 12: return launch_fuse_kp<HC, 12>(a, stage, s);
        default: return launch_fuse_kp<HC, 17>(a, stage, s);
    }
}

}  // namespace

int hf_fuse_chunk_for(int H) {
    if (H <= 8) return 8;
    if (H <= 16) return 16;
    return 32;
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

int hf_fuse_vblock_q(int V, int hchunk) {
    const int vb = (int)(kQStageBytes / ((size_t)hchunk * sizeof(float4)));
    return vb < 1 ? 1 : (vb < V ? vb : V);
}

int hf_fuse_vblock_c(int V) { return V < kCamStageViews ? V : kCamStageViews; }

cudaError_t hf_launch_argmin(const FuseArgs& a, int hchunk, cudaStream_t s) {
    switch (hchunk) {
        case 8: return launch_fuse_hc<8>(a, 1, s);
        case 16: return launch_fuse_hc<16>(a, 1, s);
        default: return launch_fuse_hc<32>(a, 1, s);
    }
}

cudaError_t hf_launch_refine(const FuseArgs& a, cudaStream_t s) { return launch_fuse_hc<8>(a, 2, s); }

cudaError_t hf_launch_fuse(const FuseArgs& a, int hchunk, cudaStream_t s) {
    cudaError_t e = hf_launch_argmin(a, hchunk, s);
    return e != cudaSuccess ? e : hf_launch_refine(a, s);
}

cudaError_t hf_launch_eval(const EvalArgs& a, cudaStream_t s) {
    const dim3 grid((a.N + 127) / 128), block(128);
    switch (kp_for(a.k)) {
        case 1: k_eval<1><<<grid, block, 0, s>>>(a); break;
        case 4: k_eval<4><<<grid, block, 0, s>>>(a); break;
        case 6: k_eval<6><<<grid, block, 0, s>>>(a); break;
        case 9: k_eval<9><<<grid, block, 0, s>>>(a); break;
        case 12: k_eval<12><<<grid, block, 0, s>>>(a); break;
        default: k_eval<17><<<grid, block, 0, s>>>(a); break;
    }
    return cudaGetLastError();
}

cudaError_t hf_launch_fib(int H, float* out, cudaStream_t s) {
    k_fib<<<(H + 127) / 128, 128, 0, s>>>(H, out);
    return cudaGetLastError();
}

cudaError_t hf_launch_features(const FeatArgs& a, cudaStream_t s) {
    k_features<<<(a.N + kFeatThreads - 1) / kFeatThreads, kFeatThreads, 0, s>>>(a);
    return cudaGetLastError();
}

template <int KP>
cudaError_t launch_start_select(const StartSelectArgs& a, cudaStream_t s) {
    k_start_select<KP><<<(a.f.N + kStartThreads - 1) / kStartThreads, kStartThreads, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t hf_launch_start_select(const StartSelectArgs& a, cudaStream_t s) {
    switch (kp_for(a.f.k)) {
        case 1: return launch_start_select<1>(a, s);
        case 4: return launch_start_select<4>(a, s);
        case 6: return launch_start_select<6>(a, s);
        case 9: return launch_start_select<9>(a, s);
        case 12: return launch_start_select<12>(a, s);
        default: return launch_start_select<17>(a, s);
    }
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

template <int KP>
cudaError_t launch_start_select_batch(const StartSelectArgs* sa, const BatchCtl& c, cudaStream_t s) {
    static int grid = 0;
    if (!grid) grid = persistent_grid(k_start_select_batch<KP>, kStartThreads, 0);
    k_start_select_batch<KP><<<grid, kStartThreads, 0, s>>>(sa, c);
    return cudaGetLastError();
}

cudaError_t hf_launch_start_select_batch(const StartSelectArgs* sa, const BatchCtl& c, int kp, cudaStream_t s) {
    switch (kp) {
        case 4: return launch_start_select_batch<4>(sa, c, s);
        case 9: return launch_start_select_batch<9>(sa, c, s);
        default: return launch_start_select_batch<17>(sa, c, s);
    }
}

cudaError_t hf_launch_argmin_batch(const FuseArgs* fa, const BatchCtl& c, int kp, int hc, int nt, cudaStream_t s) {
    switch (hc) {
        case 8: return launch_argmin_batch_kp<8>(fa, c, kp, nt, s);
        case 16: return launch_argmin_batch_kp<16>(fa, c, kp, nt, s);
        default: return launch_argmin_batch_kp<32>(fa, c, kp, nt, s);
    }
}

cudaError_t hf_launch_refine_batch(const FuseArgs* fa, const BatchCtl& c, int kp, int nt, cudaStream_t s) {
    switch (kp) {
        case 4: return launch_refine_batch_nt<4>(fa, c, nt, s);
        case 9: return launch_refine_batch_nt<9>(fa, c, nt, s);
        default: return launch_refine_batch_nt<17>(fa, c, nt, s);
    }
}
