// hf_phg.cu - the paper's Parallel Hair Growing consumer (Sec. 3.2) on the GPU: the occupancy and
// orientation volumes from the fused points, guide strands traced from scalp seeds in batches with
// deferred occupancy, segments grown from the occupied voxels no strand reached, and the linking of
// strands by Eq. segment_connection into connected components.
//
//   k_phg_splat          a thread per point: voxel, count, fixed-point d d^T (integer atomics, so
//                        the sums do not depend on the order of the additions)
//   k_phg_orient         a thread per voxel: the dominant eigenvector by power iteration
//   k_phg_trace_guides   a thread per seed of a batch; k_phg_count then adds the batch's strands to
//                        the voxels they entered (the deferred occupancy update)
//   k_phg_flags/_scan/_write   the segment seeds (occupied voxels no strand entered) in voxel order
//   k_phg_trace_segments a thread per seed of a batch (both halves); k_phg_count as above
//   k_phg_bin/_scan/_put the segment ends binned by cell; k_phg_link a thread per strand end (nearest
//                        compatible segment end); k_phg_union / k_phg_flatten the connected components
//
// Every quantity that decides a voxel or a stop is computed in single precision with one rounding
// per written operation (__fadd_rn, __fmul_rn, __fmaf_rn, __fdiv_rn, __fsqrt_rn: no contraction),
// so the traces, counts and labels are those of an exact replay of the same arithmetic.
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <vector>

#include "hf_internal.cuh"

namespace {

constexpr int kThreads = 256;
constexpr int kScanBlock = 1024;   // elements per block of the ordered scans

__device__ __forceinline__ long long phg_voxel(const hf_phg_cfg& g, float p0, float p1, float p2) {
    const float q0 = __fdiv_rn(__fsub_rn(p0, g.origin[0]), g.voxel);
    const float q1 = __fdiv_rn(__fsub_rn(p1, g.origin[1]), g.voxel);
    const float q2 = __fdiv_rn(__fsub_rn(p2, g.origin[2]), g.voxel);
    if (!(q0 >= 0.0f && q0 < (float)g.nx && q1 >= 0.0f && q1 < (float)g.ny && q2 >= 0.0f && q2 < (float)g.nz))
        return -1;
    return ((long long)(int)floorf(q2) * g.ny + (int)floorf(q1)) * g.nx + (int)floorf(q0);
}

// The linking grid: cells of edge `cell` >= 1.01 link_dist (so every end within link_dist of a
// point lies in one of the 27 cells around it), covering the voxel grid and one voxel beyond it on
// every side (every strand end lies within one step of the voxel grid); cells clamp at the border.
struct LinkGrid {
    float o0, o1, o2, cell;
    int nx, ny, nz;
};
__device__ __forceinline__ int3 phg_cell(const LinkGrid& G, float p0, float p1, float p2) {
    const float q0 = (p0 - G.o0) / G.cell, q1 = (p1 - G.o1) / G.cell, q2 = (p2 - G.o2) / G.cell;
    const int c0 = (int)fminf(fmaxf(floorf(q0), 0.0f), (float)(G.nx - 1));
    const int c1 = (int)fminf(fmaxf(floorf(q1), 0.0f), (float)(G.ny - 1));
    const int c2 = (int)fminf(fmaxf(floorf(q2), 0.0f), (float)(G.nz - 1));
    return make_int3(c0, c1, c2);
}

// ------------------------------------------------------------------ A: splat
__global__ void k_phg_splat(hf_phg_cfg g, long long n, const float* __restrict__ pts, const float* __restrict__ dirs,
                            const uint8_t* __restrict__ valid, int* __restrict__ occ,
                            unsigned long long* __restrict__ T) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        if (valid && !valid[i]) continue;
        const float p0 = pts[3 * i], p1 = pts[3 * i + 1], p2 = pts[3 * i + 2];
        const float d0 = dirs[3 * i], d1 = dirs[3 * i + 1], d2 = dirs[3 * i + 2];
        if (!(isfinite(p0) && isfinite(p1) && isfinite(p2) && isfinite(d0) && isfinite(d1) && isfinite(d2))) continue;
        const long long c = phg_voxel(g, p0, p1, p2);
        if (c < 0) continue;
        atomicAdd(occ + c, 1);
        const float pr[6] = {__fmul_rn(d0, d0), __fmul_rn(d0, d1), __fmul_rn(d0, d2),
                             __fmul_rn(d1, d1), __fmul_rn(d1, d2), __fmul_rn(d2, d2)};
#pragma unroll
        for (int e = 0; e < 6; ++e)   // two's complement: an unsigned add is the signed sum
            atomicAdd(T + 6 * c + e, (unsigned long long)__float2ll_rn(__fmul_rn(pr[e], 1073741824.0f)));
    }
}

// ------------------------------------------------------------------ B: orientation
__global__ void k_phg_orient(long long nvox, const int* __restrict__ occ, const long long* __restrict__ T,
                             float* __restrict__ ori, float4* __restrict__ vrec) {
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < nvox;
         c += (long long)gridDim.x * blockDim.x) {
        float o0 = 0.0f, o1 = 0.0f, o2 = 0.0f;
        if (occ[c] > 0) {
            const long long* t = T + 6 * c;
            const float m00 = __ll2float_rn(t[0]), m01 = __ll2float_rn(t[1]), m02 = __ll2float_rn(t[2]);
            const float m11 = __ll2float_rn(t[3]), m12 = __ll2float_rn(t[4]), m22 = __ll2float_rn(t[5]);
            int a = 0;
            float ma = m00;
            if (m11 > ma) {
                a = 1;
                ma = m11;
            }
            if (m22 > ma) a = 2;
            float x0 = a == 0 ? m00 : (a == 1 ? m01 : m02);
            float x1 = a == 0 ? m01 : (a == 1 ? m11 : m12);
            float x2 = a == 0 ? m02 : (a == 1 ? m12 : m22);
            float nn = __fsqrt_rn(__fmaf_rn(x0, x0, __fmaf_rn(x1, x1, __fmul_rn(x2, x2))));
            if (nn > 0.0f) {
                float r = __fdiv_rn(1.0f, nn);
                x0 = __fmul_rn(x0, r);
                x1 = __fmul_rn(x1, r);
                x2 = __fmul_rn(x2, r);
                for (int it = 0; it < 12; ++it) {
                    const float y0 = __fmaf_rn(m00, x0, __fmaf_rn(m01, x1, __fmul_rn(m02, x2)));
                    const float y1 = __fmaf_rn(m01, x0, __fmaf_rn(m11, x1, __fmul_rn(m12, x2)));
                    const float y2 = __fmaf_rn(m02, x0, __fmaf_rn(m12, x1, __fmul_rn(m22, x2)));
                    nn = __fsqrt_rn(__fmaf_rn(y0, y0, __fmaf_rn(y1, y1, __fmul_rn(y2, y2))));
                    if (!(nn > 0.0f)) break;
                    r = __fdiv_rn(1.0f, nn);
                    x0 = __fmul_rn(y0, r);
                    x1 = __fmul_rn(y1, r);
                    x2 = __fmul_rn(y2, r);
                }
                const bool neg = x2 < 0.0f || (x2 == 0.0f && (x1 < 0.0f || (x1 == 0.0f && x0 < 0.0f)));
                o0 = neg ? -x0 : x0;
                o1 = neg ? -x1 : x1;
                o2 = neg ? -x2 : x2;
            }
        }
        ori[3 * c] = o0;
        ori[3 * c + 1] = o1;
        ori[3 * c + 2] = o2;
        vrec[c] = make_float4(o0, o1, o2, __int_as_float(occ[c]));   // one 16-byte read per trace step
    }
}

// ------------------------------------------------------------------ C, D: tracing
// One trace: vertex k goes to out[3 dir k] and its voxel (-1 outside) to vox[dir k] (dir = +1 or
// -1); returns the vertex count (0 for a guide that met no occupied voxel); *dl the last step's
// direction; *stop the reason.  vrec[c] = (orientation, point count as int bits).
__device__ int phg_trace(const hf_phg_cfg& g, const float4* __restrict__ vrec, const int* __restrict__ crowd,
                         float p0, float p1, float p2, float d0, float d1, float d2, int walk, float* out, int* vox,
                         int dir, float* dl, int* stop) {
    int nv = 1;
    bool met = walk == 0;
    out[0] = p0;
    out[1] = p1;
    out[2] = p2;
    int st = HF_PHG_MAXLEN;
    long long c = -1;
    int t = 0;
    for (; t < g.max_steps; ++t) {
        c = phg_voxel(g, p0, p1, p2);
        vox[dir * (nv - 1)] = (int)c;
        if (c < 0) {
            st = met ? HF_PHG_OUTSIDE : HF_PHG_NO_ROOT;
            break;
        }
        const float4 vr = vrec[c];
        const int cr = crowd[c];
        if (__float_as_int(vr.w) == 0) {
            if (!met && t < walk) {
                p0 = __fmaf_rn(g.step, d0, p0);
                p1 = __fmaf_rn(g.step, d1, p1);
                p2 = __fmaf_rn(g.step, d2, p2);
                float* v = out + 3 * dir * nv++;
                v[0] = p0;
                v[1] = p1;
                v[2] = p2;
                continue;
            }
            st = met ? HF_PHG_EMPTY : HF_PHG_NO_ROOT;
            break;
        }
        met = true;
        if (cr >= g.occ_cap) {
            st = HF_PHG_CROWDED;
            break;
        }
        float o0 = vr.x, o1 = vr.y, o2 = vr.z;
        float sd = __fmaf_rn(o0, d0, __fmaf_rn(o1, d1, __fmul_rn(o2, d2)));
        if (sd < 0.0f) {
            o0 = -o0;
            o1 = -o1;
            o2 = -o2;
            sd = -sd;
        }
        if (sd < g.cos_turn) {
            st = HF_PHG_TURN;
            break;
        }
        d0 = o0;
        d1 = o1;
        d2 = o2;
        p0 = __fmaf_rn(g.step, d0, p0);
        p1 = __fmaf_rn(g.step, d1, p1);
        p2 = __fmaf_rn(g.step, d2, p2);
        float* v = out + 3 * dir * nv++;
        v[0] = p0;
        v[1] = p1;
        v[2] = p2;
    }
    if (t == g.max_steps) vox[dir * (nv - 1)] = (int)phg_voxel(g, p0, p1, p2);   // the last vertex's voxel
    if (!met) nv = 0;
    dl[0] = d0;
    dl[1] = d1;
    dl[2] = d2;
    *stop = st;
    return nv;
}

// bvox: per strand of the batch, the voxels of its vertices (stride vstride)
__global__ void k_phg_trace_guides(hf_phg_cfg g, const float4* __restrict__ vrec, const int* __restrict__ crowd,
                                   long long b0, long long b1, const float* __restrict__ seeds,
                                   const float* __restrict__ normals, float* __restrict__ gverts,
                                   int* __restrict__ glen, int* __restrict__ gstop, float* __restrict__ gtan,
                                   int* __restrict__ bvox, int vstride) {
    const long long i = b0 + blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= b1) return;
    int stop;
    glen[i] = phg_trace(g, vrec, crowd, seeds[3 * i], seeds[3 * i + 1], seeds[3 * i + 2], normals[3 * i],
                        normals[3 * i + 1], normals[3 * i + 2], g.root_steps,
                        gverts + (size_t)3 * (g.max_steps + 1) * i, bvox + (size_t)vstride * (i - b0), 1,
                        gtan + 3 * i, &stop);
    gstop[i] = stop;
}

// Two neighbouring lanes per seed: the even lane traces the backward half (written from the middle
// slot down), the odd lane the forward half (from the middle slot up); the odd lane then moves the
// polyline to the front.
__global__ void k_phg_trace_segments(hf_phg_cfg g, const float4* __restrict__ vrec, const int* __restrict__ crowd,
                                     long long b0, long long b1, const long long* __restrict__ svox,
                                     float* __restrict__ sverts, int* __restrict__ slen, float* __restrict__ stan,
                                     int* __restrict__ bvox, int vstride) {
    const long long tid = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    const long long k = b0 + (tid >> 1);
    const int half = (int)(tid & 1);
    if (k >= b1) return;   // both lanes of a pair
    const unsigned pm = 3u << (threadIdx.x & 30);
    const int L = g.max_steps;
    float* sv = sverts + (size_t)3 * (2 * L + 1) * k;
    int* bv = bvox + (size_t)vstride * (k - b0);
    float* tn = stan + 6 * k;
    const long long c = svox[k];
    if (crowd[c] > 0) {   // an earlier batch reached this voxel
        if (half) slen[k] = 0;
        for (int q = 0; q < 3; ++q) tn[3 * half + q] = 0.0f;
        return;
    }
    const long long cx = c % g.nx, cy = (c / g.nx) % g.ny, cz = c / ((long long)g.nx * g.ny);
    const float s0 = __fmaf_rn(__fadd_rn((float)cx, 0.5f), g.voxel, g.origin[0]);
    const float s1 = __fmaf_rn(__fadd_rn((float)cy, 0.5f), g.voxel, g.origin[1]);
    const float s2 = __fmaf_rn(__fadd_rn((float)cz, 0.5f), g.voxel, g.origin[2]);
    const float4 vr = vrec[c];
    const float sg = half ? 1.0f : -1.0f;
    int stop;
    const int nh = phg_trace(g, vrec, crowd, s0, s1, s2, sg * vr.x, sg * vr.y, sg * vr.z, 0, sv + 3 * L, bv + L,
                             half ? 1 : -1, tn + 3 * half, &stop);
    const int nb = __shfl_sync(pm, nh, threadIdx.x & 30);
    __syncwarp(pm);   // both halves written
    if (half) {
        const int first = L - nb + 1, n = nb + nh - 1;
        for (int q = 0; q < 3 * n; ++q) sv[q] = sv[3 * first + q];   // to the front (first >= 0, upward copy)
        for (int q = 0; q < n; ++q) bv[q] = bv[first + q];
        slen[k] = n;
    }
}

// Deferred occupancy: one more strand in every occupied voxel a polyline of [b0, b1) entered
// (consecutive vertices in one voxel count once).  A thread per vertex slot (vstride per polyline):
// vertex k counts when it is a voxel other than vertex k - 1's; the integer sums do not depend on
// the order.
__global__ void k_phg_count(const int* __restrict__ occ, const int* __restrict__ len, long long b0, long long b1,
                            const int* __restrict__ bvox, int vstride, int* __restrict__ crowd) {
    const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    const long long i = b0 + t / vstride;
    const int k = (int)(t % vstride);
    if (i >= b1 || k >= len[i]) return;
    const int* v = bvox + (size_t)vstride * (i - b0);
    const int c = v[k];
    if (c >= 0 && (k == 0 || v[k - 1] != c) && occ[c] > 0) atomicAdd(crowd + c, 1);
}

// ------------------------------------------------------------------ ordered compaction and scans
// per block of kScanBlock elements: the count of flagged elements (segment seeds: occupied voxels
// no strand entered)
__global__ void k_phg_flags(long long nvox, const int* __restrict__ occ, const int* __restrict__ crowd,
                            int* __restrict__ bsum) {
    int cnt = 0;
    const long long base = (long long)blockIdx.x * kScanBlock;
    for (int q = threadIdx.x; q < kScanBlock; q += blockDim.x) {
        const long long c = base + q;
        cnt += c < nvox && occ[c] > 0 && crowd[c] == 0;
    }
    __shared__ int s[kThreads];
    s[threadIdx.x] = cnt;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) s[threadIdx.x] += s[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) bsum[blockIdx.x] = s[0];
}

// exclusive scan of n block sums in place by one CTA; the total to *total
__global__ void k_phg_scan_top(int* __restrict__ bsum, long long n, long long* __restrict__ total) {
    __shared__ long long s[kThreads];
    long long carry = 0;
    for (long long base = 0; base < n; base += blockDim.x) {
        const long long i = base + threadIdx.x;
        const long long v = i < n ? bsum[i] : 0;
        s[threadIdx.x] = v;
        __syncthreads();
        for (int w = 1; w < (int)blockDim.x; w <<= 1) {   // inclusive Hillis-Steele
            const long long u = threadIdx.x >= w ? s[threadIdx.x - w] : 0;
            __syncthreads();
            s[threadIdx.x] += u;
            __syncthreads();
        }
        if (i < n) bsum[i] = (int)(carry + s[threadIdx.x] - v);
        carry += s[blockDim.x - 1];
        __syncthreads();
    }
    if (threadIdx.x == 0) *total = carry;
}

// the flagged voxels of each block written in voxel order from the block's offset
__global__ void k_phg_write(long long nvox, const int* __restrict__ occ, const int* __restrict__ crowd,
                            const int* __restrict__ boff, long long* __restrict__ svox) {
    __shared__ int wsum[kThreads / 32];
    __shared__ int run;
    const long long base = (long long)blockIdx.x * kScanBlock;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) run = boff[blockIdx.x];
    __syncthreads();
    for (int q0 = 0; q0 < kScanBlock; q0 += blockDim.x) {
        const long long c = base + q0 + threadIdx.x;
        const bool f = c < nvox && occ[c] > 0 && crowd[c] == 0;
        const unsigned b = __ballot_sync(0xffffffffu, f);
        if (lane == 0) wsum[warp] = __popc(b);
        __syncthreads();
        int off = run;
        for (int w = 0; w < warp; ++w) off += wsum[w];
        if (f) svox[off + __popc(b & ((1u << lane) - 1u))] = c;
        __syncthreads();
        if (threadIdx.x == 0) {
            int t = 0;
            for (int w = 0; w < (int)blockDim.x / 32; ++w) t += wsum[w];
            run += t;
        }
        __syncthreads();
    }
}

// ------------------------------------------------------------------ E: linking
struct EndRef {
    const float* p;
    const float* t;
    long long strand;
};

__device__ __forceinline__ bool end_of(long long e, long long S, int L, const float* gverts, const int* glen,
                                       const float* gtan, const float* sverts, const int* slen, const float* stan,
                                       EndRef& r) {
    if (e < S) {
        const int n = glen[e];
        if (n <= 0) return false;
        r.p = gverts + (size_t)3 * (L + 1) * e + 3 * (n - 1);
        r.t = gtan + 3 * e;
        r.strand = e;
        return true;
    }
    const long long k = (e - S) >> 1;
    const int side = (int)((e - S) & 1);
    const int n = slen[k];
    if (n <= 0) return false;
    r.p = sverts + (size_t)3 * (2 * L + 1) * k + (side ? 3 * (n - 1) : 0);
    r.t = stan + 6 * k + 3 * side;
    r.strand = S + k;
    return true;
}

__device__ __forceinline__ long long cell_index(const LinkGrid& G, int3 c) {
    return ((long long)c.z * G.ny + c.y) * G.nx + c.x;
}

// segment ends per cell
__global__ void k_phg_bin(hf_phg_cfg g, LinkGrid G, long long S, long long K, const float* __restrict__ sverts,
                          const int* __restrict__ slen, int* __restrict__ ccount) {
    const long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (q >= 2 * K) return;
    const long long k = q >> 1;
    const int n = slen[k];
    if (n <= 0) return;
    const float* p = sverts + (size_t)3 * (2 * g.max_steps + 1) * k + ((q & 1) ? 3 * (n - 1) : 0);
    atomicAdd(ccount + cell_index(G, phg_cell(G, p[0], p[1], p[2])), 1);
}

// exclusive scan of the cell counts: per block of kScanBlock cells, then the block offsets added
__global__ void k_phg_scan_blocks(int* __restrict__ a, long long n, int* __restrict__ bsum) {
    __shared__ int s[kScanBlock];
    const long long base = (long long)blockIdx.x * kScanBlock;
    for (int q = threadIdx.x; q < kScanBlock; q += blockDim.x) s[q] = base + q < n ? a[base + q] : 0;
    __syncthreads();
    if (threadIdx.x == 0) {   // a serial scan of 1024 values: small next to the rest
        int run = 0;
        for (int q = 0; q < kScanBlock; ++q) {
            const int v = s[q];
            s[q] = run;
            run += v;
        }
        bsum[blockIdx.x] = run;
    }
    __syncthreads();
    for (int q = threadIdx.x; q < kScanBlock; q += blockDim.x)
        if (base + q < n) a[base + q] = s[q];
}

__global__ void k_phg_scan_add(int* __restrict__ a, long long n, const int* __restrict__ boff) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i < n) a[i] += boff[i / kScanBlock];
}

// each segment end into its cell's slice of the list, with what the queries need: (position, end
// index) and (outward tangent, strand index)
__global__ void k_phg_put(hf_phg_cfg g, LinkGrid G, long long S, long long K, const float* __restrict__ sverts,
                          const int* __restrict__ slen, const float* __restrict__ stan, const int* __restrict__ cstart,
                          int* __restrict__ cursor, float4* __restrict__ list) {
    const long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (q >= 2 * K) return;
    const long long k = q >> 1;
    const int n = slen[k];
    if (n <= 0) return;
    const float* p = sverts + (size_t)3 * (2 * g.max_steps + 1) * k + ((q & 1) ? 3 * (n - 1) : 0);
    const float* t = stan + 6 * k + 3 * (q & 1);
    const long long c = cell_index(G, phg_cell(G, p[0], p[1], p[2]));
    const long long slot = cstart[c] + atomicAdd(cursor + c, 1);   // order within a cell does not matter below
    list[2 * slot] = make_float4(p[0], p[1], p[2], __int_as_float((int)q));
    list[2 * slot + 1] = make_float4(t[0], t[1], t[2], __int_as_float((int)(S + k)));
}

// every strand end: the nearest compatible end of another segment (Eq. segment_connection), ties
// to the lower end
__global__ void k_phg_link(hf_phg_cfg g, LinkGrid G, long long S, long long K, const float* __restrict__ gverts,
                           const int* __restrict__ glen, const float* __restrict__ gtan,
                           const float* __restrict__ sverts, const int* __restrict__ slen,
                           const float* __restrict__ stan, const int* __restrict__ cstart,
                           const int* __restrict__ ccount, const float4* __restrict__ list,
                           long long* __restrict__ match) {
    const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (e >= S + 2 * K) return;
    const int L = g.max_steps;
    EndRef me;
    long long best = -1;
    if (end_of(e, S, L, gverts, glen, gtan, sverts, slen, stan, me)) {
        const float pe0 = me.p[0], pe1 = me.p[1], pe2 = me.p[2];
        const float te0 = me.t[0], te1 = me.t[1], te2 = me.t[2];
        const float L2 = __fmul_rn(g.link_dist, g.link_dist);
        const int3 c = phg_cell(G, pe0, pe1, pe2);
        float bd = 0.0f;
        for (int z = max(c.z - 1, 0); z <= min(c.z + 1, G.nz - 1); ++z)
            for (int y = max(c.y - 1, 0); y <= min(c.y + 1, G.ny - 1); ++y)
                for (int x = max(c.x - 1, 0); x <= min(c.x + 1, G.nx - 1); ++x) {
                    const long long ci = cell_index(G, make_int3(x, y, z));
                    const int s0 = cstart[ci], n = ccount[ci];
                    for (int u = 0; u < n; ++u) {
                        const float4 cp = list[2 * (s0 + u)], ct = list[2 * (s0 + u) + 1];
                        if (__float_as_int(ct.w) == me.strand) continue;
                        const long long q = __float_as_int(cp.w);
                        const float dx = __fsub_rn(pe0, cp.x), dy = __fsub_rn(pe1, cp.y), dz = __fsub_rn(pe2, cp.z);
                        const float d2 = __fmaf_rn(dx, dx, __fmaf_rn(dy, dy, __fmul_rn(dz, dz)));
                        if (!(d2 < L2)) continue;
                        const float dt = __fmaf_rn(te0, ct.x, __fmaf_rn(te1, ct.y, __fmul_rn(te2, ct.z)));
                        if (!(-dt > g.link_cos)) continue;
                        if (best < 0 || d2 < bd || (d2 == bd && q < best)) {
                            best = q;
                            bd = d2;
                        }
                    }
                }
    }
    match[e] = best;
}

// Connected components as a lock-free union-find over the links.  Every parent pointer points to a
// smaller index (a link hooks the larger root under the smaller with a compare-and-swap, and path
// halving only shortens such chains), so each component's root is its smallest member whatever the
// order of the threads: label = the component minimum, the oracle's labels exactly.
__device__ __forceinline__ int uf_find(int* __restrict__ p, int x) {
    for (int it = 0; it < (1 << 20); ++it) {   // chains are short; the cap only bounds the loop
        const int q = p[x];
        if (q == x) return x;
        const int r = p[q];
        if (r != q) p[x] = r;   // halve: x now points to its grandparent (a smaller index)
        x = r;
    }
    return x;
}

__global__ void k_phg_union(long long S, long long nends, const long long* __restrict__ match, int* __restrict__ label,
                            int* __restrict__ failed) {
    const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (e >= nends || match[e] < 0) return;
    int a = (int)(e < S ? e : S + ((e - S) >> 1)), b = (int)(S + (match[e] >> 1));
    for (int it = 0; it < (1 << 20); ++it) {
        a = uf_find(label, a);
        b = uf_find(label, b);
        if (a == b) return;
        if (a > b) {
            const int t = a;
            a = b;
            b = t;
        }
        const int old = atomicCAS(label + b, b, a);   // hook root b under the smaller root a
        if (old == b) return;
        b = old;   // b was hooked meanwhile: retry from its new parent
    }
    *failed = 1;
}

// every label to its root (after the unions: the structure no longer changes)
__global__ void k_phg_flatten(long long n, int* __restrict__ label, int* __restrict__ failed) {
    const long long x = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (x >= n) return;
    int l = label[x];
    for (int it = 0; it < (1 << 20); ++it) {
        const int m = label[l];
        if (m == l) {
            label[x] = l;
            return;
        }
        l = m;
    }
    *failed = 1;
}

__global__ void k_phg_iota(long long n, int* __restrict__ label) {
    const long long x = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (x < n) label[x] = (int)x;
}

unsigned grid_for(long long n, int threads) {
    const long long b = (n + threads - 1) / threads;
    return (unsigned)(b < 1 ? 1 : (b > 148LL * 64 ? 148LL * 64 : b));
}
unsigned grid_all(long long n, int threads) { return (unsigned)((n + threads - 1) / threads); }

}  // namespace

// ------------------------------------------------------------------ C ABI
extern "C" int hair_fuse_phg(hf_ctx* c, const hf_phg_cfg* cfg, long long N, const float* pts, const float* dirs,
                             const uint8_t* valid, long long S, const float* seeds, const float* normals,
                             hf_phg_out* out, int mem_kind) {
    if (!c || !cfg || !out) return HF_ERR_INVALID_ARG;
    if (mem_kind != HF_HOST && mem_kind != HF_DEVICE) return hf_set_err(c, HF_ERR_INVALID_ARG, "bad mem_kind");
    const hf_phg_cfg g = *cfg;
    const long long nvox = (long long)g.nx * g.ny * g.nz;
    const long long ncell = (long long)(g.nx + 2) * (g.ny + 2) * (g.nz + 2);
    if (g.nx < 1 || g.ny < 1 || g.nz < 1 || ncell >= (1LL << 31) ||
        !(isfinite(g.origin[0]) && isfinite(g.origin[1]) && isfinite(g.origin[2])) ||
        !(isfinite(g.voxel) && g.voxel > 0.0f) || !(g.step > 0.0f && g.step <= g.voxel) || g.max_steps < 1 ||
        g.max_steps > 4096 || g.root_steps < 0 || !(g.cos_turn >= -1.0f && g.cos_turn <= 1.0f) || g.occ_cap < 1 ||
        g.batch < 1 || !(isfinite(g.link_dist) && g.link_dist >= 0.0f && g.link_dist <= 8.0f * g.voxel) ||
        !(g.link_cos >= -1.0f && g.link_cos <= 1.0f))
        return hf_set_err(c, HF_ERR_INVALID_ARG,
                          "phg: grid >= 1 and < 2^31 cells, voxel > 0, 0 < step <= voxel, max_steps in [1, 4096], "
                          "root_steps >= 0, cos values in [-1, 1], occ_cap >= 1, batch >= 1, 0 <= link_dist <= "
                          "8 voxel");
    if (N < 0 || S < 0 || out->seg_cap < 0 || (N > 0 && (!pts || !dirs)) || (S > 0 && (!seeds || !normals)) ||
        !out->occ || !out->ori || (S > 0 && (!out->gverts || !out->glen)) ||
        (out->seg_cap > 0 && (!out->slen || !out->sverts)) || !out->label || !out->n_seg)
        return hf_set_err(c, HF_ERR_INVALID_ARG, "phg: null or negative argument");
    if (S + out->seg_cap >= (1LL << 31)) return hf_set_err(c, HF_ERR_SHAPE, "phg: more than 2^31 strands");
    if (nvox >= (1LL << 31) || (double)nvox * (2 * g.max_steps + 1) > 1e15)
        return hf_set_err(c, HF_ERR_SHAPE, "phg: grid too large");
    const int L = g.max_steps;
    const long long cap = out->seg_cap;
    // the linking grid: cells of at least 1.01 link_dist over the voxel grid and one voxel around it
    LinkGrid G;
    G.cell = fmaxf(g.voxel, 1.01f * g.link_dist);
    G.o0 = g.origin[0] - g.voxel;
    G.o1 = g.origin[1] - g.voxel;
    G.o2 = g.origin[2] - g.voxel;
    G.nx = (int)ceil((double)(g.nx + 2) * g.voxel / G.cell) + 1;
    G.ny = (int)ceil((double)(g.ny + 2) * g.voxel / G.cell) + 1;
    G.nz = (int)ceil((double)(g.nz + 2) * g.voxel / G.cell) + 1;
    const long long nlc = (long long)G.nx * G.ny * G.nz;
    const long long bmax = g.batch < (S > cap ? S : cap) ? g.batch : (S > cap ? S : cap);   // strands per batch
    const int vstride = 2 * L + 1;
    // scratch: device copies of host arrays, the tensors, the scans and the links
    struct Part {
        size_t off, bytes;
    };
    size_t total = 0;
    auto part = [&](size_t bytes) {
        Part p{total, bytes};
        total += (bytes + 255) & ~(size_t)255;
        return p;
    };
    const bool host = mem_kind == HF_HOST;
    const long long nblk_v = (nvox + kScanBlock - 1) / kScanBlock, nblk_c = (nlc + kScanBlock - 1) / kScanBlock;
    const Part pT = part(sizeof(long long) * 6 * nvox), pCrowd = part(out->crowd && !host ? 0 : sizeof(int) * nvox),
               pB = part(sizeof(int) * (size_t)(nblk_v > nblk_c ? nblk_v : nblk_c)), pTot = part(sizeof(long long)),
               pCnt = part(sizeof(int) * nlc), pCur = part(sizeof(int) * nlc), pList = part(sizeof(float4) * 4 * cap),
               pVrec = part(sizeof(float4) * nvox), pBvox = part(sizeof(int) * vstride * (size_t)(bmax > 0 ? bmax : 1)),
               pMatch = part(sizeof(long long) * (S + 2 * cap)), pChg = part(sizeof(int)),
               pGstop = part(out->gstop && !host ? 0 : sizeof(int) * S),
               pGtan = part(out->gtan && !host ? 0 : sizeof(float) * 3 * S),
               pSvox = part(out->svox && !host ? 0 : sizeof(long long) * cap),
               pStan = part(out->stan && !host ? 0 : sizeof(float) * 6 * cap);
    Part pIn[5] = {}, pOut[6] = {};
    if (host) {
        pIn[0] = part(sizeof(float) * 3 * N);
        pIn[1] = part(sizeof(float) * 3 * N);
        pIn[2] = part(valid ? (size_t)N : 0);
        pIn[3] = part(sizeof(float) * 3 * S);
        pIn[4] = part(sizeof(float) * 3 * S);
        pOut[0] = part(sizeof(int) * nvox);
        pOut[1] = part(sizeof(float) * 3 * nvox);
        pOut[2] = part(sizeof(float) * 3 * (L + 1) * S);
        pOut[3] = part(sizeof(int) * S);
        pOut[4] = part(sizeof(float) * 3 * (2 * L + 1) * cap);
        pOut[5] = part(sizeof(int) * (S + cap) + sizeof(int) * cap);
    }
    int rc;
    if ((rc = hf_ensure(c, c->phg, total))) return rc;
    char* base = (char*)c->phg.p;
    auto at = [&](const Part& p) { return (void*)(base + p.off); };
    cudaStream_t st = c->stream;
    cudaError_t e = cudaSuccess;
    const float *d_pts = pts, *d_dirs = dirs, *d_seeds = seeds, *d_normals = normals;
    const uint8_t* d_valid = valid;
    int *occ = out->occ, *glen = out->glen, *slen = out->slen, *label = out->label;
    float *ori = out->ori, *gverts = out->gverts, *sverts = out->sverts;
    if (host) {
        e = cudaMemcpyAsync(at(pIn[0]), pts, pIn[0].bytes, cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(at(pIn[1]), dirs, pIn[1].bytes, cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess && valid) e = cudaMemcpyAsync(at(pIn[2]), valid, pIn[2].bytes, cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(at(pIn[3]), seeds, pIn[3].bytes, cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(at(pIn[4]), normals, pIn[4].bytes, cudaMemcpyHostToDevice, st);
        if (e != cudaSuccess) return hf_cuda_err(c, e, "phg inputs");
        d_pts = (const float*)at(pIn[0]);
        d_dirs = (const float*)at(pIn[1]);
        d_valid = valid ? (const uint8_t*)at(pIn[2]) : nullptr;
        d_seeds = (const float*)at(pIn[3]);
        d_normals = (const float*)at(pIn[4]);
        occ = (int*)at(pOut[0]);
        ori = (float*)at(pOut[1]);
        gverts = (float*)at(pOut[2]);
        glen = (int*)at(pOut[3]);
        sverts = (float*)at(pOut[4]);
        label = (int*)at(pOut[5]);
        slen = label + S + cap;
    }
    int* crowd = out->crowd && !host ? out->crowd : (int*)at(pCrowd);
    int* gstop = out->gstop && !host ? out->gstop : (int*)at(pGstop);
    float* gtan = out->gtan && !host ? out->gtan : (float*)at(pGtan);
    long long* svox = out->svox && !host ? (long long*)out->svox : (long long*)at(pSvox);
    float* stan = out->stan && !host ? out->stan : (float*)at(pStan);
    long long* T = (long long*)at(pT);
    float4* vrec = (float4*)at(pVrec);
    int* bvox = (int*)at(pBvox);
    int* bsum = (int*)at(pB);
    long long* tot = (long long*)at(pTot);
    // A, B
    e = cudaMemsetAsync(occ, 0, sizeof(int) * nvox, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(T, 0, sizeof(long long) * 6 * nvox, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(crowd, 0, sizeof(int) * nvox, st);
    if (e != cudaSuccess) return hf_cuda_err(c, e, "phg clear");
    if (N > 0 && (rc = run_launch(c, "k_phg_splat", [&] {
                      k_phg_splat<<<grid_for(N, kThreads), kThreads, 0, st>>>(g, N, d_pts, d_dirs, d_valid, occ,
                                                                              (unsigned long long*)T);
                      return cudaGetLastError();
                  })))
        return rc;
    if ((rc = run_launch(c, "k_phg_orient", [&] {
             k_phg_orient<<<grid_for(nvox, kThreads), kThreads, 0, st>>>(nvox, occ, T, ori, vrec);
             return cudaGetLastError();
         })))
        return rc;
    // C: guide strands, batch by batch
    for (long long b0 = 0; b0 < S; b0 += g.batch) {
        const long long b1 = b0 + g.batch < S ? b0 + g.batch : S;
        if ((rc = run_launch(c, "k_phg_trace_guides", [&] {
                 k_phg_trace_guides<<<grid_all(b1 - b0, 128), 128, 0, st>>>(g, vrec, crowd, b0, b1, d_seeds,
                                                                           d_normals, gverts, glen, gstop, gtan, bvox,
                                                                           vstride);
                 return cudaGetLastError();
             })))
            return rc;
        if ((rc = run_launch(c, "k_phg_count", [&] {
                 k_phg_count<<<grid_all((b1 - b0) * vstride, 128), 128, 0, st>>>(occ, glen, b0, b1, bvox, vstride, crowd);
                 return cudaGetLastError();
             })))
            return rc;
    }
    // D: the segment seeds in voxel order
    if ((rc = run_launch(c, "k_phg_flags", [&] {
             k_phg_flags<<<(unsigned)nblk_v, kThreads, 0, st>>>(nvox, occ, crowd, bsum);
             return cudaGetLastError();
         })))
        return rc;
    if ((rc = run_launch(c, "k_phg_scan_top", [&] {
             k_phg_scan_top<<<1, kThreads, 0, st>>>(bsum, nblk_v, tot);
             return cudaGetLastError();
         })))
        return rc;
    long long K = 0;
    e = cudaMemcpyAsync(&K, tot, sizeof(long long), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return hf_cuda_err(c, e, "phg seed count");
    if (host) {
        *out->n_seg = K;
    } else if ((e = cudaMemcpyAsync(out->n_seg, &K, sizeof(long long), cudaMemcpyHostToDevice, st)) != cudaSuccess) {
        return hf_cuda_err(c, e, "phg seed count");
    }
    if (K > cap) return hf_set_err(c, HF_ERR_SHAPE, "phg: %lld segment seeds exceed seg_cap %lld", K, cap);
    if (K > 0 && (rc = run_launch(c, "k_phg_write", [&] {
                      k_phg_write<<<(unsigned)nblk_v, kThreads, 0, st>>>(nvox, occ, crowd, bsum, svox);
                      return cudaGetLastError();
                  })))
        return rc;
    for (long long b0 = 0; b0 < K; b0 += g.batch) {
        const long long b1 = b0 + g.batch < K ? b0 + g.batch : K;
        if ((rc = run_launch(c, "k_phg_trace_segments", [&] {
                 k_phg_trace_segments<<<grid_all(2 * (b1 - b0), 128), 128, 0, st>>>(g, vrec, crowd, b0, b1, svox,
                                                                             sverts, slen, stan, bvox, vstride);
                 return cudaGetLastError();
             })))
            return rc;
        if ((rc = run_launch(c, "k_phg_count", [&] {
                 k_phg_count<<<grid_all((b1 - b0) * vstride, 128), 128, 0, st>>>(occ, slen, b0, b1, bvox, vstride, crowd);
                 return cudaGetLastError();
             })))
            return rc;
    }
    // E: bin the segment ends, link every end, components
    int* ccount = (int*)at(pCnt);
    int* cstart = (int*)at(pCur);   // the counts' exclusive scan
    float4* list = (float4*)at(pList);
    long long* match = (long long*)at(pMatch);
    int* changed = (int*)at(pChg);
    const long long nends = S + 2 * K, nstr = S + K;
    e = cudaMemsetAsync(ccount, 0, sizeof(int) * nlc, st);
    if (e != cudaSuccess) return hf_cuda_err(c, e, "phg link clear");
    if (K > 0 && (rc = run_launch(c, "k_phg_bin", [&] {
                      k_phg_bin<<<grid_all(2 * K, kThreads), kThreads, 0, st>>>(g, G, S, K, sverts, slen, ccount);
                      return cudaGetLastError();
                  })))
        return rc;
    e = cudaMemcpyAsync(cstart, ccount, sizeof(int) * nlc, cudaMemcpyDeviceToDevice, st);
    if (e != cudaSuccess) return hf_cuda_err(c, e, "phg link scan");
    if ((rc = run_launch(c, "k_phg_scan_cells", [&] {
             k_phg_scan_blocks<<<(unsigned)nblk_c, kThreads, 0, st>>>(cstart, nlc, bsum);
             k_phg_scan_top<<<1, kThreads, 0, st>>>(bsum, nblk_c, tot);
             k_phg_scan_add<<<grid_all(nlc, kThreads), kThreads, 0, st>>>(cstart, nlc, bsum);
             return cudaGetLastError();
         })))
        return rc;
    // the cursor reuses the counts
    e = cudaMemsetAsync(ccount, 0, sizeof(int) * nlc, st);
    if (e != cudaSuccess) return hf_cuda_err(c, e, "phg link clear");
    if (K > 0 && (rc = run_launch(c, "k_phg_put", [&] {
                      k_phg_put<<<grid_all(2 * K, kThreads), kThreads, 0, st>>>(g, G, S, K, sverts, slen, stan,
                                                                              cstart, ccount, list);
                      return cudaGetLastError();
                  })))
        return rc;
    if (nends > 0 && (rc = run_launch(c, "k_phg_link", [&] {
                          k_phg_link<<<grid_all(nends, 128), 128, 0, st>>>(g, G, S, K, gverts, glen, gtan, sverts,
                                                                         slen, stan, cstart, ccount, list, match);
                          return cudaGetLastError();
                      })))
        return rc;
    if (nstr > 0) {
        if ((rc = run_launch(c, "k_phg_iota", [&] {
                 k_phg_iota<<<grid_all(nstr, kThreads), kThreads, 0, st>>>(nstr, label);
                 return cudaGetLastError();
             })))
            return rc;
        e = cudaMemsetAsync(changed, 0, sizeof(int), st);
        if (e != cudaSuccess) return hf_cuda_err(c, e, "phg components");
        if ((rc = run_launch(c, "k_phg_union", [&] {
                 if (nends > 0)
                     k_phg_union<<<grid_all(nends, kThreads), kThreads, 0, st>>>(S, nends, match, label, changed);
                 k_phg_flatten<<<grid_all(nstr, kThreads), kThreads, 0, st>>>(nstr, label, changed);
                 return cudaGetLastError();
             })))
            return rc;
        int h = 0;
        e = cudaMemcpyAsync(&h, changed, sizeof(int), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return hf_cuda_err(c, e, "phg components");
        if (h) return hf_set_err(c, HF_ERR_CUDA, "phg: a union-find chain exceeded its bound");
    }
    if (host) {
        struct Cp {
            void* dst;
            const void* src;
            size_t bytes;
        };
        std::vector<Cp> cps = {{out->occ, occ, sizeof(int) * nvox},
                               {out->ori, ori, sizeof(float) * 3 * nvox},
                               {out->gverts, gverts, sizeof(float) * 3 * (L + 1) * S},
                               {out->glen, glen, sizeof(int) * S},
                               {out->sverts, sverts, sizeof(float) * 3 * (2 * L + 1) * K},
                               {out->slen, slen, sizeof(int) * K},
                               {out->label, label, sizeof(int) * (S + K)},
                               {out->crowd, crowd, sizeof(int) * nvox},
                               {out->gstop, gstop, sizeof(int) * S},
                               {out->gtan, gtan, sizeof(float) * 3 * S},
                               {out->svox, svox, sizeof(long long) * K},
                               {out->stan, stan, sizeof(float) * 6 * K}};
        for (const Cp& q : cps)
            if (q.dst && q.bytes && e == cudaSuccess) e = cudaMemcpyAsync(q.dst, q.src, q.bytes, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return hf_cuda_err(c, e, "phg outputs");
    }
    return HF_OK;
}
