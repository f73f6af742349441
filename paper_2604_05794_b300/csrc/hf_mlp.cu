// hf_mlp.cu - the learned proposal network: features, training (forward, backward, Adam) and
// inference, all on the tensor-core GEMM of hf_gemm.cu.  The paper has no counterpart; the
// network maps per-point multi-view orientation features to an initial direction for a short
// refinement, and is trained on directions the plain fusion produces.
//
// Network: x (51 features, zero-padded to 64) -> 256 -> 256 -> 3, GELU (erf form) after the two
// hidden layers, BF16 operands, FP32 accumulation and FP32 master weights.
// Parameter vector (f32, hf_mlp_param_count() entries), in this order:
//   W1 [256 x 64] (columns 51..63 stay 0), b1 [256], W2 [256 x 256], b2 [256], W3 [3 x 256], b3 [3].
// Loss per sample: 1 - (y_hat . t)^2 with y_hat = y / |y| (sign-invariant), averaged over the batch.
#include <cuda_bf16.h>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <vector>

#include "hf_gemm.cuh"
#include "hf_internal.cuh"
#include "hf_mlp.cuh"

namespace {

constexpr int kIn = 64, kHid = 256, kOut3 = 16;   // padded widths
constexpr int kFeatViews = 16;
constexpr long long kW1 = 0, kB1 = kW1 + kHid * kIn, kW2 = kB1 + kHid, kB2 = kW2 + kHid * kHid, kW3 = kB2 + kHid,
                    kB3 = kW3 + 3 * kHid, kParams = kB3 + 3;

__device__ __forceinline__ uint16_t bf16_bits(float x) { return __bfloat16_as_ushort(__float2bfloat16_rn(x)); }
__device__ __forceinline__ float bf16_val(uint16_t b) { return __bfloat162float(__ushort_as_bfloat16(b)); }

__host__ __device__ inline uint64_t splitmix(uint64_t x) {
    x += 0x9E3779B97F4A7C15ULL;
    x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ULL;
    x = (x ^ (x >> 27)) * 0x94D049BB133111EBULL;
    return x ^ (x >> 31);
}

// ---------------------------------------------------------------- parameters
// Uniform(-1/sqrt(fan_in), 1/sqrt(fan_in)) for every weight and bias, from a counter-based hash.
__global__ void k_init(float* P, uint64_t seed) {
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < kParams; e += (long long)gridDim.x * blockDim.x) {
        float fan;
        bool zero = false;
        if (e < kB1) {
            fan = 51.0f;
            zero = (e - kW1) % kIn >= 51;
        } else if (e < kW2) fan = 51.0f;
        else if (e < kW3) fan = 256.0f;
        else fan = 256.0f;
        const double u = (double)(splitmix(seed ^ splitmix((uint64_t)e)) >> 11) * (1.0 / 9007199254740992.0);
        P[e] = zero ? 0.0f : (float)((2.0 * u - 1.0) / sqrt((double)fan));
    }
}

// bf16 working copies (and transposes, and the padded layer-3 forms) of the f32 masters
__global__ void k_pack(const float* __restrict__ P, MlpDev d) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < kHid * kIn) d.W1b[t] = bf16_bits(P[kW1 + t]);
    if (t < kHid * kHid) {
        const int r = t / kHid, c = t % kHid;
        const uint16_t b = bf16_bits(P[kW2 + t]);
        d.W2b[t] = b;
        d.W2Tb[c * kHid + r] = b;
    }
    if (t < kOut3 * kHid) {   // W3 padded to 16 rows; its transpose padded to 64 columns
        const int r = t / kHid, c = t % kHid;
        const uint16_t b = r < 3 ? bf16_bits(P[kW3 + r * kHid + c]) : 0;
        d.W3pb[t] = b;
        if (r < 3) d.w3f[r * kHid + c] = bf16_val(b);
    }
    if (t < kHid * kIn) {
        const int r = t / kIn, c = t % kIn;   // W3T[r][c] = W3[c][r]
        d.W3Tb[t] = c < 3 ? bf16_bits(P[kW3 + c * kHid + r]) : 0;
    }
    if (t < kOut3) d.b3p[t] = t < 3 ? P[kB3 + t] : 0.0f;
}

// ---------------------------------------------------------------- training-step kernels
// batch b <- sample hash(seed, step, b) mod n (with replacement), x rows and their transpose
__global__ void k_gather(const uint16_t* __restrict__ X, const float* __restrict__ T, long long n, int B, uint64_t seed,
                         const long long* __restrict__ step, MlpDev d) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= B) return;
    const long long j = (long long)(splitmix(seed ^ splitmix(((uint64_t)*step << 20) ^ (uint64_t)b)) % (uint64_t)n);
    const uint4* src = reinterpret_cast<const uint4*>(X + j * kIn);
    uint4* dst = reinterpret_cast<uint4*>(d.Xb + (size_t)b * kIn);
#pragma unroll
    for (int q = 0; q < kIn / 8; ++q) dst[q] = src[q];
    for (int c = 0; c < kIn; ++c) d.XTb[(size_t)c * B + b] = X[j * kIn + c];
    for (int c = 0; c < 3; ++c) d.Tb[b * 3 + c] = T[j * 3 + c];
}

// loss 1 - (y_hat . t)^2 and its gradient with respect to y (mean over the batch)
__global__ void k_loss(int B, MlpDev d) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    float L = 0.0f, g[3] = {0.0f, 0.0f, 0.0f};
    if (b < B) {
        const float y0 = d.Z3[b * kOut3], y1 = d.Z3[b * kOut3 + 1], y2 = d.Z3[b * kOut3 + 2];
        const float t0 = d.Tb[b * 3], t1 = d.Tb[b * 3 + 1], t2 = d.Tb[b * 3 + 2];
        const float n2 = y0 * y0 + y1 * y1 + y2 * y2;
        L = 1.0f;
        if (n2 > 0.0f) {
            const float inv = rsqrtf(n2);
            const float s = (y0 * t0 + y1 * t1 + y2 * t2) * inv;   // y_hat . t
            L = 1.0f - s * s;
            // dL/dy = -2 s / |y| (t - s y_hat)
            const float k = -2.0f * s * inv / (float)B;
            g[0] = k * (t0 - s * y0 * inv);
            g[1] = k * (t1 - s * y1 * inv);
            g[2] = k * (t2 - s * y2 * inv);
        }
#pragma unroll
        for (int c = 0; c < 64; ++c) d.dZ3[(size_t)b * 64 + c] = c < 3 ? bf16_bits(g[c]) : 0;
#pragma unroll
        for (int c = 0; c < kOut3; ++c) d.dZ3T[(size_t)c * B + b] = c < 3 ? bf16_bits(g[c]) : 0;
    }
    // block sums of the loss and of the bias gradient -> bparts[block][4] (summed in order later)
    __shared__ float red[4][32];
    float v[4] = {L / (float)B, g[0], g[1], g[2]};
#pragma unroll
    for (int q = 0; q < 4; ++q)
        for (int o = 16; o > 0; o >>= 1) v[q] += __shfl_xor_sync(0xffffffffu, v[q], o);
    if ((threadIdx.x & 31) == 0)
        for (int q = 0; q < 4; ++q) red[q][threadIdx.x >> 5] = v[q];
    __syncthreads();
    if (threadIdx.x < 4) {
        float s = 0.0f;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[threadIdx.x][w];
        d.bparts[blockIdx.x * 4 + threadIdx.x] = s;
    }
}

// sums of the per-block loss / layer-3 bias partials, in block order
__global__ void k_loss_sum(int nblocks, MlpDev d, float* __restrict__ G, const long long* __restrict__ step,
                           float* loss_hist) {
    if (threadIdx.x >= 4) return;
    float s = 0.0f;
    for (int b = 0; b < nblocks; ++b) s += d.bparts[b * 4 + threadIdx.x];
    if (threadIdx.x == 0) loss_hist[*step] = s;
    else G[kB3 + threadIdx.x - 1] = s;
}

// dZ = dH * gelu'(Z); bf16 copies (row-major and transposed) for the GEMMs, f32 column sums -> db
__global__ void k_gelu_back(int B, const float* __restrict__ dH, const float* __restrict__ Z, uint16_t* dZ, uint16_t* dZT,
                            float* __restrict__ dbpart) {
    const int c = threadIdx.x;                     // column (256 threads)
    const int r0 = blockIdx.x * 32;                // 32 rows per block
    float acc = 0.0f;
    for (int r = r0; r < r0 + 32 && r < B; ++r) {
        const size_t o = (size_t)r * kHid + c;
        const float z = Z[o];
        const float cdf = 0.5f * (1.0f + erff(z * 0.70710678118654752f));
        const float pdf = 0.39894228040143268f * expf(-0.5f * z * z);
        const float g = dH[o] * (cdf + z * pdf);
        const uint16_t gb = bf16_bits(g);
        dZ[o] = gb;
        dZT[(size_t)c * B + r] = gb;
        acc += g;
    }
    dbpart[blockIdx.x * kHid + c] = acc;   // summed in block order by k_sum_parts
}

// out[e] = sum over p of parts[p * n + e], p in increasing order
__global__ void k_sum_parts(const float* __restrict__ parts, int nparts, long long n, float* __restrict__ out) {
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        float s = 0.0f;
        for (int q = 0; q < nparts; ++q) s += parts[(size_t)q * n + e];
        out[e] = s;
    }
}

__global__ void k_w3_grad(const float* __restrict__ dW3T, float* __restrict__ G) {   // [256][16] -> W3 [3][256]
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < 3 * kHid) G[kW3 + t] = dW3T[(t % kHid) * kOut3 + t / kHid];
}

// Adam (beta 0.9 / 0.999, eps 1e-8) on the f32 masters; the step counter lives on the device
__global__ void k_adam(float* __restrict__ P, const float* __restrict__ G, float* __restrict__ M, float* __restrict__ Vv,
                       const long long* __restrict__ step, float lr) {
    const long long t = *step + 1;
    const float c1 = 1.0f - powf(0.9f, (float)t), c2 = 1.0f - powf(0.999f, (float)t);
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < kParams; e += (long long)gridDim.x * blockDim.x) {
        const float g = G[e];
        const float m = 0.9f * M[e] + 0.1f * g;
        const float v = 0.999f * Vv[e] + 0.001f * g * g;
        M[e] = m;
        Vv[e] = v;
        P[e] -= lr * (m / c1) / (sqrtf(v / c2) + 1e-8f);
    }
}

__global__ void k_step_inc(long long* step) { ++*step; }

// ---------------------------------------------------------------- features
// bounding box of the points: lo (3), hi (3); finite coordinates only.  Block partials are merged
// with integer atomics on the order-preserving encoding of floats (exact, order independent).
__device__ __forceinline__ unsigned fkey(float x) {
    const unsigned u = __float_as_uint(x);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float fval(unsigned k) { return __uint_as_float((k & 0x80000000u) ? (k & 0x7fffffffu) : ~k); }

__global__ void k_bbox_init(unsigned* keys) {
    if (threadIdx.x < 6) keys[threadIdx.x] = threadIdx.x < 3 ? 0xffffffffu : 0u;
}

__global__ void k_bbox(const float* __restrict__ pts, int N, unsigned* keys) {
    float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x)
        for (int q = 0; q < 3; ++q) {
            const float v = pts[3 * i + q];
            if (isfinite(v)) {
                lo[q] = fminf(lo[q], v);
                hi[q] = fmaxf(hi[q], v);
            }
        }
    for (int q = 0; q < 3; ++q)
        for (int o = 16; o > 0; o >>= 1) {
            lo[q] = fminf(lo[q], __shfl_xor_sync(0xffffffffu, lo[q], o));
            hi[q] = fmaxf(hi[q], __shfl_xor_sync(0xffffffffu, hi[q], o));
        }
    if ((threadIdx.x & 31) == 0)
        for (int q = 0; q < 3; ++q) {
            if (lo[q] <= hi[q]) {
                atomicMin(keys + q, fkey(lo[q]));
                atomicMax(keys + 3 + q, fkey(hi[q]));
            }
        }
}

__global__ void k_bbox_final(const unsigned* keys, float* box) {
    if (threadIdx.x < 6) box[threadIdx.x] = fval(keys[threadIdx.x]);
}

}  // namespace

long long hf_mlp_param_count() { return kParams; }

cudaError_t hf_launch_init(float* P, uint64_t seed, cudaStream_t s) {
    k_init<<<128, 256, 0, s>>>(P, seed);
    return cudaGetLastError();
}

cudaError_t hf_launch_pack(const float* P, const MlpDev& d, cudaStream_t s) {
    k_pack<<<(kHid * kHid + 255) / 256, 256, 0, s>>>(P, d);
    return cudaGetLastError();
}

cudaError_t hf_launch_bbox_init(unsigned* keys, cudaStream_t s) {
    k_bbox_init<<<1, 32, 0, s>>>(keys);
    return cudaGetLastError();
}

cudaError_t hf_launch_bbox(const float* pts, int N, float* box, cudaStream_t s) {
    unsigned* keys = reinterpret_cast<unsigned*>(box + 8);   // 6 keys after the 6 (+2 spare) box floats
    k_bbox_init<<<1, 32, 0, s>>>(keys);
    k_bbox<<<296, 256, 0, s>>>(pts, N, keys);
    k_bbox_final<<<1, 32, 0, s>>>(keys, box);
    return cudaGetLastError();
}

// One training step on the device (no host synchronisation, capturable in a CUDA graph).
cudaError_t hf_train_step(const MlpTrain& t, cudaStream_t s) {
    const MlpDev& d = t.d;
    const int B = t.B;
    cudaError_t e = cudaSuccess;
    k_gather<<<(B + 127) / 128, 128, 0, s>>>(t.X, t.T, t.n_samples, B, t.seed, t.step, d);
    GemmArgs g{};
    g.errw = t.errw;
    // forward
    g.M = B; g.N = kHid; g.K = kIn; g.kchunks_per_split = 1; g.bias = t.P + kB1;
    g.Z = d.Z1; g.ldz = kHid; g.H = d.H1; g.ldh = kHid; g.HT = d.H1T; g.ldht = B;
    if ((e = hf_gemm_tn(EPI_GELU_TRAIN, 256, t.tm[TM_X], t.tm[TM_W1], g, 1, s))) return e;
    g.K = kHid; g.kchunks_per_split = kHid / 64; g.bias = t.P + kB2;
    g.Z = d.Z2; g.H = d.H2; g.HT = d.H2T;
    if ((e = hf_gemm_tn(EPI_GELU_TRAIN, 256, t.tm[TM_H1], t.tm[TM_W2], g, 1, s))) return e;
    GemmArgs g3{};
    g3.errw = t.errw; g3.M = B; g3.N = kOut3; g3.K = kHid; g3.kchunks_per_split = kHid / 64; g3.C = d.Z3; g3.ldc = kOut3;
    g3.bias = d.b3p;
    if ((e = hf_gemm_tn(EPI_STORE, 16, t.tm[TM_H2], t.tm[TM_W3P], g3, 1, s))) return e;
    const int lb = (B + 255) / 256;
    k_loss<<<lb, 256, 0, s>>>(B, d);
    k_loss_sum<<<1, 32, 0, s>>>(lb, d, t.G, t.step, t.loss_hist);
    // backward: weight gradients as split-K sums over the batch (at most 64 splits), partial tiles
    // summed in a fixed order so that training is bitwise reproducible
    const int kc = B / 64, per = (kc + 63) / 64, splits = (kc + per - 1) / per;
    const int gb = (B + 31) / 32;   // blocks of k_gelu_back
    auto reduce = [&](long long n, float* out) {
        k_sum_parts<<<(unsigned)((n + 255) / 256 < 1184 ? (n + 255) / 256 : 1184), 256, 0, s>>>(d.parts, splits, n, out);
    };
    GemmArgs w{};
    w.errw = t.errw; w.M = kHid; w.K = B; w.kchunks_per_split = per; w.C = d.parts;
    w.N = kOut3; w.ldc = kOut3; w.split_stride = (long long)kHid * kOut3;
    if ((e = hf_gemm_tn(EPI_PARTIAL, 16, t.tm[TM_H2T], t.tm[TM_DZ3T], w, splits, s))) return e;
    reduce((long long)kHid * kOut3, d.dW3T);
    GemmArgs h{};
    h.errw = t.errw; h.M = B; h.N = kHid; h.K = 64; h.kchunks_per_split = 1; h.C = d.dH; h.ldc = kHid;
    if ((e = hf_gemm_tn(EPI_STORE, 256, t.tm[TM_DZ3], t.tm[TM_W3T], h, 1, s))) return e;
    k_gelu_back<<<gb, kHid, 0, s>>>(B, d.dH, d.Z2, d.dZ2, d.dZ2T, d.bparts);
    k_sum_parts<<<1, kHid, 0, s>>>(d.bparts, gb, kHid, t.G + kB2);
    w.N = kHid; w.ldc = kHid; w.split_stride = (long long)kHid * kHid;
    if ((e = hf_gemm_tn(EPI_PARTIAL, 256, t.tm[TM_DZ2T], t.tm[TM_H1T], w, splits, s))) return e;
    reduce((long long)kHid * kHid, t.G + kW2);
    h.K = kHid; h.kchunks_per_split = kHid / 64;
    if ((e = hf_gemm_tn(EPI_STORE, 256, t.tm[TM_DZ2], t.tm[TM_W2T], h, 1, s))) return e;
    k_gelu_back<<<gb, kHid, 0, s>>>(B, d.dH, d.Z1, d.dZ1, d.dZ1T, d.bparts);
    k_sum_parts<<<1, kHid, 0, s>>>(d.bparts, gb, kHid, t.G + kB1);
    w.N = kIn; w.ldc = kIn; w.split_stride = (long long)kHid * kIn;
    if ((e = hf_gemm_tn(EPI_PARTIAL, 64, t.tm[TM_DZ1T], t.tm[TM_XT], w, splits, s))) return e;
    reduce((long long)kHid * kIn, t.G + kW1);
    k_w3_grad<<<(3 * kHid + 255) / 256, 256, 0, s>>>(d.dW3T, t.G);
    if (t.lr > 0.0f) {
        k_adam<<<256, 256, 0, s>>>(t.P, t.G, t.M, t.V, t.step, t.lr);
        if ((e = hf_launch_pack(t.P, d, s))) return e;
    }
    k_step_inc<<<1, 1, 0, s>>>(t.step);
    return cudaGetLastError();
}

// Inference: x [n x 64] bf16 -> directions [n x 3], the whole network in one kernel.
cudaError_t hf_mlp_infer(const MlpDev& d, const float* P, const uint16_t* x, int n, float* dir_out, uint32_t* errw,
                         cudaStream_t s, bool raw, unsigned long long wait_ns) {
    CUtensorMap tx, tw1, tw2;
    cudaError_t e = hf_make_tmap_bf16(&tx, x, n, kIn, 128);
    if (e == cudaSuccess) e = hf_make_tmap_bf16(&tw1, d.W1b, kHid, kIn, 256);
    if (e == cudaSuccess) e = hf_make_tmap_bf16(&tw2, d.W2b, kHid, kHid, 256);
    if (e != cudaSuccess) return e;
    GemmArgs g{};
    g.errw = errw; g.M = n; g.N = kHid; g.K = kIn; g.bias = P + kB1;
    g.w3 = d.w3f; g.b3 = P + kB3; g.dir_out = dir_out; g.head_raw = raw ? 1 : 0; g.wait_ns = wait_ns;
    return hf_mlp_fused(tx, tw1, tw2, g, P + kB2, s);
}
