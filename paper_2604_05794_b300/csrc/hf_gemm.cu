// hf_gemm.cu - the tensor-core GEMM of the learned proposal network (BF16 operands, FP32 accumulate
// in tensor memory), for sm_100-family GPUs.
//
//   C[M x N] = A[M x K] . B[N x K]^T      A, B row-major bf16 ("TN"), K a multiple of 64
//
// One CTA of 256 threads computes a 128 x BN tile: thread 0 keeps a ring of up to three 128 x 64
// and BN x 64 operand tiles filled by TMA (128-byte swizzle) and issues tcgen05.mma (K = 16 per
// instruction) into a TMEM accumulator of BN columns; the eight warps then read the TMEM lanes of
// their quarter (rows) and half of the columns back with tcgen05.ld and run the epilogue, storing
// 16-byte row pieces.  gridDim.z splits K (partial tiles, or partial sums added
// atomically).  Every mbarrier wait is bounded; on expiry the CTA records HF_DEV_ERR_TIMEOUT,
// drains its outstanding copies (bounded as well), frees its TMEM and writes nothing.
#include <cudaTypedefs.h>
#include <cuda_bf16.h>

#include <mutex>

#include "hf_gemm.cuh"
#include "hf_internal.cuh"
#include <algorithm>

#include "hf_tc.cuh"

using namespace hf_tc;

namespace {

constexpr int kMaxStages = 3;   // ring depth: min(3, K chunks per CTA), set at launch
constexpr uint32_t kATileBytes = 128 * 128;   // 128 rows x 64 bf16

__device__ __forceinline__ float gelu_erf(float x) { return 0.5f * x * (1.0f + erff(x * 0.70710678118654752f)); }

// FP32 pairs: packed fma / mul / add (each lane rounded like the scalar instruction).
typedef unsigned long long g2_t;
__device__ __forceinline__ g2_t g2(float a, float b) {
    g2_t r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ void g2u(g2_t r, float& a, float& b) { asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(r)); }
__device__ __forceinline__ g2_t g2fma(g2_t a, g2_t b, g2_t c) {
    g2_t d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
__device__ __forceinline__ g2_t g2mul(g2_t a, g2_t b) {
    g2_t d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ g2_t g2add(g2_t a, g2_t b) {
    g2_t d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ g2_t g2s(float a) { return g2(a, a); }
__device__ __forceinline__ float fma_sat(float a, float b, float c) {   // clamped to [0, 1]
    float d;
    asm("fma.rn.sat.f32 %0, %1, %2, %3;" : "=f"(d) : "f"(a), "f"(b), "f"(c));
    return d;
}

// GELU of the inference epilogues: x Phi(x), Phi the standard normal CDF, from a polynomial on the
// clamped input.  t = sat(x / 10 + 1/2) clamps x to [-5, 5] (1 - Phi(5) = 2.9e-7), w8 = 8 t - 4
// (= 4 x / 5 there), q = w8^2 - 8 in [-8, 8], Phi = 1/2 + w8 R(q) with R of degree 12, fitted by
// gen_gelu_poly.py (Lawson's reweighted least squares, coefficients rounded to FP32).  For every
// FP32 x, |gelu_poly(x) - x Phi(x)| <= 4.1e-7 |x| (the generator's FP32 emulation of this exact
// sequence over a dense sweep, against FP64 erf): far below the bf16 rounding that follows (relative spacing
// 3.9e-3).  Fused multiply-adds only, no special-function unit; two values per packed instruction.
__device__ constexpr float kGeluC[13] = {
    1.767047942e-01f,  -1.098382473e-02f, 1.006262843e-03f,  -9.872522060e-05f, 9.593048162e-06f,
    -8.886037790e-07f, 7.842153593e-08f,  -6.620918480e-09f, 4.703698542e-10f,  -2.552603615e-11f,
    2.115369728e-12f,  -2.318493704e-13f, 1.046213846e-14f};
__device__ __forceinline__ g2_t gelu_poly2(g2_t X) {
    float xa, xb;
    g2u(X, xa, xb);
    const g2_t T = g2(fma_sat(xa, 0.1f, 0.5f), fma_sat(xb, 0.1f, 0.5f));
    const g2_t W = g2fma(T, g2s(8.0f), g2s(-4.0f));
    const g2_t Q = g2fma(W, W, g2s(-8.0f));
    g2_t R = g2fma(g2s(kGeluC[12]), Q, g2s(kGeluC[11]));
#pragma unroll
    for (int j = 10; j >= 0; --j) R = g2fma(R, Q, g2s(kGeluC[j]));
    return g2mul(X, g2fma(W, R, g2s(0.5f)));
}
__device__ __forceinline__ float gelu_poly(float x) {
    float a, b;
    g2u(gelu_poly2(g2(x, x)), a, b);
    return a;
}
// two FP32 values rounded to bf16 (RNE) and packed, the first in the low half
__device__ __forceinline__ uint32_t bf16x2_bits(float lo, float hi) {
    uint32_t d;
    asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(d) : "f"(hi), "f"(lo));
    return d;
}
__device__ __forceinline__ uint16_t bf16_bits(float x) { return __bfloat16_as_ushort(__float2bfloat16_rn(x)); }
__device__ __forceinline__ float bf16_round(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }

__device__ __forceinline__ void st_f32x16(float* dst, const float* v, bool vec) {
    if (vec) {
        float4* d4 = reinterpret_cast<float4*>(dst);
#pragma unroll
        for (int q = 0; q < 4; ++q) d4[q] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
    } else {
#pragma unroll
        for (int q = 0; q < 16; ++q) dst[q] = v[q];
    }
}

__device__ __forceinline__ void st_bf16x16(uint16_t* dst, const uint16_t* h, bool vec) {
    if (vec) {
        uint32_t w[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) w[q] = (uint32_t)h[2 * q] | ((uint32_t)h[2 * q + 1] << 16);
        uint4* d4 = reinterpret_cast<uint4*>(dst);
        d4[0] = make_uint4(w[0], w[1], w[2], w[3]);
        d4[1] = make_uint4(w[4], w[5], w[6], w[7]);
    } else {
#pragma unroll
        for (int q = 0; q < 16; ++q) dst[q] = h[q];
    }
}

__device__ __forceinline__ void st_bf16x16w(uint16_t* dst, const uint32_t* w, bool vec) {
    if (vec) {
        uint4* d4 = reinterpret_cast<uint4*>(dst);
        d4[0] = make_uint4(w[0], w[1], w[2], w[3]);
        d4[1] = make_uint4(w[4], w[5], w[6], w[7]);
    } else {
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            dst[2 * q] = (uint16_t)(w[q] & 0xffffu);
            dst[2 * q + 1] = (uint16_t)(w[q] >> 16);
        }
    }
}

template <int BN>
__host__ __device__ constexpr uint32_t tmem_cols() {
    return BN <= 32 ? 32 : BN;
}

template <int BN, int EPI>
__global__ void __launch_bounds__(256) k_gemm_tn(const __grid_constant__ CUtensorMap ta,
                                                 const __grid_constant__ CUtensorMap tb, GemmArgs g) {
    constexpr uint32_t kBTileBytes = BN * 128;
    extern __shared__ unsigned char smem_raw[];
    const int kStages = g.stages;
    unsigned char* base = smem_raw + ((1024 - (saddr(smem_raw) & 1023)) & 1023);
    unsigned char* sA = base;
    unsigned char* sB = base + kStages * kATileBytes;
    uint64_t* full = reinterpret_cast<uint64_t*>(sB + kStages * kBTileBytes);
    uint64_t* empty = full + kStages;
    uint64_t* done = empty + kStages;
    uint32_t* tslot = reinterpret_cast<uint32_t*>(done + 1);
    float* consts = reinterpret_cast<float*>(tslot + 4);   // bias [BN] (and W3 [3][256], b3 [3] for the head)

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int m0 = blockIdx.x * 128, n0 = blockIdx.y * BN;
    const int kc0 = blockIdx.z * g.kchunks_per_split;
    const int nk = min(g.kchunks_per_split, g.K / 64 - kc0);

    if (threadIdx.x == 0) {
        for (int s = 0; s < kStages; ++s) {
            mbar_init(full + s, 1);
            mbar_init(empty + s, 1);
        }
        mbar_init(done, 1);
        fence_mbar_init();
    }
    if (warp == 0) {
        tmem_alloc(tslot, tmem_cols<BN>());
        tmem_relinquish();
    }
    if (g.bias)
        for (int q = threadIdx.x; q < BN; q += blockDim.x) consts[q] = g.bias[n0 + q];
    if constexpr (EPI == EPI_HEAD)
        for (int q = threadIdx.x; q < 3 * 256 + 3; q += blockDim.x) consts[BN + q] = q < 768 ? g.w3[q] : g.b3[q - 768];
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = *tslot;

    __shared__ int s_ok;
    const uint64_t wait_ns = g.wait_ns ? g.wait_ns : kWaitTimeoutNs;
    if (threadIdx.x == 0) {
        bool ok = true;
        int issued = 0;   // chunks whose loads were issued
        const uint32_t idesc = idesc_bf16_f32(128, BN);
        for (; issued < kStages && issued < nk; ++issued) {
            mbar_expect_tx(full + issued, kATileBytes + kBTileBytes);
            tma_load_2d(sA + issued * kATileBytes, &ta, full + issued, (kc0 + issued) * 64, m0);
            tma_load_2d(sB + issued * kBTileBytes, &tb, full + issued, (kc0 + issued) * 64, n0);
        }
        int c = 0;
        for (; c < nk; ++c) {
            const int s = c % kStages;
            const uint32_t ph = (c / kStages) & 1;
            if (!mbar_wait(full + s, ph, wait_ns)) {
                ok = false;
                break;
            }
            fence_after();
            const uint32_t a0 = saddr(sA + s * kATileBytes), b0 = saddr(sB + s * kBTileBytes);
#pragma unroll
            for (int kk = 0; kk < 4; ++kk)
                mma_bf16(tmem, sdesc_sw128(a0 + kk * 32), sdesc_sw128(b0 + kk * 32), idesc, (c > 0 || kk > 0) ? 1u : 0u);
            mma_commit(empty + s);
            if (issued < nk) {
                // the stage is reused: wait until the MMAs that read it are done
                if (!mbar_wait(empty + s, ph, wait_ns)) {
                    ok = false;
                    ++c;
                    break;
                }
                mbar_expect_tx(full + s, kATileBytes + kBTileBytes);
                tma_load_2d(sA + s * kATileBytes, &ta, full + s, (kc0 + issued) * 64, m0);
                tma_load_2d(sB + s * kBTileBytes, &tb, full + s, (kc0 + issued) * 64, n0);
                ++issued;
            }
        }
        mma_commit(done);
        if (!ok) {
            // drain the copies still in flight (bounded) before the CTA can exit
            for (int q = c; q < issued; ++q) mbar_wait(full + (q % kStages), (q / kStages) & 1, kWaitTimeoutNs);
            atomicOr(g.errw, HF_DEV_ERR_TIMEOUT);
        }
        s_ok = ok ? 1 : 0;
    }
    __syncthreads();
    bool ok = s_ok != 0;
    if (!mbar_wait(done, 0, wait_ns)) {
        ok = false;
        if (lane == 0) atomicOr(g.errw, HF_DEV_ERR_TIMEOUT);
        // the committed MMAs complete by themselves: wait for them (bounded) before the tensor
        // memory they write is released
        mbar_wait(done, 0, kWaitTimeoutNs);
    }
    fence_after();

    // eight warps: warp w reads TMEM lane quarter (w & 3), i.e. rows, and column half (w >> 2)
    const int quarter = warp & 3, half = warp >> 2;
    const int lrow = quarter * 32 + lane;
    const int row = m0 + lrow;
    const bool wr = ok && row < g.M;
    const uint32_t tl = tmem + ((uint32_t)(quarter * 32) << 16);
    constexpr int kCols = BN >= 32 ? BN / 2 : BN;   // columns per warp
    const int cbeg = BN >= 32 ? half * kCols : 0;
    const bool active = BN >= 32 || half == 0;
    bool vec = false;   // 16-byte row stores when the destination allows them
    if constexpr (EPI == EPI_STORE || EPI == EPI_PARTIAL)
        vec = ((reinterpret_cast<uintptr_t>(g.C) & 15) == 0) && (g.ldc & 3) == 0 && (g.split_stride & 3) == 0;
    if constexpr (EPI == EPI_GELU)
        vec = ((reinterpret_cast<uintptr_t>(g.H) & 15) == 0) && (g.ldh & 7) == 0;
    if constexpr (EPI == EPI_GELU_TRAIN)
        vec = ((reinterpret_cast<uintptr_t>(g.H) & 15) == 0) && (g.ldh & 7) == 0 &&
              ((reinterpret_cast<uintptr_t>(g.Z) & 15) == 0) && (g.ldz & 3) == 0;
    float y0 = 0.0f, y1 = 0.0f, y2 = 0.0f;   // EPI_HEAD accumulators
    if (active) {
#pragma unroll 1
        for (int c0 = cbeg; c0 < cbeg + kCols; c0 += 16) {
            float v[16];
            tmem_ld16(tl + c0, v);   // all lanes, unconditionally (warp-collective)
            if (!wr) continue;
            const int n = n0 + c0;
            if constexpr (EPI == EPI_STORE) {
#pragma unroll
                for (int q = 0; q < 16; ++q) v[q] += g.bias ? consts[c0 + q] : 0.0f;
                st_f32x16(g.C + (size_t)row * g.ldc + n, v, vec);
            } else if constexpr (EPI == EPI_ATOMIC) {
                const bool add_bias = g.bias && blockIdx.z == 0;
#pragma unroll
                for (int q = 0; q < 16; ++q)
                    atomicAdd(g.C + (size_t)row * g.ldc + n + q, v[q] + (add_bias ? g.bias[n + q] : 0.0f));
            } else if constexpr (EPI == EPI_PARTIAL) {
                st_f32x16(g.C + (size_t)blockIdx.z * g.split_stride + (size_t)row * g.ldc + n, v, vec);
            } else if constexpr (EPI == EPI_GELU_TRAIN) {
                uint16_t h[16];
#pragma unroll
                for (int q = 0; q < 16; ++q) {
                    v[q] += consts[c0 + q];
                    h[q] = bf16_bits(gelu_erf(v[q]));
                    g.HT[(size_t)(n + q) * g.ldht + row] = h[q];
                }
                st_f32x16(g.Z + (size_t)row * g.ldz + n, v, vec);
                st_bf16x16(g.H + (size_t)row * g.ldh + n, h, vec);
            } else if constexpr (EPI == EPI_GELU) {
                uint16_t h[16];
#pragma unroll
                for (int q = 0; q < 16; ++q) h[q] = bf16_bits(gelu_poly(v[q] + consts[c0 + q]));
                st_bf16x16(g.H + (size_t)row * g.ldh + n, h, vec);
            } else {   // EPI_HEAD: h2 = bf16(gelu(z2)), y = W3 h2 (FP32, in column order within each half)
#pragma unroll
                for (int q = 0; q < 16; ++q) {
                    const float h = bf16_round(gelu_poly(v[q] + consts[c0 + q]));
                    y0 = fmaf(consts[BN + n + q], h, y0);
                    y1 = fmaf(consts[BN + 256 + n + q], h, y1);
                    y2 = fmaf(consts[BN + 512 + n + q], h, y2);
                }
            }
        }
    }
    if constexpr (EPI == EPI_HEAD) {
        // the second column half hands its partial sums to the first through shared memory
        float* part = consts + BN + 3 * 256 + 4;
        if (half == 1) {
            part[3 * lrow] = y0;
            part[3 * lrow + 1] = y1;
            part[3 * lrow + 2] = y2;
        }
        __syncthreads();
        if (half == 0 && wr) {
            y0 += part[3 * lrow] + consts[BN + 768];
            y1 += part[3 * lrow + 1] + consts[BN + 769];
            y2 += part[3 * lrow + 2] + consts[BN + 770];
            const float nn = sqrtf(y0 * y0 + y1 * y1 + y2 * y2);
            float d0 = 0.0f, d1 = 0.0f, d2 = 1.0f;
            if (g.head_raw) {
                d0 = y0;
                d1 = y1;
                d2 = y2;
            } else if (nn > 0.0f) {
                d0 = y0 / nn;
                d1 = y1 / nn;
                d2 = y2 / nn;
            }
            g.dir_out[3 * (size_t)row] = d0;
            g.dir_out[3 * (size_t)row + 1] = d1;
            g.dir_out[3 * (size_t)row + 2] = d2;
        }
    }
    fence_before();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, tmem_cols<BN>());
}

// ---------------------------------------------------------------- persistent inference GEMM
// C = A . B^T with N = 256 and K <= 256 for the proposal network's inference (EPI_GELU, EPI_HEAD):
// one CTA per SM walks the 128-row tiles blockIdx.x, blockIdx.x + gridDim.x, ...  B (the layer's
// weights, K/64 chunks of 256 x 64) stays in shared memory; A streams through a three-stage TMA
// ring; the accumulator is double-buffered in tensor memory (2 x 256 columns), so the MMAs of the
// next tile run while the epilogue drains the previous one.  Warp 16 (one thread) issues the TMA
// loads and the MMAs; warps 0-7 drain the even tiles (buffer 0), warps 8-15 the odd ones (buffer
// 1): warp w reads TMEM lane quarter w % 4 (rows) and column half (w / 4) % 2.  For the head, the
// second column half hands its partial 256->3 sums to the first through shared memory (two
// mbarriers per group).  All waits are bounded; on expiry the CTA records HF_DEV_ERR_TIMEOUT and
// winds down.
constexpr int kPStages = 3;
constexpr int kPThreads = 17 * 32;
constexpr uint32_t kPBChunk = 256 * 128;   // 256 rows x 64 bf16

template <int EPI>
__global__ void __launch_bounds__(kPThreads, 1) k_gemm_persist(const __grid_constant__ CUtensorMap ta,
                                                               const __grid_constant__ CUtensorMap tb, GemmArgs g) {
    extern __shared__ unsigned char smem_raw[];
    const int nk = g.K / 64;
    unsigned char* base = smem_raw + ((1024 - (saddr(smem_raw) & 1023)) & 1023);
    unsigned char* sB = base;                                  // nk x 32 KB
    unsigned char* sA = sB + nk * kPBChunk;                     // kPStages x 16 KB
    uint64_t* afull = reinterpret_cast<uint64_t*>(sA + kPStages * kATileBytes);
    uint64_t* aempty = afull + kPStages;
    uint64_t* bfull = aempty + kPStages;
    uint64_t* accf = bfull + 1;    // [2] MMA -> epilogue group
    uint64_t* acce = accf + 2;     // [2] epilogue group (8 warps) -> MMA
    uint64_t* hbar = acce + 2;     // [2] head: second column half wrote its partial sums (4 warps)
    uint64_t* hfree = hbar + 2;    // [2] head: first column half read them (4 warps)
    uint64_t* done = hfree + 2;
    uint32_t* tslot = reinterpret_cast<uint32_t*>(done + 1);
    float* consts = reinterpret_cast<float*>(tslot + 4);   // bias [256] (and W3 [3][256], b3 [3] for the head)
    float* part = consts + 256 + 3 * 256 + 4;              // head: [2 groups][128 rows][3]

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int tiles = (g.M + 127) / 128;
    if (threadIdx.x == 0) {
        for (int s = 0; s < kPStages; ++s) {
            mbar_init(afull + s, 1);
            mbar_init(aempty + s, 1);
        }
        mbar_init(bfull, 1);
        for (int b = 0; b < 2; ++b) {
            mbar_init(accf + b, 1);
            mbar_init(acce + b, 8);
            mbar_init(hbar + b, 4);
            mbar_init(hfree + b, 4);
        }
        mbar_init(done, 1);
        fence_mbar_init();
    }
    if (warp == 0) {
        tmem_alloc(tslot, 512);
        tmem_relinquish();
    }
    for (int q = threadIdx.x; q < 256; q += blockDim.x) consts[q] = g.bias ? g.bias[q] : 0.0f;
    if constexpr (EPI == EPI_HEAD)
        for (int q = threadIdx.x; q < 3 * 256 + 3; q += blockDim.x) consts[256 + q] = q < 768 ? g.w3[q] : g.b3[q - 768];
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = *tslot;

    if (warp == 16) {
        // The whole warp runs the producer / MMA loop (its values stay warp-uniform); the elected
        // lane issues the copies and the MMAs, and lane 0's verdict on each wait holds for all.  A
        // loop run by one lane alone issues several times slower while the epilogue warps compute.
        auto agree = [](bool x) { return __shfl_sync(0xffffffffu, x ? 1 : 0, 0) != 0; };
        bool ok = true;
        const uint32_t idesc = idesc_bf16_f32(128, 256);
        const int my_tiles = blockIdx.x < tiles ? (tiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;
        const long long total = (long long)my_tiles * nk;
        long long g_load = 0, g_use = 0;
        // the weights, once
        if (elect_one()) {
            mbar_expect_tx(bfull, nk * kPBChunk);
            for (int c = 0; c < nk; ++c) tma_load_2d(sB + c * kPBChunk, &tb, bfull, c * 64, 0);
        }
        __syncwarp();
        auto top_up = [&]() -> bool {   // keep up to kPStages A chunks in flight
            while (g_load < total && g_load < g_use + kPStages) {
                const int s = (int)(g_load % kPStages);
                if (!agree(mbar_wait(aempty + s, (uint32_t)(((g_load / kPStages) & 1) ^ 1), kWaitTimeoutNs))) return false;
                const int t = blockIdx.x + (int)(g_load / nk) * gridDim.x, c = (int)(g_load % nk);
                if (elect_one()) {
                    mbar_expect_tx(afull + s, kATileBytes);
                    tma_load_2d(sA + s * kATileBytes, &ta, afull + s, c * 64, t * 128);
                }
                __syncwarp();
                ++g_load;
            }
            return true;
        };
        ok = top_up() && agree(mbar_wait(bfull, 0, kWaitTimeoutNs));
        int lt = 0;
        for (int t = blockIdx.x; ok && t < tiles; t += gridDim.x, ++lt) {
            const int b = lt & 1;
            if (!agree(mbar_wait(acce + b, (uint32_t)(((lt >> 1) & 1) ^ 1), kWaitTimeoutNs))) {
                ok = false;
                break;
            }
            fence_after();
            for (int c = 0; c < nk; ++c) {
                if (!top_up()) {
                    ok = false;
                    break;
                }
                const int s = (int)(g_use % kPStages);
                if (!agree(mbar_wait(afull + s, (uint32_t)((g_use / kPStages) & 1), kWaitTimeoutNs))) {
                    ok = false;
                    break;
                }
                fence_after();
                const uint32_t a0 = saddr(sA + s * kATileBytes), b0 = saddr(sB + c * kPBChunk);
                if (elect_one()) {
#pragma unroll
                    for (int kk = 0; kk < 4; ++kk)
                        mma_bf16(tmem + b * 256, sdesc_sw128(a0 + kk * 32), sdesc_sw128(b0 + kk * 32), idesc,
                                 (c > 0 || kk > 0) ? 1u : 0u);
                    mma_commit(aempty + s);
                }
                __syncwarp();
                ++g_use;
            }
            if (!ok) break;
            if (elect_one()) mma_commit(accf + b);
            __syncwarp();
        }
        // wind down: every issued MMA complete, every issued copy landed (bounded)
        if (elect_one()) mma_commit(done);
        __syncwarp();
        mbar_wait(done, 0, kWaitTimeoutNs);
        for (long long q = g_use; q < g_load; ++q)
            mbar_wait(afull + (int)(q % kPStages), (uint32_t)((q / kPStages) & 1), kWaitTimeoutNs);
        if (!ok && lane == 0) atomicOr(g.errw, HF_DEV_ERR_TIMEOUT);
    } else {
        const int grp = warp >> 3, quarter = warp & 3, half = (warp >> 2) & 1;
        const int lrow = quarter * 32 + lane;
        const uint32_t tl = tmem + (uint32_t)grp * 256 + ((uint32_t)(quarter * 32) << 16) + (uint32_t)half * 128;
        const bool vec = ((reinterpret_cast<uintptr_t>(g.H) & 15) == 0) && (g.ldh & 7) == 0;
        float* pg = part + grp * 128 * 3;
        int k = 0;   // this group's tile count
        for (int t = blockIdx.x + grp * gridDim.x; t < tiles; t += 2 * gridDim.x, ++k) {
            if (!mbar_wait(accf + grp, (uint32_t)(k & 1), kWaitTimeoutNs)) {
                if (lane == 0) atomicOr(g.errw, HF_DEV_ERR_TIMEOUT);
                break;
            }
            fence_after();
            const int row = t * 128 + lrow;
            const bool wr = row < g.M;
            const int cbase = half * 128;
            g2_t Y0 = g2s(0.0f), Y1 = g2s(0.0f), Y2 = g2s(0.0f);
            // the next 16 columns are in flight from tensor memory while these are processed
            uint32_t nxt[16];
            tmem_ld16_issue(tl, nxt);
            tmem_ld_wait(nxt);
#pragma unroll 2
            for (int c0 = 0; c0 < 128; c0 += 16) {
                float v[16];
#pragma unroll
                for (int q = 0; q < 16; ++q) v[q] = __uint_as_float(nxt[q]);
                if (c0 + 16 < 128) tmem_ld16_issue(tl + c0 + 16, nxt);
                const int n = cbase + c0;
                if constexpr (EPI == EPI_GELU) {
                    uint32_t w[8];
#pragma unroll
                    for (int q = 0; q < 16; q += 2) {
                        const float2 b = *reinterpret_cast<const float2*>(consts + n + q);
                        float ga, gb;
                        g2u(gelu_poly2(g2add(g2(v[q], v[q + 1]), g2(b.x, b.y))), ga, gb);
                        w[q >> 1] = bf16x2_bits(ga, gb);
                    }
                    if (wr) st_bf16x16w(g.H + (size_t)row * g.ldh + n, w, vec);
                } else {
                    // packed partial sums over the even and the odd columns
#pragma unroll
                    for (int q = 0; q < 16; q += 2) {
                        const float2 b = *reinterpret_cast<const float2*>(consts + n + q);
                        float ga, gb;
                        g2u(gelu_poly2(g2add(g2(v[q], v[q + 1]), g2(b.x, b.y))), ga, gb);
                        const uint32_t hb = bf16x2_bits(ga, gb);
                        const g2_t H = g2(__uint_as_float(hb << 16), __uint_as_float(hb & 0xffff0000u));
                        const float2 w0 = *reinterpret_cast<const float2*>(consts + 256 + n + q);
                        const float2 w1 = *reinterpret_cast<const float2*>(consts + 512 + n + q);
                        const float2 w2 = *reinterpret_cast<const float2*>(consts + 768 + n + q);
                        Y0 = g2fma(g2(w0.x, w0.y), H, Y0);
                        Y1 = g2fma(g2(w1.x, w1.y), H, Y1);
                        Y2 = g2fma(g2(w2.x, w2.y), H, Y2);
                    }
                }
                if (c0 + 16 < 128) tmem_ld_wait(nxt);
            }
            // the buffer is drained: the MMAs of a later tile may overwrite it
            fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(acce + grp);
            if constexpr (EPI == EPI_HEAD) {
                float y0, y1, y2, o0, o1, o2;
                g2u(Y0, y0, o0);
                g2u(Y1, y1, o1);
                g2u(Y2, y2, o2);
                y0 += o0;
                y1 += o1;
                y2 += o2;
                if (half == 1) {
                    // hand the partial sums over (once the first half has read the previous ones)
                    if (!mbar_wait(hfree + grp, (uint32_t)((k & 1) ^ 1), kWaitTimeoutNs)) {
                        if (lane == 0) atomicOr(g.errw, HF_DEV_ERR_TIMEOUT);
                        break;
                    }
                    pg[3 * lrow] = y0;
                    pg[3 * lrow + 1] = y1;
                    pg[3 * lrow + 2] = y2;
                    __syncwarp();
                    if (lane == 0) mbar_arrive(hbar + grp);
                } else {
                    if (!mbar_wait(hbar + grp, (uint32_t)(k & 1), kWaitTimeoutNs)) {
                        if (lane == 0) atomicOr(g.errw, HF_DEV_ERR_TIMEOUT);
                        break;
                    }
                    y0 += pg[3 * lrow] + consts[1024];
                    y1 += pg[3 * lrow + 1] + consts[1025];
                    y2 += pg[3 * lrow + 2] + consts[1026];
                    __syncwarp();
                    if (lane == 0) mbar_arrive(hfree + grp);
                    if (wr) {
                        const float nn = sqrtf(y0 * y0 + y1 * y1 + y2 * y2);
                        float d0 = 0.0f, d1 = 0.0f, d2 = 1.0f;
                        if (g.head_raw) {
                            d0 = y0;
                            d1 = y1;
                            d2 = y2;
                        } else if (nn > 0.0f) {
                            d0 = y0 / nn;
                            d1 = y1 / nn;
                            d2 = y2 / nn;
                        }
                        g.dir_out[3 * (size_t)row] = d0;
                        g.dir_out[3 * (size_t)row + 1] = d1;
                        g.dir_out[3 * (size_t)row + 2] = d2;
                    }
                }
            }
        }
    }
    fence_before();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, 512);
}

template <int EPI>
cudaError_t launch_persist(const CUtensorMap& ta, const CUtensorMap& tb, const GemmArgs& g, cudaStream_t s) {
    // at least 120 KB, so that one CTA holds an SM (it allocates all 512 tensor-memory columns)
    size_t smem = 1024 + (size_t)(g.K / 64) * kPBChunk + kPStages * kATileBytes + 256 +
                  (256 + 3 * 256 + 4 + 2 * 128 * 3) * 4;
    if (smem < 120 * 1024) smem = 120 * 1024;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaError_t e = cudaStreamIsCapturing(s, &cs);
    if (e == cudaSuccess && cs == cudaStreamCaptureStatusNone)
        e = cudaFuncSetAttribute(k_gemm_persist<EPI>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    static int sms = 0;
    if (!sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (sms <= 0) sms = 1;
    }
    const int tiles = (g.M + 127) / 128;
    k_gemm_persist<EPI><<<tiles < sms ? tiles : sms, kPThreads, smem, s>>>(ta, tb, g);
    return cudaGetLastError();
}

template <int BN, int EPI>
cudaError_t launch_bn_epi(const CUtensorMap& ta, const CUtensorMap& tb, const GemmArgs& g, int splits, cudaStream_t s) {
    const size_t smem = 1024 + (size_t)g.stages * (kATileBytes + BN * 128) + 256 + (BN + 3 * 256 + 4 + 3 * 128) * 4;
    // the attribute is set outside stream capture (an eager launch comes first)
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaError_t e = cudaStreamIsCapturing(s, &cs);
    if (e == cudaSuccess && cs == cudaStreamCaptureStatusNone)
        e = cudaFuncSetAttribute(k_gemm_tn<BN, EPI>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const dim3 grid((g.M + 127) / 128, g.N / BN, splits);
    k_gemm_tn<BN, EPI><<<grid, 256, smem, s>>>(ta, tb, g);
    return cudaGetLastError();
}

template <int EPI>
cudaError_t launch_epi(int bn, const CUtensorMap& ta, const CUtensorMap& tb, const GemmArgs& g, int splits, cudaStream_t s) {
    switch (bn) {
        case 16: return launch_bn_epi<16, EPI>(ta, tb, g, splits, s);
        case 64: return launch_bn_epi<64, EPI>(ta, tb, g, splits, s);
        case 128: return launch_bn_epi<128, EPI>(ta, tb, g, splits, s);
        default: return launch_bn_epi<256, EPI>(ta, tb, g, splits, s);
    }
}

PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;
std::once_flag g_encode_once;

}  // namespace

cudaError_t hf_make_tmap_bf16(CUtensorMap* map, const void* base, long long rows, long long cols, int box_rows) {
    std::call_once(g_encode_once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            g_encode = (PFN_cuTensorMapEncodeTiled_v12000)p;
    });
    if (!g_encode) return cudaErrorNotSupported;
    if (cols % 64 || ((uintptr_t)base & 15) || box_rows < 1 || box_rows > 256) return cudaErrorInvalidValue;
    const cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)cols * 2};
    const cuuint32_t box[2] = {64, (cuuint32_t)box_rows};
    const cuuint32_t estr[2] = {1, 1};
    CUresult r = g_encode(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box, estr,
                          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

cudaError_t hf_make_tmap_bf16_rows32(CUtensorMap* map, const void* base, long long rows, int box_rows) {
    std::call_once(g_encode_once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            g_encode = (PFN_cuTensorMapEncodeTiled_v12000)p;
    });
    if (!g_encode) return cudaErrorNotSupported;
    if (((uintptr_t)base & 15) || box_rows < 1 || box_rows > 256 || rows < 1) return cudaErrorInvalidValue;
    const cuuint64_t dims[2] = {16, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {32};
    const cuuint32_t box[2] = {16, (cuuint32_t)box_rows};
    const cuuint32_t estr[2] = {1, 1};
    CUresult r = g_encode(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box, estr,
                          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_32B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

cudaError_t hf_gemm_tn(int epi, int bn, const CUtensorMap& ta, const CUtensorMap& tb, const GemmArgs& g, int splits,
                       cudaStream_t s) {
    if (g.K % 64 || g.N % bn || g.kchunks_per_split < 1 || splits < 1) return cudaErrorInvalidValue;
    GemmArgs ga = g;
    // BN = 256 tiles keep two stages so that two CTAs fit on an SM
    const int max_stages = bn >= 256 ? 2 : kMaxStages;
    ga.stages = g.kchunks_per_split < max_stages ? g.kchunks_per_split : max_stages;
    switch (epi) {
        case EPI_STORE: return launch_epi<EPI_STORE>(bn, ta, tb, ga, splits, s);
        case EPI_ATOMIC: return launch_epi<EPI_ATOMIC>(bn, ta, tb, ga, splits, s);
        case EPI_GELU_TRAIN: return launch_epi<EPI_GELU_TRAIN>(bn, ta, tb, ga, splits, s);
        case EPI_GELU: return launch_epi<EPI_GELU>(bn, ta, tb, ga, splits, s);
        case EPI_PARTIAL: return launch_epi<EPI_PARTIAL>(bn, ta, tb, ga, splits, s);
        default: return launch_epi<EPI_HEAD>(bn, ta, tb, ga, splits, s);
    }
}

cudaError_t hf_gemm_persist(int epi, const CUtensorMap& ta, const CUtensorMap& tb, const GemmArgs& g, cudaStream_t s) {
    if (g.N != 256 || g.K % 64 || g.K < 64 || g.K > 256 || g.M < 1) return cudaErrorInvalidValue;
    return epi == EPI_HEAD ? launch_persist<EPI_HEAD>(ta, tb, g, s) : launch_persist<EPI_GELU>(ta, tb, g, s);
}

namespace {
int gemm_bf16(const uint16_t* A, const uint16_t* B, float* C, int M, int N, int K, unsigned long long wait_ns, void* stream) {
    if (!A || !B || !C || M < 1 || N < 16 || K < 64 || K % 64 || N % 16)
        return hf_set_err(nullptr, HF_ERR_INVALID_ARG, "need M >= 1, N a multiple of 16, K a multiple of 64");
    const int bn = N % 256 == 0 ? 256 : N % 128 == 0 ? 128 : N % 64 == 0 ? 64 : 16;
    CUtensorMap ta, tb;
    cudaError_t e = hf_make_tmap_bf16(&ta, A, M, K, 128);
    if (e == cudaSuccess) e = hf_make_tmap_bf16(&tb, B, N, K, bn);
    if (e != cudaSuccess) return hf_set_err(nullptr, HF_ERR_INVALID_ARG, "tensor map: %s", cudaGetErrorString(e));
    uint32_t* errw = nullptr;
    e = cudaMallocAsync((void**)&errw, sizeof(uint32_t), (cudaStream_t)stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(errw, 0, sizeof(uint32_t), (cudaStream_t)stream);
    GemmArgs g{};
    g.M = M;
    g.N = N;
    g.K = K;
    g.kchunks_per_split = K / 64;
    g.C = C;
    g.ldc = N;
    g.errw = errw;
    g.wait_ns = wait_ns;
    if (e == cudaSuccess) e = hf_gemm_tn(EPI_STORE, bn, ta, tb, g, 1, (cudaStream_t)stream);
    uint32_t host_err = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&host_err, errw, sizeof host_err, cudaMemcpyDeviceToHost, (cudaStream_t)stream);
    if (errw) cudaFreeAsync(errw, (cudaStream_t)stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize((cudaStream_t)stream);
    if (e != cudaSuccess) return hf_set_err(nullptr, HF_ERR_CUDA, "gemm: %s", cudaGetErrorString(e));
    if (host_err) return hf_set_err(nullptr, HF_ERR_TIMEOUT, "gemm: a bounded device wait expired");
    return HF_OK;
}
__global__ void k_gelu_eval(const float* __restrict__ x, float* __restrict__ y, long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        y[i] = gelu_poly(x[i]);
}
}  // namespace

extern "C" int hair_fuse_gelu_eval(const float* x, float* y, long long n, void* stream) {
    if (n < 0 || (n > 0 && (!x || !y))) return hf_set_err(nullptr, HF_ERR_INVALID_ARG, "need n >= 0 and device x, y");
    if (n == 0) return HF_OK;
    const long long blocks = std::min<long long>((n + 255) / 256, 148LL * 16);
    k_gelu_eval<<<(unsigned)blocks, 256, 0, (cudaStream_t)stream>>>(x, y, n);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return hf_set_err(nullptr, HF_ERR_CUDA, "gelu_eval: %s", cudaGetErrorString(e));
    return HF_OK;
}

extern "C" int hair_fuse_gemm_bf16(const uint16_t* A, const uint16_t* B, float* C, int M, int N, int K, void* stream) {
    return gemm_bf16(A, B, C, M, N, K, 0, stream);
}

extern "C" int hair_fuse_gemm_bf16_bounded(const uint16_t* A, const uint16_t* B, float* C, int M, int N, int K,
                                           unsigned long long wait_ns, void* stream) {
    return gemm_bf16(A, B, C, M, N, K, wait_ns, stream);
}
