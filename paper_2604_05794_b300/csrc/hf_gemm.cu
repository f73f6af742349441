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
    if constexpr (EPI == EPI_GELU_TRAIN)
        vec = ((reinterpret_cast<uintptr_t>(g.H) & 15) == 0) && (g.ldh & 7) == 0 &&
              ((reinterpret_cast<uintptr_t>(g.Z) & 15) == 0) && (g.ldz & 3) == 0;
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
            }
        }
    }
    fence_before();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, tmem_cols<BN>());
}

// ---------------------------------------------------------------- fused inference network
// The whole forward pass of the proposal network per 128-row tile in one persistent kernel: the
// hidden layer never leaves the SM.  Each layer runs as two N = 128 halves ("steps"), each into one
// of two 128-column tensor-memory accumulator regions (step s uses region s mod 2); the epilogue
// writes the bf16 layer-1 activations of tile t into activation region t mod 2 (columns 256..383
// or 384..511), from where layer 2 reads its A operand (tcgen05.mma with A in tensor memory).
// Steps are software-pipelined by one tile: layer 1 of tile t + 1, then layer 2 of tile t, so
// that while the epilogue drains step s the tensor cores already compute step s + 1 and no step
// waits on the activations it depends on.  Warp 16 loads (TMA: the weights once, the feature
// tiles through a two-stage ring) and issues the MMAs; warps 0-15 drain each step, warp w covering
// TMEM lanes 32 (w % 4) .. + 31 (rows) and the 32 columns 32 (w / 4) .. + 31 of the region.  The
// head (256 -> 3) sums in packed FP32 per warp; column groups 1..3 hand their partial sums to
// group 0 through shared memory.  All waits are bounded; on expiry the CTA records
// HF_DEV_ERR_TIMEOUT and winds down.
constexpr int kFXStages = 2;
constexpr int kFThreads = 17 * 32;
constexpr uint32_t kFW1Bytes = 256 * 128;        // 256 rows x 64 bf16
constexpr uint32_t kFW2Bytes = 4 * 256 * 128;    // 4 K chunks of 256 rows x 64 bf16
constexpr uint32_t kFHCol = 256;                 // tensor-memory columns of the activation regions
constexpr size_t kFSmemBytes = 1024 + kFW1Bytes + kFW2Bytes + kFXStages * kATileBytes + 256 +
                               (512 + 3 * 256 + 4) * 4 + 3 * 128 * 3 * 4;

__global__ void __launch_bounds__(kFThreads, 1) k_mlp_fused(const __grid_constant__ CUtensorMap tx,
                                                            const __grid_constant__ CUtensorMap tw1,
                                                            const __grid_constant__ CUtensorMap tw2, GemmArgs g,
                                                            const float* __restrict__ b2) {
    extern __shared__ unsigned char smem_raw[];
    unsigned char* base = smem_raw + ((1024 - (saddr(smem_raw) & 1023)) & 1023);
    unsigned char* sW1 = base;
    unsigned char* sW2 = sW1 + kFW1Bytes;
    unsigned char* sX = sW2 + kFW2Bytes;
    uint64_t* xfull = reinterpret_cast<uint64_t*>(sX + kFXStages * kATileBytes);
    uint64_t* xempty = xfull + kFXStages;
    uint64_t* wfull = xempty + kFXStages;
    uint64_t* accf = wfull + 1;    // [2] MMA step done -> epilogue
    uint64_t* acce = accf + 2;     // [2] region read (16 warps) -> MMA
    uint64_t* hfull = acce + 2;    // [2] a tile's layer-1 activations written (16 warps) -> MMA
    uint64_t* hbar = hfull + 2;    // head partial sums written (12 warps)
    uint64_t* hfree = hbar + 1;    // head partial sums read (4 warps)
    uint64_t* done = hfree + 1;
    uint64_t* never = done + 1;    // test mode: a barrier nothing completes
    uint32_t* tslot = reinterpret_cast<uint32_t*>(never + 1);
    float* consts = reinterpret_cast<float*>(base + kFW1Bytes + kFW2Bytes + kFXStages * kATileBytes + 256);
    float* cb1 = consts;              // [256]
    float* cb2 = consts + 256;        // [256]
    float* cw3 = consts + 512;        // [3][256], then b3 [3]
    float* part = consts + 512 + 3 * 256 + 4;   // [3 column groups][128 rows][3]

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int tiles = (g.M + 127) / 128;
    const int my_tiles = (int)blockIdx.x < tiles ? (tiles - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
    if (threadIdx.x == 0) {
        for (int q = 0; q < kFXStages; ++q) {
            mbar_init(xfull + q, 1);
            mbar_init(xempty + q, 1);
        }
        mbar_init(wfull, 1);
        for (int r = 0; r < 2; ++r) {
            mbar_init(accf + r, 1);
            mbar_init(acce + r, 16);
            mbar_init(hfull + r, 16);
        }
        mbar_init(hbar, 12);
        mbar_init(hfree, 4);
        mbar_init(done, 1);
        mbar_init(never, 1);
        fence_mbar_init();
    }
    if (warp == 0) {
        tmem_alloc(tslot, 512);
        tmem_relinquish();
    }
    for (int q = threadIdx.x; q < 256; q += blockDim.x) {
        cb1[q] = g.bias[q];
        cb2[q] = b2[q];
    }
    for (int q = threadIdx.x; q < 3 * 256 + 3; q += blockDim.x) cw3[q] = q < 768 ? g.w3[q] : g.b3[q - 768];
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = *tslot;
    // the pipeline's waits: the default limit, or the caller's (hinted, so that a short one expires
    // deterministically); the wind-down after an expiry always allows kWaitTimeoutNs
    const uint64_t wait_ns = g.wait_ns ? g.wait_ns : kWaitTimeoutNs;
    auto pwait = [&](uint64_t* b, uint32_t parity) -> bool {
        return g.wait_ns ? mbar_wait_hinted(b, parity, wait_ns) : mbar_wait(b, parity, kWaitTimeoutNs);
    };

    if (warp == 16) {
        // the whole warp runs the loop (warp-uniform state); the elected lane issues
        auto agree = [](bool x) { return __shfl_sync(0xffffffffu, x ? 1 : 0, 0) != 0; };
        const uint32_t idesc = idesc_bf16_f32(128, 128);
        int loaded = 0, used = 0;   // feature tiles whose loads were issued / that were consumed
        int step = 0;
        if (elect_one()) {
            mbar_expect_tx(wfull, kFW1Bytes + kFW2Bytes);
            tma_load_2d(sW1, &tw1, wfull, 0, 0);
            for (int c = 0; c < 4; ++c) tma_load_2d(sW2 + c * kFW1Bytes, &tw2, wfull, c * 64, 0);
        }
        __syncwarp();
        auto top_up = [&]() -> bool {
            while (loaded < my_tiles && loaded < used + kFXStages) {
                const int q = loaded % kFXStages;
                if (!agree(pwait(xempty + q, (uint32_t)(((loaded / kFXStages) & 1) ^ 1)))) return false;
                if (elect_one()) {
                    mbar_expect_tx(xfull + q, kATileBytes);
                    tma_load_2d(sX + q * kATileBytes, &tx, xfull + q, 0, ((int)blockIdx.x + loaded * (int)gridDim.x) * 128);
                }
                __syncwarp();
                ++loaded;
            }
            return true;
        };
        // wait until accumulator region step % 2 is free (the step two before it drained)
        auto region = [&]() -> bool {
            if (!agree(pwait(acce + (step & 1), (uint32_t)(((step >> 1) & 1) ^ 1)))) return false;
            fence_after();
            return true;
        };
        // layer 1 of the next feature tile: two steps from the feature ring
        auto layer1 = [&]() -> bool {
            const int q = used % kFXStages;
            if (!agree(pwait(xfull + q, (uint32_t)((used / kFXStages) & 1)))) return false;
            fence_after();
            const uint32_t a0 = saddr(sX + q * kATileBytes);
            for (int j = 0; j < 2; ++j, ++step) {
                if (!region()) return false;
                if (elect_one()) {
                    const uint32_t d = tmem + (uint32_t)(step & 1) * 128, b0 = saddr(sW1) + (uint32_t)j * 16384;
#pragma unroll
                    for (int kk = 0; kk < 4; ++kk)
                        mma_bf16(d, sdesc_sw128(a0 + kk * 32), sdesc_sw128(b0 + kk * 32), idesc, kk > 0 ? 1u : 0u);
                    if (j == 1) mma_commit(xempty + q);
                    mma_commit(accf + (step & 1));
                }
                __syncwarp();
            }
            ++used;
            return top_up();
        };
        // layer 2 of local tile lt: two steps from its activations in tensor memory
        auto layer2 = [&](int lt) -> bool {
            if (!agree(pwait(hfull + (lt & 1), (uint32_t)((lt >> 1) & 1)))) return false;
            fence_after();
            const uint32_t a = tmem + kFHCol + (uint32_t)(lt & 1) * 128;
            for (int j = 0; j < 2; ++j, ++step) {
                if (!region()) return false;
                if (elect_one()) {
                    const uint32_t d = tmem + (uint32_t)(step & 1) * 128;
#pragma unroll
                    for (int c = 0; c < 4; ++c) {
                        const uint32_t b0 = saddr(sW2) + (uint32_t)c * kFW1Bytes + (uint32_t)j * 16384;
#pragma unroll
                        for (int kk = 0; kk < 4; ++kk)
                            mma_bf16_ts(d, a + (uint32_t)(c * 4 + kk) * 8, sdesc_sw128(b0 + kk * 32), idesc,
                                        (c > 0 || kk > 0) ? 1u : 0u);
                    }
                    mma_commit(accf + (step & 1));
                }
                __syncwarp();
            }
            return true;
        };
        bool ok = top_up() && agree(pwait(wfull, 0));
        if (ok && my_tiles > 0) ok = layer1();
        // test mode: with the first tile's layer-1 steps in flight, wait for what never comes, so
        // that the limit expires with tensor-core work, copies and epilogue waits outstanding
        if (ok && g.wait_ns && !agree(pwait(never, 0))) ok = false;
        for (int lt = 0; ok && lt < my_tiles; ++lt) {
            if (lt + 1 < my_tiles) ok = layer1();
            if (ok) ok = layer2(lt);
        }
        // wind down: every issued MMA complete, every issued copy landed (bounded)
        if (elect_one()) mma_commit(done);
        __syncwarp();
        mbar_wait(done, 0, kWaitTimeoutNs);
        mbar_wait(wfull, 0, kWaitTimeoutNs);   // the weight copies, if their wait gave up
        for (int u = used; u < loaded; ++u)
            mbar_wait(xfull + u % kFXStages, (uint32_t)((u / kFXStages) & 1), kWaitTimeoutNs);
        if (!ok && lane == 0) atomicOr(g.errw, HF_DEV_ERR_TIMEOUT);
    } else {
        const int quarter = warp & 3, grp = warp >> 2;
        const int lrow = quarter * 32 + lane;
        const uint32_t lanes = tmem + ((uint32_t)(quarter * 32) << 16);
        int step = 0;
        // this warp's 32 columns of the next step's accumulator; the region is released at once
        auto drain = [&](uint32_t (&va)[16], uint32_t (&vb)[16]) -> bool {
            const int r = step & 1;
            if (!pwait(accf + r, (uint32_t)((step >> 1) & 1))) return false;
            fence_after();
            const uint32_t ta = lanes + (uint32_t)r * 128 + (uint32_t)grp * 32;
            tmem_ld16_issue(ta, va);
            tmem_ld16_issue(ta + 16, vb);
            tmem_ld_wait(va);
            tmem_ld_wait(vb);
            fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(acce + r);
            ++step;
            return true;
        };
        // bf16 pairs of GELU(accumulator + bias) for the 32 columns (bias at the first one)
        auto act = [&](const uint32_t (&va)[16], const uint32_t (&vb)[16], const float* bias, uint32_t (&w)[16]) {
#pragma unroll
            for (int i = 0; i < 16; ++i) {
                const uint32_t xa = i < 8 ? va[2 * i] : vb[2 * i - 16];
                const uint32_t xb = i < 8 ? va[2 * i + 1] : vb[2 * i - 15];
                const float2 b = *reinterpret_cast<const float2*>(bias + 2 * i);
                float ga, gb;
                g2u(gelu_poly2(g2add(g2(__uint_as_float(xa), __uint_as_float(xb)), g2(b.x, b.y))), ga, gb);
                w[i] = bf16x2_bits(ga, gb);
            }
        };
        // layer 1 of local tile lt: its activations into activation region lt % 2
        auto e1 = [&](int lt) -> bool {
            for (int j = 0; j < 2; ++j) {
                uint32_t va[16], vb[16], w[16];
                if (!drain(va, vb)) return false;
                const int n0 = j * 128 + grp * 32;
                act(va, vb, cb1 + n0, w);
                const uint32_t hc = lanes + kFHCol + (uint32_t)(lt & 1) * 128 + (uint32_t)(n0 >> 1);
                const uint32_t lo[8] = {w[0], w[1], w[2], w[3], w[4], w[5], w[6], w[7]};
                const uint32_t hi[8] = {w[8], w[9], w[10], w[11], w[12], w[13], w[14], w[15]};
                tmem_st8(hc, lo);
                tmem_st8(hc + 8, hi);
                tmem_st_wait();
            }
            fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(hfull + (lt & 1));
            return true;
        };
        // layer 2 and the head of local tile lt
        auto e2 = [&](int lt) -> bool {
            g2_t Y0 = g2s(0.0f), Y1 = g2s(0.0f), Y2 = g2s(0.0f);   // head sums over even / odd units
            for (int j = 0; j < 2; ++j) {
                uint32_t va[16], vb[16], w[16];
                if (!drain(va, vb)) return false;
                const int n0 = j * 128 + grp * 32;
                act(va, vb, cb2 + n0, w);
#pragma unroll
                for (int i = 0; i < 16; ++i) {
                    const g2_t H = g2(__uint_as_float(w[i] << 16), __uint_as_float(w[i] & 0xffff0000u));
                    const float2 w0 = *reinterpret_cast<const float2*>(cw3 + n0 + 2 * i);
                    const float2 w1 = *reinterpret_cast<const float2*>(cw3 + 256 + n0 + 2 * i);
                    const float2 w2 = *reinterpret_cast<const float2*>(cw3 + 512 + n0 + 2 * i);
                    Y0 = g2fma(g2(w0.x, w0.y), H, Y0);
                    Y1 = g2fma(g2(w1.x, w1.y), H, Y1);
                    Y2 = g2fma(g2(w2.x, w2.y), H, Y2);
                }
            }
            float y0, y1, y2, o0, o1, o2;
            g2u(Y0, y0, o0);
            g2u(Y1, y1, o1);
            g2u(Y2, y2, o2);
            y0 += o0;
            y1 += o1;
            y2 += o2;
            if (grp != 0) {
                // hand the partial sums over (once group 0 has read the previous tile's)
                if (!pwait(hfree, (uint32_t)((lt & 1) ^ 1))) return false;
                float* pp = part + ((grp - 1) * 128 + lrow) * 3;
                pp[0] = y0;
                pp[1] = y1;
                pp[2] = y2;
                __syncwarp();
                if (lane == 0) mbar_arrive(hbar);
                return true;
            }
            if (!pwait(hbar, (uint32_t)(lt & 1))) return false;
#pragma unroll
            for (int q = 0; q < 3; ++q) {
                const float* pp = part + (q * 128 + lrow) * 3;
                y0 += pp[0];
                y1 += pp[1];
                y2 += pp[2];
            }
            y0 += cw3[768];
            y1 += cw3[769];
            y2 += cw3[770];
            __syncwarp();
            if (lane == 0) mbar_arrive(hfree);
            const int row = ((int)blockIdx.x + lt * (int)gridDim.x) * 128 + lrow;
            if (row < g.M) {
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
            return true;
        };
        bool ok = true;
        if (my_tiles > 0) ok = e1(0);
        for (int lt = 0; ok && lt < my_tiles; ++lt) {
            if (lt + 1 < my_tiles) ok = e1(lt + 1);
            if (ok) ok = e2(lt);
        }
        if (!ok && lane == 0) atomicOr(g.errw, HF_DEV_ERR_TIMEOUT);
    }
    fence_before();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, 512);
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
        default: return launch_epi<EPI_PARTIAL>(bn, ta, tb, ga, splits, s);
    }
}

cudaError_t hf_mlp_fused(const CUtensorMap& tx, const CUtensorMap& tw1, const CUtensorMap& tw2, const GemmArgs& g,
                         const float* b2, cudaStream_t s) {
    if (g.M <= 0) return cudaSuccess;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaError_t e = cudaStreamIsCapturing(s, &cs);
    if (e == cudaSuccess && cs == cudaStreamCaptureStatusNone)
        e = cudaFuncSetAttribute(k_mlp_fused, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kFSmemBytes);
    if (e != cudaSuccess) return e;
    static int sms = 0;
    if (!sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (sms <= 0) sms = 1;
    }
    const int tiles = (g.M + 127) / 128;
    k_mlp_fused<<<tiles < sms ? tiles : sms, kFThreads, kFSmemBytes, s>>>(tx, tw1, tw2, g, b2);
    return cudaGetLastError();
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
