// hf_gabor.cu - orientation and confidence maps from images with a Gabor filter bank (the step
// before the fusion, Sec. 3.1: O and C "using Gabor filters"), on the tensor cores.
//
// The bank: 64 orientations theta_k = k pi / 64, a 15 x 15 window (offsets u right, v down), along
// a = u cos + v sin, across b = -u sin + v cos, envelope exp(-a^2 / 2 sa^2 - b^2 / 2 sb^2); even
// kernel envelope cos(2 pi b / lambda) minus its window mean, odd kernel envelope sin(2 pi b /
// lambda); bfloat16.  Per pixel F_k = sqrt(e_k^2 + o_k^2) of the window correlations (zero outside
// the image), theta = theta_k* for the largest F (first on ties), C = 1 - mean F / F_k*.
//
// As a GEMM: D[pixel][filter] = sum over the 15 window rows dy and 16 taps dx of
// A_r[pixel][dx] . B[dy][filter][dx], with A_r[pixel][dx] = I(r - 7, pixel + dx - 7) the "window row"
// r = row + dy of the pixel's run (bf16, zero outside the image, tap 15 zero).  k_gabor: a
// persistent CTA per SM walks down runs of rows of 128-column strips; four builder warps write each
// window row of the strip once, straight from the image, into a ring of 16 boxes in tensor memory
// (lane = pixel, 8 columns of bf16 pairs: one box is the A operand of one K = 16 MMA step), and an
// MMA warp issues, for every output row (a tile of 128 pixels), 15 tcgen05.mma (M = 128 pixels,
// N = 128 filters: 64 even then 64 odd; A from tensor memory, B from shared memory) over the sliding
// window of the 15 window rows it needs, against the bank held in shared memory (loaded once with
// TMA, 32-byte swizzle).  With A in tensor memory an MMA reads only the 4 KB bank box from shared
// memory.  Three accumulators in tensor memory serve three epilogue groups of four warps, which
// read a pixel per lane and reduce its 64 energies to the angle and the confidence.  Every mbarrier
// wait is bounded (2 s): on expiry the CTA records HF_DEV_ERR_TIMEOUT, drains its MMAs and returns.
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <vector>

#include "hf_gemm.cuh"
#include "hf_internal.cuh"
#include "hf_tc.cuh"

using namespace hf_tc;

namespace {

constexpr int kGOri = 64, kGR = 7, kGWin = 15, kGTaps = 16, kGN = 128;
constexpr int kGBox = 128 * kGTaps * 2;   // bytes of one bank box: 128 filters x 32 bytes
constexpr int kGGroups = 3;               // epilogue groups of four warps, one accumulator each
constexpr int kGRing = 16;                // window-row boxes held in tensor memory (a power of two)
constexpr int kGBoxCols = kGTaps / 2;     // tensor-memory columns of one window-row box (2 bf16 each)
constexpr int kGACol = kGGroups * kGN;    // first tensor-memory column of the ring
static_assert(kGACol + kGRing * kGBoxCols <= 512, "accumulators and ring exceed the 512 tensor-memory columns");
static_assert((kGRing & (kGRing - 1)) == 0 && kGRing >= kGWin + 1, "ring: a power of two above the window");
constexpr int kGBuild = 4;                // builder warps: a thread per pixel row (tensor-memory lane) of a box
constexpr int kGThreads = (4 * kGGroups + kGBuild + 1) * 32;   // epilogue warps, builders, the MMA warp
constexpr int kGMmaWarp = 4 * kGGroups + kGBuild;
constexpr float kPiF = 3.14159265358979f;

struct GaborArgs {
    int V, H, W, Hp, Wt, tx;   // images, rows, columns, padded rows, padded columns, tiles per row
    int chunk, nch;            // rows per unit, units per column strip
    int units;                 // V x tx x nch work units: (image, 128-column strip, run of rows)
    const float* img;          // V x H x W
    float* theta;
    float* conf;
    uint32_t* errw;
};

// A work unit: the output rows [y0, y0 + n) of one 128-column strip of one image; its window rows are
// the padded rows y0 .. y0 + n + 13 of the strip (image rows y0 - 7 .. y0 + n + 6).
struct Unit {
    int v, y0, n, tx;
};
__device__ __forceinline__ Unit unit_of(const GaborArgs& a, int u) {
    Unit r;
    const int ch = u % a.nch, st = u / a.nch;
    r.tx = st % a.tx;
    r.v = st / a.tx;
    r.y0 = ch * a.chunk;
    r.n = min(a.chunk, a.H - r.y0);
    return r;
}

// packed FP32 pairs (fma .f32x2: each lane rounded like the scalar instruction); a pair read from
// tensor memory already sits in adjacent registers
typedef unsigned long long g_f32x2;
__device__ __forceinline__ g_f32x2 gpk(float a, float b) {
    g_f32x2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ void gupk(g_f32x2 r, float& a, float& b) {
    asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(r));
}
__device__ __forceinline__ g_f32x2 gfma2(g_f32x2 a, g_f32x2 b, g_f32x2 c) {
    g_f32x2 d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
// three-input maximum (one instruction)
__device__ __forceinline__ float gmax3(float a, float b, float c) {
    float d;
    asm("max.f32 %0, %1, %2, %3;" : "=f"(d) : "f"(a), "f"(b), "f"(c));
    return d;
}
// MUFU reciprocal square root without the subnormal path (every argument here is >= 1e-30, normal).
__device__ __forceinline__ float rsqrt_ftz(float x) {
    float r;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// The 15 taps I(r - 7, x + dx - 7), dx < 15, of pixel column x in padded row r of unit U (0 outside).
__device__ __forceinline__ void load_taps(const GaborArgs& a, const Unit& U, int r, int x, float (&t)[kGWin]) {
    const int yi = U.y0 + r - kGR;
    const bool row_in = yi >= 0 && yi < a.H;
    const float* src = a.img + ((size_t)U.v * a.H + (row_in ? yi : 0)) * a.W;
    if (row_in && x >= kGR && x + kGR < a.W) {   // the whole window inside the image
#pragma unroll
        for (int dx = 0; dx < kGWin; ++dx) t[dx] = __ldg(src + x + dx - kGR);
    } else {
#pragma unroll
        for (int dx = 0; dx < kGWin; ++dx) {
            const int xx = x + dx - kGR;
            t[dx] = row_in && xx >= 0 && xx < a.W ? __ldg(src + xx) : 0.0f;
        }
    }
}

__global__ void __launch_bounds__(kGThreads, 1) k_gabor(const __grid_constant__ CUtensorMap tb, GaborArgs a) {
    extern __shared__ unsigned char smem_raw[];
    unsigned char* base = smem_raw + ((1024 - (saddr(smem_raw) & 1023)) & 1023);
    unsigned char* sB = base;                      // 15 boxes: the bank, one window row each
    uint64_t* aempty = reinterpret_cast<uint64_t*>(sB + kGWin * kGBox);   // [kGRing] MMAs -> builders
    uint64_t* bfull = aempty + kGRing;
    uint64_t* accf = bfull + 1;           // [kGGroups] MMA -> epilogue group
    uint64_t* tready = accf + kGGroups;   // [kGGroups] epilogue group + builders -> MMA
    uint64_t* done = tready + kGGroups;
    uint32_t* tslot = reinterpret_cast<uint32_t*>(done + 1);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int s = 0; s < kGRing; ++s) mbar_init(aempty + s, 1);
        mbar_init(bfull, 1);
        for (int b = 0; b < kGGroups; ++b) {
            mbar_init(accf + b, 1);
            mbar_init(tready + b, 4 + kGBuild);
        }
        mbar_init(done, 1);
        fence_mbar_init();
    }
    if (warp == 0) {
        tmem_alloc(tslot, 512);
        tmem_relinquish();
    }
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = *tslot;
    // Tensor memory: columns 128 g .. 128 g + 127 accumulate the tiles of epilogue group g; columns
    // kGACol + 8 s .. + 7 hold ring slot s, a window-row box as the MMAs' A operand (lane = pixel,
    // two bf16 taps per column, tap 0 in the low half).  The CTA takes units blockIdx.x, +
    // gridDim.x, ...; down a unit, output row y uses the window rows y .. y + 14, so every window
    // row is built once and freed after the last output row that uses it.  Boxes are numbered in
    // build order; box q lives in slot q % kGRing.
    if (warp >= 4 * kGGroups && warp < kGMmaWarp) {
        // Builder warp q writes lanes 32 q .. 32 q + 31 of every box (a warp reaches only its own
        // quarter of the lanes): taps in bf16 (round to nearest even), tap 15 zero.  The taps of the
        // next box are loaded before the wait for the slot of this one.
        const int q = warp & 3, p = q * 32 + lane;
        const uint32_t tq = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)kGACol;
        if (q == 0 && lane == 0) {
            mbar_expect_tx(bfull, kGWin * kGBox);
            for (int dy = 0; dy < kGWin; ++dy) tma_load_2d(sB + dy * kGBox, &tb, bfull, 0, dy * kGN);
        }
        int u = blockIdx.x, r = 0, sl = 0, tb = 0;
        uint32_t ph = 0;
        Unit U = u < a.units ? unit_of(a, u) : Unit{};
        bool have = u < a.units, ok = true;
        float t[kGWin];
        if (have) load_taps(a, U, 0, U.tx * 128 + p, t);
        while (have) {
            uint32_t w[8];
#pragma unroll
            for (int k = 0; k < 8; ++k) {   // two taps per cvt: tap 2k in the low half
                const float hi = 2 * k + 1 < kGWin ? t[2 * k + 1] : 0.0f;
                asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(w[k]) : "f"(hi), "f"(t[2 * k]));
            }
            const int rb = r;   // the box being written: padded row rb of its unit
            if (++r == U.n + kGWin - 1) {
                r = 0;
                u += gridDim.x;
                if (u < a.units) U = unit_of(a, u);
            }
            const bool next = u < a.units;
            if (next) load_taps(a, U, r, U.tx * 128 + p, t);
            uint32_t okw = 1;
            if (lane == 0) okw = mbar_wait(aempty + sl, ph ^ 1u, kWaitTimeoutNs) ? 1u : 0u;
            okw = __shfl_sync(0xffffffffu, okw, 0);
            if (!okw) {
                ok = false;
                break;
            }
            fence_after();
            tmem_st8(tq + (uint32_t)(sl * kGBoxCols), w);
            tmem_st_wait();
            fence_before();   // the MMAs read what these stores wrote
            __syncwarp();
            if (rb >= kGWin - 1) {   // the newest window row of the unit's output row rb - 14
                if (lane == 0) mbar_arrive(tready + tb);
                tb = tb + 1 == kGGroups ? 0 : tb + 1;
            }
            if (++sl == kGRing) {
                sl = 0;
                ph ^= 1u;
            }
            have = next;
        }
        if (!ok && lane == 0) atomicOr(a.errw, HF_DEV_ERR_TIMEOUT);
    } else if (warp == kGMmaWarp) {
        // The whole warp runs the loop (its values stay warp-uniform) and the elected lane issues:
        // a loop run by one lane alone issues several times slower while the epilogue warps
        // compute.  The issue sequence of a tile is straight-line code with compile-time operand
        // offsets and one barrier wait; each extra wait between MMAs stalls the tensor pipe.
        bool ok = __shfl_sync(0xffffffffu, mbar_wait(bfull, 0, kWaitTimeoutNs) ? 1 : 0, 0) != 0;
        const uint32_t idesc = idesc_bf16_f32(128, kGN), sBa = saddr(sB), ta = tmem + (uint32_t)kGACol;
        uint32_t base = 0;    // box number of the unit's first window row (per CTA: below 2^31)
        int b = 0;            // the epilogue group (accumulator) of the next tile
        uint32_t accph = 0;   // parity of that accumulator's use
        for (int u = blockIdx.x; ok && u < a.units; u += gridDim.x) {
            const Unit U = unit_of(a, u);
            for (int y = 0; y < U.n; ++y) {
                // one wait per tile: its accumulator drained by the epilogue group and its newest
                // window row (box base + y + 14, hence every older one) written by all builders
                ok = __shfl_sync(0xffffffffu, mbar_wait(tready + b, accph, kWaitTimeoutNs) ? 1 : 0, 0) != 0;
                if (!ok) break;
                fence_after();
                const uint32_t d = tmem + (uint32_t)(b * kGN), s0 = base + (uint32_t)y;
                if (elect_one()) {
                    mma_bf16_ts(d, ta + (s0 & (kGRing - 1)) * kGBoxCols, sdesc_sw32(sBa), idesc, 0u);
                    mma_commit(aempty + (s0 & (kGRing - 1)));   // window row y: that was its last use
#pragma unroll
                    for (int dy = 1; dy < kGWin; ++dy)
                        mma_bf16_ts(d, ta + ((s0 + (uint32_t)dy) & (kGRing - 1)) * kGBoxCols,
                                    sdesc_sw32(sBa + (uint32_t)(dy * kGBox)), idesc, 1u);
                    mma_commit(accf + b);
                }
                __syncwarp();
                if (++b == kGGroups) {
                    b = 0;
                    accph ^= 1u;
                }
            }
            if (!ok) break;
            if (elect_one())
                for (int r = 0; r < kGWin - 1; ++r)   // the unit's last 14 window rows
                    mma_commit(aempty + ((base + (uint32_t)(U.n + r)) & (kGRing - 1)));
            __syncwarp();
            base += (uint32_t)(U.n + kGWin - 1);
        }
        // wind down: every issued MMA complete (bounded)
        if (elect_one()) mma_commit(done);
        __syncwarp();
        mbar_wait(done, 0, kWaitTimeoutNs);
        if (!ok && lane == 0) atomicOr(a.errw, HF_DEV_ERR_TIMEOUT);
    } else {
        // group g = warp / 4 takes this CTA's tiles g, g + 3, ... (in the producer's order: unit by
        // unit, row by row), in tensor-memory buffer g; warp w reads lanes 32 (w % 4) .. + 31: pixel
        // 32 (w % 4) + lane of the tile
        const int grp = warp >> 2, quarter = warp & 3;
        const uint32_t tl = tmem + (uint32_t)grp * kGN + ((uint32_t)(quarter * 32) << 16);
        int u = blockIdx.x, y = grp;
        Unit U = u < a.units ? unit_of(a, u) : Unit{};
        while (u < a.units && y >= U.n) {   // units shorter than the offset (tiny images)
            y -= U.n;
            u += gridDim.x;
            if (u < a.units) U = unit_of(a, u);
        }
        if (lane == 0) mbar_arrive(tready + grp);   // the accumulator starts out free
        for (long long k = 0; u < a.units; ++k) {
            if (!mbar_wait_idle(accf + grp, (uint32_t)(k & 1), kWaitTimeoutNs)) {
                if (lane == 0) atomicOr(a.errw, HF_DEV_ERR_TIMEOUT);
                break;
            }
            fence_after();
            // per orientation: F^2 = e^2 + o^2 (+ 1e-30, so that the reciprocal root stays finite)
            // in packed pairs and F = F^2 rsqrt(F^2) in scalar FMAs; the argmax as a maximum of
            // keys: F^2 bits with the low 6 cleared, then 63 - k (the first of equal values wins;
            // the cleared bits move F by < 2^-18 F, inside the oracle's tie margin).  F^2 >= 1e-30
            // is a positive normal float, and so is its key, so keys order as floats: one
            // three-input max per pair.  Two chains of sums and maxima; the next 16 orientations
            // load from tensor memory while these reduce, and the accumulator is released to the
            // MMAs as soon as its last columns are in registers.
            float kmax0 = 0.0f, kmax1 = 0.0f;
            float sacc0 = 0.0f, sacc1 = 0.0f;
            const g_f32x2 tiny = gpk(1e-30f, 1e-30f);
            uint32_t ev[2][16], od[2][16];
            tmem_ld16_issue(tl, ev[0]);
            tmem_ld16_issue(tl + kGOri, od[0]);
            tmem_ld_wait(ev[0]);
            tmem_ld_wait(od[0]);
            constexpr int kCh = kGOri / 16;
#pragma unroll
            for (int ch = 0; ch < kCh; ++ch) {
                const int cur = ch & 1, c = ch * 16;
                if (ch + 1 < kCh) {
                    tmem_ld16_issue(tl + c + 16, ev[cur ^ 1]);
                    tmem_ld16_issue(tl + kGOri + c + 16, od[cur ^ 1]);
                }
#pragma unroll
                for (int q = 0; q < 16; q += 2) {
                    const g_f32x2 e = gpk(__uint_as_float(ev[cur][q]), __uint_as_float(ev[cur][q + 1]));
                    const g_f32x2 o = gpk(__uint_as_float(od[cur][q]), __uint_as_float(od[cur][q + 1]));
                    float f0, f1;
                    gupk(gfma2(e, e, gfma2(o, o, tiny)), f0, f1);
                    sacc0 = fmaf(f0, rsqrt_ftz(f0), sacc0);
                    sacc1 = fmaf(f1, rsqrt_ftz(f1), sacc1);
                    const float k0 = __uint_as_float((__float_as_uint(f0) & 0xFFFFFFC0u) | (uint32_t)(63 - (c + q)));
                    const float k1 = __uint_as_float((__float_as_uint(f1) & 0xFFFFFFC0u) | (uint32_t)(62 - (c + q)));
                    if ((q >> 1) & 1)
                        kmax1 = gmax3(kmax1, k0, k1);
                    else
                        kmax0 = gmax3(kmax0, k0, k1);
                }
                if (ch + 1 < kCh) {
                    tmem_ld_wait(ev[cur ^ 1]);
                    tmem_ld_wait(od[cur ^ 1]);
                    if (ch + 2 == kCh) {   // every column read: later MMAs may overwrite the buffer
                        fence_before();
                        __syncwarp();
                        if (lane == 0) mbar_arrive(tready + grp);
                    }
                }
            }
            const uint32_t kmax = __float_as_uint(fmaxf(kmax0, kmax1));
            const float sum = sacc0 + sacc1, best2 = __uint_as_float(kmax & 0xFFFFFFC0u);
            const int kb = 63 - (int)(kmax & 63u);
            const int x = U.tx * 128 + quarter * 32 + lane;
            if (x < a.W) {
                const float best = sqrtf(best2);
                const size_t o = ((size_t)U.v * a.H + U.y0 + y) * a.W + x;
                a.theta[o] = (float)kb * (kPiF / (float)kGOri);
                a.conf[o] = best > 0.0f ? 1.0f - sum * (1.0f / (float)kGOri) / best : 0.0f;
            }
            y += kGGroups;   // this group's next tile
            while (u < a.units && y >= U.n) {
                y -= U.n;
                u += gridDim.x;
                if (u < a.units) U = unit_of(a, u);
            }
        }
    }
    fence_before();
    __syncthreads();
    fence_after();
    if (warp == 0) tmem_dealloc(tmem, 512);
}

uint16_t bf16_host(float x) {
    uint32_t u;
    memcpy(&u, &x, 4);
    if ((u & 0x7f800000u) == 0x7f800000u) return (uint16_t)(u >> 16);
    return (uint16_t)((u + 0x7fffu + ((u >> 16) & 1u)) >> 16);
}

// The bank as bf16 bits: out[k][0 even / 1 odd][v][u], k < 64, v, u < 15.
void gabor_bank(const hf_gabor_cfg& g, std::vector<uint16_t>& out) {
    const int w = kGWin, n = w * w;
    out.assign((size_t)kGOri * 2 * n, 0);
    std::vector<double> ev(n);
    for (int k = 0; k < kGOri; ++k) {
        const double th = 3.14159265358979323846 * k / kGOri, c = cos(th), s = sin(th);
        double mean = 0.0;
        for (int v = -kGR; v <= kGR; ++v)
            for (int u = -kGR; u <= kGR; ++u) {
                const double aa = u * c + v * s, bb = -u * s + v * c;
                const double env = exp(-aa * aa / (2.0 * g.sigma_along * g.sigma_along) -
                                       bb * bb / (2.0 * g.sigma_across * g.sigma_across));
                const int q = (v + kGR) * w + (u + kGR);
                ev[q] = env * cos(2.0 * 3.14159265358979323846 * bb / g.lambda);
                mean += ev[q];
                out[(size_t)(2 * k + 1) * n + q] = bf16_host((float)(env * sin(2.0 * 3.14159265358979323846 * bb / g.lambda)));
            }
        mean /= n;
        for (int q = 0; q < n; ++q) out[(size_t)(2 * k) * n + q] = bf16_host((float)(ev[q] - mean));
    }
}

bool cfg_ok(const hf_gabor_cfg* g) {
    return g && g->n_theta == kGOri && g->radius == kGR && isfinite(g->sigma_along) && g->sigma_along > 0.0f &&
           isfinite(g->sigma_across) && g->sigma_across > 0.0f && isfinite(g->lambda) && g->lambda > 0.0f;
}

int sync_check_errw(hf_ctx* c) {
    uint32_t w = 0;
    cudaError_t e = cudaMemcpyAsync(&w, c->errw.p, sizeof(uint32_t), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return hf_cuda_err(c, e, "gabor");
    if (w) {
        cudaMemsetAsync(c->errw.p, 0, sizeof(uint32_t), c->stream);
        cudaStreamSynchronize(c->stream);
        return hf_set_err(c, (w & HF_DEV_ERR_TIMEOUT) ? HF_ERR_TIMEOUT : HF_ERR_CUDA, "gabor: device error word 0x%x", w);
    }
    return HF_OK;
}

}  // namespace

// ------------------------------------------------------------------ C ABI
extern "C" int hair_fuse_gabor_bank(const hf_gabor_cfg* cfg, float* out) {
    if (!cfg_ok(cfg) || !out) return HF_ERR_INVALID_ARG;
    std::vector<uint16_t> b;
    gabor_bank(*cfg, b);
    for (size_t q = 0; q < b.size(); ++q) {
        const uint32_t u = (uint32_t)b[q] << 16;
        memcpy(out + q, &u, 4);
    }
    return HF_OK;
}

extern "C" int hair_fuse_gabor(hf_ctx* c, const hf_gabor_cfg* cfg, int V, int H, int W, const float* images,
                               float* theta_out, float* conf_out, int mem_kind) {
    if (!c) return HF_ERR_INVALID_ARG;
    if (!cfg_ok(cfg))
        return hf_set_err(c, HF_ERR_INVALID_ARG, "gabor: n_theta 64, radius 7, positive finite sigmas and lambda");
    if (mem_kind != HF_HOST && mem_kind != HF_DEVICE && mem_kind != HF_HOST_ASYNC)
        return hf_set_err(c, HF_ERR_INVALID_ARG, "bad mem_kind");
    const bool staged = mem_kind != HF_DEVICE;   // host images and maps go through device staging
    if (V < 1 || H < 1 || W < 1 || !images || !theta_out || !conf_out)
        return hf_set_err(c, HF_ERR_INVALID_ARG, "gabor: V, H, W >= 1 and non-null arrays");
    const int Hp = H + 2 * kGR, tx = (W + 127) / 128, Wt = tx * 128;
    if ((long long)V * Hp * Wt >= (1LL << 31) - 1) return hf_set_err(c, HF_ERR_SHAPE, "gabor: more than 2^31 padded pixels");
    const size_t npx = (size_t)V * H * W;
    int rc;
    // scratch: staged host images and outputs
    const size_t ibytes = staged ? npx * 4 : 0, obytes = staged ? 2 * npx * 4 : 0;
    const float* img = images;
    float *th = theta_out, *cf = conf_out;
    cudaStream_t st = c->stream;
    cudaError_t e = cudaSuccess;
    if (staged) {
        auto al = [](size_t x) { return (x + 1023) & ~(size_t)1023; };
        if ((rc = hf_ensure(c, c->gabor, al(ibytes) + obytes))) return rc;
        float* di = (float*)c->gabor.p;
        e = cudaMemcpyAsync(di, images, npx * 4, cudaMemcpyHostToDevice, st);
        if (e != cudaSuccess) return hf_cuda_err(c, e, "gabor images");
        img = di;
        th = (float*)((char*)c->gabor.p + al(ibytes));
        cf = th + npx;
    }
    // the bank as B[dy][filter n][dx] (n < 64 even kernel of orientation n, n >= 64 odd of n - 64),
    // built on the host once per (sigma along, sigma across, lambda) and kept on the device
    const size_t bbytes = (size_t)kGWin * kGN * kGTaps * 2;
    const float key[3] = {cfg->sigma_along, cfg->sigma_across, cfg->lambda};
    if (!c->gbank_ok || memcmp(key, c->gbank_key, sizeof key) != 0) {
        c->gbank_ok = false;
        if ((rc = hf_ensure(c, c->gbank, bbytes))) return rc;
        std::vector<uint16_t> bank;
        gabor_bank(*cfg, bank);
        std::vector<uint16_t> B((size_t)kGWin * kGN * kGTaps, 0);
        for (int dy = 0; dy < kGWin; ++dy)
            for (int n = 0; n < kGN; ++n)
                for (int dx = 0; dx < kGWin; ++dx) {
                    const int k = n % kGOri, ph = n / kGOri;
                    B[((size_t)dy * kGN + n) * kGTaps + dx] = bank[((size_t)(2 * k + ph) * kGWin + dy) * kGWin + dx];
                }
        // stream-ordered after any launch still reading the previous bank; B is a host vector
        // about to go out of scope, so wait for the copy
        e = cudaMemcpyAsync(c->gbank.p, B.data(), bbytes, cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return hf_cuda_err(c, e, "gabor bank");
        memcpy(c->gbank_key, key, sizeof key);
        c->gbank_ok = true;
    }
    const uint16_t* Bd = (const uint16_t*)c->gbank.p;
    CUtensorMap tb;
    if ((e = hf_make_tmap_bf16_rows32(&tb, Bd, (long long)kGWin * kGN, 128)) != cudaSuccess)
        return hf_cuda_err(c, e, "gabor tensor map");
    int sms = 148;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device);
    // runs of rows: enough units for eight per SM, each run at least 64 rows where the image allows
    const long long strips = (long long)V * tx;
    int nch = (int)((8LL * sms + strips - 1) / strips);
    nch = nch < 1 ? 1 : (nch > (H + 63) / 64 ? (H + 63) / 64 : nch);
    nch = nch < 1 ? 1 : nch;
    const int chunk = (H + nch - 1) / nch;
    nch = (H + chunk - 1) / chunk;
    if (strips * nch >= (1LL << 31)) return hf_set_err(c, HF_ERR_SHAPE, "gabor: too many work units");
    GaborArgs ga{V, H, W, Hp, Wt, tx, chunk, nch, (int)(strips * nch), img, th, cf, (uint32_t*)c->errw.p};
    // the bank and the barriers need about 62 KB; asking for more keeps a second CTA off the SM (each
    // takes all 512 tensor-memory columns)
    size_t smem = 1024 + (size_t)kGWin * kGBox + (kGRing + 2 + 2 * kGGroups) * 8 + 16;
    smem = smem < 160 * 1024 ? 160 * 1024 : smem;
    if ((rc = run_launch(c, "k_gabor", [&] {
             cudaError_t e2 = cudaFuncSetAttribute(k_gabor, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
             if (e2 != cudaSuccess) return e2;
             const long long grid = ga.units < sms ? ga.units : sms;
             k_gabor<<<(unsigned)grid, kGThreads, smem, st>>>(tb, ga);
             return cudaGetLastError();
         })))
        return rc;
    if (staged) {
        e = cudaMemcpyAsync(theta_out, th, npx * 4, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(conf_out, cf, npx * 4, cudaMemcpyDeviceToHost, st);
        if (e != cudaSuccess) return hf_cuda_err(c, e, "gabor outputs");
        if (mem_kind == HF_HOST) return sync_check_errw(c);
    }
    return HF_OK;
}
