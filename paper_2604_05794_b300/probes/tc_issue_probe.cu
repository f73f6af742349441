// tc_issue_probe.cu - what a tcgen05.mma issue stream can afford on this GPU (stand-alone program,
// not part of the library).  One CTA per SM; warp 0 issues tiles of 15 MMAs of 128 x 128 x 16
// (bf16 in, f32 accumulate: the Gabor kernel's tile) into three accumulators in rotation, with two
// commits per tile, in the variants below; the other 15 warps either idle or run an epilogue-like
// mix of FMA, MUFU and integer work.  Prints cycles per tile (960 = 64 cycles per MMA, the peak).
//
//   nvcc -gencode arch=compute_103a,code=sm_103a -O3 -std=c++17 \
//        -o /tmp/tc_issue_probe paper_2604_05794_b300/probes/tc_issue_probe.cu && /tmp/tc_issue_probe
//
// Every wait is bounded; the operands are zeros (only the issue rate is measured).
#include <cstdio>
#include <cstdlib>

#include "../csrc/hf_tc.cuh"

using namespace hf_tc;

enum : int {
    A_SMEM = 1,      // A from shared memory (no swizzle, K-major) instead of tensor memory
    WAIT_START = 2,  // one mbarrier wait (on a completed phase) before each tile
    WAIT_LAST = 4,   // one more before each tile's last MMA
    WARP = 8,        // the whole warp runs the loop, the elected lane issues (else lane 0 alone)
    MATH = 16,       // warps 2-15 compute while warp 0 issues (warp 1 too unless GATE)
    GATE = 32,       // warp 1 does the per-tile mbarrier wait and meets warp 0 at a named barrier
};

__device__ __forceinline__ float rsq(float x) {
    float r;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

template <int MODE>
__device__ __forceinline__ bool issue_tile(uint32_t tmem, uint32_t sBa, uint32_t sAa, uint64_t* bars, uint64_t* ready,
                                           uint32_t base, int b) {
    const uint32_t idesc = idesc_bf16_f32(128, 128), ta = tmem + 384u, d = tmem + (uint32_t)(b * 128);
    bool ok = true;
#pragma unroll
    for (int dy = 0; dy < 15; ++dy) {
        if ((MODE & WAIT_LAST) && dy == 14) ok &= mbar_wait(ready, 1, kWaitTimeoutNs);
        const uint32_t sl = (base + (uint32_t)dy) & 15u;
        if (MODE & A_SMEM)
            mma_bf16(d, sdesc_none(sAa + sl * 4096u, 128, 256), sdesc_sw32(sBa + (uint32_t)dy * 4096u), idesc, dy > 0);
        else
            mma_bf16_ts(d, ta + sl * 8u, sdesc_sw32(sBa + (uint32_t)dy * 4096u), idesc, dy > 0);
        if (dy == 0) mma_commit(bars + 3 + (base & 15u));
    }
    mma_commit(bars + b);
    return ok;
}

template <int MODE>
__global__ void __launch_bounds__(512, 1) k_probe(int tiles, unsigned long long* out, float* sink, unsigned* err) {
    extern __shared__ unsigned char smem_raw[];
    unsigned char* base = smem_raw + ((1024 - (saddr(smem_raw) & 1023)) & 1023);
    unsigned char* sB = base;                 // 15 boxes of 4 KB (B)
    unsigned char* sA = base + 65536;         // 16 boxes of 4 KB (A in shared memory)
    uint64_t* bars = reinterpret_cast<uint64_t*>(base + 131072);   // 3 accumulator + 16 slot barriers
    uint64_t* ready = bars + 19;
    uint64_t* done = ready + 1;
    uint32_t* tslot = reinterpret_cast<uint32_t*>(done + 1);
    volatile int* stop = reinterpret_cast<volatile int*>(tslot + 1);
    for (int i = threadIdx.x; i < 131072 / 4; i += blockDim.x) reinterpret_cast<uint32_t*>(base)[i] = 0u;
    fence_proxy_async();
    if (threadIdx.x == 0) {
        for (int i = 0; i < 19; ++i) mbar_init(bars + i, 1);
        mbar_init(ready, 1);   // never arrived: waiting for the phase before the first completes at once
        mbar_init(done, 1);
        fence_mbar_init();
        *stop = 0;
    }
    if (threadIdx.x < 32) {
        tmem_alloc(tslot, 512);
        tmem_relinquish();
    }
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = *tslot;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (warp == 0) {
        const uint32_t sBa = saddr(sB), sAa = saddr(sA);
        const unsigned long long t0 = clock64();
        bool ok = true;
        int b = 0;
        if (MODE & WARP) {
            for (int t = 0; t < tiles; ++t) {
                if (MODE & GATE) asm volatile("bar.sync 1, 64;" ::: "memory");   // warp 1 waited for us
                if (MODE & WAIT_START) ok &= mbar_wait(ready, 1, kWaitTimeoutNs);
                fence_after();
                if (elect_one()) ok &= issue_tile<MODE>(tmem, sBa, sAa, bars, ready, (uint32_t)t, b);
                __syncwarp();
                b = b == 2 ? 0 : b + 1;
            }
        } else if (lane == 0) {
            for (int t = 0; t < tiles; ++t) {
                if (MODE & WAIT_START) ok &= mbar_wait(ready, 1, kWaitTimeoutNs);
                fence_after();
                ok &= issue_tile<MODE>(tmem, sBa, sAa, bars, ready, (uint32_t)t, b);
                b = b == 2 ? 0 : b + 1;
            }
        }
        __syncwarp();
        if (lane == 0) {
            mma_commit(done);
            if (!mbar_wait(done, 0, kWaitTimeoutNs) || !ok) atomicOr(err, 1u);
            out[blockIdx.x] = clock64() - t0;
            *stop = 1;
        }
    } else if ((MODE & GATE) && warp == 1) {
        // the same number of named-barrier meetings as warp 0's tiles, so neither can be left waiting
        bool ok = true;
        for (int t = 0; t < tiles; ++t) {
            ok &= mbar_wait(ready, 1, kWaitTimeoutNs);
            asm volatile("bar.sync 1, 64;" ::: "memory");
        }
        if (!ok && lane == 0) atomicOr(err, 1u);
    } else if (MODE & MATH) {
        // an epilogue-like mix per step: FMAs, a reciprocal root, a key and a maximum
        float s0 = 0.0f, k0 = 0.0f, x = 1.0f + lane;
        for (int it = 0; it < 20000000 && !*stop; ++it) {
#pragma unroll
            for (int q = 0; q < 16; ++q) {
                const float f = fmaf(x, x, fmaf(x + q, x, 1e-30f));
                s0 = fmaf(f, rsq(f), s0);
                k0 = fmaxf(k0, __uint_as_float((__float_as_uint(f) & 0xFFFFFFC0u) | (uint32_t)q));
                x = fmaf(x, 0.999f, 1e-3f);
            }
        }
        if (s0 == 12345.0f) sink[0] = k0;
    }
    fence_before();
    __syncthreads();
    fence_after();
    if (threadIdx.x < 32) tmem_dealloc(tmem, 512);
}

template <int MODE>
void run(const char* name, int sms, unsigned long long* out, float* sink, unsigned* err) {
    const int tiles = 3000;
    const int smem = 160 * 1024;   // also keeps a second CTA (and a second tensor-memory allocation) off the SM
    cudaFuncSetAttribute(k_probe<MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    for (int rep = 0; rep < 2; ++rep) {   // the first run warms up
        k_probe<MODE><<<sms, 512, smem>>>(tiles, out, sink, err);
        const cudaError_t e = cudaDeviceSynchronize();
        if (e != cudaSuccess) {
            printf("CUDA error %s\n", cudaGetErrorString(e));
            exit(1);
        }
    }
    unsigned long long h[1024];
    cudaMemcpy(h, out, sizeof(unsigned long long) * sms, cudaMemcpyDeviceToHost);
    double avg = 0.0;
    for (int i = 0; i < sms; ++i) avg += (double)h[i];
    printf("%-58s %7.1f cycles per tile\n", name, avg / sms / tiles);
}

int main() {
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, 0);
    if (sms <= 0 || sms > 1024) return 1;
    unsigned long long* out;
    unsigned* err;
    float* sink;
    cudaMalloc(&out, sizeof(unsigned long long) * sms);
    cudaMalloc(&err, 4);
    cudaMalloc(&sink, 4);
    cudaMemset(err, 0, 4);
    run<0>("A in tensor memory, no waits", sms, out, sink, err);
    run<WAIT_START>("A in tensor memory, one wait per tile", sms, out, sink, err);
    run<WAIT_START | WAIT_LAST>("A in tensor memory, two waits per tile", sms, out, sink, err);
    run<A_SMEM>("A in shared memory, no waits", sms, out, sink, err);
    run<A_SMEM | WAIT_START>("A in shared memory, one wait per tile", sms, out, sink, err);
    run<WAIT_START | MATH>("one wait, 15 warps computing, lane 0 issues", sms, out, sink, err);
    run<WAIT_START | MATH | WARP>("one wait, 15 warps computing, warp runs loop + elect.sync", sms, out, sink, err);
    run<GATE | WARP>("wait in a gate warp, bar.sync per tile", sms, out, sink, err);
    run<GATE | MATH | WARP>("wait in a gate warp, bar.sync per tile, 14 warps computing", sms, out, sink, err);
    unsigned herr = 0;
    cudaMemcpy(&herr, err, 4, cudaMemcpyDeviceToHost);
    printf("wait failures: %u\n", herr);
    return herr ? 2 : 0;
}
