// hf_batchtiles.cuh - the persistent work loop of the batched kernels, shared by hf_kernels.cu and
// hf_batch_kernels.cu.
#pragma once

#include "hf_internal.cuh"

namespace hf_bt {

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

}  // namespace hf_bt
