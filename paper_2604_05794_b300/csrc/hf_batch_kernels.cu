// hf_batch_kernels.cu - the batched persistent cost kernels over the (scene, tile) items of every
// scene of a batch: the argmin (K2), the refinement (K3, one launch per lane count, over the scenes
// that share it) and the learned path's selection.  The tile bodies are those of the single-scene
// kernels (hf_cost.cuh), so a batched result is bit-identical to the scene fused alone.
#include "hf_batchtiles.cuh"
#include "hf_cost.cuh"

namespace {

using namespace hf_bt;
using namespace hf_cost;

// resident CTAs per SM the register budget is sized for: 16 warps per SM (12 for the widest patch)
template <int KP, int NT>
struct MinCtasB {
    static constexpr int value = (KP <= 9 ? 512 : 384) / NT;
};

// tiles of a scene for the refinement: 32 / L points per warp
template <int L>
__device__ __forceinline__ int refine_tiles(int cnt) {
    const int ppc = (int)(blockDim.x >> 5) * (32 / L);
    return (cnt + ppc - 1) / ppc;
}

__device__ __forceinline__ int thread_tiles(int cnt) { return (cnt + (int)blockDim.x - 1) / (int)blockDim.x; }

template <int KP, int NT>
__global__ void __launch_bounds__(NT, 512 / NT) k_argmin_batch(const CostArgs* __restrict__ fa, BatchCtl c) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    batch_tiles(fa, c, [](const CostArgs& a) { return thread_tiles(a.list ? *a.list_count : a.N); },
                [&](const CostArgs& a, int t) { argmin_tile<KP, NT>(a, t, smem_raw); });
}

template <int KP, int L, int NT>
__global__ void __launch_bounds__(NT, MinCtasB<KP, NT>::value) k_refine_batch(const CostArgs* __restrict__ fa, BatchCtl c) {
    batch_tiles(fa, c, [](const CostArgs& a) { return refine_tiles<L>(a.list ? *a.list_count : a.N); },
                [](const CostArgs& a, int t) { refine_tile_l<KP, L, PairsFor<KP>::value>(a, t); });
}

template <int KP, int NT>
__global__ void __launch_bounds__(NT) k_refine_t_batch(const CostArgs* __restrict__ fa, BatchCtl c) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    batch_tiles(fa, c, [](const CostArgs& a) { return thread_tiles(a.list ? *a.list_count : a.N); },
                [&](const CostArgs& a, int t) { refine_stage_tile<KP, NT>(a, t, smem_raw); });
}

template <int KP>
__global__ void __launch_bounds__(128) k_select_batch(const LearnArgs* __restrict__ la, BatchCtl c) {
    batch_tiles(la, c, [](const LearnArgs& a) { return thread_tiles(a.f.N); },
                [](const LearnArgs& a, int t) { select_tile<KP>(a, t); });
}

template <int KP, int NT>
cudaError_t launch_argmin(const CostArgs* fa, const BatchCtl& c, cudaStream_t s) {
    const size_t sm = argmin_smem_bytes<KP, NT>();
    cudaError_t e = set_smem(k_argmin_batch<KP, NT>, sm, s);
    if (e != cudaSuccess) return e;
    static int grid = 0;
    if (!grid) grid = persistent_grid(k_argmin_batch<KP, NT>, NT, sm);
    k_argmin_batch<KP, NT><<<grid, NT, sm, s>>>(fa, c);
    return cudaGetLastError();
}

template <int KP, int L, int NT>
cudaError_t launch_refine(const CostArgs* fa, const BatchCtl& c, cudaStream_t s) {
    static int grid = 0;
    if (!grid) grid = persistent_grid(k_refine_batch<KP, L, NT>, NT, 0);
    k_refine_batch<KP, L, NT><<<grid, NT, 0, s>>>(fa, c);
    return cudaGetLastError();
}

template <int KP, int NT>
cudaError_t launch_refine_t(const CostArgs* fa, const BatchCtl& c, cudaStream_t s) {
    const size_t sm = refine_smem_bytes<KP, NT>();
    cudaError_t e = set_smem(k_refine_t_batch<KP, NT>, sm, s);
    if (e != cudaSuccess) return e;
    static int grid = 0;
    if (!grid) grid = persistent_grid(k_refine_t_batch<KP, NT>, NT, sm);
    k_refine_t_batch<KP, NT><<<grid, NT, sm, s>>>(fa, c);
    return cudaGetLastError();
}

template <int KP>
cudaError_t launch_select(const LearnArgs* la, const BatchCtl& c, cudaStream_t s) {
    static int grid = 0;
    if (!grid) grid = persistent_grid(k_select_batch<KP>, 128, 0);
    k_select_batch<KP><<<grid, 128, 0, s>>>(la, c);
    return cudaGetLastError();
}

template <int KP>
cudaError_t argmin_nt(const CostArgs* fa, const BatchCtl& c, int nt, cudaStream_t s) {
    switch (nt) {
        case 64: return launch_argmin<KP, 64>(fa, c, s);
        case 256: return launch_argmin<KP, 256>(fa, c, s);
        default: return launch_argmin<KP, 128>(fa, c, s);
    }
}

template <int KP, int L>
cudaError_t refine_nt(const CostArgs* fa, const BatchCtl& c, int nt, cudaStream_t s) {
    switch (nt) {
        case 64: return launch_refine<KP, L, 64>(fa, c, s);
        case 256: return launch_refine<KP, L, 256>(fa, c, s);
        default: return launch_refine<KP, L, 128>(fa, c, s);
    }
}

template <int KP>
cudaError_t refine_l(const CostArgs* fa, const BatchCtl& c, int L, int nt, cudaStream_t s) {
    if (L == 0) {   // a point per thread
        switch (nt) {
            case 64: return launch_refine_t<KP, 64>(fa, c, s);
            case 256: return launch_refine_t<KP, 256>(fa, c, s);
            default: return launch_refine_t<KP, 128>(fa, c, s);
        }
    }
    switch (L) {
        case 4: return refine_nt<KP, 4>(fa, c, nt, s);
        case 8: return refine_nt<KP, 8>(fa, c, nt, s);
        case 16: return refine_nt<KP, 16>(fa, c, nt, s);
        default: return refine_nt<KP, 32>(fa, c, nt, s);
    }
}

}  // namespace

cudaError_t hf_launch_argmin_batch(const CostArgs* fa, const BatchCtl& c, int kp, int nt, cudaStream_t s) {
    switch (kp) {
        case 4: return argmin_nt<4>(fa, c, nt, s);
        case 9: return argmin_nt<9>(fa, c, nt, s);
        default: return argmin_nt<17>(fa, c, nt, s);
    }
}

cudaError_t hf_launch_refine_batch(const CostArgs* fa, const BatchCtl& c, int kp, int L, int nt, cudaStream_t s) {
    switch (kp) {
        case 4: return refine_l<4>(fa, c, L, nt, s);
        case 9: return refine_l<9>(fa, c, L, nt, s);
        default: return refine_l<17>(fa, c, L, nt, s);
    }
}

cudaError_t hf_launch_select_batch(const LearnArgs* la, const BatchCtl& c, int kp, cudaStream_t s) {
    switch (kp) {
        case 4: return launch_select<4>(la, c, s);
        case 9: return launch_select<9>(la, c, s);
        default: return launch_select<17>(la, c, s);
    }
}
