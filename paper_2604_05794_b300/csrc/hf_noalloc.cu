// hf_noalloc.cu - direction fusion for callers that cannot allocate device memory.
//
// Some callers must not call cudaMalloc: plugin hosts whose enqueue hooks forbid allocation,
// processes whose device memory is owned by a framework's caching allocator, or real-time code
// with a fixed memory budget.  hair_fuse_fuse_directions_noalloc() serves them: the caller passes
// every input and output as device memory, and the scratch the fusion needs between its kernels
// (per point-view samples, the points' view-set masks, the hypothesis table, the argmin's
// hand-off to the refinement, a few per-scene constants)
// lives in one file-scope __device__ array of fixed size.  Every GPU that loads this library
// holds that array until the process exits.
//
// Host code never dereferences the array's symbol: the symbol is only a host-side stand-in for
// the device array, so its device address is looked up with cudaGetSymbolAddress once per device
// (with that device current) and that address is what the kernels receive.
#include <mutex>

#include "hf_internal.cuh"

namespace {

// Limits of the static scratch (see the header for the caller-facing statement).
constexpr long long kMaxPointViews = 1LL << 20;   // N * V, V rounded up to even (views stored in pairs)
constexpr long long kMaxPoints = 1LL << 18;       // N
constexpr int kMaxViews = 1024;                   // V
constexpr long long kMaxTable = 1LL << 16;        // V * Hq (the argmin's hypothesis-pair table)

constexpr size_t align256(size_t x) { return (x + 255) / 256 * 256; }
// samples and projection ratios: N V entries each
constexpr size_t kSampBytes = align256((size_t)kMaxPointViews * sizeof(float2));
constexpr size_t kAbBytes = align256((size_t)kMaxPointViews * sizeof(float2));
// view-set masks: N rows of ceil(V / 64) words, at most N words when V <= 64 and fewer beyond
constexpr size_t kMaskBytes = align256((size_t)kMaxPoints * sizeof(unsigned long long));
constexpr size_t kQtabBytes = align256((size_t)kMaxTable * sizeof(float4));
constexpr size_t kBestBytes = align256((size_t)kMaxPoints * sizeof(int32_t));   // argmin -> refinement
constexpr size_t kVthrBytes = align256(kMaxViews * sizeof(float));
constexpr size_t kHypsBytes = align256(HF_MAX_H * 3 * sizeof(float));
constexpr size_t kRotBytes = align256(HF_MAX_T * sizeof(float2));
constexpr size_t kWorkBytes = 256;
constexpr size_t kErrBytes = 256;
constexpr size_t kScratchBytes = kSampBytes + kAbBytes + kMaskBytes + kQtabBytes + kBestBytes + kVthrBytes + kHypsBytes +
                                 kRotBytes + kWorkBytes + kErrBytes;
// the size the header states
static_assert(kScratchBytes == 20988672, "static scratch size differs from the documented 20,988,672 bytes");

// The shared scratch: 20,988,672 bytes (20.0 MiB), reused (and overwritten) by every call on this device.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
unsigned char* g_scratch_dev[kMaxDevices] = {nullptr};

// the message is read back with hair_fuse_last_error(NULL)
int fail(int code, const char* msg) { return hf_set_err(nullptr, code, "%s", msg); }

// Device address of the scratch on the current device; looked up on the first call per device.
int scratch_for_current_device(unsigned char** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail(HF_ERR_CUDA, cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices) return fail(HF_ERR_CUDA, "device ordinal beyond the supported range");
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_dev[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || p == nullptr) {
            cudaGetLastError();
            return fail(HF_ERR_CUDA, "cudaGetSymbolAddress of the static scratch failed");
        }
        g_scratch_dev[dev] = (unsigned char*)p;
    }
    *out = g_scratch_dev[dev];
    return HF_OK;
}

}  // namespace

extern "C" int hair_fuse_fuse_directions_noalloc(const hf_config* cfg, int N, int V, int width, int height,
                                                 const float* cams, const float* angle, const void* conf,
                                                 int conf_dtype, const float* xyz, const int32_t* nbr,
                                                 const float* hyps, float* dir_out, float* cost_out,
                                                 int32_t* idx_out, uint8_t* status_out, void* cuda_stream) {
    if (!cfg) return fail(HF_ERR_INVALID_ARG, "null cfg");
    const int H = cfg->H, k = cfg->k, T = cfg->T, top_k = cfg->top_k_views;
    if (H < 1 || H > HF_MAX_H || k < 0 || k > HF_MAX_K || T < 0 || T > HF_MAX_T || top_k < 0 || top_k > HF_MAX_TOPK)
        return fail(HF_ERR_INVALID_ARG, "configuration outside the documented limits");
    if (N < 1 || V < 1 || width < 1 || height < 1 || k >= N)
        return fail(HF_ERR_INVALID_ARG, "need N >= 1, V >= 1, width, height >= 1 and k < N");
    if (!cams || !angle || !conf || !xyz || (k > 0 && !nbr) || !dir_out)
        return fail(HF_ERR_INVALID_ARG, "null input or dir_out pointer");
    if (conf_dtype != HF_F32 && conf_dtype != HF_F16) return fail(HF_ERR_INVALID_ARG, "conf_dtype must be HF_F32 or HF_F16");
    if ((long long)N * 2 * hf_view_pairs(V) > kMaxPointViews)
        return fail(HF_ERR_SHAPE, "N * V (V rounded up to even) exceeds the static scratch limit of 1048576 point-views");
    if (N > kMaxPoints) return fail(HF_ERR_SHAPE, "N exceeds the static scratch limit of 262144 points");
    if (V > kMaxViews) return fail(HF_ERR_SHAPE, "V exceeds the static scratch limit of 1024 views");
    if ((long long)V * hf_hq(H) > kMaxTable)
        return fail(HF_ERR_SHAPE, "V * H (H rounded up to a multiple of 32) exceeds the static scratch limit of 65536");
    if ((long long)width * height > (1LL << 31)) return fail(HF_ERR_SHAPE, "map larger than 2^31 pixels");
    const int Vw = hf_mask_words(V), Hpad = hf_hpad(H);
    if ((size_t)N * Vw * sizeof(unsigned long long) > kMaskBytes)
        return fail(HF_ERR_SHAPE, "the view-set masks exceed the static scratch");

    unsigned char* base = nullptr;
    int rc = scratch_for_current_device(&base);
    if (rc) return rc;
    float2* samp = (float2*)base;
    float2* ab = (float2*)(base + kSampBytes);
    unsigned char* at = base + kSampBytes + kAbBytes;
    unsigned long long* vmask = (unsigned long long*)at;
    at += kMaskBytes;
    float4* qtab = (float4*)at;
    at += kQtabBytes;
    int32_t* best = (int32_t*)at;
    at += kBestBytes;
    float* vthr = (float*)at;
    at += kVthrBytes;
    float* hy = (float*)at;
    at += kHypsBytes;
    float2* rot = (float2*)at;
    at += kRotBytes;
    unsigned long long* work = (unsigned long long*)at;
    uint32_t* errw = (uint32_t*)((unsigned char*)work + kWorkBytes);
    cudaStream_t s = (cudaStream_t)cuda_stream;

    // the counter and the error word keep the previous call's values: clear them
    cudaError_t e = cudaMemsetAsync(work, 0, kWorkBytes + kErrBytes, s);
    if (e == cudaSuccess && k > 0) e = hf_launch_check_nbr(nbr, (long long)N * k, N, errw, s);
    uint32_t host_err = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&host_err, errw, sizeof host_err, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return fail(HF_ERR_CUDA, cudaGetErrorString(e));
    if (host_err & HF_DEV_ERR_BAD_NBR) return fail(HF_ERR_INVALID_ARG, "a neighbour index is outside [0, N)");

    PrepArgs pr{cams, V, hyps, H, Hpad, T, hy, vthr, rot, errw, qtab, hf_hq(H)};
    e = hf_launch_prep(pr, s);
    ProjectArgs pa{xyz, N, cams, V, width, height, angle, conf, conf_dtype == HF_F16 ? 1 : 0, top_k, samp, ab, vmask, work};
    if (e == cudaSuccess) e = hf_launch_project(pa, s);
    CostArgs fa{};
    fa.pts = xyz;
    fa.N = N;
    fa.nbr = nbr;
    fa.k = k;
    fa.cams = cams;
    fa.V = V;
    fa.samp = samp;
    fa.ab = ab;
    fa.vmask = vmask;
    fa.Vw = Vw;
    fa.vthr = vthr;
    fa.hyps = hy;
    fa.H = H;
    fa.Hpad = Hpad;
    fa.rot = rot;
    fa.T = T;
    fa.L = hf_cost_lanes(top_k > 0 && top_k < V ? top_k : V, k);
    fa.qtab = qtab;
    fa.Hq = hf_hq(H);
    fa.best_idx = best;
    fa.dir_out = dir_out;
    fa.cost_out = cost_out;
    fa.idx_out = idx_out;
    fa.status_out = status_out;
    if (e == cudaSuccess) e = hf_launch_fuse(fa, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&host_err, errw, sizeof host_err, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return fail(HF_ERR_CUDA, cudaGetErrorString(e));
    if (host_err & HF_DEV_ERR_BAD_HYP) return fail(HF_ERR_INVALID_ARG, "a hypothesis is not unit length (|h| - 1 > 1e-3)");
    return HF_OK;
}
