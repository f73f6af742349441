// hf_api.cu - the C ABI: argument checks, device memory owned by the context, launches on the
// context's stream, error latching and per-kernel event timing.
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <string>

#include "hf_internal.cuh"

namespace {
thread_local std::string g_create_err;


cudaMemcpyKind kind_in(int mem_kind) { return mem_kind == HF_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice; }

int check_kind(hf_ctx* c, int mem_kind) {
    if (mem_kind != HF_HOST && mem_kind != HF_DEVICE) return hf_set_err(c, HF_ERR_INVALID_ARG, "mem_kind must be HF_HOST or HF_DEVICE");
    return HF_OK;
}

// Uploads also take HF_HOST_ASYNC: pinned host memory copied without waiting.
int check_upload_kind(hf_ctx* c, int mem_kind) {
    if (mem_kind != HF_HOST && mem_kind != HF_DEVICE && mem_kind != HF_HOST_ASYNC)
        return hf_set_err(c, HF_ERR_INVALID_ARG, "mem_kind must be HF_HOST, HF_DEVICE or HF_HOST_ASYNC");
    return HF_OK;
}

// Wait for the stream, then report and clear the device error word.
int sync_and_check(hf_ctx* c) {
    cudaError_t e = cudaMemcpyAsync(c->errw_host, c->errw.p, sizeof(uint32_t), cudaMemcpyDeviceToHost, c->stream);
    if (e != cudaSuccess) return hf_cuda_err(c, e, "read device error word");
    e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return hf_cuda_err(c, e, "stream synchronize");
    const uint32_t w = *c->errw_host;
    if (w) {
        cudaMemsetAsync(c->errw.p, 0, sizeof(uint32_t), c->stream);
        cudaStreamSynchronize(c->stream);
        if (w & HF_DEV_ERR_TIMEOUT) return hf_set_err(c, HF_ERR_TIMEOUT, "a bounded device wait expired");
        if (w & HF_DEV_ERR_BAD_HYP) return hf_set_err(c, HF_ERR_INVALID_ARG, "a hypothesis is not unit length (|h| - 1 > 1e-3)");
        if (w & HF_DEV_ERR_BAD_NBR) return hf_set_err(c, HF_ERR_INVALID_ARG, "a neighbour index is outside [0, N)");
        return hf_set_err(c, HF_ERR_CUDA, "device error word 0x%x", w);
    }
    return HF_OK;
}

int ready(hf_ctx* c) {
    if (!c) return HF_ERR_INVALID_ARG;
    if (c->V <= 0) return hf_set_err(c, HF_ERR_NOT_UPLOADED, "views not uploaded");
    if (c->N <= 0) return hf_set_err(c, HF_ERR_NOT_UPLOADED, "points not uploaded");
    return HF_OK;
}

// K1 over the uploaded scene into the context's scratch
int run_project(hf_ctx* c) {
    const int Vw = hf_mask_words(c->V);
    int rc;
    if ((rc = hf_ensure(c, c->samp, (size_t)c->N * hf_view_pairs(c->V) * sizeof(float4)))) return rc;
    if ((rc = hf_ensure(c, c->ab, (size_t)c->N * hf_view_pairs(c->V) * sizeof(float4)))) return rc;
    if ((rc = hf_ensure(c, c->vmask, (size_t)c->N * Vw * sizeof(unsigned long long)))) return rc;
    if ((rc = hf_ensure(c, c->work, sizeof(unsigned long long)))) return rc;
    cudaError_t e = cudaMemsetAsync(c->work.p, 0, sizeof(unsigned long long), c->stream);
    if (e != cudaSuccess) return hf_cuda_err(c, e, "clear work counter");
    ProjectArgs pa{(const float*)c->pts.p, c->N, (const float*)c->cams.p, c->V, c->W, c->Hh,
                   (const float*)c->angle.p, c->conf.p, c->conf_dtype == HF_F16 ? 1 : 0, c->cfg.top_k_views,
                   (float2*)c->samp.p, (float2*)c->ab.p, (unsigned long long*)c->vmask.p, (unsigned long long*)c->work.p, nullptr,
                   (const float2*)c->amap.p};
    return run_launch(c, "k_project", [&] { return hf_launch_project(pa, c->stream); });
}
}  // namespace

int hf_set_err(hf_ctx* c, int code, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (c) c->err = buf;
    else g_create_err = buf;
    return code;
}

int hf_cuda_err(hf_ctx* c, cudaError_t e, const char* what) {
    return hf_set_err(c, e == cudaErrorMemoryAllocation ? HF_ERR_OOM : HF_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

// Allocation-failure hook: with g_fail_after = n >= 0 the (n + 1)-th device allocation of a context
// from then on reports out-of-memory (once); -1 disables it.
static std::atomic<int> g_fail_after{-1};

int hf_ensure(hf_ctx* c, DevBuf& b, size_t bytes) {
    if (bytes <= b.cap) return HF_OK;
    if (b.p) {
        cudaError_t e = cudaStreamSynchronize(c->stream);
        if (e != cudaSuccess) return hf_cuda_err(c, e, "synchronize before reallocation");
        cudaFree(b.p);
        c->dev_bytes -= (long long)b.cap;
        b.p = nullptr;
        b.cap = 0;
    }
    for (int n = g_fail_after.load(); n >= 0;) {   // the hook: count this allocation down
        if (g_fail_after.compare_exchange_weak(n, n - 1)) {
            if (n == 0) return hf_set_err(c, HF_ERR_OOM, "cudaMalloc of %zu bytes failed: injected out-of-memory", bytes);
            break;
        }
    }
    cudaError_t e = cudaMalloc(&b.p, bytes);
    if (e != cudaSuccess) {
        b.p = nullptr;
        cudaGetLastError();
        return hf_set_err(c, HF_ERR_OOM, "cudaMalloc of %zu bytes failed: %s", bytes, cudaGetErrorString(e));
    }
    b.cap = bytes;
    c->dev_bytes += (long long)bytes;
    return HF_OK;
}

CostArgs hf_cost_args(const hf_ctx* c) {
    CostArgs a{};
    a.pts = (const float*)c->pts.p;
    a.N = c->N;
    a.nbr = (const int32_t*)c->nbr.p;
    a.k = c->k;
    a.cams = (const float*)c->cams.p;
    a.V = c->V;
    a.samp = (const float2*)c->samp.p;
    a.ab = (const float2*)c->ab.p;
    a.vmask = (const unsigned long long*)c->vmask.p;
    a.Vw = hf_mask_words(c->V);
    a.vthr = (const float*)c->vthr.p;
    a.hyps = (const float*)c->hyps.p;
    a.H = c->cfg.H;
    a.Hpad = hf_hpad(c->cfg.H);
    a.rot = (const float2*)c->rot.p;
    a.T = c->cfg.T;
    const int tk = c->cfg.top_k_views;
    a.L = hf_cost_lanes(tk > 0 && tk < c->V ? tk : c->V, c->k);
    a.qtab = (const float4*)c->qtab.p;
    a.Hq = hf_hq(c->cfg.H);
    a.best_idx = (int32_t*)c->best.p;
    return a;
}

extern "C" {

int hair_fuse_create(hf_ctx** out, const hf_config* cfg, void* cuda_stream) {
    if (!out || !cfg) return hf_set_err(nullptr, HF_ERR_INVALID_ARG, "null out or cfg");
    *out = nullptr;
    if (cfg->H < 1 || cfg->H > HF_MAX_H) return hf_set_err(nullptr, HF_ERR_INVALID_ARG, "H=%d outside [1, %d]", cfg->H, HF_MAX_H);
    if (cfg->k < 0 || cfg->k > HF_MAX_K) return hf_set_err(nullptr, HF_ERR_INVALID_ARG, "k=%d outside [0, %d]", cfg->k, HF_MAX_K);
    if (cfg->T < 0 || cfg->T > HF_MAX_T) return hf_set_err(nullptr, HF_ERR_INVALID_ARG, "T=%d outside [0, %d]", cfg->T, HF_MAX_T);
    if (cfg->top_k_views < 0 || cfg->top_k_views > HF_MAX_TOPK)
        return hf_set_err(nullptr, HF_ERR_INVALID_ARG, "top_k_views=%d outside [0, %d]", cfg->top_k_views, HF_MAX_TOPK);
    hf_ctx* c = new hf_ctx();
    c->cfg = *cfg;
    c->stream = (cudaStream_t)cuda_stream;
    cudaError_t e = cudaGetDevice(&c->device);
    if (e == cudaSuccess) e = cudaMallocHost(&c->errw_host, sizeof(uint32_t));
    if (e != cudaSuccess) {
        hf_set_err(nullptr, HF_ERR_CUDA, "CUDA unavailable: %s", cudaGetErrorString(e));
        cudaGetLastError();
        delete c;
        return HF_ERR_CUDA;
    }
    int rc = hf_ensure(c, c->errw, sizeof(uint32_t));
    if (rc == HF_OK) {
        e = cudaMemsetAsync(c->errw.p, 0, sizeof(uint32_t), c->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
        if (e != cudaSuccess) rc = hf_cuda_err(c, e, "init error word");
    }
    if (rc != HF_OK) {
        hf_set_err(nullptr, rc, "%s", c->err.c_str());
        hair_fuse_destroy(c);
        return rc;
    }
    *out = c;
    return HF_OK;
}

int hair_fuse_set_stream(hf_ctx* c, void* cuda_stream) {
    if (!c) return HF_ERR_INVALID_ARG;
    c->stream = (cudaStream_t)cuda_stream;
    return HF_OK;
}

int hair_fuse_upload_views(hf_ctx* c, int V, int width, int height, const float* cams, const float* angle,
                           const void* conf, int conf_dtype, int mem_kind) {
    if (!c) return HF_ERR_INVALID_ARG;
    int rc;
    if ((rc = check_upload_kind(c, mem_kind))) return rc;
    if (V < 1 || width < 1 || height < 1) return hf_set_err(c, HF_ERR_INVALID_ARG, "V, width, height must be >= 1");
    if (!cams || !angle || !conf) return hf_set_err(c, HF_ERR_INVALID_ARG, "null view pointer");
    if (conf_dtype != HF_F32 && conf_dtype != HF_F16) return hf_set_err(c, HF_ERR_INVALID_ARG, "conf_dtype must be HF_F32 or HF_F16");
    if ((long long)width * height > (1LL << 31)) return hf_set_err(c, HF_ERR_SHAPE, "map larger than 2^31 pixels");
    if (width > (1 << 22) || height > (1 << 22)) return hf_set_err(c, HF_ERR_SHAPE, "map side above 2^22 pixels");
    const size_t npx = (size_t)V * width * height;
    const size_t cb = conf_dtype == HF_F16 ? 2 : 4;
    if ((rc = hf_ensure(c, c->cams, (size_t)V * 16 * sizeof(float)))) return rc;
    if ((rc = hf_ensure(c, c->angle, npx * sizeof(float)))) return rc;
    if ((rc = hf_ensure(c, c->conf, npx * cb))) return rc;
    if ((rc = hf_ensure(c, c->amap, npx * sizeof(float2)))) return rc;
    cudaError_t e = cudaMemcpyAsync(c->cams.p, cams, (size_t)V * 16 * sizeof(float), kind_in(mem_kind), c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(c->angle.p, angle, npx * sizeof(float), kind_in(mem_kind), c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(c->conf.p, conf, npx * cb, kind_in(mem_kind), c->stream);
    if (e != cudaSuccess) return hf_cuda_err(c, e, "upload views");
    // the kernels gather (angle, confidence) pairs: one interleaved copy makes each an 8-byte read
    if ((rc = run_launch(c, "k_interleave", [&] {
             return hf_launch_interleave((const float*)c->angle.p, c->conf.p, conf_dtype == HF_F16 ? 1 : 0, npx,
                                         (float2*)c->amap.p, c->stream);
         })))
        return rc;
    if (mem_kind == HF_HOST && (e = cudaStreamSynchronize(c->stream)) != cudaSuccess) return hf_cuda_err(c, e, "upload views");
    c->V = V;
    c->W = width;
    c->Hh = height;
    c->conf_dtype = conf_dtype;
    ++c->views_gen;
    return HF_OK;
}

int hair_fuse_upload_points(hf_ctx* c, int N, const float* xyz, const int32_t* nbr, int mem_kind) {
    if (!c) return HF_ERR_INVALID_ARG;
    int rc;
    if ((rc = check_upload_kind(c, mem_kind))) return rc;
    const int k = c->cfg.k;
    if (N < 1) return hf_set_err(c, HF_ERR_INVALID_ARG, "N must be >= 1");
    if (k >= N) return hf_set_err(c, HF_ERR_INVALID_ARG, "k=%d must be < N=%d", k, N);
    if (!xyz || (k > 0 && !nbr)) return hf_set_err(c, HF_ERR_INVALID_ARG, "null point pointer");
    if ((rc = hf_ensure(c, c->pts, (size_t)N * 3 * sizeof(float)))) return rc;
    if (k > 0 && (rc = hf_ensure(c, c->nbr, (size_t)N * k * sizeof(int32_t)))) return rc;
    c->N = 0;
    cudaError_t e = cudaMemcpyAsync(c->pts.p, xyz, (size_t)N * 3 * sizeof(float), kind_in(mem_kind), c->stream);
    if (e == cudaSuccess && k > 0) e = cudaMemcpyAsync(c->nbr.p, nbr, (size_t)N * k * sizeof(int32_t), kind_in(mem_kind), c->stream);
    if (e != cudaSuccess) return hf_cuda_err(c, e, "upload points");
    if (k > 0) {
        rc = run_launch(c, "k_check_nbr", [&] { return hf_launch_check_nbr((const int32_t*)c->nbr.p, (long long)N * k, N, (uint32_t*)c->errw.p, c->stream); });
        if (rc) return rc;
        rc = run_launch(c, "k_order_nbr", [&] { return hf_launch_order_nbr((int32_t*)c->nbr.p, N, k, c->stream); });
        if (rc) return rc;
    }
    if ((rc = sync_and_check(c))) return rc;
    c->N = N;
    c->k = k;
    return HF_OK;
}

namespace {

// Fusion of the points first .. first + count - 1 (all points when ranged is false): every point is
// projected (the range's neighbours need their samples), the argmin and refinement run on the range,
// and outputs are written to rows 0 .. count - 1.
int fuse_impl(hf_ctx* c, const float* hyps, bool ranged, int first, int count, float* dir_out, float* cost_out,
              int32_t* idx_out, uint8_t* status_out, int mem_kind) {
    int rc;
    if ((rc = ready(c))) return rc;
    if ((rc = check_kind(c, mem_kind))) return rc;
    if (!dir_out) return hf_set_err(c, HF_ERR_INVALID_ARG, "dir_out is required");
    const int H = c->cfg.H, T = c->cfg.T, V = c->V;
    if (ranged && (first < 0 || count < 0 || (long long)first + count > c->N))
        return hf_set_err(c, HF_ERR_INVALID_ARG, "range [%d, %d + %d) outside [0, %d)", first, first, count, c->N);
    if (!ranged) {
        first = 0;
        count = c->N;
    }
    if (count == 0) return HF_OK;
    const int R = count;
    const int Hpad = hf_hpad(H);
    const float* hyps_dev = nullptr;
    if (hyps && mem_kind == HF_HOST) {
        for (int m = 0; m < H; ++m) {
            const double n = std::sqrt((double)hyps[3 * m] * hyps[3 * m] + (double)hyps[3 * m + 1] * hyps[3 * m + 1] +
                                       (double)hyps[3 * m + 2] * hyps[3 * m + 2]);
            if (!(std::fabs(n - 1.0) <= 1e-3)) return hf_set_err(c, HF_ERR_INVALID_ARG, "hypothesis %d is not unit length (|h| = %g)", m, n);
        }
        if ((rc = hf_ensure(c, c->evald, (size_t)H * 3 * sizeof(float)))) return rc;
        cudaError_t e = cudaMemcpyAsync(c->evald.p, hyps, (size_t)H * 3 * sizeof(float), cudaMemcpyHostToDevice, c->stream);
        if (e != cudaSuccess) return hf_cuda_err(c, e, "copy hypotheses");
        hyps_dev = (const float*)c->evald.p;
    } else if (hyps) {
        hyps_dev = hyps;
    }
    if ((rc = hf_ensure(c, c->vthr, (size_t)V * sizeof(float)))) return rc;
    if ((rc = hf_ensure(c, c->hyps, (size_t)Hpad * 3 * sizeof(float)))) return rc;
    if ((rc = hf_ensure(c, c->rot, (size_t)(T > 0 ? T : 1) * sizeof(float2)))) return rc;
    if ((rc = hf_ensure(c, c->qtab, (size_t)V * hf_hq(H) * sizeof(float4)))) return rc;
    if ((rc = hf_ensure(c, c->best, (size_t)c->N * sizeof(int32_t)))) return rc;
    PrepArgs pr{(const float*)c->cams.p, V, hyps_dev, H, Hpad, T, (float*)c->hyps.p, (float*)c->vthr.p,
                (float2*)c->rot.p, (uint32_t*)c->errw.p, (float4*)c->qtab.p, hf_hq(H)};
    if ((rc = run_launch(c, "k_prep", [&] { return hf_launch_prep(pr, c->stream); }))) return rc;
    if ((rc = run_project(c))) return rc;

    float *d_dir = dir_out, *d_cost = cost_out;
    int32_t* d_idx = idx_out;
    uint8_t* d_status = status_out;
    if (mem_kind == HF_HOST) {
        const size_t bytes = (size_t)R * (3 * sizeof(float) + sizeof(float) + sizeof(int32_t) + 1);
        if ((rc = hf_ensure(c, c->outs, bytes))) return rc;
        char* base = (char*)c->outs.p;
        d_dir = (float*)base;
        d_cost = cost_out ? (float*)(base + (size_t)R * 12) : nullptr;
        d_idx = idx_out ? (int32_t*)(base + (size_t)R * 16) : nullptr;
        d_status = status_out ? (uint8_t*)(base + (size_t)R * 20) : nullptr;
    }
    CostArgs fa = hf_cost_args(c);
    fa.dir_out = d_dir;
    fa.cost_out = d_cost;
    fa.idx_out = d_idx;
    fa.status_out = d_status;
    if (ranged) {
        if ((rc = hf_ensure(c, c->rlist, 16 + (size_t)R * sizeof(int32_t)))) return rc;
        int* cnt = (int*)c->rlist.p;
        int32_t* lst = (int32_t*)((char*)c->rlist.p + 16);
        if ((rc = run_launch(c, "k_iota", [&] { return hf_launch_iota(lst, cnt, first, R, c->stream); }))) return rc;
        fa.list = lst;
        fa.list_count = cnt;
        fa.out_first = first;
    }
    if ((rc = run_launch(c, "k_argmin", [&] { return hf_launch_argmin(fa, c->stream); }))) return rc;
    if ((rc = run_launch(c, "k_refine", [&] { return hf_launch_refine(fa, c->stream); }))) return rc;
    if (mem_kind == HF_HOST) {
        cudaError_t e = cudaMemcpyAsync(dir_out, d_dir, (size_t)R * 12, cudaMemcpyDeviceToHost, c->stream);
        if (e == cudaSuccess && cost_out) e = cudaMemcpyAsync(cost_out, d_cost, (size_t)R * 4, cudaMemcpyDeviceToHost, c->stream);
        if (e == cudaSuccess && idx_out) e = cudaMemcpyAsync(idx_out, d_idx, (size_t)R * 4, cudaMemcpyDeviceToHost, c->stream);
        if (e == cudaSuccess && status_out) e = cudaMemcpyAsync(status_out, d_status, (size_t)R, cudaMemcpyDeviceToHost, c->stream);
        if (e != cudaSuccess) return hf_cuda_err(c, e, "copy outputs");
        return sync_and_check(c);
    }
    return HF_OK;
}

}  // namespace

int hair_fuse_fuse_directions(hf_ctx* c, const float* hyps, float* dir_out, float* cost_out, int32_t* idx_out,
                              uint8_t* status_out, int mem_kind) {
    return fuse_impl(c, hyps, false, 0, 0, dir_out, cost_out, idx_out, status_out, mem_kind);
}

int hair_fuse_fuse_range(hf_ctx* c, int first, int count, const float* hyps, float* dir_out, float* cost_out,
                         int32_t* idx_out, uint8_t* status_out, int mem_kind) {
    return fuse_impl(c, hyps, true, first, count, dir_out, cost_out, idx_out, status_out, mem_kind);
}

int hair_fuse_eval_costs(hf_ctx* c, int M, const float* dirs, float* cost_out, int mem_kind) {
    int rc;
    if ((rc = ready(c))) return rc;
    if ((rc = check_kind(c, mem_kind))) return rc;
    if (M < 1 || !dirs || !cost_out) return hf_set_err(c, HF_ERR_INVALID_ARG, "M >= 1 and non-null dirs, cost_out required");
    const int V = c->V, N = c->N;
    // thresholds (and the hypotheses, unused here) come from the prep kernel
    const int Hpad = hf_hpad(c->cfg.H);
    if ((rc = hf_ensure(c, c->vthr, (size_t)V * sizeof(float)))) return rc;
    if ((rc = hf_ensure(c, c->hyps, (size_t)Hpad * 3 * sizeof(float)))) return rc;
    if ((rc = hf_ensure(c, c->rot, (size_t)(c->cfg.T > 0 ? c->cfg.T : 1) * sizeof(float2)))) return rc;
    PrepArgs pr{(const float*)c->cams.p, V, nullptr, c->cfg.H, Hpad, c->cfg.T, (float*)c->hyps.p, (float*)c->vthr.p,
                (float2*)c->rot.p, (uint32_t*)c->errw.p, nullptr, 0};
    if ((rc = run_launch(c, "k_prep", [&] { return hf_launch_prep(pr, c->stream); }))) return rc;
    if ((rc = run_project(c))) return rc;
    const float* d_dirs = dirs;
    float* d_cost = cost_out;
    const size_t nd = (size_t)N * M;
    if (mem_kind == HF_HOST) {
        if ((rc = hf_ensure(c, c->evald, nd * 3 * sizeof(float)))) return rc;
        if ((rc = hf_ensure(c, c->outs, nd * sizeof(float)))) return rc;
        cudaError_t e = cudaMemcpyAsync(c->evald.p, dirs, nd * 12, cudaMemcpyHostToDevice, c->stream);
        if (e != cudaSuccess) return hf_cuda_err(c, e, "copy directions");
        d_dirs = (const float*)c->evald.p;
        d_cost = (float*)c->outs.p;
    }
    EvalArgs ea{hf_cost_args(c), d_dirs, M, d_cost};
    if ((rc = run_launch(c, "k_eval", [&] { return hf_launch_eval(ea, c->stream); }))) return rc;
    if (mem_kind == HF_HOST) {
        cudaError_t e = cudaMemcpyAsync(cost_out, d_cost, nd * 4, cudaMemcpyDeviceToHost, c->stream);
        if (e != cudaSuccess) return hf_cuda_err(c, e, "copy costs");
        return sync_and_check(c);
    }
    return HF_OK;
}

int hair_fuse_fibonacci_hemisphere(int H, float* out) {
    if (H < 1 || H > HF_MAX_H || !out) return hf_set_err(nullptr, HF_ERR_INVALID_ARG, "H outside [1, %d] or null out", HF_MAX_H);
    float* d = nullptr;
    cudaError_t e = cudaMalloc(&d, (size_t)H * 3 * sizeof(float));
    if (e == cudaSuccess) e = hf_launch_fib(H, d, nullptr);
    if (e == cudaSuccess) e = cudaMemcpy(out, d, (size_t)H * 3 * sizeof(float), cudaMemcpyDeviceToHost);
    if (d) cudaFree(d);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return hf_set_err(nullptr, HF_ERR_CUDA, "fibonacci hemisphere: %s", cudaGetErrorString(e));
    }
    return HF_OK;
}

int hair_fuse_fail_alloc_after(int n) {
    g_fail_after.store(n < 0 ? -1 : n);
    return HF_OK;
}

int hair_fuse_sync(hf_ctx* c) {
    if (!c) return HF_ERR_INVALID_ARG;
    return sync_and_check(c);
}

int hair_fuse_profile(hf_ctx* c, int enable) {
    if (!c) return HF_ERR_INVALID_ARG;
    cudaStreamSynchronize(c->stream);
    for (auto& r : c->prof_recs) {
        cudaEventDestroy(r.beg);
        cudaEventDestroy(r.end);
    }
    c->prof_recs.clear();
    c->prof = enable != 0;
    return HF_OK;
}

int hair_fuse_profile_read(hf_ctx* c, hf_kernel_time* out, int max_entries) {
    if (!c) return HF_ERR_INVALID_ARG;
    cudaError_t e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return hf_cuda_err(c, e, "synchronize for profile");
    std::map<std::string, std::pair<int, double>> agg;
    std::vector<std::string> order;
    for (auto& r : c->prof_recs) {
        float ms = 0.0f;
        cudaEventElapsedTime(&ms, r.beg, r.end);
        if (!agg.count(r.name)) order.push_back(r.name);
        agg[r.name].first += 1;
        agg[r.name].second += ms;
    }
    int n = 0;
    for (auto& name : order) {
        if (out && n < max_entries) {
            std::snprintf(out[n].name, sizeof out[n].name, "%s", name.c_str());
            out[n].launches = agg[name].first;
            out[n].total_ms = agg[name].second;
        }
        ++n;
    }
    return n;
}

int hair_fuse_work(hf_ctx* c, long long* point_views) {
    if (!c || !point_views) return HF_ERR_INVALID_ARG;
    *point_views = 0;
    if (!c->work.p) return HF_OK;
    unsigned long long w = 0;
    cudaError_t e = cudaMemcpyAsync(&w, c->work.p, sizeof w, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return hf_cuda_err(c, e, "read work counter");
    *point_views = (long long)w;
    return HF_OK;
}

int hair_fuse_stats(const hf_ctx* c, long long* device_bytes, long long* launches) {
    if (!c) return HF_ERR_INVALID_ARG;
    if (device_bytes) *device_bytes = c->dev_bytes;
    if (launches) *launches = c->launches;
    return HF_OK;
}

void hair_fuse_destroy(hf_ctx* c) {
    if (!c) return;
    cudaStreamSynchronize(c->stream);
    for (auto& r : c->prof_recs) {
        cudaEventDestroy(r.beg);
        cudaEventDestroy(r.end);
    }
    DevBuf* bufs[] = {&c->cams, &c->angle, &c->conf, &c->amap, &c->depth, &c->dmap, &c->vmap, &c->fprec, &c->phg, &c->gabor, &c->gbank, &c->rlist, &c->pts, &c->nbr, &c->samp, &c->ab, &c->vmask,
                      &c->vthr, &c->qtab, &c->best, &c->hyps, &c->rot, &c->outs, &c->evald, &c->errw, &c->work, &c->feat, &c->prop, &c->lmisc};
    for (DevBuf* b : bufs)
        if (b->p) cudaFree(b->p);
    if (c->errw_host) cudaFreeHost(c->errw_host);
    delete c;
}

const char* hair_fuse_last_error(const hf_ctx* c) {
    if (!c) return g_create_err.c_str();
    return c->err.c_str();
}

}  // extern "C"
