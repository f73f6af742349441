// hf_mlp_api.cu - C ABI of the learned proposal network and of the learned fusion path.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "hf_gemm.cuh"
#include "hf_internal.cuh"
#include "hf_mlp.cuh"

struct hf_mlp {
    cudaStream_t stream = nullptr;
    int max_batch = 0;
    std::string err;
    void* block = nullptr;                  // one allocation, carved below
    float *P = nullptr, *G = nullptr, *M = nullptr, *V = nullptr;
    MlpDev d{};
    long long* step = nullptr;
    float* loss_hist = nullptr;
    long long loss_cap = 0;
    uint32_t* errw = nullptr;
    uint32_t* errw_host = nullptr;
    int tm_batch = 0;                       // batch size the tensor maps were encoded for
    unsigned long long wait_ns = 0;         // limit of the inference kernel's waits (0: the default)
    CUtensorMap tm[TM_COUNT];
    cudaStream_t cap_stream = nullptr;      // non-blocking stream the training step is captured on
    cudaGraphExec_t graph = nullptr;        // captured training step and what it was captured for
    const void* g_X = nullptr;
    const void* g_T = nullptr;
    long long g_n = 0;
    int g_B = 0;
    uint64_t g_seed = 0;
    float g_lr = 0.0f;
};

namespace {

int mlp_err(hf_mlp* m, int code, const char* fmt, const char* detail = "") {
    char buf[512];
    std::snprintf(buf, sizeof buf, fmt, detail);
    if (m) m->err = buf;
    return hf_set_err(nullptr, code, "%s", buf);
}

int mlp_cuda(hf_mlp* m, cudaError_t e, const char* what) {
    cudaGetLastError();
    char buf[256];
    std::snprintf(buf, sizeof buf, "%s: %s", what, cudaGetErrorString(e));
    return mlp_err(m, e == cudaErrorMemoryAllocation ? HF_ERR_OOM : HF_ERR_CUDA, "%s", buf);
}

int mlp_sync_check(hf_mlp* m) {
    cudaError_t e = cudaMemcpyAsync(m->errw_host, m->errw, sizeof(uint32_t), cudaMemcpyDeviceToHost, m->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(m->stream);
    if (e != cudaSuccess) return mlp_cuda(m, e, "synchronize");
    if (*m->errw_host) {
        cudaMemsetAsync(m->errw, 0, sizeof(uint32_t), m->stream);
        cudaStreamSynchronize(m->stream);
        return mlp_err(m, HF_ERR_TIMEOUT, "%s", "a bounded device wait expired in the network kernels");
    }
    return HF_OK;
}

// tensor maps of the training buffers for batch size B
cudaError_t encode_maps(hf_mlp* m, int B) {
    if (m->tm_batch == B) return cudaSuccess;
    const MlpDev& d = m->d;
    struct { int id; const void* p; long long rows, cols; int box; } spec[TM_COUNT] = {
        {TM_X, d.Xb, B, 64, 128},      {TM_W1, d.W1b, 256, 64, 256},   {TM_H1, d.H1, B, 256, 128},
        {TM_W2, d.W2b, 256, 256, 256}, {TM_H2, d.H2, B, 256, 128},     {TM_W3P, d.W3pb, 16, 256, 16},
        {TM_H2T, d.H2T, 256, B, 128},  {TM_DZ3T, d.dZ3T, 16, B, 16},   {TM_DZ3, d.dZ3, B, 64, 128},
        {TM_W3T, d.W3Tb, 256, 64, 256}, {TM_DZ2T, d.dZ2T, 256, B, 128}, {TM_H1T, d.H1T, 256, B, 256},
        {TM_DZ2, d.dZ2, B, 256, 128},  {TM_W2T, d.W2Tb, 256, 256, 256}, {TM_DZ1T, d.dZ1T, 256, B, 128},
        {TM_XT, d.XTb, 64, B, 64}};
    for (auto& s : spec) {
        cudaError_t e = hf_make_tmap_bf16(&m->tm[s.id], s.p, s.rows, s.cols, s.box);
        if (e != cudaSuccess) return e;
    }
    m->tm_batch = B;
    return cudaSuccess;
}

MlpTrain train_args(hf_mlp* m, const uint16_t* X, const float* T, long long n, int B, uint64_t seed, float lr) {
    MlpTrain t{};
    t.d = m->d;
    std::memcpy(t.tm, m->tm, sizeof t.tm);
    t.P = m->P;
    t.G = m->G;
    t.M = m->M;
    t.V = m->V;
    t.X = X;
    t.T = T;
    t.n_samples = n;
    t.B = B;
    t.seed = seed;
    t.step = m->step;
    t.loss_hist = m->loss_hist;
    t.lr = lr;
    t.errw = m->errw;
    return t;
}

int check_batch(hf_mlp* m, int B) {
    if (B < 128 || B % 128 || B > m->max_batch)
        return mlp_err(m, HF_ERR_INVALID_ARG, "%s", "batch must be a multiple of 128 and at most max_batch");
    return HF_OK;
}


// loss history covers steps [0, loss_cap); grow (keeping values) when a run goes further
int ensure_loss(hf_mlp* m, long long upto) {
    if (upto <= m->loss_cap) return HF_OK;
    long long cap = m->loss_cap ? m->loss_cap : 1024;
    while (cap < upto) cap *= 2;
    float* nb = nullptr;
    cudaError_t e = cudaMalloc(&nb, cap * sizeof(float));
    if (e == cudaSuccess) e = cudaMemsetAsync(nb, 0, cap * sizeof(float), m->stream);
    if (e == cudaSuccess && m->loss_hist)
        e = cudaMemcpyAsync(nb, m->loss_hist, m->loss_cap * sizeof(float), cudaMemcpyDeviceToDevice, m->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(m->stream);
    if (e != cudaSuccess) {
        if (nb) cudaFree(nb);
        return mlp_cuda(m, e, "loss history");
    }
    if (m->loss_hist) cudaFree(m->loss_hist);
    m->loss_hist = nb;
    m->loss_cap = cap;
    if (m->graph) {   // the captured step refers to the old history buffer
        cudaGraphExecDestroy(m->graph);
        m->graph = nullptr;
    }
    return HF_OK;
}

}  // namespace

extern "C" {

long long hair_fuse_mlp_param_count(void) { return hf_mlp_param_count(); }

int hair_fuse_mlp_create(hf_mlp** out, int max_batch, void* cuda_stream) {
    if (!out) return hf_set_err(nullptr, HF_ERR_INVALID_ARG, "null out");
    *out = nullptr;
    if (max_batch < 128 || max_batch % 128 || max_batch > 65536)
        return hf_set_err(nullptr, HF_ERR_INVALID_ARG, "max_batch must be a multiple of 128 in [128, 65536]");
    hf_mlp* m = new hf_mlp();
    m->stream = (cudaStream_t)cuda_stream;
    m->max_batch = max_batch;
    const long long np = hf_mlp_param_count(), B = max_batch;
    // sizes in bytes of every carved buffer, each rounded to 256 bytes
    const size_t sz[] = {(size_t)np * 4, (size_t)np * 4, (size_t)np * 4, (size_t)np * 4,                 // P G M V
                         256 * 64 * 2, 256 * 256 * 2, 256 * 256 * 2, 16 * 256 * 2, 256 * 64 * 2,        // bf16 weights
                         3 * 256 * 4, 16 * 4,                                                            // w3f b3p
                         (size_t)B * 64 * 2, (size_t)B * 64 * 2, (size_t)B * 3 * 4,                      // Xb XTb Tb
                         (size_t)B * 256 * 4, (size_t)B * 256 * 4, (size_t)B * 16 * 4,                   // Z1 Z2 Z3
                         (size_t)B * 256 * 2, (size_t)B * 256 * 2, (size_t)B * 256 * 2, (size_t)B * 256 * 2,   // H1 H1T H2 H2T
                         (size_t)B * 64 * 2, (size_t)16 * B * 2, (size_t)B * 256 * 4,                    // dZ3 dZ3T dH
                         (size_t)B * 256 * 2, (size_t)B * 256 * 2, (size_t)B * 256 * 2, (size_t)B * 256 * 2,   // dZ2 dZ2T dZ1 dZ1T
                         256 * 16 * 4, 8, 4,                                                             // dW3T step errw
                         (size_t)64 * 256 * 256 * 4, (size_t)(B / 32 + 1) * 256 * 4};                    // parts bparts
    const int nbuf = sizeof sz / sizeof sz[0];
    size_t total = 0;
    for (int q = 0; q < nbuf; ++q) total += (sz[q] + 255) / 256 * 256;
    cudaError_t e = cudaMalloc(&m->block, total);
    if (e == cudaSuccess) e = cudaMemsetAsync(m->block, 0, total, m->stream);
    if (e == cudaSuccess) e = cudaMallocHost(&m->errw_host, sizeof(uint32_t));
    if (e == cudaSuccess) e = cudaStreamSynchronize(m->stream);
    if (e != cudaSuccess) {
        int rc = mlp_cuda(nullptr, e, "network buffers");
        if (m->block) cudaFree(m->block);
        delete m;
        return rc;
    }
    void* p[64];
    size_t off = 0;
    for (int q = 0; q < nbuf; ++q) {
        p[q] = (char*)m->block + off;
        off += (sz[q] + 255) / 256 * 256;
    }
    int q = 0;
    m->P = (float*)p[q++]; m->G = (float*)p[q++]; m->M = (float*)p[q++]; m->V = (float*)p[q++];
    MlpDev& d = m->d;
    d.W1b = (uint16_t*)p[q++]; d.W2b = (uint16_t*)p[q++]; d.W2Tb = (uint16_t*)p[q++]; d.W3pb = (uint16_t*)p[q++];
    d.W3Tb = (uint16_t*)p[q++]; d.w3f = (float*)p[q++]; d.b3p = (float*)p[q++];
    d.Xb = (uint16_t*)p[q++]; d.XTb = (uint16_t*)p[q++]; d.Tb = (float*)p[q++];
    d.Z1 = (float*)p[q++]; d.Z2 = (float*)p[q++]; d.Z3 = (float*)p[q++];
    d.H1 = (uint16_t*)p[q++]; d.H1T = (uint16_t*)p[q++]; d.H2 = (uint16_t*)p[q++]; d.H2T = (uint16_t*)p[q++];
    d.dZ3 = (uint16_t*)p[q++]; d.dZ3T = (uint16_t*)p[q++]; d.dH = (float*)p[q++];
    d.dZ2 = (uint16_t*)p[q++]; d.dZ2T = (uint16_t*)p[q++]; d.dZ1 = (uint16_t*)p[q++]; d.dZ1T = (uint16_t*)p[q++];
    d.dW3T = (float*)p[q++];
    m->step = (long long*)p[q++];
    m->errw = (uint32_t*)p[q++];
    d.parts = (float*)p[q++];
    d.bparts = (float*)p[q++];
    *out = m;
    return HF_OK;
}

void hair_fuse_mlp_destroy(hf_mlp* m) {
    if (!m) return;
    cudaStreamSynchronize(m->stream);
    if (m->graph) cudaGraphExecDestroy(m->graph);
    if (m->cap_stream) cudaStreamDestroy(m->cap_stream);
    if (m->block) cudaFree(m->block);
    if (m->loss_hist) cudaFree(m->loss_hist);
    if (m->errw_host) cudaFreeHost(m->errw_host);
    delete m;
}

int hair_fuse_mlp_init(hf_mlp* m, uint64_t seed) {
    if (!m) return HF_ERR_INVALID_ARG;
    const size_t np = (size_t)hf_mlp_param_count();
    cudaError_t e = hf_launch_init(m->P, seed, m->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(m->M, 0, np * 4, m->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(m->V, 0, np * 4, m->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(m->step, 0, 8, m->stream);
    if (e == cudaSuccess) e = hf_launch_pack(m->P, m->d, m->stream);
    if (e != cudaSuccess) return mlp_cuda(m, e, "init");
    return mlp_sync_check(m);
}

int hair_fuse_mlp_set_params(hf_mlp* m, const float* params, int mem_kind) {
    if (!m || !params) return HF_ERR_INVALID_ARG;
    cudaError_t e = cudaMemcpyAsync(m->P, params, hf_mlp_param_count() * 4,
                                    mem_kind == HF_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, m->stream);
    if (e == cudaSuccess) e = hf_launch_pack(m->P, m->d, m->stream);
    if (e != cudaSuccess) return mlp_cuda(m, e, "set params");
    return mlp_sync_check(m);
}

int hair_fuse_mlp_get_params(hf_mlp* m, float* params, int mem_kind) {
    if (!m || !params) return HF_ERR_INVALID_ARG;
    cudaError_t e = cudaMemcpyAsync(params, m->P, hf_mlp_param_count() * 4,
                                    mem_kind == HF_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, m->stream);
    if (e != cudaSuccess) return mlp_cuda(m, e, "get params");
    return mlp_sync_check(m);
}

int hair_fuse_mlp_train(hf_mlp* m, const uint16_t* X, const float* T, long long n_samples, int batch, int steps, float lr,
                        uint64_t seed, int use_graph, float* loss_out) {
    if (!m || !X || !T || n_samples < 1 || steps < 0 || !(lr >= 0.0f)) return mlp_err(m, HF_ERR_INVALID_ARG, "%s", "bad training arguments");
    int rc;
    if ((rc = check_batch(m, batch))) return rc;
    long long step0 = 0;
    cudaError_t e = cudaMemcpyAsync(&step0, m->step, 8, cudaMemcpyDeviceToHost, m->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(m->stream);
    if (e != cudaSuccess) return mlp_cuda(m, e, "read step");
    if ((rc = ensure_loss(m, step0 + steps))) return rc;
    if ((e = encode_maps(m, batch))) return mlp_cuda(m, e, "tensor maps");
    const MlpTrain t = train_args(m, X, T, n_samples, batch, seed, lr);
    int done = 0;
    if (steps > 0) {   // the first step runs eagerly (sets kernel attributes before any capture)
        if ((e = hf_train_step(t, m->stream))) return mlp_cuda(m, e, "train step");
        done = 1;
    }
    if (use_graph && done < steps) {
        const bool same = m->graph && m->g_X == X && m->g_T == T && m->g_n == n_samples && m->g_B == batch &&
                          m->g_seed == seed && m->g_lr == lr;
        if (!same) {
            if (m->graph) cudaGraphExecDestroy(m->graph);
            m->graph = nullptr;
            // capture on a stream of our own (the caller's may be the legacy default stream, which
            // cannot be captured); the graph is launched on the caller's stream
            cudaGraph_t g = nullptr;
            if (!m->cap_stream) e = cudaStreamCreateWithFlags(&m->cap_stream, cudaStreamNonBlocking);
            if (e == cudaSuccess) e = cudaStreamSynchronize(m->stream);
            if (e == cudaSuccess) e = cudaStreamBeginCapture(m->cap_stream, cudaStreamCaptureModeThreadLocal);
            if (e == cudaSuccess) {
                cudaError_t e2 = hf_train_step(t, m->cap_stream);
                e = cudaStreamEndCapture(m->cap_stream, &g);
                if (e == cudaSuccess) e = e2;
            }
            if (e == cudaSuccess) e = cudaGraphInstantiate(&m->graph, g, 0);
            if (g) cudaGraphDestroy(g);
            if (e != cudaSuccess) return mlp_cuda(m, e, "capture training step");
            m->g_X = X; m->g_T = T; m->g_n = n_samples; m->g_B = batch; m->g_seed = seed; m->g_lr = lr;
        }
        for (; done < steps; ++done)
            if ((e = cudaGraphLaunch(m->graph, m->stream))) return mlp_cuda(m, e, "graph launch");
    }
    for (; done < steps; ++done)
        if ((e = hf_train_step(t, m->stream))) return mlp_cuda(m, e, "train step");
    if (loss_out && steps > 0) {
        e = cudaMemcpyAsync(loss_out, m->loss_hist + step0, steps * sizeof(float), cudaMemcpyDeviceToHost, m->stream);
        if (e != cudaSuccess) return mlp_cuda(m, e, "read losses");
    }
    return mlp_sync_check(m);
}

int hair_fuse_mlp_grads(hf_mlp* m, const uint16_t* X, const float* T, long long n_samples, int batch, uint64_t seed,
                        float* grads_out, float* loss_out, uint16_t* xb_out, float* tb_out) {
    if (!m || !X || !T || !grads_out) return mlp_err(m, HF_ERR_INVALID_ARG, "%s", "bad gradient arguments");
    int rc;
    if ((rc = check_batch(m, batch))) return rc;
    long long step0 = 0;
    cudaError_t e = cudaMemcpyAsync(&step0, m->step, 8, cudaMemcpyDeviceToHost, m->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(m->stream);
    if (e != cudaSuccess) return mlp_cuda(m, e, "read step");
    if ((rc = ensure_loss(m, step0 + 1))) return rc;
    if ((e = encode_maps(m, batch))) return mlp_cuda(m, e, "tensor maps");
    MlpTrain t = train_args(m, X, T, n_samples, batch, seed, 0.0f);
    e = cudaMemsetAsync(m->loss_hist + step0, 0, sizeof(float), m->stream);
    if (e == cudaSuccess) e = hf_train_step(t, m->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(grads_out, m->G, hf_mlp_param_count() * 4, cudaMemcpyDeviceToHost, m->stream);
    if (e == cudaSuccess && loss_out) e = cudaMemcpyAsync(loss_out, m->loss_hist + step0, 4, cudaMemcpyDeviceToHost, m->stream);
    if (e == cudaSuccess && xb_out) e = cudaMemcpyAsync(xb_out, m->d.Xb, (size_t)batch * 64 * 2, cudaMemcpyDeviceToHost, m->stream);
    if (e == cudaSuccess && tb_out) e = cudaMemcpyAsync(tb_out, m->d.Tb, (size_t)batch * 3 * 4, cudaMemcpyDeviceToHost, m->stream);
    // the gradient step counts as a step (its batch index comes from the counter): undo that
    if (e == cudaSuccess) e = cudaMemcpyAsync(m->step, &step0, 8, cudaMemcpyHostToDevice, m->stream);
    if (e != cudaSuccess) return mlp_cuda(m, e, "gradients");
    return mlp_sync_check(m);
}

namespace {
int mlp_forward(hf_mlp* m, const uint16_t* X, int n, float* dir_out, int mem_kind, bool raw) {
    if (!m || !X || !dir_out || n < 1) return mlp_err(m, HF_ERR_INVALID_ARG, "%s", "bad forward arguments");
    const uint16_t* xd = X;
    float* od = dir_out;
    void* tmp = nullptr;
    cudaError_t e = cudaSuccess;
    if (mem_kind == HF_HOST) {
        e = cudaMalloc(&tmp, (size_t)n * (64 * 2 + 12));
        if (e == cudaSuccess) e = cudaMemcpyAsync(tmp, X, (size_t)n * 128, cudaMemcpyHostToDevice, m->stream);
        xd = (const uint16_t*)tmp;
        od = (float*)((char*)tmp + (size_t)n * 128);
    }
    if (e == cudaSuccess) e = hf_mlp_infer(m->d, m->P, xd, n, od, m->errw, m->stream, raw, m->wait_ns);
    if (e == cudaSuccess && mem_kind == HF_HOST) e = cudaMemcpyAsync(dir_out, od, (size_t)n * 12, cudaMemcpyDeviceToHost, m->stream);
    if (mem_kind == HF_HOST) {
        cudaError_t e2 = cudaStreamSynchronize(m->stream);
        if (tmp) cudaFree(tmp);
        if (e == cudaSuccess) e = e2;
    }
    if (e != cudaSuccess) return mlp_cuda(m, e, "forward");
    return mem_kind == HF_HOST ? mlp_sync_check(m) : HF_OK;
}
}  // namespace

int hair_fuse_mlp_forward(hf_mlp* m, const uint16_t* X, int n, float* dir_out, int mem_kind) {
    return mlp_forward(m, X, n, dir_out, mem_kind, false);
}

int hair_fuse_mlp_forward_raw(hf_mlp* m, const uint16_t* X, int n, float* y_out, int mem_kind) {
    return mlp_forward(m, X, n, y_out, mem_kind, true);
}

int hair_fuse_mlp_save(hf_mlp* m, const char* path) {
    if (!m || !path) return HF_ERR_INVALID_ARG;
    const long long np = hf_mlp_param_count();
    float* h = new float[3 * np];
    long long step = 0;
    cudaError_t e = cudaMemcpyAsync(h, m->P, np * 4, cudaMemcpyDeviceToHost, m->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(h + np, m->M, np * 4, cudaMemcpyDeviceToHost, m->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(h + 2 * np, m->V, np * 4, cudaMemcpyDeviceToHost, m->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&step, m->step, 8, cudaMemcpyDeviceToHost, m->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(m->stream);
    if (e != cudaSuccess) {
        delete[] h;
        return mlp_cuda(m, e, "save");
    }
    FILE* f = std::fopen(path, "wb");
    bool ok = f != nullptr;
    const char magic[8] = {'H', 'F', 'M', 'L', 'P', '0', '0', '1'};
    if (ok) ok = std::fwrite(magic, 1, 8, f) == 8 && std::fwrite(&np, 8, 1, f) == 1 && std::fwrite(&step, 8, 1, f) == 1 &&
                 std::fwrite(h, 4, 3 * np, f) == (size_t)(3 * np);
    if (f) std::fclose(f);
    delete[] h;
    return ok ? HF_OK : mlp_err(m, HF_ERR_INVALID_ARG, "cannot write %s", path);
}

int hair_fuse_mlp_load(hf_mlp* m, const char* path) {
    if (!m || !path) return HF_ERR_INVALID_ARG;
    const long long np = hf_mlp_param_count();
    FILE* f = std::fopen(path, "rb");
    if (!f) return mlp_err(m, HF_ERR_INVALID_ARG, "cannot open %s", path);
    char magic[8];
    long long cnt = 0, step = 0;
    float* h = new float[3 * np];
    bool ok = std::fread(magic, 1, 8, f) == 8 && std::memcmp(magic, "HFMLP001", 8) == 0 && std::fread(&cnt, 8, 1, f) == 1 &&
              cnt == np && std::fread(&step, 8, 1, f) == 1 && std::fread(h, 4, 3 * np, f) == (size_t)(3 * np);
    std::fclose(f);
    if (!ok) {
        delete[] h;
        return mlp_err(m, HF_ERR_INVALID_ARG, "%s is not a proposal-network checkpoint of this layout", path);
    }
    cudaError_t e = cudaMemcpyAsync(m->P, h, np * 4, cudaMemcpyHostToDevice, m->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(m->M, h + np, np * 4, cudaMemcpyHostToDevice, m->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(m->V, h + 2 * np, np * 4, cudaMemcpyHostToDevice, m->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(m->step, &step, 8, cudaMemcpyHostToDevice, m->stream);
    if (e == cudaSuccess) e = hf_launch_pack(m->P, m->d, m->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(m->stream);
    delete[] h;
    if (e != cudaSuccess) return mlp_cuda(m, e, "load");
    return mlp_sync_check(m);
}

const char* hair_fuse_mlp_last_error(const hf_mlp* m) { return m ? m->err.c_str() : hair_fuse_last_error(nullptr); }

int hair_fuse_mlp_set_wait_limit(hf_mlp* m, unsigned long long wait_ns) {
    if (!m) return HF_ERR_INVALID_ARG;
    m->wait_ns = wait_ns;
    return HF_OK;
}

}  // extern "C"

// ------------------------------------------------------------------ features and the learned path
namespace {
int learned_scratch(hf_ctx* c, long long N) {
    int rc;
    if ((rc = hf_ensure(c, c->feat, (size_t)N * 64 * 2))) return rc;
    if ((rc = hf_ensure(c, c->prop, (size_t)N * 3 * 4))) return rc;
    if ((rc = hf_ensure(c, c->lmisc, 256 + 64 * 8 + (size_t)N * 8))) return rc;
    return HF_OK;
}

// The projection's outputs (samples, ratios, view-set masks, work counter) for the current scene.
int projection_buffers(hf_ctx* c) {
    const int N = c->N, V = c->V;
    int rc;
    if ((rc = hf_ensure(c, c->samp, (size_t)N * hf_view_pairs(V) * sizeof(float4)))) return rc;
    if ((rc = hf_ensure(c, c->ab, (size_t)N * hf_view_pairs(V) * sizeof(float4)))) return rc;
    if ((rc = hf_ensure(c, c->vmask, (size_t)N * hf_mask_words(V) * sizeof(unsigned long long)))) return rc;
    if ((rc = hf_ensure(c, c->work, sizeof(unsigned long long)))) return rc;
    return HF_OK;
}

// The projection of the uploaded points with the view part of the features written to x, folding
// the points into the bounding box at box_keys (which the caller resets); work counts its (point,
// view) pairs.
ProjectArgs feature_projection(hf_ctx* c, uint16_t* x, unsigned* box_keys, unsigned long long* work) {
    return ProjectArgs{(const float*)c->pts.p, c->N, (const float*)c->cams.p, c->V, c->W, c->Hh,
                       (const float*)c->angle.p, c->conf.p, c->conf_dtype == HF_F16 ? 1 : 0, c->cfg.top_k_views,
                       (float2*)c->samp.p, (float2*)c->ab.p, (unsigned long long*)c->vmask.p, work, box_keys,
                       (const float2*)c->amap.p, x};
}
}  // namespace

extern "C" int hair_fuse_features(hf_ctx* c, uint16_t* x_out, int mem_kind) {
    if (!c || !x_out) return HF_ERR_INVALID_ARG;
    if (c->V <= 0 || c->N <= 0) return hf_set_err(c, HF_ERR_NOT_UPLOADED, "views or points not uploaded");
    if (mem_kind != HF_HOST && mem_kind != HF_DEVICE) return hf_set_err(c, HF_ERR_INVALID_ARG, "bad mem_kind");
    int rc;
    if ((rc = learned_scratch(c, c->N))) return rc;
    if ((rc = projection_buffers(c))) return rc;
    // the same kernels as the learned path: the projection (view part, bounding box), then the
    // position part; its own work counter, so the last fusion's count stays readable
    char* lm = (char*)c->lmisc.p;
    unsigned* box_keys = reinterpret_cast<unsigned*>(lm + 32);
    unsigned long long* work = reinterpret_cast<unsigned long long*>(lm + 88);
    // the kernels store 8 and 16 bytes at a time: an unaligned device destination gets a copy
    const bool direct = mem_kind == HF_DEVICE && (reinterpret_cast<uintptr_t>(x_out) & 15) == 0;
    uint16_t* x = direct ? x_out : (uint16_t*)c->feat.p;
    cudaError_t e = hf_launch_bbox_init(box_keys, c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(work, 0, 8, c->stream);
    if (e == cudaSuccess) e = hf_launch_project(feature_projection(c, x, box_keys, work), c->stream);
    if (e == cudaSuccess) e = hf_launch_featpos(FeatArgs{(const float*)c->pts.p, c->N, nullptr, x, box_keys}, c->stream);
    c->launches += 3;
    if (e == cudaSuccess && !direct)
        e = cudaMemcpyAsync(x_out, x, (size_t)c->N * 128, mem_kind == HF_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice,
                            c->stream);
    if (e != cudaSuccess) return hf_cuda_err(c, e, "features");
    if (mem_kind == HF_HOST) {
        e = cudaStreamSynchronize(c->stream);
        if (e != cudaSuccess) return hf_cuda_err(c, e, "features");
    }
    return HF_OK;
}

extern "C" int hair_fuse_fuse_learned(hf_ctx* c, hf_mlp* m, int T_short, float alpha_short, float tau, float* dir_out,
                                      float* cost_out, int32_t* idx_out, uint8_t* status_out, int* n_fallback,
                                      int mem_kind) {
    if (!c || !m || !dir_out) return HF_ERR_INVALID_ARG;
    if (c->V <= 0 || c->N <= 0) return hf_set_err(c, HF_ERR_NOT_UPLOADED, "views or points not uploaded");
    if (T_short < 0 || T_short > HF_MAX_T || !(alpha_short > 0.0f) || !(tau == tau))
        return hf_set_err(c, HF_ERR_INVALID_ARG, "T_short in [0, %d], alpha_short > 0 and a finite tau required", HF_MAX_T);
    if (mem_kind != HF_HOST && mem_kind != HF_DEVICE) return hf_set_err(c, HF_ERR_INVALID_ARG, "bad mem_kind");
    const int N = c->N, V = c->V, H = c->cfg.H, T = c->cfg.T;
    int rc;
    if ((rc = learned_scratch(c, N))) return rc;
    // per-scene constants and the projection / gather (shared with the plain path)
    const int Hpad = hf_hpad(H);
    if ((rc = hf_ensure(c, c->vthr, (size_t)V * sizeof(float)))) return rc;
    if ((rc = hf_ensure(c, c->hyps, (size_t)Hpad * 3 * sizeof(float)))) return rc;
    if ((rc = hf_ensure(c, c->rot, (size_t)(T > 0 ? T : 1) * sizeof(float2)))) return rc;
    if ((rc = hf_ensure(c, c->qtab, (size_t)V * hf_hq(H) * sizeof(float4)))) return rc;
    if ((rc = hf_ensure(c, c->best, (size_t)N * sizeof(int32_t)))) return rc;
    if ((rc = projection_buffers(c))) return rc;
    if ((rc = hf_ensure(c, c->outs, (size_t)N * 21))) return rc;
    char* lm = (char*)c->lmisc.p;
    float* box = (float*)lm;
    int* count = (int*)(lm + 64);                                        // fallback points
    int* acc_count = (int*)(lm + 68);                                    // accepted proposals
    unsigned long long* fb_work = (unsigned long long*)(lm + 72);       // their (point, view) pairs
    unsigned long long* acc_work = (unsigned long long*)(lm + 80);      // those of the accepted proposals
    float2* rot_s = (float2*)(lm + 128);
    int32_t* list = (int32_t*)(lm + 256 + 64 * 8);
    int32_t* acc_list = list + N;
    char* so = (char*)c->outs.p;
    float* d_dir = mem_kind == HF_HOST ? (float*)so : dir_out;
    float* d_cost = (mem_kind == HF_HOST || !cost_out) ? (float*)(so + (size_t)N * 12) : cost_out;
    int32_t* d_idx = mem_kind == HF_HOST ? (int32_t*)(so + (size_t)N * 16) : idx_out;
    uint8_t* d_status = mem_kind == HF_HOST ? (uint8_t*)(so + (size_t)N * 20) : status_out;
    cudaStream_t s = c->stream;

    PrepArgs pr{(const float*)c->cams.p, V, nullptr, H, Hpad, T, (float*)c->hyps.p, (float*)c->vthr.p,
                (float2*)c->rot.p, (uint32_t*)c->errw.p, (float4*)c->qtab.p, hf_hq(H)};
    unsigned* box_keys = reinterpret_cast<unsigned*>(box + 8);
    if ((rc = run_launch(c, "k_prep", [&] {
             cudaError_t e2 = hf_launch_prep(pr, s);
             return e2 != cudaSuccess ? e2 : hf_launch_bbox_init(box_keys, s);
         })))
        return rc;
    cudaError_t e = cudaMemsetAsync(c->work.p, 0, 8, s);
    if (e != cudaSuccess) return hf_cuda_err(c, e, "clear work counter");
    // the projection also writes the view part of the features and folds the points into the
    // bounding box their position part is normalised by
    const ProjectArgs pa = feature_projection(c, (uint16_t*)c->feat.p, box_keys, (unsigned long long*)c->work.p);
    if ((rc = run_launch(c, "k_project", [&] { return hf_launch_project(pa, s); }))) return rc;
    // proposal: the features' position part -> network
    const FeatArgs fa{(const float*)c->pts.p, N, nullptr, (uint16_t*)c->feat.p, box_keys};
    if ((rc = run_launch(c, "k_featpos", [&] { return hf_launch_featpos(fa, s); }))) return rc;
    if ((rc = run_launch(c, "k_mlp", [&] {
             return hf_mlp_infer(m->d, m->P, (const uint16_t*)c->feat.p, N, (float*)c->prop.p,
                                 (uint32_t*)c->errw.p, s, false, m->wait_ns);
         })))
        return rc;
    // the proposal's cost decides: above tau -> the plain fusion (fallback list), else the short
    // refinement from the proposal
    CostArgs base = hf_cost_args(c);
    base.dir_out = d_dir;
    base.cost_out = d_cost;
    base.idx_out = d_idx;
    base.status_out = d_status;
    LearnArgs la{base, (const float*)c->prop.p, tau, list, count, fb_work, acc_work, acc_list, acc_count};
    if ((rc = run_launch(c, "k_select", [&] {
             cudaError_t e2 = cudaMemsetAsync(count, 0, 24, s);   // counts, fb_work, acc_work
             if (e2 == cudaSuccess) e2 = hf_launch_rot(rot_s, T_short, (double)alpha_short, s);
             return e2 != cudaSuccess ? e2 : hf_launch_select(la, s);
         })))
        return rc;
    CostArgs fs = base;   // the accepted proposals: T_short rounds from the proposal, a point per thread
    fs.L = 0;
    fs.list = acc_list;
    fs.list_count = acc_count;
    fs.start_dir = (const float*)c->prop.p;
    fs.rot = rot_s;
    fs.T = T_short;
    if ((rc = run_launch(c, "k_refine_short", [&] { return hf_launch_refine(fs, s); }))) return rc;
    CostArgs fb = base;   // the fallback points: the plain fusion
    fb.list = list;
    fb.list_count = count;
    fb.fell_back = 1;
    if ((rc = run_launch(c, "k_argmin_fallback", [&] { return hf_launch_argmin(fb, s); }))) return rc;
    if ((rc = run_launch(c, "k_refine_fallback", [&] { return hf_launch_refine(fb, s); }))) return rc;
    c->learned_ran = true;
    if (mem_kind == HF_HOST) {
        e = cudaMemcpyAsync(dir_out, d_dir, (size_t)N * 12, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess && cost_out) e = cudaMemcpyAsync(cost_out, d_cost, (size_t)N * 4, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess && idx_out) e = cudaMemcpyAsync(idx_out, d_idx, (size_t)N * 4, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess && status_out) e = cudaMemcpyAsync(status_out, d_status, (size_t)N, cudaMemcpyDeviceToHost, s);
        if (e != cudaSuccess) return hf_cuda_err(c, e, "copy outputs");
    }
    if (n_fallback) {
        e = cudaMemcpyAsync(n_fallback, count, sizeof(int), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return hf_cuda_err(c, e, "read fallback count");
    }
    if (mem_kind == HF_HOST || n_fallback) return hair_fuse_sync(c);
    return HF_OK;
}

cudaError_t hf_mlp_infer_rows(hf_mlp* m, const uint16_t* x, long long n, float* dir_out, uint32_t* errw, cudaStream_t s) {
    if (n <= 0 || n > 0x7fffffffLL) return cudaErrorInvalidValue;
    return hf_mlp_infer(m->d, m->P, x, (int)n, dir_out, errw, s, false, m->wait_ns);
}

cudaStream_t hf_mlp_stream(hf_mlp* m) { return m->stream; }

extern "C" int hair_fuse_learned_work(hf_ctx* c, long long* fallback_point_views, long long* accepted_point_views) {
    if (!c) return HF_ERR_INVALID_ARG;
    if (c->N <= 0 || !c->lmisc.p || !c->learned_ran) return hf_set_err(c, HF_ERR_NOT_UPLOADED, "no learned fusion has run");
    unsigned long long w[2] = {0, 0};
    cudaError_t e = cudaMemcpyAsync(w, (const char*)c->lmisc.p + 72, sizeof w, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return hf_cuda_err(c, e, "read work counters");
    if (fallback_point_views) *fallback_point_views = (long long)w[0];
    if (accepted_point_views) *accepted_point_views = (long long)w[1];
    return HF_OK;
}
