// hf_batch.cu - batched serving: many uploaded scenes of uneven size fused together.
//
// Every stage of the fusion (constants, projection + gather, features, proposal network, short
// refinement, fallback selection, hypothesis argmin, refinement) is ONE launch over all scenes of
// the batch: a persistent grid takes (scene, tile) items from a global counter (hf_kernels.cu), the
// proposal network runs once over the concatenated feature rows of all scenes, and the whole stage
// sequence is captured in one CUDA graph that each run replays.  The tile shape of the cost
// kernels (hypothesis chunk, points per CTA) and the scene order are picked by timing the
// candidates on the batch itself (autotuning, first run).  The CTA finishing a scene's last tile
// stamps the global timer, which gives per-scene completion latencies.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "hf_internal.cuh"
#include "hf_mlp.cuh"

namespace {

// stages of a run; the refinement stages run one launch per lane class (a point per thread, or 4, 8,
// 16, 32 lanes per point), each with its own item counter
enum { ST_PROJECT, ST_FEATURES, ST_SELECT, ST_SHORT, ST_ARGMIN, ST_MAIN, ST_MLP, ST_COUNT };
const char* const kStageName[ST_COUNT] = {"k_project_batch", "k_featpos_batch", "k_select_batch", "k_refine_short_batch",
                                          "k_argmin_batch", "k_refine_batch", "k_mlp"};
constexpr int kClasses = 5;   // a point per thread (L = 0), then 4, 8, 16, 32 lanes per point
int class_of(int L) { return L == 0 ? 0 : L <= 4 ? 1 : L <= 8 ? 2 : L <= 16 ? 3 : 4; }
// item counter of a stage (and lane class)
int counter_of(int stage, int cls) {
    switch (stage) {
        case ST_PROJECT: return 0;
        case ST_FEATURES: return 1;
        case ST_SELECT: return 2;
        case ST_ARGMIN: return 3;
        case ST_SHORT: return 4 + cls;
        default: return 4 + kClasses + cls;
    }
}
constexpr int kCounters = 4 + 2 * kClasses;
static_assert(kCounters <= 16, "sixteen item counters");

// device control block (bytes); [0, kZeroEnd) is cleared by k_prep_batch at the start of a run
constexpr size_t kNextOff = 0;                                   // u32 [16] item counters
constexpr size_t kDoneOff = 64;                                  // u32 [2][HF_MAX_BATCH]: short, main
constexpr size_t kCountOff = kDoneOff + 2 * HF_MAX_BATCH * 4;    // i32 [HF_MAX_BATCH]: fallback list lengths
constexpr size_t kAccOff = kCountOff + HF_MAX_BATCH * 4;         // i32 [HF_MAX_BATCH]: accepted list lengths
constexpr size_t kWorkOff = kAccOff + HF_MAX_BATCH * 4;          // u64 [HF_MAX_BATCH]: (point, view) pairs
constexpr size_t kFbWorkOff = kWorkOff + HF_MAX_BATCH * 8;       // u64 [HF_MAX_BATCH]: those of fallback points
constexpr size_t kAccWorkOff = kFbWorkOff + HF_MAX_BATCH * 8;    // u64 [HF_MAX_BATCH]: of accepted proposals
constexpr size_t kStampOff = kAccWorkOff + HF_MAX_BATCH * 8;     // u64 [2][HF_MAX_BATCH]: completion times
constexpr size_t kZeroEnd = kStampOff + 2 * HF_MAX_BATCH * 8;
constexpr size_t kT0Off = kZeroEnd;                              // u64 batch start
constexpr size_t kBoxOff = kT0Off + 8;                           // u32 [HF_MAX_BATCH][6]
constexpr size_t kRotOff = kBoxOff + HF_MAX_BATCH * 24;          // float2 [HF_MAX_T]
constexpr size_t kErrOff = kRotOff + HF_MAX_T * 8;               // u32 error word
constexpr size_t kCtlBytes = kErrOff + 8;
static_assert(kWorkOff % 8 == 0 && kStampOff % 8 == 0 && kT0Off % 8 == 0 && kRotOff % 8 == 0, "alignment");

struct BatchScene {
    hf_ctx* c = nullptr;
    float* dir = nullptr;
    float* cost = nullptr;
    int32_t* idx = nullptr;
    uint8_t* status = nullptr;
    long long off = 0;   // first row in the concatenated feature / proposal / list arrays
    double work = 0.0;   // relative cost of the scene, for heaviest-first ordering
};

// per-position argument arrays, uploaded as one block
struct ArgBlock {
    PrepArgs prep[HF_MAX_BATCH];
    ProjectArgs proj[HF_MAX_BATCH];
    FeatArgs feat[HF_MAX_BATCH];
    LearnArgs sel[HF_MAX_BATCH];
    CostArgs shrt[HF_MAX_BATCH];
    CostArgs main[HF_MAX_BATCH];
};

}  // namespace

struct hf_batch {
    std::vector<BatchScene> sc;
    std::vector<int> pos;   // position -> scene index
    hf_mlp* mlp = nullptr;
    hf_batch_cfg cfg{};
    cudaStream_t user = nullptr;    // caller's stream (ordering only)
    cudaStream_t stream = nullptr;  // the batch's own non-blocking stream (captured)
    cudaEvent_t ev_in = nullptr, ev_out = nullptr, t_beg = nullptr, t_end = nullptr;
    int kp = 9, nt = 128, order = 1;   // nt: threads per CTA of the cost kernels; order: 1 heaviest first, 2 as given, 3 lightest first
    struct Class {
        int L, first, count, hmax;   // lanes per point, positions [first, first + count), largest H
    };
    std::vector<Class> cls;          // the lane classes present, positions grouped by class
    bool tuned = false, configured = false;
    bool tuned_from_cache = false;   // the launch shape came from an earlier batch of the same class
    long long total = 0;
    char* ctl = nullptr;
    ArgBlock* args = nullptr;   // device
    ArgBlock* args_h = nullptr; // pinned host copy
    uint16_t* x = nullptr;
    float* prop = nullptr;
    int32_t* list = nullptr;       // fallback points, per scene from its row offset
    int32_t* acc_list = nullptr;   // accepted proposals, likewise
    cudaGraphExec_t gexec = nullptr;
    long long launches = 0;   // kernels enqueued (graph replays counted by their kernels)
    std::string err;
};

namespace {

int b_err(hf_batch* b, int code, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    std::vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    b->err = buf;
    return code;
}

int b_cuda(hf_batch* b, cudaError_t e, const char* what) {
    return b_err(b, HF_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

void drop_graph(hf_batch* b) {
    if (b->gexec) cudaGraphExecDestroy(b->gexec);
    b->gexec = nullptr;
}

// Fill and upload the argument arrays for the current scene order.
int configure(hf_batch* b) {
    const int ns = (int)b->sc.size();
    b->pos.resize(ns);
    for (int p = 0; p < ns; ++p) b->pos[p] = p;
    // per-point work x points: the scene's share of a stage
    auto load = [&](int u) { return b->sc[u].work * (double)b->sc[u].c->N; };
    if (b->order == 1)
        std::stable_sort(b->pos.begin(), b->pos.end(), [&](int u, int v) { return load(u) > load(v); });
    else if (b->order == 3)
        std::stable_sort(b->pos.begin(), b->pos.end(), [&](int u, int v) { return load(u) < load(v); });
    // positions grouped by lane class (one launch per class), the order kept inside a class
    auto lanes = [&](int u) { return hf_cost_args(b->sc[u].c).L; };
    std::stable_sort(b->pos.begin(), b->pos.end(), [&](int u, int v) { return lanes(u) < lanes(v); });
    b->cls.clear();
    for (int p = 0; p < ns; ++p) {
        const int L = lanes(b->pos[p]), H = b->sc[b->pos[p]].c->cfg.H;
        if (b->cls.empty() || b->cls.back().L != L) b->cls.push_back({L, p, 0, 0});
        b->cls.back().count++;
        b->cls.back().hmax = std::max(b->cls.back().hmax, H);
    }
    const bool learned = b->mlp != nullptr;
    unsigned* box = reinterpret_cast<unsigned*>(b->ctl + kBoxOff);
    int* count = reinterpret_cast<int*>(b->ctl + kCountOff);
    int* acc = reinterpret_cast<int*>(b->ctl + kAccOff);
    unsigned long long* work = reinterpret_cast<unsigned long long*>(b->ctl + kWorkOff);
    unsigned long long* fb_work = reinterpret_cast<unsigned long long*>(b->ctl + kFbWorkOff);
    unsigned long long* acc_work = reinterpret_cast<unsigned long long*>(b->ctl + kAccWorkOff);
    float2* rot_s = reinterpret_cast<float2*>(b->ctl + kRotOff);
    uint32_t* errw = reinterpret_cast<uint32_t*>(b->ctl + kErrOff);
    ArgBlock& A = *b->args_h;
    std::memset(&A, 0, sizeof A);
    for (int p = 0; p < ns; ++p) {
        const BatchScene& s = b->sc[b->pos[p]];
        hf_ctx* c = s.c;
        const int N = c->N, V = c->V, H = c->cfg.H, T = c->cfg.T;
        A.prep[p] = PrepArgs{(const float*)c->cams.p, V, nullptr, H, hf_hpad(H), T, (float*)c->hyps.p,
                             (float*)c->vthr.p, (float2*)c->rot.p, errw, (float4*)c->qtab.p, hf_hq(H)};
        A.proj[p] = ProjectArgs{(const float*)c->pts.p, N, (const float*)c->cams.p, V, c->W, c->Hh,
                                (const float*)c->angle.p, c->conf.p, c->conf_dtype == HF_F16 ? 1 : 0,
                                c->cfg.top_k_views, (float2*)c->samp.p, (float2*)c->ab.p, (unsigned long long*)c->vmask.p, work + p,
                                learned ? box + 6 * p : nullptr, (const float2*)c->amap.p,
                                learned ? b->x + (size_t)s.off * 64 : nullptr};
        A.feat[p] = FeatArgs{(const float*)c->pts.p, N, nullptr, b->x + (size_t)s.off * 64, box + 6 * p};
        CostArgs m = hf_cost_args(c);
        m.dir_out = s.dir;
        m.cost_out = s.cost;
        m.idx_out = s.idx;
        m.status_out = s.status;
        if (learned) {
            // the proposal's cost sorts the points into the fallback and the accepted list
            A.sel[p] = LearnArgs{m, b->prop + (size_t)s.off * 3, b->cfg.tau, b->list + s.off, count + p, fb_work + p,
                                 acc_work + p, b->acc_list + s.off, acc + p};
            CostArgs f = m;   // accepted: T_short rounds from the proposal, a point per thread
            f.L = 0;
            f.list = b->acc_list + s.off;
            f.list_count = acc + p;
            f.start_dir = b->prop + (size_t)s.off * 3;
            f.rot = rot_s;
            f.T = b->cfg.T_short;
            A.shrt[p] = f;
            m.list = b->list + s.off;   // fallback: the plain fusion
            m.list_count = count + p;
            m.fell_back = 1;
        }
        A.main[p] = m;
    }
    cudaError_t e = cudaMemcpyAsync(b->args, b->args_h, sizeof(ArgBlock), cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return b_cuda(b, e, "upload batch arguments");
    b->configured = true;
    return HF_OK;
}

// work distribution of a stage over positions [first, first + count) (all positions when count < 0)
BatchCtl ctl_for(hf_batch* b, int stage, int stamp_slot, int cls = 0, int first = 0, int count = -1) {
    BatchCtl c{};
    c.next = reinterpret_cast<unsigned*>(b->ctl + kNextOff) + counter_of(stage, cls);
    c.ns = count < 0 ? (int)b->sc.size() : count;
    if (stamp_slot >= 0) {
        c.done = reinterpret_cast<unsigned*>(b->ctl + kDoneOff) + stamp_slot * HF_MAX_BATCH + first;
        c.stamp = reinterpret_cast<unsigned long long*>(b->ctl + kStampOff) + stamp_slot * HF_MAX_BATCH + first;
    }
    return c;
}

cudaError_t launch_prep(hf_batch* b, bool reset) {
    BatchReset r{};
    if (reset) {
        r.zero = reinterpret_cast<unsigned*>(b->ctl);
        r.nzero = (int)(kZeroEnd / 4);
        r.box_keys = reinterpret_cast<unsigned*>(b->ctl + kBoxOff);
        r.t0 = reinterpret_cast<unsigned long long*>(b->ctl + kT0Off);
        if (b->mlp) {
            r.rot_s = reinterpret_cast<float2*>(b->ctl + kRotOff);
            r.T_short = b->cfg.T_short;
            r.alpha_short = (double)b->cfg.alpha_short;
        }
    }
    return hf_launch_prep_batch(b->args->prep, (int)b->sc.size(), r, b->stream);
}

cudaError_t launch_stage(hf_batch* b, int stage) {
    cudaStream_t s = b->stream;
    ArgBlock* A = b->args;
    switch (stage) {
        case ST_PROJECT: return hf_launch_project_batch(A->proj, ctl_for(b, ST_PROJECT, -1), b->mlp != nullptr, s);
        case ST_FEATURES: return hf_launch_featpos_batch(A->feat, ctl_for(b, ST_FEATURES, -1), s);
        case ST_MLP:
            return hf_mlp_infer_rows(b->mlp, b->x, b->total, b->prop, reinterpret_cast<uint32_t*>(b->ctl + kErrOff), s);
        case ST_SELECT: return hf_launch_select_batch(A->sel, ctl_for(b, ST_SELECT, -1), b->kp, s);
        case ST_ARGMIN: return hf_launch_argmin_batch(A->main, ctl_for(b, ST_ARGMIN, -1), b->kp, b->nt, s);
        case ST_SHORT: return hf_launch_refine_batch(A->shrt, ctl_for(b, ST_SHORT, 0), b->kp, 0, b->nt, s);
        case ST_MAIN: {
            for (const auto& k : b->cls) {
                const BatchCtl c = ctl_for(b, stage, 1, class_of(k.L), k.first, k.count);
                const cudaError_t e = hf_launch_refine_batch(A->main + k.first, c, b->kp, k.L, b->nt, s);
                if (e != cudaSuccess) return e;
            }
            return cudaSuccess;
        }
        default: return cudaErrorInvalidValue;
    }
}

// launches of a stage
int stage_launches(const hf_batch* b, int stage) {
    return stage == ST_MLP ? 2 : stage == ST_MAIN ? (int)b->cls.size() : 1;
}

// kernels of one run (the network's two GEMMs included)
int kernels_per_run(const hf_batch* b) {
    const int nc = (int)b->cls.size();
    return b->mlp ? 8 + nc : 3 + nc;
}

// the whole run: constants (and counter reset), then every stage in order; with ev (profiling,
// eager only) an event is recorded after the constants and after every stage
cudaError_t enqueue(hf_batch* b, cudaEvent_t* ev = nullptr, int* stages_out = nullptr, int* n_out = nullptr) {
    if (ev) cudaEventRecord(ev[0], b->stream);
    cudaError_t e = launch_prep(b, true);
    if (e != cudaSuccess) return e;
    if (ev) cudaEventRecord(ev[1], b->stream);
    const bool learned = b->mlp != nullptr;
    const int plain_stages[] = {ST_PROJECT, ST_ARGMIN, ST_MAIN};
    const int learned_stages[] = {ST_PROJECT, ST_FEATURES, ST_MLP, ST_SELECT, ST_SHORT, ST_ARGMIN, ST_MAIN};
    const int* st = learned ? learned_stages : plain_stages;
    const int n = learned ? 7 : 3;
    for (int q = 0; q < n && e == cudaSuccess; ++q) {
        e = launch_stage(b, st[q]);
        if (ev) cudaEventRecord(ev[2 + q], b->stream);
    }
    if (stages_out)
        for (int q = 0; q < n; ++q) stages_out[q] = st[q];
    if (n_out) *n_out = n;
    b->launches += kernels_per_run(b);
    return e;
}

// time one stage re-run (its item counter cleared first); min of reps, ms
int time_stage(hf_batch* b, int stage, int reps, float* ms) {
    float best = INFINITY;
    for (int r = 0; r < reps; ++r) {
        cudaError_t e = cudaSuccess;
        for (int q = 0; q < kClasses && e == cudaSuccess; ++q)
            e = cudaMemsetAsync(reinterpret_cast<unsigned*>(b->ctl + kNextOff) + counter_of(stage, q), 0, 4, b->stream);
        // the selection appends to the lists and adds to the work counts: they start empty
        if (e == cudaSuccess && stage == ST_SELECT) e = cudaMemsetAsync(b->ctl + kCountOff, 0, 2 * HF_MAX_BATCH * 4, b->stream);
        if (e == cudaSuccess && stage == ST_SELECT) e = cudaMemsetAsync(b->ctl + kFbWorkOff, 0, 2 * HF_MAX_BATCH * 8, b->stream);
        if (e == cudaSuccess) e = cudaEventRecord(b->t_beg, b->stream);
        if (e == cudaSuccess) e = launch_stage(b, stage);
        if (e == cudaSuccess) e = cudaEventRecord(b->t_end, b->stream);
        if (e == cudaSuccess) e = cudaEventSynchronize(b->t_end);
        float t = 0.0f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&t, b->t_beg, b->t_end);
        if (e != cudaSuccess) return b_cuda(b, e, "autotune timing");
        best = std::min(best, t);
    }
    *ms = best;
    return HF_OK;
}

int run_eager(hf_batch* b) {
    cudaError_t e = enqueue(b);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return b_cuda(b, e, "batch run");
    return HF_OK;
}

// Autotuner: candidate launch shapes timed on the batch itself.  The stages are re-run in pipeline
// order, so every buffer a timed stage reads holds what the full run left there.  The lanes per
// point follow from each scene's view count (they fix the order of the sums, so they are not tuned:
// a batched result stays bit-identical to the scene run alone).
// Tuned shapes are kept per process for batches of one shape class: learned or plain, patch width,
// scene count, total points and total views each within a factor of two, and the caller's fixed
// choices; a later batch of the class takes them without timing.
using TuneKey = std::tuple<int, int, int, int, int, int, int>;
std::map<TuneKey, std::pair<int, int>>& tune_cache() {
    static std::map<TuneKey, std::pair<int, int>> m;
    return m;
}
std::mutex& tune_mutex() {
    static std::mutex m;
    return m;
}
TuneKey tune_key(const hf_batch* b) {
    long long pts = 0, views = 0;
    for (const auto& s : b->sc) {
        pts += s.c->N;
        views += s.c->V;
    }
    auto lg = [](long long x) { int e = 0; while (x > 1) { x >>= 1; ++e; } return e; };
    return TuneKey{b->mlp ? 1 : 0, b->kp, (int)b->sc.size(), lg(pts), lg(views), b->cfg.cta_threads, b->cfg.order};
}

int autotune(hf_batch* b) {
    int rc;
    const int nts[] = {64, 128, 256};
    const bool learned = b->mlp != nullptr;
    const TuneKey key = tune_key(b);
    {
        std::lock_guard<std::mutex> lock(tune_mutex());
        const auto it = tune_cache().find(key);
        if (it != tune_cache().end()) {
            b->nt = it->second.first;
            b->order = it->second.second;
            if ((rc = configure(b))) return rc;
            b->tuned = b->tuned_from_cache = true;
            return HF_OK;
        }
    }
    if ((rc = configure(b)) || (rc = run_eager(b))) return rc;
    // threads per CTA of the cost kernels (the short refinement, the argmin and the refinement)
    float best = INFINITY;
    int best_nt = b->nt;
    for (int nt : nts) {
        if (b->cfg.cta_threads && nt != b->cfg.cta_threads) continue;
        b->nt = nt;
        float t = 0.0f, t2 = 0.0f, t3 = 0.0f;
        if (learned && (rc = time_stage(b, ST_SHORT, 2, &t2))) return rc;
        if ((rc = time_stage(b, ST_ARGMIN, 2, &t3))) return rc;
        if ((rc = time_stage(b, ST_MAIN, 2, &t))) return rc;
        if (t + t2 + t3 < best) {
            best = t + t2 + t3;
            best_nt = nt;
        }
    }
    b->nt = best_nt;
    // scene order: heaviest first (best balance at the end of a stage) against lightest first (small
    // scenes complete early); lightest first unless it costs more than 1 % of throughput
    if (!b->cfg.order) {
        float tt[2] = {0.0f, 0.0f};
        const int modes[2] = {1, 3};
        for (int q = 0; q < 2; ++q) {
            b->order = modes[q];
            if ((rc = configure(b)) || (rc = run_eager(b))) return rc;
            cudaError_t e = cudaEventRecord(b->t_beg, b->stream);
            if (e == cudaSuccess) e = enqueue(b);
            if (e == cudaSuccess) e = cudaEventRecord(b->t_end, b->stream);
            if (e == cudaSuccess) e = cudaEventSynchronize(b->t_end);
            if (e == cudaSuccess) e = cudaEventElapsedTime(&tt[q], b->t_beg, b->t_end);
            if (e != cudaSuccess) return b_cuda(b, e, "autotune order");
        }
        b->order = tt[1] <= 1.01f * tt[0] ? 3 : 1;
    }
    if ((rc = configure(b)) || (rc = run_eager(b))) return rc;
    b->tuned = true;
    std::lock_guard<std::mutex> lock(tune_mutex());
    tune_cache()[key] = {b->nt, b->order};
    return HF_OK;
}

int check_errw(hf_batch* b) {
    uint32_t w = 0;
    cudaError_t e = cudaMemcpyAsync(&w, b->ctl + kErrOff, 4, cudaMemcpyDeviceToHost, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return b_cuda(b, e, "read device error word");
    if (w) {
        cudaMemsetAsync(b->ctl + kErrOff, 0, 4, b->stream);
        cudaStreamSynchronize(b->stream);
        if (w & HF_DEV_ERR_TIMEOUT) return b_err(b, HF_ERR_TIMEOUT, "a bounded device wait expired");
        return b_err(b, HF_ERR_CUDA, "device error word 0x%x", w);
    }
    return HF_OK;
}

thread_local std::string g_batch_create_err;

}  // namespace

extern "C" int hair_fuse_batch_create(hf_batch** out, hf_ctx* const* scenes, int n_scenes, hf_mlp* mlp,
                                      const hf_batch_cfg* cfg, void* cuda_stream) {
    auto fail = [&](int code, const char* msg) {
        g_batch_create_err = msg;
        return code;
    };
    if (!out || !scenes) return fail(HF_ERR_INVALID_ARG, "out and scenes are required");
    *out = nullptr;
    if (n_scenes < 1 || n_scenes > HF_MAX_BATCH) return fail(HF_ERR_SHAPE, "n_scenes must be in [1, 64]");
    hf_batch_cfg c{};
    if (cfg) c = *cfg;
    if (mlp && (c.T_short < 1 || c.T_short > HF_MAX_T || !(c.alpha_short > 0.0f) || !(c.tau == c.tau)))
        return fail(HF_ERR_INVALID_ARG, "learned batch: T_short in [1, 24], alpha_short > 0 and a non-NaN tau required");
    if (c.cta_threads && c.cta_threads != 64 && c.cta_threads != 128 && c.cta_threads != 256)
        return fail(HF_ERR_INVALID_ARG, "cta_threads: 0, 64, 128 or 256");
    if (c.order < 0 || c.order > 3) return fail(HF_ERR_INVALID_ARG, "order: 0, 1, 2 or 3");
    long long total = 0;
    int max_k = 0;
    for (int s = 0; s < n_scenes; ++s) {
        hf_ctx* x = scenes[s];
        if (!x) return fail(HF_ERR_INVALID_ARG, "a scene is null");
        if (x->V <= 0 || x->N <= 0) return fail(HF_ERR_NOT_UPLOADED, "a scene has no views or no points uploaded");
        for (int t = 0; t < s; ++t)
            if (scenes[t] == x) return fail(HF_ERR_INVALID_ARG, "a scene appears twice");
        total += x->N;
        max_k = std::max(max_k, x->k);
    }
    if (total > (1LL << 30)) return fail(HF_ERR_SHAPE, "more than 2^30 points in a batch");
    hf_batch* b = new hf_batch();
    b->mlp = mlp;
    b->cfg = c;
    b->user = (cudaStream_t)cuda_stream;
    b->total = total;
    b->kp = hf_batch_kp_for(max_k);
    b->nt = c.cta_threads ? c.cta_threads : 128;
    b->order = c.order ? c.order : 1;
    b->sc.resize(n_scenes);
    int rc = HF_OK;
    cudaError_t e = cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_in, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_out, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreate(&b->t_beg);
    if (e == cudaSuccess) e = cudaEventCreate(&b->t_end);
    if (e == cudaSuccess) e = cudaMalloc(&b->ctl, kCtlBytes);
    if (e == cudaSuccess) e = cudaMemset(b->ctl, 0, kCtlBytes);
    if (e == cudaSuccess) e = cudaMalloc(&b->args, sizeof(ArgBlock));
    if (e == cudaSuccess) e = cudaMallocHost(&b->args_h, sizeof(ArgBlock));
    if (e == cudaSuccess && mlp) {
        e = cudaMalloc(&b->x, (size_t)total * 64 * sizeof(uint16_t));
        if (e == cudaSuccess) e = cudaMalloc(&b->prop, (size_t)total * 3 * sizeof(float));
        if (e == cudaSuccess) e = cudaMalloc(&b->list, (size_t)total * sizeof(int32_t));
        if (e == cudaSuccess) e = cudaMalloc(&b->acc_list, (size_t)total * sizeof(int32_t));
    }
    if (e != cudaSuccess) {
        hair_fuse_batch_destroy(b);
        return fail(e == cudaErrorMemoryAllocation ? HF_ERR_OOM : HF_ERR_CUDA, cudaGetErrorString(e));
    }
    long long off = 0;
    for (int s = 0; s < n_scenes && rc == HF_OK; ++s) {
        hf_ctx* x = scenes[s];
        BatchScene& bs = b->sc[s];
        bs.c = x;
        bs.off = off;
        off += x->N;
        // per-(point, view) work: hypotheses, refinement candidates, patch members
        bs.work = (double)x->V * (x->cfg.H + 6.0 * x->cfg.T) * (x->k + 1);
        const int N = x->N, V = x->V, T = x->cfg.T;
        const int Hpad = hf_hpad(x->cfg.H);
        if (!rc) rc = hf_ensure(x, x->samp, (size_t)N * hf_view_pairs(V) * sizeof(float4));
        if (!rc) rc = hf_ensure(x, x->ab, (size_t)N * hf_view_pairs(V) * sizeof(float4));
        if (!rc) rc = hf_ensure(x, x->vmask, (size_t)N * hf_mask_words(V) * sizeof(unsigned long long));
        if (!rc) rc = hf_ensure(x, x->vthr, (size_t)V * sizeof(float));
        if (!rc) rc = hf_ensure(x, x->hyps, (size_t)Hpad * 3 * sizeof(float));
        if (!rc) rc = hf_ensure(x, x->rot, (size_t)(T > 0 ? T : 1) * sizeof(float2));
        if (!rc) rc = hf_ensure(x, x->qtab, (size_t)V * hf_hq(x->cfg.H) * sizeof(float4));
        if (!rc) rc = hf_ensure(x, x->best, (size_t)N * sizeof(int32_t));
        if (!rc && cudaStreamSynchronize(x->stream) != cudaSuccess) rc = HF_ERR_CUDA;   // uploads complete
        if (rc) g_batch_create_err = "scene " + std::to_string(s) + ": " + x->err;
    }
    if (rc == HF_OK && mlp && cudaStreamSynchronize(hf_mlp_stream(mlp)) != cudaSuccess) {
        rc = HF_ERR_CUDA;
        g_batch_create_err = "proposal network stream";
    }
    if (rc != HF_OK) {
        hair_fuse_batch_destroy(b);
        return rc;
    }
    *out = b;
    return HF_OK;
}

extern "C" int hair_fuse_batch_set_outputs(hf_batch* b, int scene, float* dir_out, float* cost_out, int32_t* idx_out,
                                           uint8_t* status_out) {
    if (!b) return HF_ERR_INVALID_ARG;
    if (scene < 0 || scene >= (int)b->sc.size()) return b_err(b, HF_ERR_INVALID_ARG, "scene %d out of range", scene);
    if (!dir_out) return b_err(b, HF_ERR_INVALID_ARG, "dir_out is required");
    if (b->mlp && !cost_out) return b_err(b, HF_ERR_INVALID_ARG, "the learned batch needs cost_out (fallback selection)");
    BatchScene& s = b->sc[scene];
    s.dir = dir_out;
    s.cost = cost_out;
    s.idx = idx_out;
    s.status = status_out;
    b->configured = false;
    drop_graph(b);
    return HF_OK;
}

extern "C" int hair_fuse_batch_run(hf_batch* b, int use_graph) {
    if (!b) return HF_ERR_INVALID_ARG;
    for (size_t s = 0; s < b->sc.size(); ++s)
        if (!b->sc[s].dir) return b_err(b, HF_ERR_INVALID_ARG, "scene %d has no outputs set", (int)s);
    int rc;
    // order after the caller's stream
    cudaError_t e = cudaEventRecord(b->ev_in, b->user);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(b->stream, b->ev_in, 0);
    if (e != cudaSuccess) return b_cuda(b, e, "order after the caller's stream");
    if (b->cfg.autotune && !b->tuned) {
        if ((rc = autotune(b))) return rc;
    } else if (!b->configured) {
        if ((rc = configure(b))) return rc;
    }
    if (use_graph) {
        if (!b->gexec) {
            // one eager run first: function attributes and grid sizes are settled outside capture
            if ((rc = run_eager(b))) return rc;
            cudaGraph_t g = nullptr;
            e = cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal);
            if (e != cudaSuccess) return b_cuda(b, e, "begin capture");
            cudaError_t e2 = enqueue(b);
            b->launches -= kernels_per_run(b);   // captured, not run
            e = cudaStreamEndCapture(b->stream, &g);
            if (e2 != cudaSuccess || e != cudaSuccess) {
                if (g) cudaGraphDestroy(g);
                return b_cuda(b, e2 != cudaSuccess ? e2 : e, "capture batch");
            }
            e = cudaGraphInstantiate(&b->gexec, g, 0);
            cudaGraphDestroy(g);
            if (e != cudaSuccess) return b_cuda(b, e, "instantiate batch graph");
        }
        e = cudaGraphLaunch(b->gexec, b->stream);
        b->launches += kernels_per_run(b);
    } else {
        e = enqueue(b);
    }
    if (e != cudaSuccess) return b_cuda(b, e, "launch batch");
    e = cudaEventRecord(b->ev_out, b->stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(b->user, b->ev_out, 0);
    if (e != cudaSuccess) return b_cuda(b, e, "order the caller's stream after the batch");
    return HF_OK;
}

extern "C" int hair_fuse_batch_sync(hf_batch* b) {
    if (!b) return HF_ERR_INVALID_ARG;
    return check_errw(b);
}

extern "C" int hair_fuse_batch_latency(hf_batch* b, double* ms_out) {
    if (!b || !ms_out) return HF_ERR_INVALID_ARG;
    const int ns = (int)b->sc.size();
    std::vector<unsigned long long> st(2 * HF_MAX_BATCH + 1);
    cudaError_t e = cudaMemcpyAsync(st.data(), b->ctl + kStampOff, 2 * HF_MAX_BATCH * 8, cudaMemcpyDeviceToHost, b->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&st[2 * HF_MAX_BATCH], b->ctl + kT0Off, 8, cudaMemcpyDeviceToHost, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return b_cuda(b, e, "read completion stamps");
    const unsigned long long t0 = st[2 * HF_MAX_BATCH];
    for (int p = 0; p < ns; ++p) {
        const unsigned long long done = std::max(st[p], st[HF_MAX_BATCH + p]);
        ms_out[b->pos[p]] = done > t0 ? (double)(done - t0) * 1e-6 : 0.0;
    }
    return HF_OK;
}

extern "C" int hair_fuse_batch_fallbacks(hf_batch* b, int* n_out) {
    if (!b || !n_out) return HF_ERR_INVALID_ARG;
    const int ns = (int)b->sc.size();
    int cnt[HF_MAX_BATCH];
    cudaError_t e = cudaMemcpyAsync(cnt, b->ctl + kCountOff, sizeof cnt, cudaMemcpyDeviceToHost, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return b_cuda(b, e, "read fallback counts");
    for (int p = 0; p < ns; ++p) n_out[b->pos[p]] = b->mlp ? cnt[p] : 0;
    return HF_OK;
}

extern "C" int hair_fuse_batch_tuning(const hf_batch* b, int* out2) {
    if (!b || !out2) return HF_ERR_INVALID_ARG;
    out2[0] = b->nt;
    out2[1] = b->order;
    return HF_OK;
}

extern "C" int hair_fuse_batch_tuned_from_cache(const hf_batch* b) {
    if (!b) return HF_ERR_INVALID_ARG;
    return b->tuned_from_cache ? 1 : 0;
}

extern "C" int hair_fuse_batch_profile_run(hf_batch* b, hf_kernel_time* out, int max_entries) {
    if (!b || (!out && max_entries > 0)) return HF_ERR_INVALID_ARG;
    for (size_t s = 0; s < b->sc.size(); ++s)
        if (!b->sc[s].dir) return b_err(b, HF_ERR_INVALID_ARG, "scene %d has no outputs set", (int)s);
    int rc;
    if (!b->configured && (rc = configure(b))) return rc;
    cudaEvent_t ev[10];
    int made = 0;
    cudaError_t e = cudaSuccess;
    for (; made < 10 && e == cudaSuccess; ++made) e = cudaEventCreate(&ev[made]);
    int st[8], n = 0;
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e == cudaSuccess) e = enqueue(b, ev, st, &n);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    int k = 0;
    if (e == cudaSuccess) {
        float t = 0.0f;
        cudaEventElapsedTime(&t, ev[0], ev[1]);
        if (k < max_entries) {
            std::snprintf(out[k].name, sizeof out[k].name, "%s", "k_prep_batch");
            out[k].launches = 1;
            out[k].total_ms = t;
        }
        ++k;
        for (int q = 0; q < n; ++q, ++k) {
            cudaEventElapsedTime(&t, ev[1 + q], ev[2 + q]);
            if (k < max_entries) {
                std::snprintf(out[k].name, sizeof out[k].name, "%s", kStageName[st[q]]);
                out[k].launches = stage_launches(b, st[q]);
                out[k].total_ms = t;
            }
        }
    }
    for (int q = 0; q < made; ++q) cudaEventDestroy(ev[q]);
    if (e != cudaSuccess) return b_cuda(b, e, "profiled batch run");
    return k;
}

extern "C" int hair_fuse_batch_stats(hf_batch* b, long long* launches, long long* point_views,
                                     long long* fallback_point_views, long long* accepted_point_views) {
    if (!b) return HF_ERR_INVALID_ARG;
    if (launches) *launches = b->launches;
    if (!point_views && !fallback_point_views && !accepted_point_views) return HF_OK;
    const int ns = (int)b->sc.size();
    unsigned long long w[3 * HF_MAX_BATCH];
    cudaError_t e = cudaMemcpyAsync(w, b->ctl + kWorkOff, sizeof w, cudaMemcpyDeviceToHost, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return b_cuda(b, e, "read work counters");
    long long pv = 0, fpv = 0, apv = 0;
    for (int p = 0; p < ns; ++p) {
        pv += (long long)w[p];
        if (b->mlp) {
            fpv += (long long)w[HF_MAX_BATCH + p];
            apv += (long long)w[2 * HF_MAX_BATCH + p];
        }
    }
    if (point_views) *point_views = pv;
    if (fallback_point_views) *fallback_point_views = fpv;
    if (accepted_point_views) *accepted_point_views = apv;
    return HF_OK;
}

extern "C" void hair_fuse_batch_destroy(hf_batch* b) {
    if (!b) return;
    if (b->stream) cudaStreamSynchronize(b->stream);
    drop_graph(b);
    cudaFree(b->ctl);
    cudaFree(b->args);
    if (b->args_h) cudaFreeHost(b->args_h);
    cudaFree(b->x);
    cudaFree(b->prop);
    cudaFree(b->list);
    cudaFree(b->acc_list);
    if (b->ev_in) cudaEventDestroy(b->ev_in);
    if (b->ev_out) cudaEventDestroy(b->ev_out);
    if (b->t_beg) cudaEventDestroy(b->t_beg);
    if (b->t_end) cudaEventDestroy(b->t_end);
    if (b->stream) cudaStreamDestroy(b->stream);
    delete b;
}

extern "C" const char* hair_fuse_batch_last_error(const hf_batch* b) {
    return b ? b->err.c_str() : g_batch_create_err.c_str();
}
