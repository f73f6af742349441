// hf_internal.cuh - internal declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <stdint.h>
#include <string>
#include <vector>

#include "../../include/hair_fuse.h"

// Device-side error word bits (latched, read back by synchronising calls).
enum : uint32_t {
    HF_DEV_ERR_BAD_HYP = 1u,      // a hypothesis is not unit length within 1e-3
    HF_DEV_ERR_BAD_NBR = 2u,      // a neighbour index outside [0, N)
    HF_DEV_ERR_TIMEOUT = 4u,      // a bounded wait expired
};

// Grow-only device buffer owned by the context.
struct DevBuf {
    void* p = nullptr;
    size_t cap = 0;
};

// Per-kernel timing record (profiling mode).
struct ProfRec {
    std::string name;
    cudaEvent_t beg, end;
};

struct hf_ctx {
    hf_config cfg{};
    cudaStream_t stream = nullptr;
    int device = 0;
    std::string err;
    // views
    int V = 0, W = 0, Hh = 0, conf_dtype = HF_F32;
    DevBuf cams, angle, conf;
    DevBuf amap;    // [V][H][W] float2 (angle, confidence as f32): one 8-byte read per gathered pixel
    // points
    int N = 0, k = 0;
    DevBuf pts, nbr;
    // scratch of the fusion path
    DevBuf samp;    // [V][N] float2: C (cos theta, sin theta) at the point's pixel, 0 when not visible
    DevBuf ab;      // [V][N] float2: projection ratios (X/Z, Y/Z); NaN when v is not in the point's view set
    DevBuf vmask;   // [N][Vw] u64: the point's view set V_i
    DevBuf vthr;    // [V] float: degenerate-offset threshold 1e-20 (fx^2 + fy^2)
    DevBuf qtab;    // [V][Hq] float4: the argmin's hypothesis-pair table
    DevBuf best;    // [N] int32: the argmin's hypothesis index
    DevBuf hyps;    // [Hpad] x 3 float
    DevBuf rot;     // [T] float2: (cos alpha_t, sin alpha_t)
    DevBuf outs;    // device outputs staged for HF_HOST calls
    DevBuf evald;   // device copy of eval directions for HF_HOST calls
    DevBuf errw;    // uint32 device error word
    DevBuf work;    // uint64 (point, view) pairs of the last projection
    DevBuf feat;    // [N x 64] bf16 proposal-network features
    DevBuf prop;    // [N x 3] proposals
    DevBuf lmisc;   // bounding box, fallback count, short-refinement steps, fallback list
    DevBuf rlist;   // point range of hair_fuse_fuse_range: count, then the indices
    DevBuf depth;   // [V][H][W] f32 staging of host depth maps (FPMVO), +inf where no hair
    DevBuf dmap;    // [V][H][W] float2 (depth, confidence) for FPMVO's depth test and view selection
    DevBuf vmap;    // [V][H][W] float2 C (cos theta, sin theta) for FPMVO's patches
    DevBuf fprec;   // FPMVO scratch: [N][K][3] float4 top-view records
    DevBuf phg;     // Parallel Hair Growing scratch: tensors, scans, links, staged host arrays
    DevBuf gabor;   // Gabor maps scratch: staged host images and outputs
    DevBuf gbank;   // the Gabor bank B[dy][filter][dx] bf16, built for gbank_key (sigma along, across, lambda)
    float gbank_key[3] = {0.0f, 0.0f, 0.0f};
    bool gbank_ok = false;
    long long views_gen = 0;   // bumped by every view upload
    long long depth_gen = -1;  // views_gen the FPMVO maps were built for
    bool learned_ran = false;  // a learned fusion has filled the work counters
    uint32_t* errw_host = nullptr;  // pinned read-back slot
    long long launches = 0;
    long long dev_bytes = 0;
    bool prof = false;
    std::vector<ProfRec> prof_recs;
};

// Error helpers -------------------------------------------------------------------------------
int hf_set_err(hf_ctx* c, int code, const char* fmt, ...);
int hf_cuda_err(hf_ctx* c, cudaError_t e, const char* what);
int hf_ensure(hf_ctx* c, DevBuf& b, size_t bytes);

// Run one launch (f returns its cudaError_t) with optional event timing on the context's stream.
template <class F>
int run_launch(hf_ctx* c, const char* name, F&& f) {
    ProfRec rec;
    if (c->prof) {
        rec.name = name;
        cudaEventCreate(&rec.beg);
        cudaEventCreate(&rec.end);
        cudaEventRecord(rec.beg, c->stream);
    }
    cudaError_t e = f();
    if (c->prof) {
        cudaEventRecord(rec.end, c->stream);
        c->prof_recs.push_back(rec);
    }
    c->launches++;
    if (e != cudaSuccess) return hf_cuda_err(c, e, name);
    return HF_OK;
}

// Kernel-launch helpers (defined in hf_kernels.cu); each returns the launch error -------------
//
// Scratch of the fusion path (per context, or the static array of the allocation-free entry):
//   samp  [V/2][N] float4  C (cos theta, sin theta) at point i's own pixel in views 2p and 2p + 1 (one
//                        16-byte element per view pair; 0 when the point does not project into the view)
//   ab    [V/2][N] float4  projection ratios (X/Z, Y/Z) of point i in views 2p and 2p + 1; NaN when the
//                        view is not in V_i (and for the missing second view of an odd V)
//                        (V/2 rounded up; element (v, i) is float2 number hf_pv(v, i, N))
//   vmask [N][Vw] u64    bit v of word v / 64: v is in the point's view set V_i; Vw = ceil(V / 64)
//   hyps  [Hpad][3] f32   the hypotheses, padded to an even count with copies of h_0
//   qtab  [V][Hq] float4  hypothesis pairs q = R_v h folded with fx, fy (the argmin's table)
//   best  [N] i32         the argmin's hypothesis index, read by the refinement
//   vthr  [V] f32         degenerate-offset threshold 1e-20 (fx^2 + fy^2) per view
//   rot   [T] float2      (cos alpha_t, sin alpha_t) of the refinement rounds
__host__ __device__ inline int hf_mask_words(int V) { return (V + 63) / 64; }
// view pairs of the samp / ab planes, and the float2 index of (view v, point i)
__host__ __device__ inline int hf_view_pairs(int V) { return (V + 1) >> 1; }
__host__ __device__ inline size_t hf_pv(int v, int i, int N) { return (((size_t)(v >> 1) * N + i) << 1) + (v & 1); }
__host__ __device__ inline int hf_hpad(int H) { return (H + 1) & ~1; }

struct ProjectArgs {
    const float* pts; int N;
    const float* cams; int V; int W; int H;
    const float* angle; const void* conf; int conf_f16;
    int top_k;
    float2* samp; float2* ab; unsigned long long* vmask;
    unsigned long long* work;   // += number of (point, view) pairs in the view sets
    unsigned* box_keys;         // optional: bounding-box keys lo[3], hi[3] folded in (see hf_launch_bbox_init)
    const float2* amap;         // optional: interleaved (angle, confidence) maps, read instead of angle / conf
    uint16_t* featx;            // optional: [N x 64] bf16 network features; the projection writes columns
                                // 0..47, the view part (hf_launch_featpos writes the rest)
};
cudaError_t hf_launch_project(const ProjectArgs& a, cudaStream_t s);
// list[q] = first + q for q < n, *count = n
cudaError_t hf_launch_iota(int32_t* list, int* count, int first, int n, cudaStream_t s);
// out[i] = (angle[i], conf[i] as f32) for npx pixels
cudaError_t hf_launch_interleave(const float* angle, const void* conf, int conf_f16, size_t npx, float2* out,
                                 cudaStream_t s);

struct PrepArgs {
    const float* cams; int V;
    const float* hyps_in;  // device H x 3, or nullptr for the Fibonacci set
    int H; int Hpad; int T;
    float* hyps;           // out Hpad x 3
    float* vthr;           // out [V]
    float2* rot;           // out [T]
    uint32_t* errw;
    float4* qtab; int Hq;  // out [V][Hq]: the argmin's hypothesis-pair table (Hq = hf_hq(H)); may be null
};
// hypotheses of the argmin's table: H rounded up to its chunk of 32
__host__ __device__ inline int hf_hq(int H) { return (H + 31) & ~31; }
cudaError_t hf_launch_prep(const PrepArgs& a, cudaStream_t s);

// The cost kernels: the argmin runs a point per thread; the refinement either also runs a point per
// thread (L = 0) or serves a point by a group of L lanes (L in {4, 8, 16, 32}) over which the views
// of its view set are dealt (hf_cost_lanes() picks from the largest view-set size).
struct CostArgs {
    const float* pts; int N;
    const int32_t* nbr; int k;
    const float* cams; int V;
    const float2* samp; const float2* ab;
    const unsigned long long* vmask; int Vw;
    const float* vthr;
    const float* hyps; int H; int Hpad;
    const float2* rot; int T;
    int L;                                               // refinement: lanes per point, 0 = a point per thread
    float* dir_out; float* cost_out; int32_t* idx_out; uint8_t* status_out;
    int32_t* nvs;                                        // optional [N]: |V_i|, -1 for a non-finite point
    const int32_t* list; const int* list_count;          // optional: only these points (device count)
    int fell_back;                                       // mark outputs HF_STATUS_FELL_BACK
    int out_first;   // outputs of point i go to row i - out_first (0: point-indexed)
    const float4* qtab; int Hq;                          // argmin: hypothesis-pair table
    int32_t* best_idx;                                   // argmin output, refinement start (hyps[best_idx[i]])
    const float* start_dir;                              // refinement start instead (learned proposals)
};
int hf_cost_lanes(int veff, int k);    // lanes per point for view sets of up to veff views
struct hf_ctx;
CostArgs hf_cost_args(const hf_ctx* c);   // the uploaded scene's arguments (outputs, list unset)
cudaError_t hf_launch_argmin(const CostArgs& a, cudaStream_t s);   // K2: -> best_idx
cudaError_t hf_launch_refine(const CostArgs& a, cudaStream_t s);   // K3: from best_idx or start_dir -> outputs
cudaError_t hf_launch_fuse(const CostArgs& a, cudaStream_t s);     // K2 then K3

// Learned path after the network: the cost c_i of the proposal start_dir; points with a view and
// c_i > tau are appended to fb_list (count *fb_count, from 0; work += |V_i| into fb_work), the
// other finite points to acc_list (count *acc_count; work into acc_work); non-finite points get
// their BAD_INPUT outputs.
struct LearnArgs {
    CostArgs f;
    const float* start_dir;
    float tau;
    int32_t* fb_list; int* fb_count;
    unsigned long long* fb_work; unsigned long long* acc_work;
    int32_t* acc_list; int* acc_count;
};
cudaError_t hf_launch_select(const LearnArgs& a, cudaStream_t s);

struct EvalArgs {
    CostArgs f;
    const float* dirs; int M;
    float* cost;     // [N][M]
};
cudaError_t hf_launch_eval(const EvalArgs& a, cudaStream_t s);

cudaError_t hf_launch_fib(int H, float* out, cudaStream_t s);

// learned proposal path
// The position part of the network features: columns 48..63 of each row of x, (p - centre) /
// half_extent of the points' bounding box and zero padding.  The view part (columns 0..47) is
// written by the projection (ProjectArgs::featx) from the samples it gathers anyway.
struct FeatArgs {
    const float* pts; int N;
    const float* box;           // bounding box lo[3], hi[3] (used when box_keys is null)
    uint16_t* x;                // [N x 64] bf16 features
    const unsigned* box_keys;   // bounding box as order-preserving keys lo[3], hi[3], or null
};
cudaError_t hf_launch_featpos(const FeatArgs& a, cudaStream_t s);
// (cos, sin) of alpha0 / 2^t for t < T, in double then rounded
cudaError_t hf_launch_rot(float2* rot, int T, double alpha0, cudaStream_t s);
cudaError_t hf_launch_check_nbr(const int32_t* nbr, long long n, int N, uint32_t* errw, cudaStream_t s);
// reorder each point's k neighbours by index distance (the cost kernels' gather order)
cudaError_t hf_launch_order_nbr(int32_t* nbr, int N, int k, cudaStream_t s);

// ------------------------------------------------------------------ batched scenes (hf_batch.cu)
#define HF_MAX_BATCH HF_MAX_BATCH_SCENES

// Work distribution of one persistent stage over a batch: next = global item counter (zeroed
// before the launch); with done set, done[p] counts finished tiles of position p and stamp[p]
// receives the global timer when its last tile finishes.
struct BatchCtl {
    unsigned* next;
    unsigned* done;
    unsigned long long* stamp;
    int ns;
};

// what k_prep_batch does besides the per-scene constants
struct BatchReset {
    unsigned* zero; int nzero;              // words cleared (counters)
    unsigned* box_keys;                     // [ns][6] set to the empty box, or null
    float2* rot_s; int T_short; double alpha_short;   // short-refinement steps, or null
    unsigned long long* t0;                 // batch start time, or null
};

int hf_batch_kp_for(int k);   // patch width instantiated for the batched kernels (4, 9 or 17)
cudaError_t hf_launch_prep_batch(const PrepArgs* pr, int ns, const BatchReset& r, cudaStream_t s);
// feat: the scenes' ProjectArgs carry featx (the learned path)
cudaError_t hf_launch_project_batch(const ProjectArgs* pa, const BatchCtl& c, bool feat, cudaStream_t s);
cudaError_t hf_launch_featpos_batch(const FeatArgs* fe, const BatchCtl& c, cudaStream_t s);
// The batched cost kernels (hf_batch_kernels.cu) over the c.ns scenes at fa / la; kp from
// hf_batch_kp_for(max k); nt threads per CTA (64, 128 or 256).  The refinement takes the scenes
// that share the lane count L.
cudaError_t hf_launch_argmin_batch(const CostArgs* fa, const BatchCtl& c, int kp, int nt, cudaStream_t s);
cudaError_t hf_launch_refine_batch(const CostArgs* fa, const BatchCtl& c, int kp, int L, int nt, cudaStream_t s);
cudaError_t hf_launch_select_batch(const LearnArgs* la, const BatchCtl& c, int kp, cudaStream_t s);

// ------------------------------------------------------------------ FPMVO (hf_fpmvo.cu)
#define HF_FPMVO_MAX_K 8
struct FpmvoArgs {
    const float* pts; int N;
    const float* cams; int V; int W; int H;
    const float2* amap;     // (angle, confidence)
    const float2* dmap;     // (depth, confidence)
    const float2* vmap;     // C (cos theta, sin theta)
    // scratch between the two kernels: K records per point of three 16-byte words, one per top view
    // and zeros past the last: (view, confidence, pixel x, pixel y), (u, w, lambda cos theta,
    // lambda sin theta), (Zp hi, Zp lo, z at the offset pixel (+inf if none), n); n of record 0 is
    // the number of top views (-1 for a non-finite point)
    float4* rec;
    int K, S, P;
    float lambda, delta, eps;
    float* dir_out; float* cost_out; int32_t* sel_out; uint8_t* status_out;
    float ds[32];           // the S depth-sample offsets delta_s
};
cudaError_t hf_launch_fpmvo_views(const FpmvoArgs& a, cudaStream_t s);   // then hf_launch_fpmvo_fuse
cudaError_t hf_launch_fpmvo_fuse(const FpmvoArgs& a, cudaStream_t s);
cudaError_t hf_launch_fpmvo_maps(const float* depth, const float2* amap, size_t npx, float2* dmap, float2* vmap,
                                 cudaStream_t s);
