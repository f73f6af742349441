/*
 * hair_fuse.h - C ABI of the B300 multi-view hair direction-fusion library.
 *
 * The library assigns each 3D hair point a strand direction by fusing per-view 2D orientation
 * evidence: EfficientMonoHair, Sec. 3.1 ("Fusion-Patch-based Multi-View Optimization"),
 * patch-based consistency step (Eqs. proj_r, sim, patchloss, patch_min, final_dout), evaluated
 * over an explicit set of candidate directions (hypotheses), followed by an argmin and a short
 * rotation pattern-search refinement.  For a point p_i and unit direction d:
 *
 *   r_v(d)  = dPi_v/dp(p_i) . d                      image offset of d in view v   (Eq. proj_r)
 *   L_v(d)  = max_{j in {i} U nbr(i), visible in v}  C_v(u_j) |<r_v/|r_v|, O_v(u_j)>|
 *                                                    (Eqs. sim, patchloss, patch_min)
 *   c_i(d)  = 1 - mean_{v in V_i} L_v(d)             (aggregation for Eq. final_dout)
 *
 * with O_v(u) = (cos theta, sin theta) from the angle map, nearest-pixel sampling at
 * (floor u, floor v), V_i the views in which p_i projects inside the image (optionally only the
 * top-K of them by confidence at p_i's pixel, Sec. 3.1.2).  The output direction is the best
 * hypothesis refined by T rounds of +-alpha rotations about the world x, y, z axes (alpha_0 =
 * sqrt(2 pi / H) / 2, halved every round, move only on a strictly lower cost), normalised, with
 * the first of z, y, x whose magnitude exceeds 1e-12 made positive.
 *
 * Conventions (all entry points):
 *  - Return 0 (HF_OK) or a negative HF_ERR_* code; hair_fuse_last_error() gives a message.
 *    No entry point aborts the process.
 *  - mem_kind HF_HOST: pointers are host memory (pageable or pinned); the call copies inputs in
 *    and, for outputs, returns after they are written back (synchronous).
 *    mem_kind HF_DEVICE: pointers are device memory of the current device; the work is queued on
 *    the context's stream and the call returns without waiting.  Device inputs must stay valid
 *    until the stream has consumed them; outputs are valid once the stream reaches that point.
 *    mem_kind HF_HOST_ASYNC (hair_fuse_upload_views, hair_fuse_upload_points, hair_fuse_gabor): pinned host
 *    memory copied on the context's stream without waiting, so that a caller can overlap the
 *    upload of one scene set with the work of another on a second stream.  The caller keeps the
 *    buffers unchanged until the stream has consumed them (hair_fuse_sync(), or any later
 *    synchronising call on the context).  Pageable memory makes the copy synchronous (CUDA's rule).
 *  - Uploads copy into buffers the context owns; the caller keeps ownership of its own buffers.
 *  - Errors found on the device (a bad hypothesis, a timed-out wait) are latched in the context
 *    and returned by the next synchronising call (an HF_HOST call or hair_fuse_sync()).
 *  - A context is used by one host thread at a time.
 */
#ifndef HAIR_FUSE_H
#define HAIR_FUSE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* return codes */
#define HF_OK 0
#define HF_ERR_INVALID_ARG (-1)   /* bad pointer, size, dtype, value (e.g. non-unit hypothesis) */
#define HF_ERR_NOT_UPLOADED (-2)  /* views or points missing, or inconsistent with each other */
#define HF_ERR_OOM (-3)           /* a device or pinned allocation failed */
#define HF_ERR_CUDA (-4)          /* a CUDA runtime call failed */
#define HF_ERR_TIMEOUT (-5)       /* a bounded device-side wait expired */
#define HF_ERR_SHAPE (-6)         /* a size exceeds a documented limit */

/* memory kinds */
#define HF_HOST 0
#define HF_DEVICE 1
#define HF_HOST_ASYNC 2

/* confidence map element types */
#define HF_F32 0
#define HF_F16 1

/* per-point status values written to status_out */
#define HF_STATUS_OK 0
#define HF_STATUS_NO_VIEWS 1    /* the point projects into no view: cost 1, direction = best of ties */
#define HF_STATUS_BAD_INPUT 2   /* non-finite coordinates: direction 0, cost NaN, index -1 */
#define HF_STATUS_FELL_BACK 3   /* learned path only: the proposal was rejected, plain fusion used */

/* limits */
#define HF_MAX_K 16       /* neighbours per point */
#define HF_MAX_T 24       /* refinement rounds */
#define HF_MAX_H 1024     /* hypotheses */
#define HF_MAX_TOPK 16    /* top-K views */

typedef struct hf_ctx hf_ctx;

typedef struct {
    int H;               /* number of hypotheses, 1..HF_MAX_H */
    int k;               /* neighbours per point in the patch, 0..HF_MAX_K */
    int T;               /* refinement rounds, 0..HF_MAX_T */
    int top_k_views;     /* 0: all views that see the point; K>0: the K most confident (Sec. 3.1.2) */
    float fallback_tau;  /* learned path: proposals with cost above tau fall back to plain fusion */
    int flags;           /* reserved, 0 */
} hf_config;

/* Create a context bound to the current CUDA device and to `cuda_stream` (a cudaStream_t; NULL =
 * the legacy default stream).  *out receives the context, or NULL on error. */
int hair_fuse_create(hf_ctx** out, const hf_config* cfg, void* cuda_stream);

/* Rebind the context to another stream (cudaStream_t). */
int hair_fuse_set_stream(hf_ctx* ctx, void* cuda_stream);

/* Upload the V calibrated views (Sec. 3.1: cameras Pi_v, orientation maps O_v, confidence C_v).
 *  cams:  V x 16 f32 per view: fx, fy, cx, cy, R (3x3 row-major, world -> camera), t (3);
 *         camera frame x right, y down, z forward; u = fx X/Z + cx, v = fy Y/Z + cy.
 *  angle: V x height x width f32, orientation angle theta in [0, pi) in pixel axes (+u right,
 *         +v down), row-major (row = v, column = u).
 *  conf:  V x height x width, f32 or IEEE half (conf_dtype HF_F32 / HF_F16), values in [0, 1].
 * Errors: V < 1, width/height < 1, null pointers, bad dtype -> HF_ERR_INVALID_ARG; a map of more
 * than 2^31 pixels or a side above 2^22 pixels -> HF_ERR_SHAPE. */
int hair_fuse_upload_views(hf_ctx* ctx, int V, int width, int height, const float* cams, const float* angle,
                           const void* conf, int conf_dtype, int mem_kind);

/* Upload the raw outer point cloud P_raw (Sec. 3.1) and each point's fusion patch.
 *  xyz: N x 3 f32 world coordinates.
 *  nbr: N x k int32, the k neighbours of each point (excluding the point itself), each in [0, N).
 * Errors: N < 1, k >= N, an index outside [0, N) -> HF_ERR_INVALID_ARG.  The indices are checked
 * by a device kernel and read back, so this call synchronises the stream for either mem_kind. */
int hair_fuse_upload_points(hf_ctx* ctx, int N, const float* xyz, const int32_t* nbr, int mem_kind);

/* Fuse the directions of all uploaded points (Eqs. proj_r .. final_dout, argmin, refinement).
 *  hyps:       H x 3 f32 unit directions (|h| within 1e-3 of 1), or NULL for the built-in
 *              Fibonacci hemisphere z_m = 1 - (m + 1/2)/H, azimuth m pi (3 - sqrt 5).
 *  dir_out:    N x 3 f32, unit direction with canonical sign.
 *  cost_out:   N f32, c_i of the returned direction (may be NULL).
 *  idx_out:    N int32, index of the best hypothesis (may be NULL).
 *  status_out: N uint8, HF_STATUS_* (may be NULL).
 * All of hyps and the outputs are of kind mem_kind.
 * Errors: nothing uploaded -> HF_ERR_NOT_UPLOADED; non-unit hypothesis -> HF_ERR_INVALID_ARG. */
int hair_fuse_fuse_directions(hf_ctx* ctx, const float* hyps, float* dir_out, float* cost_out, int32_t* idx_out,
                              uint8_t* status_out, int mem_kind);

/* Fusion of the points first .. first + count - 1 only: the partition hook for spreading one scene
 * over several GPUs (each uploads the whole scene, so the range's neighbours are available, and
 * fuses its own range).  Every point is projected; the hypothesis argmin and the refinement run on
 * the range.  Outputs have count rows: row q holds point first + q, with exactly the values
 * hair_fuse_fuse_directions gives that point.  Errors as there, plus HF_ERR_INVALID_ARG for a range
 * outside [0, N). */
int hair_fuse_fuse_range(hf_ctx* ctx, int first, int count, const float* hyps, float* dir_out, float* cost_out,
                         int32_t* idx_out, uint8_t* status_out, int mem_kind);

/* ------------------------------------------------------------------------------------------------
 * The paper's own FPMVO step (Sec. 3.1.1-3.1.3), from depth maps instead of a hypothesis set:
 *  - view v sees point i when it projects inside the image and X_z <= D_v(pixel) + eps_vis
 *    (D_v: camera-space depth of the front-most hair, +inf where none);
 *  - candidates (Eqs. 1-3): the pixel u_i^v + lambda_px (cos theta, sin theta) with theta the angle at
 *    u_i^v, its depth z (nearest pixel), S depths z + delta_s spread evenly over [-delta, delta]
 *    (both ends included), back-projected through the offset pixel; unit directions from p_i;
 *  - medoid fusion (Eqs. G, sigma): for each depth layer s, over the top-K views by the confidence
 *    at u_i^v (ties to the lower view), the candidate with the largest
 *    sum_j w_j |<d_i, d_j>| / sum_j w_j (w_j = that confidence), first on ties;
 *  - patch consistency (Eqs. proj_r, sim, patchloss, patch_min, final_dout): each layer's fused
 *    offset point is reprojected into the top-K views, r = Pi_v(p_f) - Pi_v(p_i) normalised, the
 *    largest C |<r, O>| over the P x P pixels around u_i^v, averaged over the views; the best layer
 *    wins (lowest on ties); the direction p_f - p_i normalised with the canonical sign of
 *    hair_fuse_fuse_directions; cost = 1 - that average; sel = the layer (-1 if none).
 * Status: OK, NO_VIEWS (no view sees the point or no view yields a candidate: direction 0, cost 1),
 * BAD_INPUT (non-finite point).  Limits: 1 <= K <= 8, K * S <= 32, P odd in [1, 7].
 * ------------------------------------------------------------------------------------------------ */
typedef struct {
    int K;              /* top-K views */
    int S;              /* depth samples per view */
    int P;              /* patch side in pixels (odd) */
    float lambda_px;    /* pixel offset along the orientation */
    float delta;        /* half range of the depth samples (scene units) */
    float eps_vis;      /* depth-test tolerance (scene units) */
} hf_fpmvo_cfg;

/* Depth maps of the uploaded views: V x H x W f32 (kind mem_kind), copied into the context; the
 * caller keeps ownership of depth.  Upload the views first (HF_ERR_NOT_UPLOADED otherwise);
 * uploading new views requires new depth maps. */
int hair_fuse_upload_depth(hf_ctx* ctx, const float* depth, int mem_kind);
/* FPMVO of every uploaded point into dir_out (N x 3), cost_out (N), sel_out (N int32, may be NULL),
 * status_out (N, may be NULL), all of kind mem_kind and owned by the caller; asynchronous on the
 * context's stream for HF_DEVICE outputs.  Errors: HF_ERR_NOT_UPLOADED without views, points or
 * depth maps of the current views; HF_ERR_INVALID_ARG for a configuration outside the limits above
 * (or lambda_px, delta, eps_vis negative or not finite); CUDA failures as in every other call. */
int hair_fuse_fpmvo(hf_ctx* ctx, const hf_fpmvo_cfg* cfg, float* dir_out, float* cost_out, int32_t* sel_out,
                    uint8_t* status_out, int mem_kind);

/* ------------------------------------------------------------------------------------------------
 * The paper's Parallel Hair Growing consumer (Sec. 3.2): from fused points with directions to
 * strands.  All decisions that turn positions into voxels are single-precision with one rounding per
 * operation (no fused contraction beyond the written FMAs), so results are reproducible bit for bit.
 *  A  volumes: voxel c(p) = floor((p - origin) / voxel) per axis (outside the nx x ny x nz grid: no
 *     voxel); occ[c] = number of valid points in c; T[c] = sum of rint(2^30 fl(d_a d_b)) (int64);
 *  B  ori[c] = dominant eigenvector of T[c] (12 rounds of power iteration from the column with the
 *     largest diagonal, sign z > 0, else y > 0, else x > 0), 0 for an empty voxel;
 *  C  guide strands from S scalp seeds h with normals n, in batches of `batch` seeds: d = n; per step
 *     stop outside the grid; in an empty voxel go on along d only while no occupied voxel was met and
 *     fewer than root_steps steps were taken (a guide that meets none has no strand), else stop; stop
 *     where crowd[c] >= occ_cap; o = ori[c] turned to <o, d> >= 0, stop if <o, d> < cos_turn; d = o;
 *     p += step d; at most max_steps steps.  crowd[c] (deferred occupancy) counts the strands of
 *     earlier batches that entered c: it is updated after each batch;
 *  D  segments: every occupied voxel with crowd 0 after the guides seeds one at its centre, in voxel
 *     order and in batches (a seed whose voxel an earlier batch entered is skipped: 0 vertices),
 *     traced along -ori and +ori by the rules of C without the empty walk; vertices run from the end
 *     of the backward half through the seed to the end of the forward half;
 *  E  linking (Eq. segment_connection): every strand end (a guide tip; both segment ends; outward
 *     tangent t = the last step's direction) takes the nearest end q of another segment with
 *     |p - p_q| < link_dist and <t, -t_q> > link_cos (squared distances compared, ties to the lower
 *     q); joined strands form connected components labelled by their lowest strand index (guides
 *     0 .. S-1, then segments S .. S+K-1).
 * ------------------------------------------------------------------------------------------------ */
typedef struct {
    float origin[3];      /* grid corner (scene units) */
    float voxel;          /* voxel edge > 0 */
    int nx, ny, nz;       /* grid size, (nx + 2)(ny + 2)(nz + 2) < 2^31 */
    float step;           /* tracing step, 0 < step <= voxel */
    int max_steps;        /* steps per trace, 1 .. 4096 */
    int root_steps;       /* empty-voxel steps a guide may take before its first occupied voxel */
    float cos_turn;       /* smallest cosine between consecutive step directions */
    int occ_cap;          /* strands of earlier batches that close a voxel, >= 1 */
    int batch;            /* seeds per batch, >= 1 */
    float link_dist;      /* delta_d, 0 .. 8 voxel */
    float link_cos;       /* cos(delta_theta) */
} hf_phg_cfg;

enum { HF_PHG_MAXLEN = 1, HF_PHG_OUTSIDE = 2, HF_PHG_EMPTY = 3, HF_PHG_CROWDED = 4, HF_PHG_TURN = 5,
       HF_PHG_NO_ROOT = 6 };   /* why a trace stopped */

typedef struct {          /* caller-owned outputs, all of the call's mem_kind */
    int32_t* occ;         /* nvox = nx ny nz points per voxel (index (z ny + y) nx + x) */
    float* ori;           /* nvox x 3 voxel orientations */
    int32_t* crowd;       /* nvox strands that entered each voxel, at the end (may be NULL) */
    float* gverts;        /* S x (max_steps + 1) x 3 guide-strand vertices, the seed first */
    int32_t* glen;        /* S vertex counts (0: no strand) */
    int32_t* gstop;       /* S stop reasons HF_PHG_* (may be NULL) */
    float* gtan;          /* S x 3 tip tangents (may be NULL) */
    long long seg_cap;    /* capacity of the segment arrays */
    float* sverts;        /* seg_cap x (2 max_steps + 1) x 3 segment vertices */
    int32_t* slen;        /* seg_cap vertex counts (0: skipped seed) */
    int64_t* svox;        /* seg_cap seed voxels (may be NULL) */
    float* stan;          /* seg_cap x 2 x 3 outward tangents at the start and the end (may be NULL) */
    int32_t* label;       /* S + seg_cap component labels */
    long long* n_seg;     /* 1: the number K of segment seeds */
} hf_phg_out;

/* The consumer, A to E, on the context's stream (it synchronises once to learn K and once per
 * component round).  pts, dirs: N x 3 f32 points and unit directions (P_out and P_in fused); valid:
 * N u8 (non-zero = use the point; may be NULL); seeds, normals: S x 3 f32.  All pointers of kind
 * mem_kind; inputs are read during the call, outputs written by its end.  Errors: HF_ERR_INVALID_ARG
 * for a configuration outside the limits above or a missing array; HF_ERR_SHAPE when K exceeds
 * seg_cap (n_seg still receives K) or S + seg_cap >= 2^31; CUDA failures as elsewhere. */
int hair_fuse_phg(hf_ctx* ctx, const hf_phg_cfg* cfg, long long N, const float* pts, const float* dirs,
                  const uint8_t* valid, long long S, const float* seeds, const float* normals, hf_phg_out* out,
                  int mem_kind);

/* ------------------------------------------------------------------------------------------------
 * Orientation and confidence maps from images with Gabor filters (Sec. 3.1: O and C extracted
 * "using Gabor filters"; the bank and the response below are readings of an unspecified step):
 *  bank   64 orientations theta_k = k pi / 64 on a 15 x 15 window of offsets (u right, v down);
 *         along a = u cos + v sin, across b = -u sin + v cos; envelope exp(-a^2 / (2 sigma_along^2)
 *         - b^2 / (2 sigma_across^2)); even kernel envelope cos(2 pi b / lambda) minus its window
 *         mean, odd kernel envelope sin(2 pi b / lambda); both rounded to bfloat16;
 *  F_k    sqrt(e_k^2 + o_k^2) of the window correlations with the image rounded to bfloat16 (zero
 *         outside), accumulated in FP32 on the tensor cores;
 *  theta  theta_k* for the largest F_k (first on ties), in [0, pi) in pixel axes (the angle maps'
 *         convention); C = 1 - mean_k F_k / F_k* (0 where all F are 0).
 * ------------------------------------------------------------------------------------------------ */
typedef struct {
    int n_theta;          /* 64 */
    int radius;           /* 7: a 15 x 15 window */
    float sigma_along;    /* envelope along the strand (px) */
    float sigma_across;   /* envelope across (px) */
    float lambda;         /* wavelength across the strand (px) */
} hf_gabor_cfg;

/* The bank as f32 values of its bfloat16 kernels: out[k][0 even, 1 odd][v][u], 64 x 2 x 15 x 15 (host
 * memory).  HF_ERR_INVALID_ARG for a configuration other than the above. */
int hair_fuse_gabor_bank(const hf_gabor_cfg* cfg, float* out);
/* Maps of V images (V x H x W f32) into theta_out and conf_out (V x H x W f32), all of kind
 * mem_kind (caller-owned); asynchronous for HF_DEVICE (the first call with a new sigma / lambda
 * builds the bank on the host and waits for its upload; the context keeps it).  Device scratch:
 * none for HF_DEVICE, the staged images and maps for HF_HOST and HF_HOST_ASYNC (with HF_HOST_ASYNC
 * the images are copied in, the maps computed and copied out on the context's stream without
 * waiting; a device error is reported by the next synchronising call).  The maps can be passed to
 * hair_fuse_upload_views.  Errors: HF_ERR_INVALID_ARG (configuration, sizes, null arrays),
 * HF_ERR_SHAPE (more than 2^31 padded pixels), HF_ERR_TIMEOUT (a bounded device wait expired). */
int hair_fuse_gabor(hf_ctx* ctx, const hf_gabor_cfg* cfg, int V, int H, int W, const float* images, float* theta_out,
                    float* conf_out, int mem_kind);

/* Evaluate the cost c_i(d) of M given directions for every point (no argmin, no refinement).
 *  dirs: N x M x 3 f32 (any non-zero length; the cost is scale- and sign-invariant),
 *  cost_out: N x M f32.  Both of kind mem_kind. */
int hair_fuse_eval_costs(hf_ctx* ctx, int M, const float* dirs, float* cost_out, int mem_kind);

/* Direction fusion that allocates nothing, for callers that may not call cudaMalloc: plugin
 * hosts whose enqueue hooks forbid allocation, processes whose device memory belongs to a
 * framework's caching allocator, real-time code with a fixed memory budget.  The paper has no
 * counterpart; it computes exactly what upload_views + upload_points + fuse_directions compute.
 *  - All pointers are device memory of the current device: cams, angle, conf, xyz, nbr and hyps
 *    (NULL = built-in set) as in those calls; dir_out (required), cost_out, idx_out, status_out
 *    (each may be NULL) as in hair_fuse_fuse_directions.  cfg gives H, k, T and top_k_views.
 *  - The scratch between the kernels is one static device array of 20,988,672 bytes (20.0 MiB)
 *    inside this library, which every GPU that loads the library holds until the process exits.
 *    Limits: N * V' <= 1,048,576 (V' = V rounded up to even), N <= 262,144, V <= 1024,
 *    V * Hq <= 65,536 (Hq = H rounded up to a multiple of 32); larger inputs are rejected with
 *    HF_ERR_SHAPE before any work is queued.
 *  - The first call on a device looks the array's device address up (cudaGetSymbolAddress, with
 *    that device current); make that first call before any stream capture.
 *  - Every call on a device shares the one array and leaves its contents behind; the call clears
 *    what must start at zero.  Calls whose GPU work overlaps (different host threads or streams
 *    on the same device) race on the array and corrupt each other's results.
 *  - The call runs on cuda_stream (a cudaStream_t) and waits for it before returning: it checks
 *    the neighbour indices (-> HF_ERR_INVALID_ARG) before the fusion reads through them, and
 *    reports a non-unit hypothesis (-> HF_ERR_INVALID_ARG) after it.
 *  - Messages are read with hair_fuse_last_error(NULL). */
int hair_fuse_fuse_directions_noalloc(const hf_config* cfg, int N, int V, int width, int height, const float* cams,
                                      const float* angle, const void* conf, int conf_dtype, const float* xyz,
                                      const int32_t* nbr, const float* hyps, float* dir_out, float* cost_out,
                                      int32_t* idx_out, uint8_t* status_out, void* cuda_stream);

/* The tensor-core GEMM the learned proposal network is built on (tcgen05, BF16 operands, FP32
 * accumulation in tensor memory).  The paper has no counterpart: the proposal network is an
 * addition to the method that replaces most refinement rounds.
 *  C[M x N] (f32, row-major) = A[M x K] . B[N x K]^T with A, B row-major IEEE bf16 bits.
 * All pointers are device memory (16-byte aligned); N a multiple of 16, K a multiple of 64.
 * Runs on cuda_stream and waits for it. */
int hair_fuse_gemm_bf16(const uint16_t* A, const uint16_t* B, float* C, int M, int N, int K, void* cuda_stream);

/* The same GEMM with the limit of its pipeline's bounded waits set to wait_ns nanoseconds (0: the
 * default 2 s), for exercising the timeout path (the paper has no counterpart).  When a wait runs
 * out the CTA records the expiry, waits (up to 2 s) for the copies and tensor-core operations it has
 * already issued, which complete by themselves, releases its tensor memory and writes no output;
 * the call then returns HF_ERR_TIMEOUT (C is left unspecified) and the next call starts clean. */
int hair_fuse_gemm_bf16_bounded(const uint16_t* A, const uint16_t* B, float* C, int M, int N, int K,
                                unsigned long long wait_ns, void* cuda_stream);

/* The GELU that the network's inference epilogues apply, y[i] = gelu(x[i]) for n FP32 values
 * (device pointers, n >= 0; x and y may be the same array), asynchronous on cuda_stream; for
 * testing.  gelu(x) = x Phi(x) from a polynomial on x clamped to [-5, 5]; |gelu(x) - x Phi(x)| <=
 * 4.1e-7 |x| for finite x (NaN propagates).  The paper has no counterpart (the network is not in
 * it).  Returns HF_ERR_INVALID_ARG for n < 0 or a NULL pointer with n > 0. */
int hair_fuse_gelu_eval(const float* x, float* y, long long n, void* cuda_stream);

/* ------------------------------------------------------------------------------------------------
 * Learned proposal network.  The paper has no counterpart: a small MLP maps per-point multi-view
 * orientation features to an initial direction that a short refinement finishes, replacing most of
 * the hypothesis search; points whose refined proposal costs more than a threshold fall back to the
 * plain fusion above, which also provides the training targets.
 *  features x (51, zero-padded to 64, bf16): for the 16 views v_m = floor(m V / 16),
 *    (sin 2 theta, cos 2 theta, C) at the point's pixel (zeros outside the view), then
 *    (p - centre) / half_extent of the points' bounding box (half_extent = largest half side);
 *  network: 64 -> 256 -> 256 -> 3, GELU x Phi(x) on both hidden layers (training: erff;
 *    inference: the polynomial of hair_fuse_gelu_eval), BF16 operands, FP32
 *    accumulation and FP32 master weights; proposal = y / |y|;
 *  loss per sample 1 - (y_hat . t)^2 (sign-invariant), mean over the batch; Adam (0.9, 0.999, 1e-8).
 *  Parameter vector (f32, hair_fuse_mlp_param_count() entries): W1 [256 x 64] (columns 51..63 zero),
 *  b1 [256], W2 [256 x 256], b2 [256], W3 [3 x 256], b3 [3].
 * ------------------------------------------------------------------------------------------------ */
typedef struct hf_mlp hf_mlp;

long long hair_fuse_mlp_param_count(void);
/* Network with training buffers for batches of up to max_batch (a multiple of 128, <= 65536)
 * samples, working on cuda_stream. */
int hair_fuse_mlp_create(hf_mlp** out, int max_batch, void* cuda_stream);
void hair_fuse_mlp_destroy(hf_mlp* mlp);
/* Uniform(-1/sqrt(fan_in), +1/sqrt(fan_in)) weights and biases from a counter-based hash of seed;
 * Adam state and step counter reset. */
int hair_fuse_mlp_init(hf_mlp* mlp, uint64_t seed);
int hair_fuse_mlp_set_params(hf_mlp* mlp, const float* params, int mem_kind);
int hair_fuse_mlp_get_params(hf_mlp* mlp, float* params, int mem_kind);
/* `steps` Adam steps with learning rate lr on batches of `batch` samples drawn with replacement from
 * X (n_samples x 64 bf16, device) and T (n_samples x 3 f32 unit targets, device); sample b of step s
 * is hash(seed, s, b) mod n_samples.  use_graph != 0 captures one step in a CUDA graph and replays
 * it.  loss_out (host, may be NULL) receives the mean loss of each step.  Synchronous. */
int hair_fuse_mlp_train(hf_mlp* mlp, const uint16_t* X, const float* T, long long n_samples, int batch, int steps,
                        float lr, uint64_t seed, int use_graph, float* loss_out);
/* Gradients (host, parameter-vector layout) of the mean loss on the batch the next training step
 * would draw, without updating anything; the batch itself (xb_out batch x 64 bf16, tb_out batch x 3,
 * host, may be NULL) and its loss (host, may be NULL) are returned for checking.  Synchronous. */
int hair_fuse_mlp_grads(hf_mlp* mlp, const uint16_t* X, const float* T, long long n_samples, int batch, uint64_t seed,
                        float* grads_out, float* loss_out, uint16_t* xb_out, float* tb_out);
/* Proposals dir_out (n x 3, unit) for features X (n x 64 bf16), both of kind mem_kind. */
int hair_fuse_mlp_forward(hf_mlp* mlp, const uint16_t* X, int n, float* dir_out, int mem_kind);
/* The same forward pass, writing the head's raw outputs y = W3 h2 + b3 (n x 3, before the
 * normalisation) to y_out. */
int hair_fuse_mlp_forward_raw(hf_mlp* mlp, const uint16_t* X, int n, float* y_out, int mem_kind);
/* Parameters, Adam state and step counter to / from a binary file (magic "HFMLP001"). */
int hair_fuse_mlp_save(hf_mlp* mlp, const char* path);
int hair_fuse_mlp_load(hf_mlp* mlp, const char* path);
const char* hair_fuse_mlp_last_error(const hf_mlp* mlp);
/* Test hook (no counterpart in the paper) for the inference kernel's expiry path.  wait_ns > 0
 * limits every wait of its pipeline (mbarrier waits on copies, tensor-core steps and the other
 * warps) to wait_ns nanoseconds instead of the default 2 s, and makes the producer, once it has
 * issued the first tile's layer-1 steps, wait on a barrier that nothing completes, so the limit
 * always expires there.  On expiry every warp stops; the kernel waits, up to the default limit,
 * for the copies and tensor-core work it already issued (they complete by themselves), releases
 * its tensor memory and writes no further output; the call returns HF_ERR_TIMEOUT.  wait_ns = 0
 * restores normal operation.  Applies to hair_fuse_mlp_forward(_raw), the learned fusion and the
 * batches that use this network. */
int hair_fuse_mlp_set_wait_limit(hf_mlp* mlp, unsigned long long wait_ns);

/* Features (N x 64 bf16, kind mem_kind) of the uploaded scene's points, as the learned fusion
 * computes them: the projection writes the view part (it also refreshes the context's per-view
 * samples, which the next fusion recomputes anyway), then the position part.  A device x_out that
 * is not 16-byte aligned is filled through a copy.  Errors: NULL arguments or a bad mem_kind ->
 * HF_ERR_INVALID_ARG; no views or points uploaded -> HF_ERR_NOT_UPLOADED; HF_ERR_OOM, HF_ERR_CUDA. */
int hair_fuse_features(hf_ctx* ctx, uint16_t* x_out, int mem_kind);

/* Learned fusion of all uploaded points: proposal from the network and its cost c_i; points whose
 * proposal cost exceeds tau are fused by the plain path (H hypotheses, T rounds) and get status
 * HF_STATUS_FELL_BACK; the others get T_short refinement rounds from the proposal, starting with
 * step alpha_short (radians, halved each round).  Outputs as in hair_fuse_fuse_directions
 * (idx_out = -1 for refined proposals); n_fallback (host, may be NULL; reading it synchronises)
 * receives the number of fallback points. */
int hair_fuse_fuse_learned(hf_ctx* ctx, hf_mlp* mlp, int T_short, float alpha_short, float tau, float* dir_out,
                           float* cost_out, int32_t* idx_out, uint8_t* status_out, int* n_fallback, int mem_kind);

/* ------------------------------------------------------------------------------------------------
 * Batched serving: the fusion of many uploaded scenes (contexts) of uneven point count, view count
 * and map size in one submission.  Each stage of the path is ONE persistent launch over the
 * (scene, tile) items of all scenes, the proposal network (when given) runs once over the feature
 * rows of all scenes, and the stage sequence is captured in one CUDA graph that every run replays.
 * A scene's results are bit-identical to hair_fuse_fuse_directions (mlp == NULL, built-in
 * hypotheses) or hair_fuse_fuse_learned (mlp given) on that scene alone.
 *
 * Ownership: the batch keeps pointers to the contexts and to the output buffers; both must outlive
 * it (and the contexts must not be re-uploaded while it exists).  The batch allocates its own
 * scratch (features, proposals, hidden activations, fallback lists: about 660 bytes per point of
 * the batch with a network, none without) and runs on its own stream, ordered after cuda_stream at
 * every run and ordering cuda_stream after itself.  Train or load the network before creating the
 * batch.
 * ------------------------------------------------------------------------------------------------ */
/* per-kernel (or per-stage) timing record */
typedef struct {
    char name[32];
    int launches;
    double total_ms;
} hf_kernel_time;
typedef struct hf_batch hf_batch;

#define HF_MAX_BATCH_SCENES 64

typedef struct {
    int T_short;        /* learned: refinement rounds from the proposal, 1..HF_MAX_T */
    float alpha_short;  /* learned: first rotation step (radians), halved each round */
    float tau;          /* learned: fallback threshold on the proposal's cost */
    int autotune;       /* 1: at the first run, time the candidate launch shapes on the batch and keep the fastest */
    int cta_threads;    /* threads per CTA of the cost kernels: 0 = tuned / default 128, else 64, 128, 256 */
    int order;          /* scene order of the work list: 0 = tuned (heaviest or lightest first), 1 = heaviest
                         * first, 2 = as given, 3 = lightest first (small scenes complete early) */
} hf_batch_cfg;

/* n_scenes (1..HF_MAX_BATCH_SCENES) contexts with views and points uploaded; mlp = NULL for the
 * plain fusion.  cfg may be NULL (defaults, plain only).  Errors: HF_ERR_INVALID_ARG, _SHAPE,
 * _NOT_UPLOADED, _OOM, _CUDA (message via hair_fuse_batch_last_error(NULL)). */
int hair_fuse_batch_create(hf_batch** out, hf_ctx* const* scenes, int n_scenes, hf_mlp* mlp,
                           const hf_batch_cfg* cfg, void* cuda_stream);
/* Device output buffers of scene `scene` (as in hair_fuse_fuse_directions; cost_out is required
 * with a network).  Must be set for every scene before the first run; changing them re-captures. */
int hair_fuse_batch_set_outputs(hf_batch* b, int scene, float* dir_out, float* cost_out, int32_t* idx_out,
                                uint8_t* status_out);
/* Enqueue one fusion of every scene (asynchronous).  use_graph != 0 replays the captured graph
 * (captured at the first such call, after one eager run; autotuning, if enabled, runs first). */
int hair_fuse_batch_run(hf_batch* b, int use_graph);
/* Wait for the batch and return any error latched on the device. */
int hair_fuse_batch_sync(hf_batch* b);
/* Per-scene completion time of the last run in ms after its start (device global timer: the CTA
 * finishing a scene's last tile stamps it), ms_out[n_scenes], host.  Synchronises. */
int hair_fuse_batch_latency(hf_batch* b, double* ms_out);
/* Per-scene fallback counts of the last learned run (0 for the plain fusion), host.  Synchronises. */
int hair_fuse_batch_fallbacks(hf_batch* b, int* n_out);
/* The launch shape in use: out2 = {threads per CTA of the cost kernels, scene order (1 heaviest first,
 * 2 as given, 3 lightest first)}. */
int hair_fuse_batch_tuning(const hf_batch* b, int* out2);
/* 1 when the batch took its launch shape from an earlier batch of the same shape class in this
 * process (autotune results are cached per class: learned or plain, patch width, scene count, total
 * points and total views each within a factor of two, the fixed cta_threads / order), 0 when it was
 * timed on this batch or not tuned, or a negative error code. */
int hair_fuse_batch_tuned_from_cache(const hf_batch* b);
/* One eager run with CUDA events between the stages (synchronous): per-stage records as in
 * hair_fuse_profile_read (the network's stage counts its two GEMM launches).  Returns the number of
 * stages (records beyond max_entries are dropped) or a negative error code. */
int hair_fuse_batch_profile_run(hf_batch* b, hf_kernel_time* out, int max_entries);
/* Kernel launches issued so far (graph replays counted by their kernels), and from the last run the
 * (point, view) pairs in the points' view sets of all scenes and, for the learned path, of the
 * fallback points and of the accepted proposals (any pointer may be NULL; the work counts
 * synchronise). */
int hair_fuse_batch_stats(hf_batch* b, long long* launches, long long* point_views, long long* fallback_point_views,
                          long long* accepted_point_views);
void hair_fuse_batch_destroy(hf_batch* b);
const char* hair_fuse_batch_last_error(const hf_batch* b);

/* Work of the last hair_fuse_fuse_learned call (synchronises): the (point, view) pairs in the view
 * sets of the fallback points and of the accepted (refined) proposals (either pointer may be NULL). */
int hair_fuse_learned_work(hf_ctx* ctx, long long* fallback_point_views, long long* accepted_point_views);

/* The built-in hypothesis set (host memory): H x 3 f32 Fibonacci hemisphere directions. */
int hair_fuse_fibonacci_hemisphere(int H, float* out);

/* FP32 issue-rate microbenchmark: the measured peak that the cost kernels' rooflines divide by.
 * The paper has no counterpart.  kind selects the instruction timed:
 *   HF_ISSUE_FFMA      scalar fma.rn.f32 (1 operation per lane)
 *   HF_ISSUE_FFMA2     packed fma.rn.f32x2 (2 operations per lane)
 *   HF_ISSUE_FMUL2     packed mul.rn.f32x2 (2 operations per lane)
 *   HF_ISSUE_FMAX_ABS  max(|x|, y) as the patch maximum writes it
 *   HF_ISSUE_FMAX3     three-input max.f32 (2 operations)
 *   HF_ISSUE_PATCH     the patch term's inner step for two directions and one patch member:
 *                      mul.rn.f32x2 + fma.rn.f32x2 + two max of |x| (2 evaluations, counted as
 *                      3 operations each: multiply, multiply-add, maximum)
 *   HF_ISSUE_FMAX3_ABS three-input max.f32 of a running maximum and two absolute values (2 operations)
 *   HF_ISSUE_PATCH3    the patch term's inner step for two directions and two patch members:
 *                      2 mul.rn.f32x2 + 2 fma.rn.f32x2 + two three-input maxima of |x| (4
 *                      evaluations, 12 operations)
 *   HF_ISSUE_PATCH3S   HF_ISSUE_PATCH3 with scalar products: 4 mul.rn.f32 + 4 fma.rn.f32 + two
 *                      three-input maxima of |x| (4 evaluations, 12 operations)
 * Each thread of a full-occupancy grid of 256-thread CTAs runs iters x 16 steps of 8 independent
 * chains; one short untimed launch precedes the timed one (CUDA events on cuda_stream, a cudaStream_t;
 * the call waits for it and allocates a small result buffer).  Outputs (host): instr_out = thread-level
 * instructions of the kind issued (4 per step for HF_ISSUE_PATCH, 6 for HF_ISSUE_PATCH3, 10 for
 * HF_ISSUE_PATCH3S), ops_out =
 * operations as above,
 * ms_out = the timed launch's duration; instr_out and ops_out may be NULL.
 * Errors: HF_ERR_INVALID_ARG (unknown kind, iters < 1, null ms_out), HF_ERR_OOM, HF_ERR_CUDA. */
#define HF_ISSUE_FFMA 0
#define HF_ISSUE_FFMA2 1
#define HF_ISSUE_FMUL2 2
#define HF_ISSUE_FMAX_ABS 3
#define HF_ISSUE_FMAX3 4
#define HF_ISSUE_PATCH 5
#define HF_ISSUE_FMAX3_ABS 6
#define HF_ISSUE_PATCH3 7
#define HF_ISSUE_PATCH3S 8
int hair_fuse_issue_rate(int kind, int iters, void* cuda_stream, double* instr_out, double* ops_out, float* ms_out);

/* Allocation-failure hook for testing the error paths (the paper has no counterpart): after
 * hair_fuse_fail_alloc_after(n) with n >= 0, the (n + 1)-th device allocation that a context makes
 * for its buffers from then on fails as if the device were out of memory (once; the call that needed
 * it returns HF_ERR_OOM with nothing else changed); n < 0 disables the hook.  Process-wide; meant
 * for single-threaded tests. */
int hair_fuse_fail_alloc_after(int n);

/* Wait for the context's stream and return any error latched on the device. */
int hair_fuse_sync(hf_ctx* ctx);

/* Per-kernel timing with CUDA events recorded on the context's stream around every launch.
 * hair_fuse_profile(ctx, 1) clears and enables it; hair_fuse_profile_read() synchronises and
 * fills up to max_entries records, returning how many kernels have records. */
int hair_fuse_profile(hf_ctx* ctx, int enable);
int hair_fuse_profile_read(hf_ctx* ctx, hf_kernel_time* out, int max_entries);

/* Number of (point, view) pairs in the points' view sets V_i at the last fuse or eval call
 * (synchronises the stream): the unit of work of the cost evaluation. */
int hair_fuse_work(hf_ctx* ctx, long long* point_views);

/* Bytes of device memory the context holds and the number of kernel launches it has issued
 * (kernels of this library only). */
int hair_fuse_stats(const hf_ctx* ctx, long long* device_bytes, long long* launches);

void hair_fuse_destroy(hf_ctx* ctx);

/* Message of the last error on this context (never NULL); ctx may be NULL for create errors. */
const char* hair_fuse_last_error(const hf_ctx* ctx);

#ifdef __cplusplus
}
#endif

#endif /* HAIR_FUSE_H */
