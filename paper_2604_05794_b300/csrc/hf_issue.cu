// hf_issue.cu - FP32 issue-rate microbenchmark: the measured denominator of the cost kernels'
// rooflines.  The paper has no counterpart.
//
// Each thread runs `iters` iterations of a body of 8 independent dependency chains unrolled 16
// times (128 instructions of the measured kind per iteration, so the loop's own counter, compare
// and branch are under 2 % of the issue slots).  The grid is the occupancy limit of 256-thread
// CTAs on every SM, so each SM sub-partition holds at least 8 warps with 8 chains each: enough
// independent work to cover the pipeline latencies, so the rate measured is the issue / pipe rate.
// Operands come from kernel arguments (unknown to the compiler) and every chain's value is stored
// at the end, so nothing is folded or dropped.  The instructions are written in inline PTX so that
// the measured kind is exactly the instruction the cost kernels issue.
#include "hf_internal.cuh"

namespace {

typedef unsigned long long f32x2;

__device__ __forceinline__ f32x2 pk2(float a, float b) {
    f32x2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ float lo2(f32x2 r) {
    float a, b;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(r));
    return a + b;
}

constexpr int kChains = 8;
constexpr int kUnroll = 16;
constexpr int kThreads = 256;

// kind bodies: one instruction of the kind per chain per unrolled step
template <int KIND>
__global__ void __launch_bounds__(kThreads) k_issue(int iters, float a, float b, float* out) {
    float x[kChains];
    f32x2 y[kChains];
    float m0[kChains], m1[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) {
        x[c] = 1.0f + c * 1e-3f + threadIdx.x * 1e-6f;
        y[c] = pk2(x[c], x[c] + 0.5f);
        m0[c] = x[c];
        m1[c] = x[c] + 0.25f;
    }
    const f32x2 A = pk2(a, a), B = pk2(b, b);
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
#pragma unroll
            for (int c = 0; c < kChains; ++c) {
                if (KIND == HF_ISSUE_FFMA) {
                    asm("fma.rn.f32 %0, %0, %1, %2;" : "+f"(x[c]) : "f"(a), "f"(b));
                } else if (KIND == HF_ISSUE_FFMA2) {
                    asm("fma.rn.f32x2 %0, %0, %1, %2;" : "+l"(y[c]) : "l"(A), "l"(B));
                } else if (KIND == HF_ISSUE_FMUL2) {
                    asm("mul.rn.f32x2 %0, %0, %1;" : "+l"(y[c]) : "l"(A));
                } else if (KIND == HF_ISSUE_FMAX_ABS) {
                    // m = max(|m|, a): the patch maximum's max-of-absolute-value
                    asm("{ .reg .f32 t; abs.f32 t, %0; max.f32 %0, t, %1; }" : "+f"(x[c]) : "f"(a));
                } else if (KIND == HF_ISSUE_FMAX3) {
                    // three-input maximum (sm_100 and later)
                    asm("max.f32 %0, %0, %1, %2;" : "+f"(x[c]) : "f"(a), "f"(b));
                } else if (KIND == HF_ISSUE_FMAX3_ABS) {
                    // m = max(m, |x|, |y|): two patch members folded into a running maximum
                    asm("{ .reg .f32 t, u; abs.f32 t, %1; abs.f32 u, %2; max.f32 %0, %0, t, u; }"
                        : "+f"(x[c]) : "f"(m0[c]), "f"(m1[c]));
                    m0[c] = x[c];
                } else if (KIND == HF_ISSUE_PATCH3) {
                    // four evaluations (hypotheses m, m+1 of members j, j+1): two packed products per
                    // member, then one three-input maximum of absolute values per hypothesis
                    f32x2 u, w;
                    const f32x2 S0 = pk2(m0[c], m0[c]), S1 = pk2(m1[c], m1[c]);
                    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(u) : "l"(B), "l"(S0));
                    asm("fma.rn.f32x2 %0, %1, %2, %0;" : "+l"(u) : "l"(A), "l"(S0));
                    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(w) : "l"(B), "l"(S1));
                    asm("fma.rn.f32x2 %0, %1, %2, %0;" : "+l"(w) : "l"(A), "l"(S1));
                    float u0, u1, w0, w1;
                    asm("mov.b64 {%0, %1}, %2;" : "=f"(u0), "=f"(u1) : "l"(u));
                    asm("mov.b64 {%0, %1}, %2;" : "=f"(w0), "=f"(w1) : "l"(w));
                    asm("{ .reg .f32 t, v; abs.f32 t, %1; abs.f32 v, %2; max.f32 %0, %0, t, v; }"
                        : "+f"(m0[c]) : "f"(u0), "f"(w0));
                    asm("{ .reg .f32 t, v; abs.f32 t, %1; abs.f32 v, %2; max.f32 %0, %0, t, v; }"
                        : "+f"(m1[c]) : "f"(u1), "f"(w1));
                } else if (KIND == HF_ISSUE_PATCH3S) {
                    // four evaluations as PATCH3 with scalar products: 4 mul.rn.f32 + 4 fma.rn.f32
                    // + two three-input maxima of |x|
                    float u0, u1, w0, w1;
                    asm("mul.rn.f32 %0, %1, %2;" : "=f"(u0) : "f"(b), "f"(m0[c]));
                    asm("mul.rn.f32 %0, %1, %2;" : "=f"(u1) : "f"(a), "f"(m0[c]));
                    asm("mul.rn.f32 %0, %1, %2;" : "=f"(w0) : "f"(b), "f"(m1[c]));
                    asm("mul.rn.f32 %0, %1, %2;" : "=f"(w1) : "f"(a), "f"(m1[c]));
                    asm("fma.rn.f32 %0, %1, %2, %0;" : "+f"(u0) : "f"(a), "f"(m0[c]));
                    asm("fma.rn.f32 %0, %1, %2, %0;" : "+f"(u1) : "f"(b), "f"(m0[c]));
                    asm("fma.rn.f32 %0, %1, %2, %0;" : "+f"(w0) : "f"(a), "f"(m1[c]));
                    asm("fma.rn.f32 %0, %1, %2, %0;" : "+f"(w1) : "f"(b), "f"(m1[c]));
                    asm("{ .reg .f32 t, v; abs.f32 t, %1; abs.f32 v, %2; max.f32 %0, %0, t, v; }"
                        : "+f"(m0[c]) : "f"(u0), "f"(w0));
                    asm("{ .reg .f32 t, v; abs.f32 t, %1; abs.f32 v, %2; max.f32 %0, %0, t, v; }"
                        : "+f"(m1[c]) : "f"(u1), "f"(w1));
                } else {   // HF_ISSUE_PATCH: two patch-term evaluations (hypotheses m, m+1 of one member)
                    // u = r_x s_x + r_y s_y for the pair, then the two running maxima of |u|
                    f32x2 u;
                    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(u) : "l"(B), "l"(pk2(m0[c], m1[c])));
                    asm("fma.rn.f32x2 %0, %1, %2, %0;" : "+l"(u) : "l"(A), "l"(pk2(m0[c], m1[c])));
                    float u0, u1;
                    asm("mov.b64 {%0, %1}, %2;" : "=f"(u0), "=f"(u1) : "l"(u));
                    asm("{ .reg .f32 t; abs.f32 t, %1; max.f32 %0, %0, t; }" : "+f"(m0[c]) : "f"(u0));
                    asm("{ .reg .f32 t; abs.f32 t, %1; max.f32 %0, %0, t; }" : "+f"(m1[c]) : "f"(u1));
                }
            }
        }
    }
    float s = 0.0f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c] + lo2(y[c]) + m0[c] + m1[c];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

template <int KIND>
cudaError_t run_kind(int iters, float a, float b, float* out, int grid, cudaStream_t s) {
    k_issue<KIND><<<grid, kThreads, 0, s>>>(iters, a, b, out);
    return cudaGetLastError();
}

template <int KIND>
int grid_of() {
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_issue<KIND>, kThreads, 0) != cudaSuccess || per < 1) per = 1;
    return per * (sms > 0 ? sms : 1);
}

cudaError_t launch(int kind, int iters, float a, float b, float* out, int grid, cudaStream_t s) {
    switch (kind) {
        case HF_ISSUE_FFMA: return run_kind<HF_ISSUE_FFMA>(iters, a, b, out, grid, s);
        case HF_ISSUE_FFMA2: return run_kind<HF_ISSUE_FFMA2>(iters, a, b, out, grid, s);
        case HF_ISSUE_FMUL2: return run_kind<HF_ISSUE_FMUL2>(iters, a, b, out, grid, s);
        case HF_ISSUE_FMAX_ABS: return run_kind<HF_ISSUE_FMAX_ABS>(iters, a, b, out, grid, s);
        case HF_ISSUE_FMAX3: return run_kind<HF_ISSUE_FMAX3>(iters, a, b, out, grid, s);
        case HF_ISSUE_FMAX3_ABS: return run_kind<HF_ISSUE_FMAX3_ABS>(iters, a, b, out, grid, s);
        case HF_ISSUE_PATCH3: return run_kind<HF_ISSUE_PATCH3>(iters, a, b, out, grid, s);
        case HF_ISSUE_PATCH3S: return run_kind<HF_ISSUE_PATCH3S>(iters, a, b, out, grid, s);
        default: return run_kind<HF_ISSUE_PATCH>(iters, a, b, out, grid, s);
    }
}

int grid_for(int kind) {
    switch (kind) {
        case HF_ISSUE_FFMA: return grid_of<HF_ISSUE_FFMA>();
        case HF_ISSUE_FFMA2: return grid_of<HF_ISSUE_FFMA2>();
        case HF_ISSUE_FMUL2: return grid_of<HF_ISSUE_FMUL2>();
        case HF_ISSUE_FMAX_ABS: return grid_of<HF_ISSUE_FMAX_ABS>();
        case HF_ISSUE_FMAX3: return grid_of<HF_ISSUE_FMAX3>();
        case HF_ISSUE_FMAX3_ABS: return grid_of<HF_ISSUE_FMAX3_ABS>();
        case HF_ISSUE_PATCH3: return grid_of<HF_ISSUE_PATCH3>();
        case HF_ISSUE_PATCH3S: return grid_of<HF_ISSUE_PATCH3S>();
        default: return grid_of<HF_ISSUE_PATCH>();
    }
}

// instructions of the measured kind per chain per unrolled step
int instr_per_step(int kind) {
    return kind == HF_ISSUE_PATCH ? 4 : (kind == HF_ISSUE_PATCH3 ? 6 : (kind == HF_ISSUE_PATCH3S ? 10 : 1));
}
// operations per chain per unrolled step: lanes of packed instructions count twice, a three-input
// maximum counts as two maxima; for the patch mixes, 3 operations per evaluation (multiply, fused
// multiply-add, maximum) and two or four evaluations
double ops_per_step(int kind) {
    switch (kind) {
        case HF_ISSUE_FFMA2:
        case HF_ISSUE_FMUL2: return 2.0;
        case HF_ISSUE_PATCH: return 6.0;
        case HF_ISSUE_PATCH3:
        case HF_ISSUE_PATCH3S: return 12.0;
        case HF_ISSUE_FMAX3:
        case HF_ISSUE_FMAX3_ABS: return 2.0;
        default: return 1.0;
    }
}

}  // namespace

extern "C" int hair_fuse_issue_rate(int kind, int iters, void* cuda_stream, double* instr_out, double* ops_out,
                                    float* ms_out) {
    if (kind < HF_ISSUE_FFMA || kind > HF_ISSUE_PATCH3S || iters < 1 || !ms_out)
        return HF_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    const int grid = grid_for(kind);
    float* out = nullptr;
    if (cudaMalloc(&out, (size_t)grid * kThreads * sizeof(float)) != cudaSuccess) {
        cudaGetLastError();
        return HF_ERR_OOM;
    }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int rc = HF_OK;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) rc = HF_ERR_CUDA;
    // one untimed launch (clocks up, code loaded), then the timed one
    if (rc == HF_OK && launch(kind, iters < 64 ? iters : 64, 0.999f, 1e-3f, out, grid, s) != cudaSuccess) rc = HF_ERR_CUDA;
    if (rc == HF_OK && cudaEventRecord(e0, s) != cudaSuccess) rc = HF_ERR_CUDA;
    if (rc == HF_OK && launch(kind, iters, 0.999f, 1e-3f, out, grid, s) != cudaSuccess) rc = HF_ERR_CUDA;
    if (rc == HF_OK && cudaEventRecord(e1, s) != cudaSuccess) rc = HF_ERR_CUDA;
    if (rc == HF_OK && cudaEventSynchronize(e1) != cudaSuccess) rc = HF_ERR_CUDA;
    float ms = 0.0f;
    if (rc == HF_OK && cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) rc = HF_ERR_CUDA;
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(out);
    if (rc != HF_OK) {
        cudaGetLastError();
        return rc;
    }
    const double steps = (double)grid * kThreads * (double)iters * kUnroll * kChains;
    *ms_out = ms;
    if (instr_out) *instr_out = steps * instr_per_step(kind);
    if (ops_out) *ops_out = steps * ops_per_step(kind);
    return HF_OK;
}
