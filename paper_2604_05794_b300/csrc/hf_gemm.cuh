// hf_gemm.cuh - interface of the tcgen05 GEMM (hf_gemm.cu) used by the learned proposal network.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

// Epilogues of C = A . B^T (+ bias):
enum {
    EPI_STORE = 0,        // C[row][n] = acc + bias[n] (f32)
    EPI_ATOMIC = 1,       // C[row][n] += acc (+ bias[n] from split 0): split-K partial sums (f32)
    EPI_GELU_TRAIN = 2,   // Z = acc + bias (f32), H = bf16(gelu(Z)), HT = H transposed (bf16)
    EPI_PARTIAL = 5,      // C[split z][row][n] = acc: split-K partial tiles, summed afterwards in a fixed order
};

struct GemmArgs {
    int M, N, K;              // rows of A and C, rows of B (= columns of C), reduction length (multiple of 64)
    int kchunks_per_split;    // 64-wide K chunks per CTA along gridDim.z
    float* C;
    int ldc;
    const float* bias;        // [N] or null
    float* Z;
    int ldz;
    uint16_t* H;
    int ldh;
    uint16_t* HT;
    int ldht;
    const float* w3;          // inference head: 3 x 256 f32 (values of the bf16 layer-3 weights)
    const float* b3;          // inference head: 3
    float* dir_out;           // inference: M x 3
    int head_raw;             // inference: write y itself instead of y / |y|
    uint32_t* errw;           // device error word (HF_DEV_ERR_TIMEOUT)
    long long split_stride;   // EPI_PARTIAL: elements between the partial tiles of consecutive splits
    int stages;               // set by hf_gemm_tn: operand ring depth
    unsigned long long wait_ns;   // limit of the pipeline's waits (0: kWaitTimeoutNs); the drain after an
                                  // expiry always waits up to kWaitTimeoutNs for work that completes by itself
};

// 2D bf16 tensor map of a row-major [rows x cols] matrix (cols a multiple of 64, base 16-byte
// aligned) with a {64, box_rows} box and the 128-byte swizzle.
cudaError_t hf_make_tmap_bf16(CUtensorMap* map, const void* base, long long rows, long long cols, int box_rows);

// 2D bf16 tensor map of a row-major [rows x 16] matrix (32-byte rows, base 16-byte aligned) with a
// {16, box_rows} box and the 32-byte swizzle: one box is one K = 16 step of a tcgen05 operand.
cudaError_t hf_make_tmap_bf16_rows32(CUtensorMap* map, const void* base, long long rows, int box_rows);

// C = A . B^T with the given epilogue; ta: A map (box 128 rows), tb: B map (box bn rows).
cudaError_t hf_gemm_tn(int epi, int bn, const CUtensorMap& ta, const CUtensorMap& tb, const GemmArgs& g, int splits,
                       cudaStream_t s);

// The proposal network's whole inference in one persistent kernel (the hidden layer stays in
// tensor memory): tx the features [M x 64] (box 128 rows), tw1 W1 [256 x 64] and tw2 W2
// [256 x 256] (box 256 rows); g.bias = b1, b2 the layer-2 bias, g.w3 / g.b3 the head, g.dir_out
// (M x 3), g.head_raw, g.errw, g.wait_ns (0: the default limit).
cudaError_t hf_mlp_fused(const CUtensorMap& tx, const CUtensorMap& tw1, const CUtensorMap& tw2, const GemmArgs& g,
                         const float* b2, cudaStream_t s);
