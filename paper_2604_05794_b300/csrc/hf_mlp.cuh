// hf_mlp.cuh - device buffers and launchers of the learned proposal network (hf_mlp.cu).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

// bf16 weight copies and the activation / gradient buffers of one training batch (B rows)
struct MlpDev {
    uint16_t *W1b, *W2b, *W2Tb, *W3pb, *W3Tb;   // [256x64] [256x256] [256x256]^T [16x256] [256x64]
    float *w3f, *b3p;                           // [3x256] values of the bf16 W3; [16] padded b3
    uint16_t *Xb, *XTb;                         // [B x 64], [64 x B]
    float* Tb;                                  // [B x 3] targets
    float *Z1, *Z2, *Z3;                        // [B x 256], [B x 256], [B x 16]
    uint16_t *H1, *H1T, *H2, *H2T;              // [B x 256] and transposes
    uint16_t *dZ3, *dZ3T;                       // [B x 64], [16 x B]
    float* dH;                                  // [B x 256]
    uint16_t *dZ2, *dZ2T, *dZ1, *dZ1T;          // [B x 256] and transposes
    float* dW3T;                                // [256 x 16]
    float* parts;                               // split-K partial tiles (<= 64 x 256 x 256)
    float* bparts;                              // per-block partial sums of bias gradients and loss
};

enum {
    TM_X, TM_W1, TM_H1, TM_W2, TM_H2, TM_W3P, TM_H2T, TM_DZ3T, TM_DZ3, TM_W3T, TM_DZ2T, TM_H1T, TM_DZ2, TM_W2T, TM_DZ1T,
    TM_XT, TM_COUNT
};

struct MlpTrain {
    MlpDev d;
    CUtensorMap tm[TM_COUNT];
    float *P, *G, *M, *V;           // parameters, gradients, Adam moments (f32)
    const uint16_t* X;              // training features [n_samples x 64] bf16
    const float* T;                 // training targets [n_samples x 3]
    long long n_samples;
    int B;
    uint64_t seed;
    long long* step;                // device step counter
    float* loss_hist;               // device, one mean loss per step
    float lr;                       // 0: gradients only, no update
    uint32_t* errw;
};

long long hf_mlp_param_count();
cudaError_t hf_launch_init(float* P, uint64_t seed, cudaStream_t s);
cudaError_t hf_launch_pack(const float* P, const MlpDev& d, cudaStream_t s);
// box: 14 floats of device scratch; box[0..5] receives lo[3], hi[3]
cudaError_t hf_launch_bbox(const float* pts, int N, float* box, cudaStream_t s);
// keys[0..2] = 0xffffffff, keys[3..5] = 0: empty box for the projection to fold points into
cudaError_t hf_launch_bbox_init(unsigned* keys, cudaStream_t s);
cudaError_t hf_train_step(const MlpTrain& t, cudaStream_t s);
// raw: the head's raw 3-vectors y instead of the directions y / |y|
// wait_ns: limit of the kernel's pipeline waits (0: the default)
cudaError_t hf_mlp_infer(const MlpDev& d, const float* P, const uint16_t* x, int n, float* dir_out, uint32_t* errw,
                         cudaStream_t s, bool raw = false, unsigned long long wait_ns = 0);

// the network behind the C-ABI handle (hf_mlp_api.cu): inference on n rows of features, and the
// stream the handle was created with
typedef struct hf_mlp hf_mlp;
cudaError_t hf_mlp_infer_rows(hf_mlp* m, const uint16_t* x, long long n, float* dir_out, uint32_t* errw, cudaStream_t s);
cudaStream_t hf_mlp_stream(hf_mlp* m);
