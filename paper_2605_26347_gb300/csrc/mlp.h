// Kernel-surrogate MLP (internal): parameters, buffers and the training / inference steps.
#pragma once

#include <cuda_bf16.h>
#include <stdint.h>

#include <vector>

namespace rimo {

constexpr int MLP_IN = 3, MLP_H = 128, MLP_OUT = 450;
constexpr int MLP_OUT_PAD = 464;  // layer-3 rows padded to a multiple of 16 (MMA N)
constexpr int MLP_K3 = 512;       // row stride of dY (K of dH2 = dY W3) and rows of dY^T (M of dW3)
// FP32 parameter vector: W1 [128][3], b1, W2 [128][128], b2, W3 [450][128], b3
constexpr int MLP_OFF_W1 = 0;
constexpr int MLP_OFF_B1 = MLP_OFF_W1 + MLP_H * MLP_IN;
constexpr int MLP_OFF_W2 = MLP_OFF_B1 + MLP_H;
constexpr int MLP_OFF_B2 = MLP_OFF_W2 + MLP_H * MLP_H;
constexpr int MLP_OFF_W3 = MLP_OFF_B2 + MLP_H;
constexpr int MLP_OFF_B3 = MLP_OFF_W3 + MLP_OUT * MLP_H;
constexpr int MLP_NPARAM = MLP_OFF_B3 + MLP_OUT;

struct Mlp {
    float* P = nullptr;    // FP32 master parameters
    float* G = nullptr;    // gradients
    float* Mom = nullptr;  // Adam first moments
    float* Vel = nullptr;  // Adam second moments
    __nv_bfloat16 *W2b = nullptr, *W2Tb = nullptr, *W3b = nullptr, *W3Tb = nullptr;
    float* loss = nullptr;
    int* status = nullptr;
    int t = 0;
    // activations of the last batch
    int cap = 0;
    float *Z1 = nullptr, *Z2 = nullptr, *Y = nullptr, *dH = nullptr;
    __nv_bfloat16 *H1 = nullptr, *H1T = nullptr, *H2 = nullptr, *H2T = nullptr;
    __nv_bfloat16 *dY = nullptr, *dYT = nullptr, *dZ = nullptr, *dZT = nullptr;
    std::vector<void*> owned;

    ~Mlp();
    void* alloc(size_t bytes);
    void init(uint64_t seed);
    void set_params(const float* host, cudaStream_t s);
    void pack(cudaStream_t s);
    void reserve(int B);
    void forward(const float* X, int B, cudaStream_t s);             // Y [B][464] without b3
    void grads(const float* X, const float* T, int B, cudaStream_t s);
    void step(const float* X, const float* T, int B, float lr, cudaStream_t s);
};

}  // namespace rimo
