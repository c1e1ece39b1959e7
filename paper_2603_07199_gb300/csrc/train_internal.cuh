// Definitions shared by the distillation trainer's FP32 kernels (k_train.cu)
// and its BF16 tensor-core GEMM kernels (k_train_tc.cu): the flat parameter
// layout, the per-batch device buffers and the activation of the Gate-SDF MLP
// (Sec. III-B, Eq. 3: softplus hidden layers of width 128).
#pragma once

#include <cmath>
#include <cstdint>
#include <cuda_runtime.h>

#include "common.cuh"

namespace mppi {
namespace train {

constexpr int kH = kHidden;
constexpr int kIn = 3 + kLatent;
// offsets of the parameters in the flat vector theta: W1 [128][67], b1, W2, b2, W3, b3, W4, b4, w5 [128], b5
constexpr int oW1 = 0;
constexpr int oB1 = oW1 + kH * kIn;
constexpr int oW2 = oB1 + kH;
constexpr int oB2 = oW2 + kH * kH;
constexpr int oW3 = oB2 + kH;
constexpr int oB3 = oW3 + kH * kH;
constexpr int oW4 = oB3 + kH;
constexpr int oB4 = oW4 + kH * kH;
constexpr int oW5 = oB4 + kH;
constexpr int oB5 = oW5 + kH;
constexpr int kNumParams = oB5 + 1;
__host__ __device__ constexpr int offW(int l) { return l == 2 ? oW2 : l == 3 ? oW3 : oW4; }
__host__ __device__ constexpr int offB(int l) { return l == 2 ? oB2 : l == 3 ? oB3 : oB4; }

struct TrainBufs {
    float* theta;        // parameters
    float* grad;         // reduced gradient
    float* partial;      // [n_cta][kNumParams] per-CTA gradient partials of layers 2-4
    float* opart;        // [n_out_cta][kH + 1] per-CTA partials of w5, b5
    float* l1part;       // [n_l1_cta][4][kH] per-CTA partials of W1[:, 0..2], b1
    float* b1p;          // [128] b1 + W1[:, 3:] z0
    float* z0;           // [64]
    const float4* pts;   // batch points (x, y, z, target)
    float* A[5];         // A[l]: [B][128] pre-activations of layer l (1..4)
    float* AT[5];        // AT[l]: [3][B][128] tangents of layer l (2..4)
    float* dA[5];        // adjoints of A[l]
    float* dAT[5];       // adjoints of AT[l]
    float* loss;         // [B] per-point loss
    int* err;            // device error word (bounded waits of the tensor-core kernels)
    int B;
    float beta, lam_e;
};

__device__ __forceinline__ float sp_beta(float a, float beta) {
    return fmaxf(a, 0.f) + log1pf(expf(-beta * fabsf(a))) / beta;
}
__device__ __forceinline__ float sig_beta(float a, float beta) { return 1.f / (1.f + expf(-beta * a)); }

// Input stream s of a hidden layer, element (point pt, feature k), built from the
// layer below: s = 0: sp(A), s = 1..3: sp'(A) * tangent (layer 1's tangent is W1[k, s-1]).
__device__ __forceinline__ float stream_in(const TrainBufs& T, int lower, int s, int pt, int k) {
    const float a = T.A[lower][static_cast<size_t>(pt) * kH + k];
    if (s == 0) return sp_beta(a, T.beta);
    const float t = (lower == 1) ? T.theta[oW1 + k * kIn + (s - 1)]
                                 : T.AT[lower][(static_cast<size_t>(s - 1) * T.B + pt) * kH + k];
    return sig_beta(a, T.beta) * t;
}

// BF16 tensor-core GEMMs of the hidden layers (k_train_tc.cu), launched on `s`
// with `grid` CTAs (grid <= B / 128); the same outputs as the FP32 kernels of
// k_train.cu with BF16 operands and FP32 accumulation.
cudaError_t configure_tc_train();
cudaError_t launch_fwd_hidden_tc(const TrainBufs& T, int l, int grid, cudaStream_t s);
cudaError_t launch_bwd_weight_tc(const TrainBufs& T, int l, int grid, cudaStream_t s);
cudaError_t launch_bwd_input_tc(const TrainBufs& T, int l, int grid, cudaStream_t s);

}  // namespace train
}  // namespace mppi
