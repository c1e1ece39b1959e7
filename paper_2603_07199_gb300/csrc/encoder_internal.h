// State of a depth encoder shared by its forward pass (k_encoder.cu) and its trainer
// (k_encoder_train.cu); internal to the library.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "mppi.h"

struct mppi_encoder {
    int H = 0, W = 0, max_images = 0;
    int h[5] = {0, 0, 0, 0, 0}, w[5] = {0, 0, 0, 0, 0};   // sizes of x_0 .. x_4
    cudaStream_t stream = nullptr;
    float* wt[4] = {nullptr, nullptr, nullptr, nullptr};  // [co][ci][3][3] as given
    float* bias[4] = {nullptr, nullptr, nullptr, nullptr};
    float* W5 = nullptr;
    float* b5 = nullptr;
    float* act[4] = {nullptr, nullptr, nullptr, nullptr};  // x_1 .. x_4 of the last encoded batch
    int n_sms = 152;
    int conv_path = MPPI_ENC_CONV_TC;   // which convolution kernels mppi_encode_depth runs
    int* d_err = nullptr;               // device error word of the tensor-core kernels' bounded waits
    int inject_timeout = 0;             // test hook: the next encoding's first convolution waits in vain
    uint8_t* wpack[4] = {nullptr, nullptr, nullptr, nullptr};  // conv weights, BF16 hi / lo operand stages
    uint8_t* dgpack[4] = {nullptr, nullptr, nullptr, nullptr}; // the same per parity class for input gradients (1..3)
    char err[512] = "";
};

namespace mppi {
constexpr int kEncCin[4] = {1, 16, 32, 64};
constexpr int kEncCout[4] = {16, 32, 64, 64};
// tensor-core convolution of encoder layer 0..3 (k_encoder_tc.cu); configure once per encoder;
// the weights are read from their packed form, which pack_conv_tc_weights refreshes from wt[]
// (at creation and after every optimiser step)
cudaError_t configure_conv_tc();
size_t conv_tc_packed_bytes(int layer);
size_t conv_dgrad_tc_packed_bytes(int layer);
cudaError_t pack_conv_tc_weights(const float* const* wt, uint8_t* const* out, uint8_t* const* out_dgrad,
                                 cudaStream_t s);
// inject != 0 (a test hook): the launch's first weight wait waits for a phase that never completes,
// so every CTA gives up after its bounded wait and sets *err
cudaError_t launch_conv_tc(int layer, const float* x, int n_img, int H, int W, int Ho, int Wo, const uint8_t* wpack,
                           const float* b, float scale, float* y, int* err, int inject, cudaStream_t s);
// weight gradient of layer 0..3 on the tensor cores: partial sums of `slices` pixel slices of
// stages_per_slice x conv_wgrad_tc_stage_pixels() output pixels into ws[slice][c_out][9 c_in + 1]
int conv_wgrad_tc_stage_pixels();
int conv_wgrad_tc_k_tiles(int layer);
// input gradient (ReLU mask of the input applied) of layer 1..3 on the tensor cores
cudaError_t launch_conv_dgrad_tc(int layer, const float* delta, const uint8_t* wpack, const float* x_in, int n_img,
                                 int H, int W, int Ho, int Wo, float* delta_in, int* err, cudaStream_t s);
cudaError_t launch_conv_wgrad_tc(int layer, const float* x, const float* delta, int n_img, int H, int W, int Ho, int Wo,
                                 float scale, int slices, int stages_per_slice, float* ws, int* err, cudaStream_t s);
}  // namespace mppi
