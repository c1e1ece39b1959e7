// State of a depth encoder shared by its forward pass (k_encoder.cu) and its trainer
// (k_encoder_train.cu); internal to the library.
#pragma once

#include <cuda_runtime.h>

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
    char err[512] = "";
};

namespace mppi {
constexpr int kEncCin[4] = {1, 16, 32, 64};
constexpr int kEncCout[4] = {16, 32, 64, 64};
}  // namespace mppi
