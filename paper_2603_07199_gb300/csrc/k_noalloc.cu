// Allocation-free variant of the softmax-weight and weighted-update kernels
// (mppi_softmax_update_noalloc): the costs, the noise and the nominal sequence
// come from the caller, the only scratch (the per-block partials of the
// softmax) lives in a file-scope device array, and no call allocates or frees
// memory.  For callers that cannot allocate device memory: code that runs
// inside a CUDA stream capture, real-time control loops that forbid allocation
// after start-up (cudaMalloc can synchronise the device and take unbounded
// time), and hosts whose device memory is owned by another allocator.
#include <cstdio>
#include <mutex>

#include "kernels.h"
#include "mppi.h"

namespace mppi {
namespace {

constexpr int kNaThreads = 128;                          // rollouts per partial
constexpr int kNaMaxBlocks = MPPI_NOALLOC_MAX_K / kNaThreads;
constexpr int kNaUpdThreads = 256;
constexpr int kMaxDevices = 64;

// Per-block (min J, sum exp(-(J - min) / lambda)) partials, 8 KB.  Every GPU that
// loads the library holds one copy until exit; every call on that GPU shares it.
static __device__ __align__(256) float g_noalloc_partials[2 * kNaMaxBlocks];

__device__ __forceinline__ float na_warp_min(float x) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x = fminf(x, __shfl_xor_sync(0xffffffffu, x, o));
    return x;
}
__device__ __forceinline__ float na_warp_sum(float x) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    return x;
}

// Block b: m_b = min of its 128 costs, s_b = sum exp(-(J - m_b) / lambda).
// Every block writes its own two floats, so nothing has to start at zero.
__global__ void __launch_bounds__(kNaThreads) na_partials_kernel(const float* __restrict__ J, int K, float lam,
                                                                 float* __restrict__ part) {
    __shared__ float sh[kNaThreads / 32];
    const int k = blockIdx.x * kNaThreads + threadIdx.x;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const float j = (k < K) ? J[k] : __int_as_float(0x7f800000);
    float m = na_warp_min(j);
    if (lane == 0) sh[wid] = m;
    __syncthreads();
    m = sh[0];
#pragma unroll
    for (int i = 1; i < kNaThreads / 32; ++i) m = fminf(m, sh[i]);
    __syncthreads();
    const float e = (k < K) ? expf(-(j - m) / lam) : 0.f;
    const float s = na_warp_sum(e);
    if (lane == 0) sh[wid] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        float t = sh[0];
#pragma unroll
        for (int i = 1; i < kNaThreads / 32; ++i) t += sh[i];
        part[2 * blockIdx.x] = m;
        part[2 * blockIdx.x + 1] = t;
    }
}

// Block h: rho, eta from the partials (same fixed order in every block),
// w_k = exp(-(J_k - rho) / lambda) / eta, U*_new[h] = sum_k w_k clip(U*_h + delta_{k,h}).
__global__ void __launch_bounds__(kNaUpdThreads) na_update_kernel(const float* __restrict__ J,
                                                                  const float4* __restrict__ noise,
                                                                  const float4* __restrict__ nominal, int K,
                                                                  StepParams P, const float* __restrict__ part,
                                                                  float4* __restrict__ unew, float* __restrict__ w_out) {
    __shared__ float4 sh[kNaUpdThreads / 32];
    __shared__ float s_rho, s_eta;
    const int h = blockIdx.x;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int nb = (K + kNaThreads - 1) / kNaThreads;
    if (wid == 0) {
        float m = __int_as_float(0x7f800000);
        for (int b = lane; b < nb; b += 32) m = fminf(m, part[2 * b]);
        const float rho = na_warp_min(m);
        float s = 0.f;
        for (int b = lane; b < nb; b += 32) s += part[2 * b + 1] * expf(-(part[2 * b] - rho) / P.lam);
        const float eta = na_warp_sum(s);
        if (lane == 0) {
            s_rho = rho;
            s_eta = eta;
        }
    }
    __syncthreads();
    const float rho = s_rho, eta = s_eta;
    const float4 un = nominal[h];
    float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int k = threadIdx.x; k < K; k += kNaUpdThreads) {
        const float w = expf(-(J[k] - rho) / P.lam) / eta;
        if (h == 0 && w_out != nullptr) w_out[k] = w;
        const float4 d = noise[static_cast<size_t>(h) * K + k];
        const float4 u = clip_control(P, make_float4(un.x + d.x, un.y + d.y, un.z + d.z, un.w + d.w));
        acc.x = fmaf(w, u.x, acc.x);
        acc.y = fmaf(w, u.y, acc.y);
        acc.z = fmaf(w, u.z, acc.z);
        acc.w = fmaf(w, u.w, acc.w);
    }
    acc.x = na_warp_sum(acc.x);
    acc.y = na_warp_sum(acc.y);
    acc.z = na_warp_sum(acc.z);
    acc.w = na_warp_sum(acc.w);
    if (lane == 0) sh[wid] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        float4 t = sh[0];
        for (int i = 1; i < kNaUpdThreads / 32; ++i) {
            t.x += sh[i].x; t.y += sh[i].y; t.z += sh[i].z; t.w += sh[i].w;
        }
        unew[h] = t;
    }
}

std::mutex g_scratch_mu;
float* g_scratch[kMaxDevices] = {};

// Device address of the scratch array on the current device, looked up with that
// device current (the array's name is not a device address in host code).  Outside
// a stream capture the address is looked up again on every call, so that a device
// reset (which reloads the module, possibly elsewhere) never leaves a stale address;
// inside a capture the address cached by an earlier call is used.
cudaError_t scratch_on_current_device(cudaStream_t s, float** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    e = cudaStreamIsCapturing(s, &cs);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (g_scratch[dev] == nullptr || cs == cudaStreamCaptureStatusNone) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_partials);
        if (e != cudaSuccess) return e;
        g_scratch[dev] = static_cast<float*>(p);
    }
    *out = g_scratch[dev];
    return cudaSuccess;
}

// The message goes to the calling thread's error slot, read with mppi_last_error(NULL).
int na_fail(int code, const char* msg, cudaError_t e = cudaSuccess) {
    char buf[256];
    if (e != cudaSuccess)
        snprintf(buf, sizeof(buf), "%s: %s", msg, cudaGetErrorString(e));
    else
        snprintf(buf, sizeof(buf), "%s", msg);
    set_thread_error(buf);
    return code;
}

}  // namespace
}  // namespace mppi

extern "C" int mppi_softmax_update_noalloc(const float* d_costs, const float* d_noise, const float* d_nominal, int K,
                                           int H, float lambda, float thrust_min, float thrust_max, float rate_max,
                                           float* d_new_controls, float* d_weights, void* stream) {
    using namespace mppi;
    if (!d_costs || !d_noise || !d_nominal || !d_new_controls)
        return na_fail(MPPI_E_INVALID, "mppi_softmax_update_noalloc: NULL input or output pointer");
    if (K < 1 || K > MPPI_NOALLOC_MAX_K)
        return na_fail(MPPI_E_INVALID, "mppi_softmax_update_noalloc: K out of [1, MPPI_NOALLOC_MAX_K = 131072]");
    if (H < 1 || H > MPPI_MAX_H) return na_fail(MPPI_E_INVALID, "mppi_softmax_update_noalloc: H out of [1, MPPI_MAX_H]");
    if (!(lambda > 0.f) || !(thrust_min <= thrust_max) || !(rate_max >= 0.f))
        return na_fail(MPPI_E_INVALID, "mppi_softmax_update_noalloc: lambda <= 0 or inconsistent control bounds");
    // the kernels move noise, nominal and controls as float4: misaligned buffers are refused here,
    // before anything is enqueued
    const auto misaligned = [](const void* p) { return reinterpret_cast<uintptr_t>(p) % 16 != 0; };
    if (misaligned(d_noise) || misaligned(d_nominal) || misaligned(d_new_controls))
        return na_fail(MPPI_E_INVALID, "mppi_softmax_update_noalloc: d_noise, d_nominal and d_new_controls must be "
                                       "16-byte aligned");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    float* part = nullptr;
    cudaError_t e = scratch_on_current_device(s, &part);
    if (e != cudaSuccess) return na_fail(MPPI_E_CUDA, "mppi_softmax_update_noalloc: scratch address lookup failed", e);
    StepParams P{};
    P.K = K;
    P.H = H;
    P.lam = lambda;
    P.tmin = thrust_min;
    P.tmax = thrust_max;
    P.rmax = rate_max;
    const int nb = (K + kNaThreads - 1) / kNaThreads;
    na_partials_kernel<<<nb, kNaThreads, 0, s>>>(d_costs, K, lambda, part);
    na_update_kernel<<<H, kNaUpdThreads, 0, s>>>(d_costs, reinterpret_cast<const float4*>(d_noise),
                                                 reinterpret_cast<const float4*>(d_nominal), K, P, part,
                                                 reinterpret_cast<float4*>(d_new_controls), d_weights);
    e = cudaGetLastError();
    if (e != cudaSuccess) return na_fail(MPPI_E_CUDA, "mppi_softmax_update_noalloc: launch failed", e);
    return MPPI_OK;
}
