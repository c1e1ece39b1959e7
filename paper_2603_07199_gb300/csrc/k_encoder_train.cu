// Denoising training of the depth encoder (the reconstruction term of Sec. III-B's first
// stage): encode noisy depth images, map each latent through a linear depth decoder D_psi to
// the 8 x 8 block means of the clean image (scaled by 1 / max_range), take the L1 loss, back-
// propagate through D_psi, the encoder head and the four stride-2 convolutions, and apply
// Adam to every tensor.  FP32 on the CUDA cores; every reduction runs in a fixed order, so a
// step is bit-reproducible.
//
// Kernels per step (after the encoder's own forward pass, whose activations it keeps):
//   recon_kernel        per image: target, D_psi(z), residual, sign / (n T), dL/dz
//   outer_sum_kernel    dL/dW_D, dL/db_D and dL/dW5, dL/db5 (sums over the batch)
//   head_bwd_kernel     per image: the pooled mean, dL/dm = W5^T dL/dz, and the gradient at
//                       conv 4's pre-activation (dL/dm / pixels where x4 > 0)
//   conv_wgrad_kernel   per layer: dL/dW[co][k] = sum over pixels of delta x the gathered
//                       input tap k (plus a ones column for the bias), split over blocks
//   wgrad_reduce_kernel the split partial sums, in slice order (a block per element when
//                       there are many slices)
//   conv_dgrad_kernel   per layer above the first: each input pixel gathers the output
//                       gradients of the (1, 2 or 4 per axis pair) windows that read it,
//                       times the weights, masked by the ReLU of that input
//   adam_kernel         all 12 tensors
// With the SDF term (a frozen Gate-SDF decoder g_phi and camera-frame query points with their
// exact SDF), per step also: sdf_bias_kernel (per image b1 + W1_z z), sdf_dz_kernel (32
// points per block: forward through the decoder keeping the softplus derivatives in shared
// memory, the L1 residual's sign, backward to the first layer) and sdf_dz_reduce_kernel (the
// per-image sum, W1_z^T of it added to dL/dz), before the encoder's backward pass.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <new>
#include <vector>

#include "encoder_internal.h"
#include "kernels.h"
#include "mppi.h"

namespace mppi {
namespace {

constexpr int kLat = MPPI_LATENT_DIM;
constexpr int kPool = 8;
constexpr int kNumTensors = 12;        // W1, b1, .., W4, b4, W5, b5, W_D, b_D
constexpr int kWgThreads = 256;
constexpr int kWgK = 32;               // k columns per weight-gradient block
constexpr int kWgP = 64;               // pixels per staged chunk
constexpr int kDgThreads = 128;
constexpr int kDgGroup = 16;           // input channels per data-gradient thread

// ---------------------------------------------------------------- loss and head
__global__ void __launch_bounds__(256) recon_kernel(const float* __restrict__ z, const float* __restrict__ clean,
                                                    float inv_range, int H, int W, int th, int tw,
                                                    const float* __restrict__ Wd, const float* __restrict__ bd,
                                                    float inv_count, float* __restrict__ g, float* __restrict__ dz,
                                                    float* __restrict__ loss_img) {
    __shared__ float sz[kLat];
    __shared__ float red[256];
    const int n = blockIdx.x, T = th * tw;
    if (threadIdx.x < kLat) sz[threadIdx.x] = z[n * kLat + threadIdx.x];
    __syncthreads();
    const float* img = clean + static_cast<size_t>(n) * H * W;
    float l1 = 0.f;
    for (int t = threadIdx.x; t < T; t += 256) {
        const int a = t / tw, b = t - (t / tw) * tw;
        const int y0 = a * kPool, x0 = b * kPool, y1 = min(y0 + kPool, H), x1 = min(x0 + kPool, W);
        float s = 0.f;
        for (int yy = y0; yy < y1; ++yy)
            for (int xx = x0; xx < x1; ++xx) s += img[yy * W + xx];
        const float target = s * inv_range / static_cast<float>((y1 - y0) * (x1 - x0));
        float y = bd[t];
        const float* wr = Wd + static_cast<size_t>(t) * kLat;
#pragma unroll 8
        for (int c = 0; c < kLat; ++c) y = fmaf(wr[c], sz[c], y);
        const float r = y - target;
        g[static_cast<size_t>(n) * T + t] = (r > 0.f ? inv_count : (r < 0.f ? -inv_count : 0.f));
        l1 += fabsf(r);
    }
    red[threadIdx.x] = l1;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) loss_img[n] = red[0];
    if (threadIdx.x < kLat) {
        const int c = threadIdx.x;
        const float* gn = g + static_cast<size_t>(n) * T;
        float acc = 0.f;
        for (int t = 0; t < T; ++t) acc = fmaf(Wd[static_cast<size_t>(t) * kLat + c], gn[t], acc);
        dz[n * kLat + c] = acc;
    }
}

// out[r][c] = sum_i A[i][r] Bm[i][c]; out_b[r] = sum_i A[i][r] (batch order)
__global__ void __launch_bounds__(256) outer_sum_kernel(const float* __restrict__ A, const float* __restrict__ Bm,
                                                        int n, int R, int C, float* __restrict__ out,
                                                        float* __restrict__ out_b) {
    const int e = blockIdx.x * 256 + threadIdx.x;
    if (e < R * C) {
        const int r = e / C, c = e - (e / C) * C;
        float s = 0.f;
        for (int i = 0; i < n; ++i) s = fmaf(A[static_cast<size_t>(i) * R + r], Bm[static_cast<size_t>(i) * C + c], s);
        out[e] = s;
    }
    if (e < R) {
        float s = 0.f;
        for (int i = 0; i < n; ++i) s += A[static_cast<size_t>(i) * R + e];
        out_b[e] = s;
    }
}

__global__ void __launch_bounds__(kLat) head_bwd_kernel(const float* __restrict__ x4, int hw,
                                                        const float* __restrict__ W5, const float* __restrict__ dz,
                                                        float* __restrict__ m4, float* __restrict__ delta4) {
    const int n = blockIdx.x, c = threadIdx.x;
    const float* xc = x4 + (static_cast<size_t>(n) * kLat + c) * hw;
    float s = 0.f;
    for (int p = 0; p < hw; ++p) s += xc[p];
    m4[n * kLat + c] = s / static_cast<float>(hw);
    float dm = 0.f;
    for (int o = 0; o < kLat; ++o) dm = fmaf(W5[o * kLat + c], dz[n * kLat + o], dm);
    const float d = dm / static_cast<float>(hw);
    float* dc = delta4 + (static_cast<size_t>(n) * kLat + c) * hw;
    for (int p = 0; p < hw; ++p) dc[p] = xc[p] > 0.f ? d : 0.f;
}

// ---------------------------------------------------------------- convolution gradients
// Partial sums over a slice of output pixels of dW[co][k] = sum_p delta[co][p] X[k][p], with
// X[k][p] the layer input at tap k of output pixel p (k = ci 9 + ky 3 + kx, zero outside the
// image) and X[9 CI][p] = 1 for the bias.  Block: kWgK columns x all CO rows over 64-pixel
// chunks staged in shared memory (both [row][pixel], padded); thread t holds columns
// 2 (t % 16) + {0, 1} for rows (t / 16) CO / 16 + {0 .. CO / 16 - 1} and reads 4 pixels per
// 16-byte load.
template <int CI, int CO, bool kScale>
__global__ void __launch_bounds__(kWgThreads) conv_wgrad_kernel(const float* __restrict__ x,
                                                                const float* __restrict__ delta, int n_img, int H,
                                                                int W, int Ho, int Wo, float scale,
                                                                int chunks_per_slice, float* __restrict__ ws) {
    constexpr int K1 = 9 * CI + 1;
    constexpr int RT = CO / 16;                  // rows per thread
    constexpr int kLd = kWgP + 4;
    __shared__ __align__(16) float sd[CO][kLd];
    __shared__ __align__(16) float sx[kWgK][kLd];
    const int hwo = Ho * Wo;
    const long long P = static_cast<long long>(n_img) * hwo;
    const long long n_chunks = (P + kWgP - 1) / kWgP;
    const int k0 = blockIdx.x * kWgK;
    const int kp = threadIdx.x % 16, rg = threadIdx.x / 16;
    float acc[RT][2];
#pragma unroll
    for (int j = 0; j < RT; ++j) acc[j][0] = acc[j][1] = 0.f;
    const long long c_begin = static_cast<long long>(blockIdx.y) * chunks_per_slice;
    const long long c_end = min(c_begin + chunks_per_slice, n_chunks);
    for (long long ch = c_begin; ch < c_end; ++ch) {
        const long long p0 = ch * kWgP;
        __syncthreads();
        for (int e = threadIdx.x; e < CO * kWgP; e += kWgThreads) {
            const int co = e / kWgP, pp = e - (e / kWgP) * kWgP;
            const long long p = p0 + pp;
            float v = 0.f;
            if (p < P) {
                const int n = static_cast<int>(p / hwo);
                const int pix = static_cast<int>(p - static_cast<long long>(n) * hwo);
                v = delta[(static_cast<size_t>(n) * CO + co) * hwo + pix];
            }
            sd[co][pp] = v;
        }
        for (int e = threadIdx.x; e < kWgK * kWgP; e += kWgThreads) {
            const int kk = e / kWgP, pp = e - (e / kWgP) * kWgP;
            const long long p = p0 + pp;
            const int k = k0 + kk;
            float v = 0.f;
            if (p < P && k < K1) {
                if (k == 9 * CI) {
                    v = 1.f;
                } else {
                    const int n = static_cast<int>(p / hwo);
                    const int pix = static_cast<int>(p - static_cast<long long>(n) * hwo);
                    const int i = pix / Wo, j = pix - (pix / Wo) * Wo;
                    const int ci = k / 9, t = k - 9 * (k / 9);
                    const int yy = 2 * i + t / 3 - 1, xx = 2 * j + t % 3 - 1;
                    if (yy >= 0 && yy < H && xx >= 0 && xx < W) {
                        v = x[((static_cast<size_t>(n) * CI + ci) * H + yy) * W + xx];
                        if (kScale) v *= scale;
                    }
                }
            }
            sx[kk][pp] = v;
        }
        __syncthreads();
#pragma unroll 4
        for (int pp = 0; pp < kWgP; pp += 4) {
            const float4 x0 = *reinterpret_cast<const float4*>(&sx[2 * kp][pp]);
            const float4 x1 = *reinterpret_cast<const float4*>(&sx[2 * kp + 1][pp]);
#pragma unroll
            for (int j = 0; j < RT; ++j) {
                const float4 d = *reinterpret_cast<const float4*>(&sd[rg * RT + j][pp]);
                acc[j][0] = fmaf(d.x, x0.x, fmaf(d.y, x0.y, fmaf(d.z, x0.z, fmaf(d.w, x0.w, acc[j][0]))));
                acc[j][1] = fmaf(d.x, x1.x, fmaf(d.y, x1.y, fmaf(d.z, x1.z, fmaf(d.w, x1.w, acc[j][1]))));
            }
        }
    }
#pragma unroll
    for (int c = 0; c < 2; ++c) {
        const int k = k0 + 2 * kp + c;
        if (k < K1) {
#pragma unroll
            for (int j = 0; j < RT; ++j)
                ws[(static_cast<size_t>(blockIdx.y) * CO + rg * RT + j) * K1 + k] = acc[j][c];
        }
    }
}

// The first layer's weight gradient (one input channel: K = 9 taps + the bias column) over a
// slice of output pixels: every thread keeps the 8 x 10 sums of half of the 16 channels
// (blockIdx.y) for its pixels (one 3 x 3 input window and 8 output gradients each), then the
// block sums them in a fixed order (warp shuffle tree, then the warps in index order) and writes
// ws[slice][co][k].  The reduction is short and the pixels many, so the CUDA cores keep it.
constexpr int kW1Threads = 256;
template <bool kScale>
__global__ void __launch_bounds__(kW1Threads) conv1_wgrad_kernel(const float* __restrict__ x,
                                                                 const float* __restrict__ delta, int n_img, int H,
                                                                 int W, int Ho, int Wo, float scale,
                                                                 long long pixels_per_slice, float* __restrict__ ws) {
    constexpr int CO = 16, K1 = 10, CH = 8;
    __shared__ float red[kW1Threads / 32][CH * K1];
    const int hw = Ho * Wo;
    const long long P = static_cast<long long>(n_img) * hw;
    const long long p_begin = static_cast<long long>(blockIdx.x) * pixels_per_slice;
    const long long p_end = min(p_begin + pixels_per_slice, P);
    const int co0 = blockIdx.y * CH;
    float acc[CH][K1];
#pragma unroll
    for (int c = 0; c < CH; ++c)
#pragma unroll
        for (int k = 0; k < K1; ++k) acc[c][k] = 0.f;
    for (long long p = p_begin + threadIdx.x; p < p_end; p += kW1Threads) {
        const int n = static_cast<int>(p / hw);
        const int rem = static_cast<int>(p - static_cast<long long>(n) * hw);
        const int i = rem / Wo, j = rem - (rem / Wo) * Wo;
        float xv[9];
#pragma unroll
        for (int t = 0; t < 9; ++t) {
            const int yy = 2 * i + t / 3 - 1, xx = 2 * j + t % 3 - 1;
            float v = 0.f;
            if (yy >= 0 && yy < H && xx >= 0 && xx < W) {
                v = __ldg(x + (static_cast<size_t>(n) * H + yy) * W + xx);
                if (kScale) v *= scale;
            }
            xv[t] = v;
        }
#pragma unroll
        for (int c = 0; c < CH; ++c) {
            const float d = __ldg(delta + (static_cast<size_t>(n) * CO + co0 + c) * hw + rem);
#pragma unroll
            for (int t = 0; t < 9; ++t) acc[c][t] = fmaf(d, xv[t], acc[c][t]);
            acc[c][9] += d;
        }
    }
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
    for (int c = 0; c < CH; ++c)
#pragma unroll
        for (int k = 0; k < K1; ++k) {
            float v = acc[c][k];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            if (lane == 0) red[warp][c * K1 + k] = v;
        }
    __syncthreads();
    if (threadIdx.x < CH * K1) {
        float v = 0.f;
#pragma unroll
        for (int w = 0; w < kW1Threads / 32; ++w) v += red[w][threadIdx.x];
        const int c = threadIdx.x / K1, k = threadIdx.x - (threadIdx.x / K1) * K1;
        ws[(static_cast<size_t>(blockIdx.x) * CO + co0 + c) * K1 + k] = v;
    }
}

// gW[co][k] (= the [co][ci][ky][kx] layout) and gb[co] from the slices' partial sums, in slice
// order: one thread per element.
__global__ void __launch_bounds__(256) wgrad_reduce_kernel(const float* __restrict__ ws, int n_slices, int CO, int K1,
                                                           float* __restrict__ gW, float* __restrict__ gb) {
    const int e = blockIdx.x * 256 + threadIdx.x;
    if (e >= CO * K1) return;
    const int co = e / K1, k = e - (e / K1) * K1;
    float s = 0.f;
    for (int q = 0; q < n_slices; ++q) s += ws[static_cast<size_t>(q) * CO * K1 + e];
    if (k < K1 - 1)
        gW[co * (K1 - 1) + k] = s;
    else
        gb[co] = s;
}

// The same for many slices: one block per element, 128 strided partial sums, a fixed tree.
__global__ void __launch_bounds__(128) wgrad_reduce_wide_kernel(const float* __restrict__ ws, int n_slices, int CO,
                                                                int K1, float* __restrict__ gW,
                                                                float* __restrict__ gb) {
    __shared__ float red[128];
    const int e = blockIdx.x;
    const int co = e / K1, k = e - (e / K1) * K1;
    float s = 0.f;
    for (int q = threadIdx.x; q < n_slices; q += 128) s += ws[static_cast<size_t>(q) * CO * K1 + e];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int o = 64; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        if (k < K1 - 1)
            gW[co * (K1 - 1) + k] = red[0];
        else
            gb[co] = red[0];
    }
}

// delta_in[n][ci][y][x] = [x_in > 0] sum_{co, ky, kx} W[co][ci][ky][kx] delta[n][co][i][j] over the
// windows (i, j) = ((y + 1 - ky) / 2, (x + 1 - kx) / 2) that read input pixel (y, x).
template <int CI, int CO>
__global__ void __launch_bounds__(kDgThreads) conv_dgrad_kernel(const float* __restrict__ delta,
                                                                const float* __restrict__ Wt,
                                                                const float* __restrict__ x_in, int n_img, int H,
                                                                int W, int Ho, int Wo, float* __restrict__ delta_in) {
    __shared__ __align__(16) float w_s[CO * 9 * kDgGroup];   // [co][tap][16 input channels]
    const int c0 = blockIdx.y * kDgGroup;
    for (int e = threadIdx.x; e < CO * 9 * kDgGroup; e += kDgThreads) {
        const int co = e / (9 * kDgGroup), rem = e - co * 9 * kDgGroup;
        const int t = rem / kDgGroup, c = rem - t * kDgGroup;
        w_s[e] = Wt[(static_cast<size_t>(co) * CI + c0 + c) * 9 + t];
    }
    __syncthreads();
    const int hw = H * W, hwo = Ho * Wo;
    const long long p = static_cast<long long>(blockIdx.x) * kDgThreads + threadIdx.x;
    if (p >= static_cast<long long>(n_img) * hw) return;
    const int n = static_cast<int>(p / hw);
    const int pix = static_cast<int>(p - static_cast<long long>(n) * hw);
    const int y = pix / W, xq = pix - (pix / W) * W;
    // taps along each axis: y odd -> ky in {0, 2}; y even -> ky = 1 (window index (y + 1 - ky) / 2)
    int kys[2], iys[2], nky = 0, kxs[2], ixs[2], nkx = 0;
    for (int k = 0; k < 3; ++k) {
        const int a = y + 1 - k;
        if ((a & 1) == 0 && a / 2 < Ho) { kys[nky] = k; iys[nky] = a / 2; ++nky; }
        const int b = xq + 1 - k;
        if ((b & 1) == 0 && b / 2 < Wo) { kxs[nkx] = k; ixs[nkx] = b / 2; ++nkx; }
    }
    float acc[kDgGroup];
#pragma unroll
    for (int c = 0; c < kDgGroup; ++c) acc[c] = 0.f;
    const float* dn = delta + static_cast<size_t>(n) * CO * hwo;
    const float4* w4 = reinterpret_cast<const float4*>(w_s);
    for (int co = 0; co < CO; ++co) {
        for (int a = 0; a < nky; ++a) {
            for (int b = 0; b < nkx; ++b) {
                const float d = dn[static_cast<size_t>(co) * hwo + iys[a] * Wo + ixs[b]];
                const int t = kys[a] * 3 + kxs[b];
#pragma unroll
                for (int c4 = 0; c4 < kDgGroup / 4; ++c4) {
                    const float4 w = w4[(co * 9 + t) * (kDgGroup / 4) + c4];
                    acc[4 * c4 + 0] = fmaf(w.x, d, acc[4 * c4 + 0]);
                    acc[4 * c4 + 1] = fmaf(w.y, d, acc[4 * c4 + 1]);
                    acc[4 * c4 + 2] = fmaf(w.z, d, acc[4 * c4 + 2]);
                    acc[4 * c4 + 3] = fmaf(w.w, d, acc[4 * c4 + 3]);
                }
            }
        }
    }
#pragma unroll
    for (int c = 0; c < kDgGroup; ++c) {
        const size_t o = (static_cast<size_t>(n) * CI + c0 + c) * hw + pix;
        delta_in[o] = x_in[o] > 0.f ? acc[c] : 0.f;
    }
}

// ---------------------------------------------------------------- SDF term (frozen decoder)
constexpr int kSdThreads = 256;
constexpr int kSdPts = 32;                 // query points per block (all of one image)
constexpr int kSdMaxFeat = 3 + 6 * MPPI_MAX_PE_LEVELS;
constexpr int kSdHidden = MPPI_HIDDEN;

struct SdfNet {
    const float* W1;        // [128][NF + 64] as given
    const float* b1;        // [128]
    const float* W[3];      // layers 2..4 as given: [out][in]
    const float* b[3];      // [128]
    const float* w5;        // [128]
    const float* b5;        // [1]
    float beta;
    int nf, pe;             // point features 3 + 6 pe
};

// Per-point records kept for the decoder's weight gradients (all NULL when it is frozen):
// layer-1 input features X [P][NF], hidden activations H [4][P][128], pre-activation
// gradients G [4][P][128] and output gradients g5 [P] (P = images x points per image).
struct SdfRecord {
    float* X;               // [P][NF + 64]: PE(p) then the image's latent
    float* H;
    float* G;
    float* g5;
    const float* z;         // [images][64]
    long long P;
};

// per image: b1'_i = b1 + W1[:, NF:] z_i
__global__ void __launch_bounds__(kSdHidden) sdf_bias_kernel(SdfNet N, const float* __restrict__ z,
                                                              float* __restrict__ b1p) {
    const int i = blockIdx.x, c = threadIdx.x;
    const int ld = N.nf + kLat;
    float acc = N.b1[c];   // (sdf_bias_kernel)
    for (int j = 0; j < kLat; ++j) acc = fmaf(N.W1[c * ld + N.nf + j], z[i * kLat + j], acc);
    b1p[i * kSdHidden + c] = acc;
}

__device__ __forceinline__ float sp_acc(float x, float beta) {
    return fmaxf(x, 0.f) + log1pf(expf(-beta * fabsf(x))) / beta;
}
__device__ __forceinline__ float sp_grad(float x, float beta) {   // logistic(beta x)
    const float e = expf(-beta * fabsf(x));
    return x >= 0.f ? 1.f / (1.f + e) : e / (1.f + e);
}

// out[p][c] = sum_r in[p][r] M[r][c] for the block's 32 points: thread rows 4 (t / 32) .. + 3,
// columns 4 (t % 32) .. + 3.
__device__ __forceinline__ void sd_gemm(const float (*in)[kSdHidden], const float* M, float acc[4][4]) {
    const int rp = threadIdx.x >> 5, cq = threadIdx.x & 31;
#pragma unroll 4
    for (int r = 0; r < kSdHidden; ++r) {
        const float4 b = *reinterpret_cast<const float4*>(M + r * kSdHidden + cq * 4);
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const float a = in[rp * 4 + i][r];
            acc[i][0] = fmaf(a, b.x, acc[i][0]);
            acc[i][1] = fmaf(a, b.y, acc[i][1]);
            acc[i][2] = fmaf(a, b.z, acc[i][2]);
            acc[i][3] = fmaf(a, b.w, acc[i][3]);
        }
    }
}

// Forward through the frozen decoder at 32 query points of image blockIdx.x / (n_points / 32),
// the signed L1 residual's coefficient, and the backward pass to the first layer's
// pre-activation; writes the block's sum of that gradient over its points and its sum of |r|.
__global__ void __launch_bounds__(kSdThreads) sdf_dz_kernel(SdfNet N, const float* __restrict__ points,
                                                            const float* __restrict__ labels, int n_points,
                                                            const float* __restrict__ b1p, float coef,
                                                            float* __restrict__ part, float* __restrict__ loss_part,
                                                            SdfRecord rec) {
    extern __shared__ __align__(16) float sm[];
    float (*h)[kSdHidden] = reinterpret_cast<float (*)[kSdHidden]>(sm);                      // [32][128]
    float (*spd)[kSdPts][kSdHidden] = reinterpret_cast<float (*)[kSdPts][kSdHidden]>(sm + kSdPts * kSdHidden);
    float* Mst = sm + 5 * kSdPts * kSdHidden;                                                 // [128][128]
    float* pe = Mst + kSdHidden * kSdHidden;                                                  // [NF][32]
    float* sres = pe + kSdMaxFeat * kSdPts;                                                   // [32]
    const int blocks_per_img = n_points / kSdPts;
    const int img = blockIdx.x / blocks_per_img;
    const long long q0 = static_cast<long long>(blockIdx.x) * kSdPts;   // first query of the block
    const int rp = threadIdx.x >> 5, cq = threadIdx.x & 31;
    if (threadIdx.x < kSdPts) {
        const float* pt = points + (q0 + threadIdx.x) * 3;
        const float px = pt[0], py = pt[1], pz = pt[2];
        pe[0 * kSdPts + threadIdx.x] = px;
        pe[1 * kSdPts + threadIdx.x] = py;
        pe[2 * kSdPts + threadIdx.x] = pz;
        for (int l = 0; l < N.pe; ++l) {
            const float sc = static_cast<float>(1 << l);
            float s0, c0, s1, c1, s2, c2;
            sincospif(sc * px, &s0, &c0);
            sincospif(sc * py, &s1, &c1);
            sincospif(sc * pz, &s2, &c2);
            float* f = pe + (3 + 6 * l) * kSdPts + threadIdx.x;
            f[0] = s0; f[kSdPts] = s1; f[2 * kSdPts] = s2;
            f[3 * kSdPts] = c0; f[4 * kSdPts] = c1; f[5 * kSdPts] = c2;
        }
    }
    __syncthreads();
    if (rec.X) {
        const int ldx = N.nf + kLat;
        for (int e = threadIdx.x; e < kSdPts * ldx; e += kSdThreads) {
            const int pnt = e / ldx, f = e - pnt * ldx;
            rec.X[(q0 + pnt) * ldx + f] = f < N.nf ? pe[f * kSdPts + pnt] : rec.z[img * kLat + f - N.nf];
        }
    }
    // layer 1: a1[p][c] = b1'_img[c] + W1[c][0:NF] pe[p]
    const int ld1 = N.nf + kLat;
    for (int e = threadIdx.x; e < kSdPts * kSdHidden; e += kSdThreads) {
        const int pnt = e / kSdHidden, c = e - pnt * kSdHidden;
        float a = b1p[img * kSdHidden + c];
        for (int f = 0; f < N.nf; ++f) a = fmaf(N.W1[c * ld1 + f], pe[f * kSdPts + pnt], a);
        h[pnt][c] = sp_acc(a, N.beta);
        spd[0][pnt][c] = sp_grad(a, N.beta);
        if (rec.H) rec.H[(q0 + pnt) * kSdHidden + c] = h[pnt][c];
    }
    // layers 2..4
    for (int l = 0; l < 3; ++l) {
        __syncthreads();
        // stage W_l transposed (M[k][o] = W[o][k]): coalesced reads, strided shared writes
        for (int e = threadIdx.x; e < kSdHidden * kSdHidden; e += kSdThreads) {
            const int o = e / kSdHidden, k = e - o * kSdHidden;
            Mst[k * kSdHidden + o] = N.W[l][e];
        }
        __syncthreads();
        float acc[4][4] = {};
        sd_gemm(h, Mst, acc);
        __syncthreads();
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const float a = acc[i][c] + N.b[l][cq * 4 + c];
                const float hv = sp_acc(a, N.beta);
                h[rp * 4 + i][cq * 4 + c] = hv;
                spd[l + 1][rp * 4 + i][cq * 4 + c] = sp_grad(a, N.beta);
                if (rec.H) rec.H[((l + 1) * rec.P + q0 + rp * 4 + i) * kSdHidden + cq * 4 + c] = hv;
            }
    }
    __syncthreads();
    // output, residual and its coefficient (one warp per 4 points, lanes over the hidden units)
    {
        const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
        for (int pnt = w; pnt < kSdPts; pnt += kSdThreads / 32) {
            float sacc = 0.f;
            for (int c = lane; c < kSdHidden; c += 32) sacc = fmaf(N.w5[c], h[pnt][c], sacc);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) sacc += __shfl_xor_sync(0xffffffffu, sacc, o);
            if (lane == 0) sres[pnt] = sacc + N.b5[0] - labels[q0 + pnt];
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        float l1 = 0.f;
        for (int pnt = 0; pnt < kSdPts; ++pnt) l1 += fabsf(sres[pnt]);
        loss_part[blockIdx.x] = l1;
    }
    // backward: g4 = coef sign(r) w5 sp'(a4); g_{l-1} = (g_l W_l) sp'(a_{l-1})
    for (int e = threadIdx.x; e < kSdPts * kSdHidden; e += kSdThreads) {
        const int pnt = e / kSdHidden, c = e - pnt * kSdHidden;
        const float r = sres[pnt];
        const float sg = r > 0.f ? coef : (r < 0.f ? -coef : 0.f);
        h[pnt][c] = sg * N.w5[c] * spd[3][pnt][c];
        if (rec.G) rec.G[(3 * rec.P + q0 + pnt) * kSdHidden + c] = h[pnt][c];
        if (rec.g5 && c == 0) rec.g5[q0 + pnt] = sg;
    }
    for (int l = 2; l >= 0; --l) {
        __syncthreads();
        for (int e = threadIdx.x; e < kSdHidden * kSdHidden / 4; e += kSdThreads)
            reinterpret_cast<float4*>(Mst)[e] = reinterpret_cast<const float4*>(N.W[l])[e];
        __syncthreads();
        float acc[4][4] = {};
        sd_gemm(h, Mst, acc);
        __syncthreads();
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const float gv = acc[i][c] * spd[l][rp * 4 + i][cq * 4 + c];
                h[rp * 4 + i][cq * 4 + c] = gv;
                if (rec.G) rec.G[(static_cast<long long>(l) * rec.P + q0 + rp * 4 + i) * kSdHidden + cq * 4 + c] = gv;
            }
    }
    __syncthreads();
    if (threadIdx.x < kSdHidden) {
        float acc = 0.f;
        for (int pnt = 0; pnt < kSdPts; ++pnt) acc += h[pnt][threadIdx.x];
        part[static_cast<size_t>(blockIdx.x) * kSdHidden + threadIdx.x] = acc;
    }
}

// per image: G = sum over its blocks of the first-layer gradient sums (block order);
// dz_i += W1[:, NF:]^T G; its SDF loss sum = sum of its blocks' |r| sums.
__global__ void __launch_bounds__(kSdHidden) sdf_dz_reduce_kernel(SdfNet N, const float* __restrict__ part,
                                                                   const float* __restrict__ loss_part,
                                                                   int blocks_per_img, float* __restrict__ dz,
                                                                   float* __restrict__ loss_img) {
    __shared__ float G[kSdHidden];
    const int i = blockIdx.x, c = threadIdx.x;
    float acc = 0.f;
    for (int q = 0; q < blocks_per_img; ++q) acc += part[(static_cast<size_t>(i) * blocks_per_img + q) * kSdHidden + c];
    G[c] = acc;
    __syncthreads();
    if (c < kLat) {
        const int ld = N.nf + kLat;
        float d = 0.f;
        for (int k = 0; k < kSdHidden; ++k) d = fmaf(N.W1[k * ld + N.nf + c], G[k], d);
        dz[i * kLat + c] += d;
    }
    if (c == 0) {
        float l1 = 0.f;
        for (int q = 0; q < blocks_per_img; ++q) l1 += loss_part[i * blocks_per_img + q];
        loss_img[i] = l1;
    }
}

constexpr size_t kSdSmem = sizeof(float) * (5 * kSdPts * kSdHidden + kSdHidden * kSdHidden + kSdMaxFeat * kSdPts +
                                            kSdPts);

// Weight gradients of the decoder: out[r][c] = sum_p A[p][r] X[p][c] over the points p of a
// slice (partials to ws[slice][R][C]), 32 x 32 outputs per block, 2 x 2 per thread.
constexpr int kGxT = 32;
constexpr int kGxP = 64;
__global__ void __launch_bounds__(256) gtx_kernel(const float* __restrict__ A, int R, const float* __restrict__ X,
                                                  int C, long long P, int chunks_per_slice, float* __restrict__ ws) {
    __shared__ float sa[kGxP][kGxT + 1];
    __shared__ float sx[kGxP][kGxT + 1];
    const int r0 = blockIdx.x * kGxT, c0 = blockIdx.y * kGxT;
    const int tr = threadIdx.x / 16, tc = threadIdx.x % 16;      // rows 2 tr + {0, 1}, columns 2 tc + {0, 1}
    float acc[2][2] = {};
    const long long n_chunks = (P + kGxP - 1) / kGxP;
    const long long cb = static_cast<long long>(blockIdx.z) * chunks_per_slice;
    const long long ce = min(cb + chunks_per_slice, n_chunks);
    for (long long ch = cb; ch < ce; ++ch) {
        const long long p0 = ch * kGxP;
        __syncthreads();
        for (int e = threadIdx.x; e < kGxP * kGxT; e += 256) {
            const int pp = e / kGxT, k = e - (e / kGxT) * kGxT;
            const long long pt = p0 + pp;
            sa[pp][k] = (pt < P && r0 + k < R) ? A[pt * R + r0 + k] : 0.f;
            sx[pp][k] = (pt < P && c0 + k < C) ? X[pt * C + c0 + k] : 0.f;
        }
        __syncthreads();
#pragma unroll 8
        for (int pp = 0; pp < kGxP; ++pp) {
            const float a0 = sa[pp][2 * tr], a1 = sa[pp][2 * tr + 1];
            const float x0 = sx[pp][2 * tc], x1 = sx[pp][2 * tc + 1];
            acc[0][0] = fmaf(a0, x0, acc[0][0]);
            acc[0][1] = fmaf(a0, x1, acc[0][1]);
            acc[1][0] = fmaf(a1, x0, acc[1][0]);
            acc[1][1] = fmaf(a1, x1, acc[1][1]);
        }
    }
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 2; ++j) {
            const int r = r0 + 2 * tr + i, c = c0 + 2 * tc + j;
            if (r < R && c < C) ws[(static_cast<size_t>(blockIdx.z) * R + r) * C + c] = acc[i][j];
        }
}

// out[e] = sum over slices of ws[slice][e], in slice order
__global__ void __launch_bounds__(256) slice_sum_kernel(const float* __restrict__ ws, int n_slices, int n,
                                                        float* __restrict__ out) {
    const int e = blockIdx.x * 256 + threadIdx.x;
    if (e >= n) return;
    float s = 0.f;
    for (int q = 0; q < n_slices; ++q) s += ws[static_cast<size_t>(q) * n + e];
    out[e] = s;
}

// out[r] = sum_p A[p][r]: one block per column, 256 strided partial sums and a fixed tree
__global__ void __launch_bounds__(256) colsum_kernel(const float* __restrict__ A, int R, long long P,
                                                     float* __restrict__ out) {
    __shared__ float red[256];
    const int r = blockIdx.x;
    float s = 0.f;
    for (long long p = threadIdx.x; p < P; p += 256) s += A[p * R + r];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[r] = red[0];
}

// ---------------------------------------------------------------- Adam
constexpr int kMaxTensors = kNumTensors + 10;   // + the SDF decoder's, when it trains
struct AdamTable {
    float* p[kMaxTensors];
    const float* g[kMaxTensors];
    float* m[kMaxTensors];
    float* v[kMaxTensors];
    int size[kMaxTensors];
};

__global__ void __launch_bounds__(256) adam_kernel(AdamTable tab, float lr, float c1, float c2) {
    const int i = blockIdx.y;
    const int e = blockIdx.x * 256 + threadIdx.x;
    if (e >= tab.size[i]) return;
    const float g = tab.g[i][e];
    const float m = 0.9f * tab.m[i][e] + 0.1f * g;
    const float v = 0.999f * tab.v[i][e] + 0.001f * g * g;
    tab.m[i][e] = m;
    tab.v[i][e] = v;
    tab.p[i][e] -= lr * (m / c1) / (sqrtf(v / c2) + 1e-8f);
}

thread_local char g_etr_err[512] = "";

}  // namespace
}  // namespace mppi

struct mppi_encoder_trainer {
    mppi_encoder* enc = nullptr;
    int batch = 0, th = 0, tw = 0, T = 0;
    float lr = 1e-3f;
    int step = 0;
    float* param[mppi::kNumTensors] = {};
    int size[mppi::kNumTensors] = {};
    float* grad[mppi::kNumTensors] = {};
    float* m[mppi::kNumTensors] = {};
    float* v[mppi::kNumTensors] = {};
    float* Wd = nullptr;
    float* bd = nullptr;
    float* z = nullptr;
    float* g = nullptr;
    float* dz = nullptr;
    float* m4 = nullptr;
    float* loss_img = nullptr;
    float* delta[2] = {nullptr, nullptr};
    float* ws = nullptr;
    size_t ws_floats = 0;
    // SDF term (frozen decoder), set by mppi_encoder_train_set_sdf
    bool sdf = false;
    float lam_recon = 1.f, lam_sdf = 0.f;
    int max_points = 0;
    mppi::SdfNet net{};
    bool train_dec = false;                 // the SDF decoder trains too (stage 1)
    float* dparam[10] = {};                 // W1, b1, W2, b2, W3, b3, W4, b4, w5, b5 (device)
    int dsize[10] = {};
    float* dgrad[10] = {};
    float* dm[10] = {};
    float* dv[10] = {};
    mppi::SdfRecord rec{};
    float* gx_ws = nullptr;
    size_t gx_ws_floats = 0;
    float* sdf_b1p = nullptr;
    float* sdf_part = nullptr;
    float* sdf_loss_part = nullptr;
    float* sdf_loss_img = nullptr;
    std::vector<void*> allocs;
    std::vector<float> h_loss;
    std::vector<float> h_loss2;
    char err[512] = "";
};

namespace {

int tfail(mppi_encoder_trainer* t, int code, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    std::snprintf(t ? t->err : mppi::g_etr_err, 512, "%s", buf);
    return code;
}

bool talloc(mppi_encoder_trainer* t, float** p, size_t n) {
    void* q = nullptr;
    if (cudaMalloc(&q, std::max<size_t>(n, 1) * sizeof(float)) != cudaSuccess) return false;
    t->allocs.push_back(q);
    *p = static_cast<float*>(q);
    return true;
}

void trainer_free(mppi_encoder_trainer* t) {
    for (void* p : t->allocs) cudaFree(p);
    t->allocs.clear();
}

int wgrad_slices(const mppi_encoder* e, int k_tiles, long long chunks) {
    const long long want = (2LL * e->n_sms + k_tiles - 1) / k_tiles;
    return static_cast<int>(std::max(1LL, std::min(want, chunks)));
}

template <int CI, int CO, bool kScale>
cudaError_t launch_wgrad(mppi_encoder_trainer* t, int l, int n, const float* x, float scale, const float* delta) {
    const mppi_encoder* e = t->enc;
    constexpr int K1 = 9 * CI + 1;
    const long long P = static_cast<long long>(n) * e->h[l + 1] * e->w[l + 1];
    if (e->conv_path == MPPI_ENC_CONV_TC) {
        // tensor cores: 128 k rows x all channels per CTA, pixel slices of whole 64-pixel stages,
        // about two CTAs per SM
        const int kt = mppi::conv_wgrad_tc_k_tiles(l);
        const long long stages = (P + mppi::conv_wgrad_tc_stage_pixels() - 1) / mppi::conv_wgrad_tc_stage_pixels();
        long long S = std::max(1LL, std::min(stages, (2LL * e->n_sms + kt - 1) / kt));
        while (static_cast<size_t>(S) * CO * K1 > t->ws_floats && S > 1) --S;
        const int cps = static_cast<int>((stages + S - 1) / S);
        S = (stages + cps - 1) / cps;
        cudaError_t ce = mppi::launch_conv_wgrad_tc(l, x, delta, n, e->h[l], e->w[l], e->h[l + 1], e->w[l + 1], scale,
                                                    static_cast<int>(S), cps, t->ws, e->d_err, e->stream);
        if (ce != cudaSuccess) return ce;
        // a block per element only when the elements are few (its strided reads are slow); otherwise a
        // thread per element reads the slices in order with coalesced loads
        if (S > 32 && CO * K1 < 4096)
            mppi::wgrad_reduce_wide_kernel<<<CO * K1, 128, 0, e->stream>>>(t->ws, static_cast<int>(S), CO, K1,
                                                                           t->grad[2 * l], t->grad[2 * l + 1]);
        else
            mppi::wgrad_reduce_kernel<<<(CO * K1 + 255) / 256, 256, 0, e->stream>>>(
                t->ws, static_cast<int>(S), CO, K1, t->grad[2 * l], t->grad[2 * l + 1]);
        return cudaGetLastError();
    }
    const int k_tiles = (K1 + mppi::kWgK - 1) / mppi::kWgK;
    const long long chunks = (P + mppi::kWgP - 1) / mppi::kWgP;
    int S = wgrad_slices(e, k_tiles, chunks);
    while (static_cast<size_t>(S) * CO * K1 > t->ws_floats && S > 1) --S;
    const int cps = static_cast<int>((chunks + S - 1) / S);
    S = static_cast<int>((chunks + cps - 1) / cps);
    mppi::conv_wgrad_kernel<CI, CO, kScale><<<dim3(k_tiles, S), mppi::kWgThreads, 0, e->stream>>>(
        x, delta, n, e->h[l], e->w[l], e->h[l + 1], e->w[l + 1], scale, cps, t->ws);
    if (S > 32)
        mppi::wgrad_reduce_wide_kernel<<<CO * K1, 128, 0, e->stream>>>(t->ws, S, CO, K1, t->grad[2 * l],
                                                                       t->grad[2 * l + 1]);
    else
        mppi::wgrad_reduce_kernel<<<(CO * K1 + 255) / 256, 256, 0, e->stream>>>(t->ws, S, CO, K1, t->grad[2 * l],
                                                                               t->grad[2 * l + 1]);
    return cudaGetLastError();
}

// The first layer's weight gradient (conv1_wgrad_kernel, slices of whole 256-pixel rounds, about
// four blocks per SM), then the slices summed in order.
cudaError_t launch_wgrad1(mppi_encoder_trainer* t, int n, const float* x, float scale, const float* delta) {
    const mppi_encoder* e = t->enc;
    constexpr int CO = 16, K1 = 10;
    const long long P = static_cast<long long>(n) * e->h[1] * e->w[1];
    const long long rounds = (P + mppi::kW1Threads - 1) / mppi::kW1Threads;
    long long S = std::max(1LL, std::min(rounds, 2LL * e->n_sms));
    while (static_cast<size_t>(S) * CO * K1 > t->ws_floats && S > 1) --S;
    const long long per = (rounds + S - 1) / S * mppi::kW1Threads;
    S = (P + per - 1) / per;
    mppi::conv1_wgrad_kernel<true><<<dim3(static_cast<unsigned>(S), 2), mppi::kW1Threads, 0, e->stream>>>(
        x, delta, n, e->h[0], e->w[0], e->h[1], e->w[1], scale, per, t->ws);
    if (S > 32)
        mppi::wgrad_reduce_wide_kernel<<<CO * K1, 128, 0, e->stream>>>(t->ws, static_cast<int>(S), CO, K1, t->grad[0],
                                                                       t->grad[1]);
    else
        mppi::wgrad_reduce_kernel<<<(CO * K1 + 255) / 256, 256, 0, e->stream>>>(t->ws, static_cast<int>(S), CO, K1,
                                                                               t->grad[0], t->grad[1]);
    return cudaGetLastError();
}

template <int CI, int CO>
cudaError_t launch_dgrad(mppi_encoder_trainer* t, int l, int n, const float* delta, float* delta_in) {
    const mppi_encoder* e = t->enc;
    if (e->conv_path == MPPI_ENC_CONV_TC)
        return mppi::launch_conv_dgrad_tc(l, delta, e->dgpack[l], e->act[l - 1], n, e->h[l], e->w[l], e->h[l + 1],
                                          e->w[l + 1], delta_in, e->d_err, e->stream);
    const long long pix = static_cast<long long>(n) * e->h[l] * e->w[l];
    const dim3 grid(static_cast<unsigned>((pix + mppi::kDgThreads - 1) / mppi::kDgThreads), CI / mppi::kDgGroup);
    mppi::conv_dgrad_kernel<CI, CO><<<grid, mppi::kDgThreads, 0, e->stream>>>(
        delta, e->wt[l], e->act[l - 1], n, e->h[l], e->w[l], e->h[l + 1], e->w[l + 1], delta_in);
    return cudaGetLastError();
}

// out[R][C] = A^T X over P points (A [P][R], X [P][C]): split over blocks, summed in slice order.
void gtx(mppi_encoder_trainer* t, const float* A, int R, const float* X, int C, long long P, float* out) {
    cudaStream_t s = t->enc->stream;
    const int tiles = ((R + mppi::kGxT - 1) / mppi::kGxT) * ((C + mppi::kGxT - 1) / mppi::kGxT);
    const long long chunks = (P + mppi::kGxP - 1) / mppi::kGxP;
    int S = static_cast<int>(std::max(1LL, std::min<long long>((2LL * t->enc->n_sms + tiles - 1) / tiles, chunks)));
    while (static_cast<size_t>(S) * R * C > t->gx_ws_floats && S > 1) --S;
    const int cps = static_cast<int>((chunks + S - 1) / S);
    S = static_cast<int>((chunks + cps - 1) / cps);
    const dim3 grid((R + mppi::kGxT - 1) / mppi::kGxT, (C + mppi::kGxT - 1) / mppi::kGxT, S);
    mppi::gtx_kernel<<<grid, 256, 0, s>>>(A, R, X, C, P, cps, t->gx_ws);
    mppi::slice_sum_kernel<<<(R * C + 255) / 256, 256, 0, s>>>(t->gx_ws, S, R * C, out);
}

struct Queries {
    const float* points;   // [n][n_points][3] camera frame (device)
    const float* labels;   // [n][n_points] (device)
    int n_points;
};

// Forward, loss and every gradient of one batch.  losses (nullable, host): total, reconstruction
// mean |r|, SDF mean |r| (0 without queries).
int check_device_error(mppi_encoder_trainer* t);

int loss_grads(mppi_encoder_trainer* t, int n, const float* d_noisy, const float* d_clean, float max_range,
               const Queries* q, float* losses) {
    mppi_encoder* e = t->enc;
    int rc = mppi_encode_depth(e, n, d_noisy, max_range, t->z);
    if (rc != MPPI_OK) return tfail(t, rc, "encoder forward failed: %s", mppi_encoder_last_error(e));
    cudaStream_t s = e->stream;
    const float inv_count = 1.f / (static_cast<float>(n) * static_cast<float>(t->T));
    const float lam_r = q ? t->lam_recon : 1.f;
    mppi::recon_kernel<<<n, 256, 0, s>>>(t->z, d_clean, 1.f / max_range, e->H, e->W, t->th, t->tw, t->Wd, t->bd,
                                         lam_r * inv_count, t->g, t->dz, t->loss_img);
    const float inv_q = q ? 1.f / (static_cast<float>(n) * static_cast<float>(q->n_points)) : 0.f;
    if (q) {
        const int bpi = q->n_points / mppi::kSdPts;
        mppi::sdf_bias_kernel<<<n, mppi::kSdHidden, 0, s>>>(t->net, t->z, t->sdf_b1p);
        mppi::SdfRecord rec{};
        if (t->train_dec) {
            rec = t->rec;
            rec.P = static_cast<long long>(n) * q->n_points;
            rec.z = t->z;
        }
        mppi::sdf_dz_kernel<<<n * bpi, mppi::kSdThreads, mppi::kSdSmem, s>>>(
            t->net, q->points, q->labels, q->n_points, t->sdf_b1p, t->lam_sdf * inv_q, t->sdf_part, t->sdf_loss_part,
            rec);
        mppi::sdf_dz_reduce_kernel<<<n, mppi::kSdHidden, 0, s>>>(t->net, t->sdf_part, t->sdf_loss_part, bpi, t->dz,
                                                                  t->sdf_loss_img);
        if (t->train_dec) {
            const long long P = rec.P;
            const int H = mppi::kSdHidden, ldx = t->net.nf + mppi::kLat;
            // dW1 = G1^T X, dW_l = G_l^T H_{l-1}, dw5 = g5^T H4; biases = column sums
            gtx(t, rec.G, H, rec.X, ldx, P, t->dgrad[0]);
            mppi::colsum_kernel<<<H, 256, 0, s>>>(rec.G, H, P, t->dgrad[1]);
            for (int l = 1; l < 4; ++l) {
                gtx(t, rec.G + static_cast<size_t>(l) * P * H, H, rec.H + static_cast<size_t>(l - 1) * P * H, H, P,
                    t->dgrad[2 * l]);
                mppi::colsum_kernel<<<H, 256, 0, s>>>(rec.G + static_cast<size_t>(l) * P * H, H, P, t->dgrad[2 * l + 1]);
            }
            gtx(t, rec.g5, 1, rec.H + static_cast<size_t>(3) * P * H, H, P, t->dgrad[8]);
            mppi::colsum_kernel<<<1, 256, 0, s>>>(rec.g5, 1, P, t->dgrad[9]);
        }
    }
    mppi::outer_sum_kernel<<<(t->T * mppi::kLat + 255) / 256, 256, 0, s>>>(t->g, t->z, n, t->T, mppi::kLat,
                                                                          t->grad[10], t->grad[11]);
    const int hw4 = e->h[4] * e->w[4];
    mppi::head_bwd_kernel<<<n, mppi::kLat, 0, s>>>(e->act[3], hw4, e->W5, t->dz, t->m4, t->delta[0]);
    mppi::outer_sum_kernel<<<(mppi::kLat * mppi::kLat + 255) / 256, 256, 0, s>>>(t->dz, t->m4, n, mppi::kLat,
                                                                                mppi::kLat, t->grad[8], t->grad[9]);
    float* cur = t->delta[0];
    float* nxt = t->delta[1];
    cudaError_t ce = cudaGetLastError();
    if (ce == cudaSuccess) ce = launch_wgrad<64, 64, false>(t, 3, n, e->act[2], 1.f, cur);
    if (ce == cudaSuccess) ce = launch_dgrad<64, 64>(t, 3, n, cur, nxt);
    std::swap(cur, nxt);
    if (ce == cudaSuccess) ce = launch_wgrad<32, 64, false>(t, 2, n, e->act[1], 1.f, cur);
    if (ce == cudaSuccess) ce = launch_dgrad<32, 64>(t, 2, n, cur, nxt);
    std::swap(cur, nxt);
    if (ce == cudaSuccess) ce = launch_wgrad<16, 32, false>(t, 1, n, e->act[0], 1.f, cur);
    if (ce == cudaSuccess) ce = launch_dgrad<16, 32>(t, 1, n, cur, nxt);
    std::swap(cur, nxt);
    if (ce == cudaSuccess) ce = launch_wgrad1(t, n, d_noisy, 1.f / max_range, cur);
    if (ce != cudaSuccess) return tfail(t, MPPI_E_CUDA, "launch failed: %s", cudaGetErrorString(ce));
    if (losses) {
        t->h_loss.resize(n);
        t->h_loss2.assign(n, 0.f);
        ce = cudaMemcpyAsync(t->h_loss.data(), t->loss_img, n * sizeof(float), cudaMemcpyDeviceToHost, s);
        if (ce == cudaSuccess && q)
            ce = cudaMemcpyAsync(t->h_loss2.data(), t->sdf_loss_img, n * sizeof(float), cudaMemcpyDeviceToHost, s);
        if (ce == cudaSuccess) ce = cudaStreamSynchronize(s);
        if (ce != cudaSuccess) return tfail(t, MPPI_E_CUDA, "loss read-back failed: %s", cudaGetErrorString(ce));
        const int rc = check_device_error(t);
        if (rc != MPPI_OK) return rc;
        double rsum = 0.0, ssum = 0.0;
        for (int i = 0; i < n; ++i) {
            rsum += t->h_loss[i];
            ssum += t->h_loss2[i];
        }
        const double l_rec = rsum * inv_count, l_sdf = ssum * inv_q;
        losses[0] = static_cast<float>(lam_r * l_rec + (q ? t->lam_sdf * l_sdf : 0.0));
        losses[1] = static_cast<float>(l_rec);
        losses[2] = static_cast<float>(l_sdf);
    }
    return MPPI_OK;
}

// After the trainer's work on the encoder's stream: MPPI_E_TIMEOUT (the word cleared) when a
// bounded wait of a tensor-core convolution gave up since the last check.  Synchronous.
int check_device_error(mppi_encoder_trainer* t) {
    mppi_encoder* e = t->enc;
    int word = 0;
    cudaError_t ce = cudaMemcpyAsync(&word, e->d_err, sizeof(int), cudaMemcpyDeviceToHost, e->stream);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(e->stream);
    if (ce == cudaSuccess && word != 0) {
        ce = cudaMemsetAsync(e->d_err, 0, sizeof(int), e->stream);
        if (ce == cudaSuccess) ce = cudaStreamSynchronize(e->stream);
        if (ce == cudaSuccess)
            return tfail(t, MPPI_E_TIMEOUT, "a tensor-core convolution gave up waiting for its MMAs (word %d)", word);
    }
    if (ce != cudaSuccess) return tfail(t, MPPI_E_CUDA, "error-word read-back failed: %s", cudaGetErrorString(ce));
    return MPPI_OK;
}

int adam_all(mppi_encoder_trainer* t, bool with_decoder) {
    t->step += 1;
    mppi::AdamTable tab{};
    int max_size = 0, nt = 0;
    for (int i = 0; i < mppi::kNumTensors; ++i, ++nt) {
        tab.p[nt] = t->param[i];
        tab.g[nt] = t->grad[i];
        tab.m[nt] = t->m[i];
        tab.v[nt] = t->v[i];
        tab.size[nt] = t->size[i];
        max_size = std::max(max_size, t->size[i]);
    }
    if (t->train_dec && with_decoder)
        for (int i = 0; i < 10; ++i, ++nt) {
            tab.p[nt] = t->dparam[i];
            tab.g[nt] = t->dgrad[i];
            tab.m[nt] = t->dm[i];
            tab.v[nt] = t->dv[i];
            tab.size[nt] = t->dsize[i];
            max_size = std::max(max_size, t->dsize[i]);
        }
    const float c1 = static_cast<float>(1.0 - std::pow(0.9, t->step));
    const float c2 = static_cast<float>(1.0 - std::pow(0.999, t->step));
    mppi::adam_kernel<<<dim3((max_size + 255) / 256, nt), 256, 0, t->enc->stream>>>(tab, t->lr, c1, c2);
    cudaError_t ce = cudaGetLastError();
    // the tensor-core convolutions read the weights in their packed form
    if (ce == cudaSuccess) ce = mppi::pack_conv_tc_weights(t->enc->wt, t->enc->wpack, t->enc->dgpack, t->enc->stream);
    if (ce != cudaSuccess) return tfail(t, MPPI_E_CUDA, "Adam launch failed: %s", cudaGetErrorString(ce));
    return MPPI_OK;
}

int read_grads(mppi_encoder_trainer* t, float* const* grads_out, bool with_decoder) {
    const int rc = check_device_error(t);
    if (rc != MPPI_OK) return rc;
    cudaError_t ce = cudaStreamSynchronize(t->enc->stream);
    for (int i = 0; i < mppi::kNumTensors && ce == cudaSuccess; ++i)
        if (grads_out[i])
            ce = cudaMemcpy(grads_out[i], t->grad[i], t->size[i] * sizeof(float), cudaMemcpyDeviceToHost);
    if (t->train_dec && with_decoder)
        for (int i = 0; i < 10 && ce == cudaSuccess; ++i)
            if (grads_out[mppi::kNumTensors + i])
                ce = cudaMemcpy(grads_out[mppi::kNumTensors + i], t->dgrad[i], t->dsize[i] * sizeof(float),
                                cudaMemcpyDeviceToHost);
    if (ce != cudaSuccess) return tfail(t, MPPI_E_CUDA, "gradient read-back failed: %s", cudaGetErrorString(ce));
    return MPPI_OK;
}

int check_queries(mppi_encoder_trainer* t, const float* d_points, const float* d_labels, int n_points) {
    if (!t->sdf) return tfail(t, MPPI_E_NOT_READY, "no SDF decoder: call mppi_encoder_train_set_sdf first");
    if (!d_points || !d_labels) return tfail(t, MPPI_E_INVALID, "NULL query pointer");
    if (n_points < mppi::kSdPts || n_points % mppi::kSdPts != 0 || n_points > t->max_points)
        return tfail(t, MPPI_E_INVALID, "n_points must be a multiple of 32 in [32, %d]", t->max_points);
    return MPPI_OK;
}

int check_batch(mppi_encoder_trainer* t, int n, const float* d_noisy, const float* d_clean, float max_range) {
    if (n < 1 || n > t->batch) return tfail(t, MPPI_E_INVALID, "n out of [1, batch = %d]", t->batch);
    if (!d_noisy || !d_clean) return tfail(t, MPPI_E_INVALID, "NULL image pointer");
    if (!(max_range > 0.f && max_range <= 3.0e38f)) return tfail(t, MPPI_E_INVALID, "max_range must be > 0");
    return MPPI_OK;
}

}  // namespace

extern "C" int mppi_encoder_get_weights(mppi_encoder* e, float* const* layers_out) {
    if (!e || !layers_out) return MPPI_E_INVALID;
    cudaError_t ce = cudaStreamSynchronize(e->stream);
    for (int l = 0; l < 4 && ce == cudaSuccess; ++l) {
        const size_t nw = static_cast<size_t>(mppi::kEncCout[l]) * mppi::kEncCin[l] * 9;
        if (layers_out[2 * l]) ce = cudaMemcpy(layers_out[2 * l], e->wt[l], nw * sizeof(float), cudaMemcpyDeviceToHost);
        if (ce == cudaSuccess && layers_out[2 * l + 1])
            ce = cudaMemcpy(layers_out[2 * l + 1], e->bias[l], mppi::kEncCout[l] * sizeof(float),
                            cudaMemcpyDeviceToHost);
    }
    if (ce == cudaSuccess && layers_out[8])
        ce = cudaMemcpy(layers_out[8], e->W5, MPPI_LATENT_DIM * MPPI_LATENT_DIM * sizeof(float), cudaMemcpyDeviceToHost);
    if (ce == cudaSuccess && layers_out[9])
        ce = cudaMemcpy(layers_out[9], e->b5, MPPI_LATENT_DIM * sizeof(float), cudaMemcpyDeviceToHost);
    if (ce != cudaSuccess) {
        std::snprintf(e->err, sizeof(e->err), "mppi_encoder_get_weights: %s", cudaGetErrorString(ce));
        return MPPI_E_CUDA;
    }
    return MPPI_OK;
}

extern "C" int mppi_encoder_train_create(mppi_encoder* enc, int batch, float lr, const float* dec_W,
                                         const float* dec_b, mppi_encoder_trainer** out) {
    using namespace mppi;
    if (!out) return tfail(nullptr, MPPI_E_INVALID, "mppi_encoder_train_create: NULL out");
    *out = nullptr;
    if (!enc || !dec_W || !dec_b) return tfail(nullptr, MPPI_E_INVALID, "mppi_encoder_train_create: NULL argument");
    if (batch < 1 || batch > enc->max_images)
        return tfail(nullptr, MPPI_E_INVALID, "mppi_encoder_train_create: batch out of [1, max_images = %d]",
                     enc->max_images);
    if (!(lr > 0.f && lr < 1e3f)) return tfail(nullptr, MPPI_E_INVALID, "mppi_encoder_train_create: lr must be > 0");
    mppi_encoder_trainer* t = new (std::nothrow) mppi_encoder_trainer();
    if (!t) return tfail(nullptr, MPPI_E_OOM, "mppi_encoder_train_create: host allocation failed");
    t->enc = enc;
    t->batch = batch;
    t->lr = lr;
    t->th = (enc->H + kPool - 1) / kPool;
    t->tw = (enc->W + kPool - 1) / kPool;
    t->T = t->th * t->tw;
    bool ok = talloc(t, &t->Wd, static_cast<size_t>(t->T) * kLat) && talloc(t, &t->bd, t->T);
    for (int l = 0; l < 4; ++l) {
        t->param[2 * l] = enc->wt[l];
        t->size[2 * l] = kEncCout[l] * kEncCin[l] * 9;
        t->param[2 * l + 1] = enc->bias[l];
        t->size[2 * l + 1] = kEncCout[l];
    }
    t->param[8] = enc->W5;
    t->size[8] = kLat * kLat;
    t->param[9] = enc->b5;
    t->size[9] = kLat;
    t->param[10] = t->Wd;
    t->size[10] = t->T * kLat;
    t->param[11] = t->bd;
    t->size[11] = t->T;
    for (int i = 0; i < kNumTensors && ok; ++i)
        ok = talloc(t, &t->grad[i], t->size[i]) && talloc(t, &t->m[i], t->size[i]) && talloc(t, &t->v[i], t->size[i]);
    size_t delta_floats = 0;
    for (int l = 0; l < 4; ++l)
        delta_floats = std::max(delta_floats, static_cast<size_t>(batch) * kEncCout[l] * enc->h[l + 1] * enc->w[l + 1]);
    // a split layer has S <= ceil(2 SMs / k_tiles) slices of CO x K1 <= 64 x 32 k_tiles floats
    // enough for the CUDA-core slicing and for the tensor-core one (the 64 -> 64 layer: 5 k tiles,
    // about two CTAs per SM, 64 x 577 partial sums each)
    t->ws_floats = std::max(static_cast<size_t>(64) * kWgK * (2 * enc->n_sms + 32),
                            static_cast<size_t>((2 * enc->n_sms + 4) / 5) * 64 * (9 * 64 + 1));
    ok = ok && talloc(t, &t->z, static_cast<size_t>(batch) * kLat) &&
         talloc(t, &t->g, static_cast<size_t>(batch) * t->T) && talloc(t, &t->dz, static_cast<size_t>(batch) * kLat) &&
         talloc(t, &t->m4, static_cast<size_t>(batch) * kLat) && talloc(t, &t->loss_img, batch) &&
         talloc(t, &t->delta[0], delta_floats) && talloc(t, &t->delta[1], delta_floats) &&
         talloc(t, &t->ws, t->ws_floats);
    if (ok) {
        ok = cudaMemcpy(t->Wd, dec_W, static_cast<size_t>(t->T) * kLat * sizeof(float), cudaMemcpyHostToDevice) ==
                 cudaSuccess &&
             cudaMemcpy(t->bd, dec_b, t->T * sizeof(float), cudaMemcpyHostToDevice) == cudaSuccess;
        for (int i = 0; i < kNumTensors && ok; ++i)
            ok = cudaMemset(t->m[i], 0, t->size[i] * sizeof(float)) == cudaSuccess &&
                 cudaMemset(t->v[i], 0, t->size[i] * sizeof(float)) == cudaSuccess;
    }
    if (!ok) {
        const cudaError_t ce = cudaGetLastError();
        trainer_free(t);
        delete t;
        return tfail(nullptr, ce == cudaErrorMemoryAllocation ? MPPI_E_OOM : MPPI_E_CUDA,
                     "mppi_encoder_train_create: device allocation or copy failed: %s", cudaGetErrorString(ce));
    }
    *out = t;
    return MPPI_OK;
}

extern "C" void mppi_encoder_train_destroy(mppi_encoder_trainer* t) {
    if (!t) return;
    cudaStreamSynchronize(t->enc->stream);
    trainer_free(t);
    delete t;
}

extern "C" const char* mppi_encoder_train_last_error(const mppi_encoder_trainer* t) {
    return t ? t->err : mppi::g_etr_err;
}

extern "C" int mppi_encoder_train_loss_grads(mppi_encoder_trainer* t, int n, const float* d_noisy,
                                             const float* d_clean, float max_range, float* loss,
                                             float* const* grads_out) {
    if (!t) return tfail(nullptr, MPPI_E_INVALID, "mppi_encoder_train_loss_grads: NULL trainer");
    int rc = check_batch(t, n, d_noisy, d_clean, max_range);
    if (rc != MPPI_OK) return rc;
    float losses[3];
    rc = loss_grads(t, n, d_noisy, d_clean, max_range, nullptr, loss ? losses : nullptr);
    if (rc != MPPI_OK) return rc;
    if (loss) *loss = losses[0];
    return grads_out ? read_grads(t, grads_out, false) : MPPI_OK;
}

extern "C" int mppi_encoder_train_step(mppi_encoder_trainer* t, int n, const float* d_noisy, const float* d_clean,
                                       float max_range, float* loss) {
    if (!t) return tfail(nullptr, MPPI_E_INVALID, "mppi_encoder_train_step: NULL trainer");
    int rc = check_batch(t, n, d_noisy, d_clean, max_range);
    if (rc != MPPI_OK) return rc;
    float losses[3];
    rc = loss_grads(t, n, d_noisy, d_clean, max_range, nullptr, loss ? losses : nullptr);
    if (rc != MPPI_OK) return rc;
    if (loss) *loss = losses[0];
    return adam_all(t, false);
}

extern "C" int mppi_encoder_train_set_sdf(mppi_encoder_trainer* t, const float* const* layers, int pe_levels,
                                          float softplus_beta, float lambda_recon, float lambda_sdf,
                                          int max_points_per_image, int train_decoder) {
    using namespace mppi;
    if (!t) return tfail(nullptr, MPPI_E_INVALID, "mppi_encoder_train_set_sdf: NULL trainer");
    if (!layers) return tfail(t, MPPI_E_INVALID, "mppi_encoder_train_set_sdf: NULL layers");
    for (int i = 0; i < 10; ++i)
        if (!layers[i]) return tfail(t, MPPI_E_INVALID, "mppi_encoder_train_set_sdf: layer array %d is NULL", i);
    if (pe_levels < 0 || pe_levels > MPPI_MAX_PE_LEVELS)
        return tfail(t, MPPI_E_INVALID, "pe_levels out of [0, MPPI_MAX_PE_LEVELS]");
    if (!(softplus_beta > 0.f && softplus_beta < 1e6f) || !(lambda_recon >= 0.f) || !(lambda_sdf >= 0.f))
        return tfail(t, MPPI_E_INVALID, "softplus_beta must be > 0 and the lambdas >= 0");
    if (max_points_per_image < kSdPts || max_points_per_image % kSdPts != 0 || max_points_per_image > (1 << 16))
        return tfail(t, MPPI_E_INVALID, "max_points_per_image must be a multiple of 32 in [32, 65536]");
    if (t->sdf) return tfail(t, MPPI_E_INVALID, "the SDF decoder is already set");
    if (cudaFuncSetAttribute(sdf_dz_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(kSdSmem)) !=
        cudaSuccess)
        return tfail(t, MPPI_E_CUDA, "shared-memory configuration of the SDF kernel failed");
    const int nf = 3 + 6 * pe_levels, ld = nf + kLat;
    const int sizes[10] = {kSdHidden * ld, kSdHidden, kSdHidden * kSdHidden, kSdHidden, kSdHidden * kSdHidden,
                           kSdHidden, kSdHidden * kSdHidden, kSdHidden, kSdHidden, 1};
    bool ok = true;
    for (int i = 0; i < 10 && ok; ++i) {
        t->dsize[i] = sizes[i];
        ok = talloc(t, &t->dparam[i], sizes[i]);
    }
    const size_t per = static_cast<size_t>(t->batch) * (max_points_per_image / kSdPts);
    ok = ok && talloc(t, &t->sdf_b1p, static_cast<size_t>(t->batch) * kSdHidden) &&
         talloc(t, &t->sdf_part, per * kSdHidden) && talloc(t, &t->sdf_loss_part, per) &&
         talloc(t, &t->sdf_loss_img, t->batch);
    if (ok && train_decoder) {
        const size_t P = static_cast<size_t>(t->batch) * max_points_per_image;
        for (int i = 0; i < 10 && ok; ++i)
            ok = talloc(t, &t->dgrad[i], sizes[i]) && talloc(t, &t->dm[i], sizes[i]) && talloc(t, &t->dv[i], sizes[i]);
        t->gx_ws_floats = static_cast<size_t>(kSdHidden) * kSdHidden * 32;
        ok = ok && talloc(t, &t->rec.X, P * ld) && talloc(t, &t->rec.H, 4 * P * kSdHidden) &&
             talloc(t, &t->rec.G, 4 * P * kSdHidden) && talloc(t, &t->rec.g5, P) && talloc(t, &t->gx_ws, t->gx_ws_floats);
        for (int i = 0; i < 10 && ok; ++i)
            ok = cudaMemset(t->dm[i], 0, sizes[i] * sizeof(float)) == cudaSuccess &&
                 cudaMemset(t->dv[i], 0, sizes[i] * sizeof(float)) == cudaSuccess;
    }
    if (!ok) return tfail(t, MPPI_E_OOM, "device allocation failed");
    cudaError_t ce = cudaSuccess;
    for (int i = 0; i < 10 && ce == cudaSuccess; ++i)
        ce = cudaMemcpy(t->dparam[i], layers[i], sizes[i] * sizeof(float), cudaMemcpyHostToDevice);
    if (ce != cudaSuccess) return tfail(t, MPPI_E_CUDA, "weight upload failed: %s", cudaGetErrorString(ce));
    t->net.W1 = t->dparam[0];
    t->net.b1 = t->dparam[1];
    for (int l = 0; l < 3; ++l) {
        t->net.W[l] = t->dparam[2 + 2 * l];
        t->net.b[l] = t->dparam[3 + 2 * l];
    }
    t->net.w5 = t->dparam[8];
    t->net.b5 = t->dparam[9];
    t->net.beta = softplus_beta;
    t->net.nf = nf;
    t->net.pe = pe_levels;
    t->train_dec = train_decoder != 0;
    t->lam_recon = lambda_recon;
    t->lam_sdf = lambda_sdf;
    t->max_points = max_points_per_image;
    t->sdf = true;
    return MPPI_OK;
}

extern "C" int mppi_encoder_train_loss_grads_sdf(mppi_encoder_trainer* t, int n, const float* d_noisy,
                                                 const float* d_clean, float max_range, const float* d_points,
                                                 const float* d_labels, int n_points, float* losses,
                                                 float* const* grads_out) {
    if (!t) return tfail(nullptr, MPPI_E_INVALID, "mppi_encoder_train_loss_grads_sdf: NULL trainer");
    int rc = check_batch(t, n, d_noisy, d_clean, max_range);
    if (rc == MPPI_OK) rc = check_queries(t, d_points, d_labels, n_points);
    if (rc != MPPI_OK) return rc;
    const Queries q{d_points, d_labels, n_points};
    rc = loss_grads(t, n, d_noisy, d_clean, max_range, &q, losses);
    if (rc != MPPI_OK) return rc;
    return grads_out ? read_grads(t, grads_out, true) : MPPI_OK;
}

extern "C" int mppi_encoder_train_step_sdf(mppi_encoder_trainer* t, int n, const float* d_noisy, const float* d_clean,
                                           float max_range, const float* d_points, const float* d_labels,
                                           int n_points, float* losses) {
    if (!t) return tfail(nullptr, MPPI_E_INVALID, "mppi_encoder_train_step_sdf: NULL trainer");
    int rc = check_batch(t, n, d_noisy, d_clean, max_range);
    if (rc == MPPI_OK) rc = check_queries(t, d_points, d_labels, n_points);
    if (rc != MPPI_OK) return rc;
    const Queries q{d_points, d_labels, n_points};
    rc = loss_grads(t, n, d_noisy, d_clean, max_range, &q, losses);
    if (rc != MPPI_OK) return rc;
    return adam_all(t, true);
}

extern "C" int mppi_encoder_train_get_decoder(mppi_encoder_trainer* t, float* W, float* b) {
    if (!t || !W || !b) return tfail(t, MPPI_E_INVALID, "mppi_encoder_train_get_decoder: NULL argument");
    cudaError_t ce = cudaStreamSynchronize(t->enc->stream);
    if (ce == cudaSuccess)
        ce = cudaMemcpy(W, t->Wd, static_cast<size_t>(t->T) * mppi::kLat * sizeof(float), cudaMemcpyDeviceToHost);
    if (ce == cudaSuccess) ce = cudaMemcpy(b, t->bd, t->T * sizeof(float), cudaMemcpyDeviceToHost);
    if (ce != cudaSuccess) return tfail(t, MPPI_E_CUDA, "decoder read-back failed: %s", cudaGetErrorString(ce));
    return MPPI_OK;
}

extern "C" int mppi_encoder_train_get_sdf_decoder(mppi_encoder_trainer* t, float* const* layers_out) {
    if (!t || !layers_out) return tfail(t, MPPI_E_INVALID, "mppi_encoder_train_get_sdf_decoder: NULL argument");
    if (!t->sdf) return tfail(t, MPPI_E_NOT_READY, "no SDF decoder set");
    cudaError_t ce = cudaStreamSynchronize(t->enc->stream);
    for (int i = 0; i < 10 && ce == cudaSuccess; ++i)
        if (layers_out[i])
            ce = cudaMemcpy(layers_out[i], t->dparam[i], t->dsize[i] * sizeof(float), cudaMemcpyDeviceToHost);
    if (ce != cudaSuccess) return tfail(t, MPPI_E_CUDA, "decoder read-back failed: %s", cudaGetErrorString(ce));
    return MPPI_OK;
}
