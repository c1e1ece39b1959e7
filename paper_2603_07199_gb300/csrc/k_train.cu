// Learned part: distil the exact gate-frame SDF into the Gate-SDF MLP on the GPU.
//
// Training set: Philox-sampled gate-frame points (70 % near the frame surface,
// a uniform surface point plus N(0, sigma^2 I); 30 % uniform in a cube) with the
// exact frame SDF as target.  Loss per batch of B points (Sec. III-B's L1 term
// plus an Eikonal term on the input gradient):
//     L = mean |s - s*| + lambda_e mean (|grad_p s| - 1)^2 .
// The input gradient is carried in forward mode (three tangent streams next to
// the values, "stream" 0 = values, 1..3 = d/dp_x, d/dp_y, d/dp_z) and the whole
// computation is differentiated in reverse mode; Adam updates FP32 master
// weights.  Kernels (FP32 on the CUDA cores, 128-point tiles, register-blocked
// GEMMs through shared memory, deterministic fixed-order reductions; the hidden
// layers' GEMMs can run instead in BF16 on the tensor cores, k_train_tc.cu):
//   sample -> [per step] first-layer bias -> forward layer 1 -> forward layers 2..4
//   -> output + loss + adjoints -> per layer 4..2: weight gradients, input
//   gradients -> layer-1 gradients -> reduce partials -> Adam.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "kernels.h"
#include "mppi.h"
#include "train_internal.cuh"

namespace mppi {
namespace {

using namespace train;

constexpr int kT = 256;
constexpr int kLd = kH + 4;

// acc[i][j] += sum_k Xs[k][row_i] Ms[k][col_j] over k < 128; rows/cols of thread (tr, tn)
// are two 4-wide strips 64 apart.
__device__ __forceinline__ int strip(int t, int i) { return (i < 4) ? t * 4 + i : 64 + t * 4 + (i - 4); }

__device__ __forceinline__ void tile_mm(const float* Xs, const float* Ms, int tr, int tn, float (&acc)[8][8]) {
#pragma unroll 4
    for (int k = 0; k < kH; ++k) {
        const float4 a0 = *reinterpret_cast<const float4*>(Xs + k * kLd + tr * 4);
        const float4 a1 = *reinterpret_cast<const float4*>(Xs + k * kLd + 64 + tr * 4);
        const float4 b0 = *reinterpret_cast<const float4*>(Ms + k * kLd + tn * 4);
        const float4 b1 = *reinterpret_cast<const float4*>(Ms + k * kLd + 64 + tn * 4);
        const float av[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
        const float bv[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
        for (int i = 0; i < 8; ++i)
#pragma unroll
            for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
    }
}

// ------------------------------------------------------------------ training points
__global__ void sample_kernel(int N, uint32_t key0, uint32_t key1, float near_frac, float sigma, float cube,
                              float a_in, float a_out, float d, float4* __restrict__ out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const uint4 w0 = philox4x32_10(make_uint4(static_cast<uint32_t>(i), 0u, 0x5EEDu, 0u), key0, key1);
    const uint4 w1 = philox4x32_10(make_uint4(static_cast<uint32_t>(i), 1u, 0x5EEDu, 0u), key0, key1);
    const float u0 = word_to_uniform(w0.x), u1 = word_to_uniform(w0.y);
    const float ua = word_to_uniform(w0.z), ub = word_to_uniform(w0.w);
    float x, y, z;
    if (u0 < near_frac) {
        // a point uniform over the frame surface: pick a part by its area, then a point on it
        const float face = (2.f * a_out) * (2.f * a_out) - (2.f * a_in) * (2.f * a_in);
        const float bar = (2.f * a_out) * (a_out - a_in), post = (a_out - a_in) * (2.f * a_in);
        const float outer = (2.f * a_out) * (2.f * d), inner = (2.f * a_in) * (2.f * d);
        const float total = 2.f * face + 4.f * outer + 4.f * inner;
        float r = u1 * total;
        if (r < 2.f * face) {
            x = (r < face) ? d : -d;
            r = (r < face) ? r : r - face;
            if (r < bar) {
                y = -a_out + 2.f * a_out * ua; z = a_in + (a_out - a_in) * ub;
            } else if (r < 2.f * bar) {
                y = -a_out + 2.f * a_out * ua; z = -(a_in + (a_out - a_in) * ub);
            } else if (r < 2.f * bar + post) {
                y = a_in + (a_out - a_in) * ua; z = -a_in + 2.f * a_in * ub;
            } else {
                y = -(a_in + (a_out - a_in) * ua); z = -a_in + 2.f * a_in * ub;
            }
        } else {
            r -= 2.f * face;
            const bool is_outer = r < 4.f * outer;
            const float half = is_outer ? a_out : a_in;
            const float part = is_outer ? outer : inner;
            const int wall = min(static_cast<int>((is_outer ? r : r - 4.f * outer) / part), 3);
            x = -d + 2.f * d * ua;
            const float t = -half + 2.f * half * ub;
            if (wall == 0) { y = half; z = t; } else if (wall == 1) { y = -half; z = t; }
            else if (wall == 2) { z = half; y = t; } else { z = -half; y = t; }
        }
        const float2 n01 = box_muller(word_to_uniform(w1.x), word_to_uniform(w1.y));
        const float2 n23 = box_muller(word_to_uniform(w1.z), word_to_uniform(w1.w));
        x += sigma * n01.x; y += sigma * n01.y; z += sigma * n23.x;
    } else {
        x = -cube + 2.f * cube * u1; y = -cube + 2.f * cube * ua; z = -cube + 2.f * cube * ub;
    }
    out[i] = make_float4(x, y, z, frame_sdf(x, y, z, a_in, a_out, d));
}

// ------------------------------------------------------------------ forward
__global__ void first_bias_kernel(TrainBufs T) {
    const int c = threadIdx.x;
    float acc = T.theta[oB1 + c];
    for (int j = 0; j < kLatent; ++j) acc = fmaf(T.theta[oW1 + c * kIn + 3 + j], T.z0[j], acc);
    T.b1p[c] = acc;
}

__global__ void fwd_layer1_kernel(TrainBufs T) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= T.B * kH) return;
    const int pt = idx / kH, c = idx - pt * kH;
    const float4 p = T.pts[pt];
    const float* w = T.theta + oW1 + c * kIn;
    T.A[1][idx] = T.b1p[c] + w[0] * p.x + w[1] * p.y + w[2] * p.z;
}

// Layer l in {2, 3, 4}: A_l = x0 W^T + b, AT_l^j = x_j W^T for the four input streams.
__global__ void __launch_bounds__(kT, 1) fwd_hidden_kernel(TrainBufs T, int l) {
    extern __shared__ __align__(16) float sm[];
    float* Xs = sm;                 // [k][row]
    float* Ms = sm + kH * kLd;      // [k][n] = W[n][k]
    const int tid = threadIdx.x, tn = tid & 15, tr = tid >> 4;
    const float* W = T.theta + offW(l);
    for (int i = tid; i < kH * kH; i += kT) {
        const int n = i / kH, k = i - n * kH;
        Ms[k * kLd + n] = W[i];
    }
    const float* bias = T.theta + offB(l);
    const int n_tiles = T.B / kTileRows;
    for (int tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
        for (int s = 0; s < 4; ++s) {
            __syncthreads();
            for (int i = tid; i < kTileRows * kH; i += kT) {
                const int m = i / kH, k = i - m * kH;
                Xs[k * kLd + m] = stream_in(T, l - 1, s, tile * kTileRows + m, k);
            }
            __syncthreads();
            float acc[8][8];
#pragma unroll
            for (int i = 0; i < 8; ++i)
#pragma unroll
                for (int j = 0; j < 8; ++j) acc[i][j] = 0.f;
            tile_mm(Xs, Ms, tr, tn, acc);
            float* dst = (s == 0) ? T.A[l] : T.AT[l] + static_cast<size_t>(s - 1) * T.B * kH;
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const size_t row = static_cast<size_t>(tile * kTileRows + strip(tr, i)) * kH;
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    const int n = strip(tn, j);
                    dst[row + n] = acc[i][j] + (s == 0 ? bias[n] : 0.f);
                }
            }
        }
    }
}

// ------------------------------------------------------------------ output layer, loss, adjoints of layer 4
// One warp per point (lane holds features lane + 32 i), 16 warps per CTA.  Also the w5 / b5
// partial gradients.
constexpr int kOutT = 512;
// the output and layer-1 kernels launch up to this many CTAs per SM (their partials are small)
constexpr int kSmallGridPerSm = 4;
__global__ void __launch_bounds__(kOutT) output_kernel(TrainBufs T) {
    __shared__ float s_w5[kOutT / 32][kH];
    __shared__ float s_b5[kOutT / 32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int nw = gridDim.x * (kOutT / 32);
    float gw5[4] = {0.f, 0.f, 0.f, 0.f}, gb5 = 0.f;
    const float invB = 1.f / static_cast<float>(T.B);
    for (int pt = blockIdx.x * (kOutT / 32) + wid; pt < T.B; pt += nw) {
        float a[4], sg[4], at[3][4], w5[4];
        float s = 0.f, g[3] = {0.f, 0.f, 0.f};
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int c = lane + 32 * i;
            a[i] = T.A[4][static_cast<size_t>(pt) * kH + c];
            sg[i] = sig_beta(a[i], T.beta);
            w5[i] = T.theta[oW5 + c];
            s = fmaf(w5[i], sp_beta(a[i], T.beta), s);
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                at[j][i] = T.AT[4][(static_cast<size_t>(j) * T.B + pt) * kH + c];
                g[j] = fmaf(w5[i], sg[i] * at[j][i], g[j]);
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            s += __shfl_xor_sync(0xffffffffu, s, o);
#pragma unroll
            for (int j = 0; j < 3; ++j) g[j] += __shfl_xor_sync(0xffffffffu, g[j], o);
        }
        s += T.theta[oB5];
        const float tgt = T.pts[pt].w;
        const float gn = sqrtf(g[0] * g[0] + g[1] * g[1] + g[2] * g[2]);
        if (lane == 0) T.loss[pt] = fabsf(s - tgt) + T.lam_e * (gn - 1.f) * (gn - 1.f);
        const float ds = (s > tgt ? 1.f : (s < tgt ? -1.f : 0.f)) * invB;
        const float kg = T.lam_e * 2.f * (gn - 1.f) / fmaxf(gn, 1e-30f) * invB;
        const float dg[3] = {kg * g[0], kg * g[1], kg * g[2]};
        gb5 += ds;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int c = lane + 32 * i;
            const float sig2 = T.beta * sg[i] * (1.f - sg[i]);
            float da = ds * w5[i] * sg[i];
            float gsum = ds * sp_beta(a[i], T.beta);
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                const float dht = dg[j] * w5[i];
                da = fmaf(dht * at[j][i], sig2, da);
                T.dAT[4][(static_cast<size_t>(j) * T.B + pt) * kH + c] = dht * sg[i];
                gsum = fmaf(dg[j], sg[i] * at[j][i], gsum);
            }
            T.dA[4][static_cast<size_t>(pt) * kH + c] = da;
            gw5[i] += gsum;
        }
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) s_w5[wid][lane + 32 * i] = gw5[i];
    if (lane == 0) s_b5[wid] = gb5;
    __syncthreads();
    if (threadIdx.x < kH) {
        float t = 0.f;
        for (int w = 0; w < kOutT / 32; ++w) t += s_w5[w][threadIdx.x];
        T.opart[static_cast<size_t>(blockIdx.x) * (kH + 1) + threadIdx.x] = t;
    }
    if (threadIdx.x == 0) {
        float t = 0.f;
        for (int w = 0; w < kOutT / 32; ++w) t += s_b5[w];
        T.opart[static_cast<size_t>(blockIdx.x) * (kH + 1) + kH] = t;
    }
}

// ------------------------------------------------------------------ backward: weight gradients of layer l
// dW_l[o][i] = sum_pt dA_l[pt][o] x0[pt][i] + sum_j dAT_l^j[pt][o] xj[pt][i];  db_l = sum_pt dA_l[pt].
__global__ void __launch_bounds__(kT, 1) bwd_weight_kernel(TrainBufs T, int l) {
    extern __shared__ __align__(16) float sm[];
    float* Ds = sm;                 // [pt][o]
    float* Xs = sm + kH * kLd;      // [pt][i]
    const int tid = threadIdx.x, tn = tid & 15, tr = tid >> 4;
    float acc[8][8];
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = 0.f;
    float db = 0.f;
    const int n_tiles = T.B / kTileRows;
    for (int tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
        for (int s = 0; s < 4; ++s) {
            __syncthreads();
            const float* src = (s == 0) ? T.dA[l] : T.dAT[l] + static_cast<size_t>(s - 1) * T.B * kH;
            for (int i = tid; i < kTileRows * kH; i += kT) {
                const int m = i / kH, k = i - m * kH;
                const int pt = tile * kTileRows + m;
                Ds[m * kLd + k] = src[static_cast<size_t>(pt) * kH + k];
                Xs[m * kLd + k] = stream_in(T, l - 1, s, pt, k);
            }
            __syncthreads();
            tile_mm(Ds, Xs, tr, tn, acc);
            if (s == 0 && tid < kH)
                for (int m = 0; m < kTileRows; ++m) db += Ds[m * kLd + tid];
        }
    }
    float* part = T.partial + static_cast<size_t>(blockIdx.x) * kNumParams;
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) part[offW(l) + strip(tr, i) * kH + strip(tn, j)] = acc[i][j];
    if (tid < kH) part[offB(l) + tid] = db;
}

// ------------------------------------------------------------------ backward: input gradients of layer l
// dx_s = d_s W_l (s = 0..3), then through the activation of layer l-1:
//   dA_{l-1} = dx_0 sp'(A) + sum_j dx_j AT_j sp''(A),   dAT_{l-1}^j = dx_j sp'(A).
__global__ void __launch_bounds__(kT, 1) bwd_input_kernel(TrainBufs T, int l) {
    extern __shared__ __align__(16) float sm[];
    float* Xs = sm;                 // [o][pt]
    float* Ms = sm + kH * kLd;      // [o][i] = W[o][i]
    const int tid = threadIdx.x, tn = tid & 15, tr = tid >> 4;
    const float* W = T.theta + offW(l);
    for (int i = tid; i < kH * kH; i += kT) {
        const int o = i / kH, k = i - o * kH;
        Ms[o * kLd + k] = W[i];
    }
    const int lower = l - 1;
    const int n_tiles = T.B / kTileRows;
    for (int tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
        float tot[8][8];
#pragma unroll
        for (int i = 0; i < 8; ++i)
#pragma unroll
            for (int j = 0; j < 8; ++j) tot[i][j] = 0.f;
        for (int s = 0; s < 4; ++s) {
            __syncthreads();
            const float* src = (s == 0) ? T.dA[l] : T.dAT[l] + static_cast<size_t>(s - 1) * T.B * kH;
            for (int i = tid; i < kTileRows * kH; i += kT) {
                const int m = i / kH, k = i - m * kH;
                Xs[k * kLd + m] = src[static_cast<size_t>(tile * kTileRows + m) * kH + k];
            }
            __syncthreads();
            float acc[8][8];
#pragma unroll
            for (int i = 0; i < 8; ++i)
#pragma unroll
                for (int j = 0; j < 8; ++j) acc[i][j] = 0.f;
            tile_mm(Xs, Ms, tr, tn, acc);
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const int pt = tile * kTileRows + strip(tr, i);
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    const int k = strip(tn, j);
                    const float a = T.A[lower][static_cast<size_t>(pt) * kH + k];
                    const float sg = sig_beta(a, T.beta);
                    if (s == 0) {
                        tot[i][j] = fmaf(acc[i][j], sg, tot[i][j]);
                    } else {
                        const float t = (lower == 1) ? T.theta[oW1 + k * kIn + (s - 1)]
                                                     : T.AT[lower][(static_cast<size_t>(s - 1) * T.B + pt) * kH + k];
                        tot[i][j] = fmaf(acc[i][j] * t, T.beta * sg * (1.f - sg), tot[i][j]);
                        T.dAT[lower][(static_cast<size_t>(s - 1) * T.B + pt) * kH + k] = acc[i][j] * sg;
                    }
                }
            }
        }
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const int pt = tile * kTileRows + strip(tr, i);
#pragma unroll
            for (int j = 0; j < 8; ++j) T.dA[lower][static_cast<size_t>(pt) * kH + strip(tn, j)] = tot[i][j];
        }
    }
}

// ------------------------------------------------------------------ layer-1 gradients
// dW1[c][k] = sum_pt dA1[pt][c] p_k + sum_pt dAT1^k[pt][c] (k < 3);  db1[c] = sum_pt dA1[pt][c].
// CTA b takes a contiguous range of points; thread (c, q) sums every kL1Phases-th point of it
// from q, and the phases are added in a fixed order.
constexpr int kL1Phases = 4;
__global__ void __launch_bounds__(kH * kL1Phases) layer1_grad_kernel(TrainBufs T) {
    __shared__ float red[kL1Phases][4][kH];
    const int c = threadIdx.x & (kH - 1), q = threadIdx.x / kH;
    const int per = (T.B + gridDim.x - 1) / gridDim.x;
    const int p0 = blockIdx.x * per, p1 = min(T.B, p0 + per);
    const size_t plane = static_cast<size_t>(T.B) * kH;
    float g0 = 0.f, g1 = 0.f, g2 = 0.f, gb = 0.f;
#pragma unroll 4
    for (int pt = p0 + q; pt < p1; pt += kL1Phases) {
        const float4 p = T.pts[pt];
        const size_t i = static_cast<size_t>(pt) * kH + c;
        const float d = T.dA[1][i];
        gb += d;
        g0 += d * p.x + T.dAT[1][i];
        g1 += d * p.y + T.dAT[1][plane + i];
        g2 += d * p.z + T.dAT[1][2 * plane + i];
    }
    red[q][0][c] = g0;
    red[q][1][c] = g1;
    red[q][2][c] = g2;
    red[q][3][c] = gb;
    __syncthreads();
    if (q == 0) {
        float r[4] = {0.f, 0.f, 0.f, 0.f};
        for (int h = 0; h < kL1Phases; ++h)
            for (int k = 0; k < 4; ++k) r[k] += red[h][k][c];
        float* part = T.l1part + static_cast<size_t>(blockIdx.x) * 4 * kH;
        for (int k = 0; k < 4; ++k) part[k * kH + c] = r[k];
    }
}

// Sum the per-CTA partials of layers 2-4 (n_lin rows of T.partial) in a fixed order.
__global__ void reduce_kernel(TrainBufs T, int n_lin) {
    const int p = oW2 + blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= oW5) return;
    float acc = 0.f;
    for (int b = 0; b < n_lin; ++b) acc += T.partial[static_cast<size_t>(b) * kNumParams + p];
    T.grad[p] = acc;
}

// The small partial areas, one warp per sum (lanes take rows lane, lane + 32, ..., then a fixed
// shuffle tree): sums 0..4 kH - 1 are W1[:, 0..2] and b1 over n_l1 rows of T.l1part (the warp
// of db1[c] also writes the latent columns dW1[c][3 + j] = db1[c] z0[j]); sums 4 kH .. 5 kH are
// w5 and b5 over n_out rows of T.opart.
constexpr int kSmallSums = 5 * kH + 1;
__global__ void reduce_small_kernel(TrainBufs T, int n_out, int n_l1) {
    const int w = blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    if (w >= kSmallSums) return;
    float acc = 0.f;
    if (w < 4 * kH) {
        const int k = w / kH, c = w - k * kH;
        for (int b = lane; b < n_l1; b += 32) acc += T.l1part[(static_cast<size_t>(b) * 4 + k) * kH + c];
    } else {
        const int q = w - 4 * kH;
        for (int b = lane; b < n_out; b += 32) acc += T.opart[static_cast<size_t>(b) * (kH + 1) + q];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (w < 3 * kH) {
        const int k = w / kH, c = w - k * kH;
        if (lane == 0) T.grad[oW1 + c * kIn + k] = acc;
    } else if (w < 4 * kH) {
        const int c = w - 3 * kH;
        if (lane == 0) T.grad[oB1 + c] = acc;
        for (int j = lane; j < kLatent; j += 32) T.grad[oW1 + c * kIn + 3 + j] = acc * T.z0[j];
    } else {
        if (lane == 0) T.grad[oW5 + (w - 4 * kH)] = acc;
    }
}

__global__ void adam_kernel(float* theta, const float* grad, float* m, float* v, int n, float lr, float b1, float b2,
                            float eps, float c1, float c2) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    const float g = grad[p];
    const float mm = b1 * m[p] + (1.f - b1) * g;
    const float vv = b2 * v[p] + (1.f - b2) * g * g;
    m[p] = mm;
    v[p] = vv;
    theta[p] -= lr * (mm / c1) / (sqrtf(vv / c2) + eps);
}

__global__ void loss_mean_kernel(const float* loss, int B, float* out) {
    __shared__ float sh[kT];
    float acc = 0.f;
    for (int i = threadIdx.x; i < B; i += kT) acc += loss[i];
    sh[threadIdx.x] = acc;
    __syncthreads();
    for (int s = kT / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[0] = sh[0] / static_cast<float>(B);
}

// Inference-only output for evaluation: s per point (one warp per point).
__global__ void eval_output_kernel(TrainBufs T, float* err) {
    const int lane = threadIdx.x & 31;
    const int pt = blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
    if (pt >= T.B) return;
    float s = 0.f;
    for (int i = 0; i < 4; ++i) {
        const int c = lane + 32 * i;
        s = fmaf(T.theta[oW5 + c], sp_beta(T.A[4][static_cast<size_t>(pt) * kH + c], T.beta), s);
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) err[pt] = fabsf(s + T.theta[oB5] - T.pts[pt].w);
}

constexpr size_t kGemmSmem = sizeof(float) * 2 * kH * kLd;

}  // namespace
}  // namespace mppi

using namespace mppi;

struct mppi_trainer {
    mppi_train_config cfg{};
    int n_sms = 0;
    int n_cta = 0;
    int step = 0;
    char err[512] = "";
    std::vector<void*> allocs;
    float* theta = nullptr;
    float* m = nullptr;
    float* v = nullptr;
    float* grad = nullptr;
    float* partial = nullptr;
    float* opart = nullptr;
    float* l1part = nullptr;
    float* b1p = nullptr;
    float* z0 = nullptr;
    float4* data = nullptr;        // training set
    float4* holdout = nullptr;     // held-out check set
    float4* batch_pts = nullptr;   // explicit batch (gradient checks)
    float* acts = nullptr;
    float* loss = nullptr;
    float* loss_mean = nullptr;
    float* errs = nullptr;
    int* dev_err = nullptr;                  // device error word of the tensor-core kernels
    int gemm = MPPI_TRAIN_GEMM_FP32;         // precision of the hidden-layer GEMMs in training
    cudaStream_t stream = nullptr;
    TrainBufs T{};
};

namespace {

thread_local char g_train_err[512] = "";

int tfail(mppi_trainer* t, int code, const char* fmt, ...) {
    char* dst = t ? t->err : g_train_err;
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(dst, 512, fmt, ap);
    va_end(ap);
    return code;
}

#define TRY(t, expr)                                                                                  \
    do {                                                                                              \
        cudaError_t e_ = (expr);                                                                      \
        if (e_ != cudaSuccess) return tfail((t), MPPI_E_CUDA, "%s: %s", #expr, cudaGetErrorString(e_)); \
    } while (0)

template <typename X>
int talloc(mppi_trainer* t, X** p, size_t count) {
    void* q = nullptr;
    if (cudaMalloc(&q, count * sizeof(X)) != cudaSuccess) {
        cudaGetLastError();
        return tfail(t, MPPI_E_OOM, "cudaMalloc(%zu) failed", count * sizeof(X));
    }
    t->allocs.push_back(q);
    *p = static_cast<X*>(q);
    return MPPI_OK;
}

// Point the per-batch buffers at `pts` (B points) and bind the activation storage.
void bind_batch(mppi_trainer* t, const float4* pts, int B) {
    TrainBufs& T = t->T;
    T.pts = pts;
    T.B = B;
    const size_t BH = static_cast<size_t>(B) * kH;
    float* a = t->acts;
    for (int l = 1; l <= 4; ++l) {
        T.A[l] = a; a += BH;
        T.dA[l] = a; a += BH;
        T.AT[l] = a; a += 3 * BH;
        T.dAT[l] = a; a += 3 * BH;
    }
}

// Forward through layer 4 for the bound batch (values and tangents); tc: the hidden
// layers' GEMMs in BF16 on the tensor cores.
int forward(mppi_trainer* t, bool tc) {
    TrainBufs& T = t->T;
    cudaStream_t s = t->stream;
    first_bias_kernel<<<1, kH, 0, s>>>(T);
    fwd_layer1_kernel<<<(T.B * kH + 255) / 256, 256, 0, s>>>(T);
    const int grid = std::min(t->n_cta, T.B / kTileRows);
    for (int l = 2; l <= 4; ++l) {
        if (tc) TRY(t, launch_fwd_hidden_tc(T, l, grid, s));
        else fwd_hidden_kernel<<<grid, kT, kGemmSmem, s>>>(T, l);
    }
    TRY(t, cudaGetLastError());
    return MPPI_OK;
}

// Loss, adjoints, gradients (reduced into T.grad) for the bound batch.
int backward(mppi_trainer* t, bool tc) {
    TrainBufs& T = t->T;
    cudaStream_t s = t->stream;
    const int grid = std::min(t->n_cta, T.B / kTileRows);
    const int out_grid = std::min(kSmallGridPerSm * t->n_cta, (T.B + kOutT / 32 - 1) / (kOutT / 32));
    output_kernel<<<out_grid, kOutT, 0, s>>>(T);
    for (int l = 4; l >= 2; --l) {
        if (tc) {
            TRY(t, launch_bwd_weight_tc(T, l, grid, s));
            TRY(t, launch_bwd_input_tc(T, l, grid, s));
        } else {
            bwd_weight_kernel<<<grid, kT, kGemmSmem, s>>>(T, l);
            bwd_input_kernel<<<grid, kT, kGemmSmem, s>>>(T, l);
        }
    }
    const int l1_grid = std::min(kSmallGridPerSm * t->n_cta, T.B / kL1Phases);
    layer1_grad_kernel<<<l1_grid, kH * kL1Phases, 0, s>>>(T);
    reduce_kernel<<<(oW5 - oW2 + 255) / 256, 256, 0, s>>>(T, grid);
    reduce_small_kernel<<<(kSmallSums + 7) / 8, 256, 0, s>>>(T, out_grid, l1_grid);
    loss_mean_kernel<<<1, kT, 0, s>>>(T.loss, T.B, t->loss_mean);
    TRY(t, cudaGetLastError());
    return MPPI_OK;
}

// After the stream has drained: a bounded wait that gave up inside a tensor-core kernel.
int check_device_error(mppi_trainer* t) {
    int e = 0;
    TRY(t, cudaMemcpy(&e, t->dev_err, sizeof(int), cudaMemcpyDeviceToHost));
    if (e != 0) {
        TRY(t, cudaMemset(t->dev_err, 0, sizeof(int)));
        return tfail(t, MPPI_E_TIMEOUT, "a tensor-core GEMM kernel gave up waiting for its MMAs (code %d)", e);
    }
    return MPPI_OK;
}

const size_t kLayerSizes[10] = {static_cast<size_t>(kH) * kIn, kH, kH * kH, kH, kH * kH, kH, kH * kH, kH, kH, 1};
const int kLayerOffsets[10] = {oW1, oB1, oW2, oB2, oW3, oB3, oW4, oB4, oW5, oB5};

}  // namespace

extern "C" {

void mppi_train_config_default(mppi_train_config* c) {
    if (!c) return;
    std::memset(c, 0, sizeof(*c));
    c->batch = 65536;
    c->n_points = 1 << 21;
    c->n_holdout = 1 << 18;
    c->lr = 1e-3f;
    c->beta1 = 0.9f;
    c->beta2 = 0.999f;
    c->eps = 1e-8f;
    c->eikonal_weight = 0.1f;
    c->softplus_beta = 100.f;
    c->near_surface_fraction = 0.7f;
    c->near_surface_sigma = 0.05f;
    c->cube_half = 4.f;
    c->gate_inner_half = 0.5f;
    c->gate_outer_half = 0.75f;
    c->gate_half_depth = 0.1f;
    c->seed = 0xD15711ull;
}

void mppi_train_destroy(mppi_trainer* t) {
    if (!t) return;
    if (t->stream) cudaStreamSynchronize(t->stream);
    for (void* p : t->allocs) cudaFree(p);
    if (t->stream) cudaStreamDestroy(t->stream);
    delete t;
}

const char* mppi_train_last_error(const mppi_trainer* t) { return t ? t->err : g_train_err; }

int mppi_train_create(const mppi_train_config* cfg, const float* const* init_layers, const float* latent,
                      mppi_trainer** out) {
    if (!cfg || !init_layers || !latent || !out) return tfail(nullptr, MPPI_E_INVALID, "NULL argument");
    *out = nullptr;
    if (cfg->batch < kTileRows || cfg->batch % kTileRows != 0 || cfg->batch > (1 << 20))
        return tfail(nullptr, MPPI_E_INVALID, "batch must be a multiple of 128 in [128, 2^20]");
    if (cfg->n_points < cfg->batch || cfg->n_points % cfg->batch != 0 || cfg->n_points > (1 << 26))
        return tfail(nullptr, MPPI_E_INVALID, "n_points must be a multiple of batch, at most 2^26");
    if (cfg->n_holdout < kTileRows || cfg->n_holdout % kTileRows != 0 || cfg->n_holdout > (1 << 22))
        return tfail(nullptr, MPPI_E_INVALID, "n_holdout must be a multiple of 128 in [128, 2^22]");
    if (!(cfg->lr > 0.f) || !(cfg->softplus_beta > 0.f) || cfg->eikonal_weight < 0.f)
        return tfail(nullptr, MPPI_E_INVALID, "lr and softplus_beta must be > 0, eikonal_weight >= 0");
    for (int i = 0; i < 10; ++i)
        if (!init_layers[i]) return tfail(nullptr, MPPI_E_INVALID, "layer pointer %d is NULL", i);
    mppi_trainer* t = new (std::nothrow) mppi_trainer();
    if (!t) return tfail(nullptr, MPPI_E_OOM, "host allocation failed");
    t->cfg = *cfg;
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&t->n_sms, cudaDevAttrMultiProcessorCount, dev);
    t->n_cta = t->n_sms > 0 ? t->n_sms : 1;
    if (cudaStreamCreateWithFlags(&t->stream, cudaStreamNonBlocking) != cudaSuccess) {
        delete t;
        return tfail(nullptr, MPPI_E_CUDA, "cudaStreamCreate failed");
    }
    const int B = cfg->batch;
    const int n_part = std::max(t->n_cta, 1);
    int rc = MPPI_OK;
    rc = rc ? rc : talloc(t, &t->theta, kNumParams);
    rc = rc ? rc : talloc(t, &t->m, kNumParams);
    rc = rc ? rc : talloc(t, &t->v, kNumParams);
    rc = rc ? rc : talloc(t, &t->grad, kNumParams);
    rc = rc ? rc : talloc(t, &t->partial, static_cast<size_t>(n_part) * kNumParams);
    rc = rc ? rc : talloc(t, &t->opart, static_cast<size_t>(kSmallGridPerSm) * n_part * (kH + 1));
    rc = rc ? rc : talloc(t, &t->l1part, static_cast<size_t>(kSmallGridPerSm) * n_part * 4 * kH);
    rc = rc ? rc : talloc(t, &t->b1p, kH);
    rc = rc ? rc : talloc(t, &t->z0, kLatent);
    rc = rc ? rc : talloc(t, &t->data, cfg->n_points);
    rc = rc ? rc : talloc(t, &t->holdout, cfg->n_holdout);
    rc = rc ? rc : talloc(t, &t->batch_pts, cfg->batch);
    rc = rc ? rc : talloc(t, &t->acts, static_cast<size_t>(B) * kH * 32);
    rc = rc ? rc : talloc(t, &t->loss, B);
    rc = rc ? rc : talloc(t, &t->loss_mean, 1);
    rc = rc ? rc : talloc(t, &t->errs, cfg->n_holdout);
    rc = rc ? rc : talloc(t, &t->dev_err, 1);
    if (rc != MPPI_OK) {
        std::snprintf(g_train_err, sizeof(g_train_err), "%s", t->err);
        mppi_train_destroy(t);
        return rc;
    }
    std::vector<float> h(kNumParams);
    for (int i = 0; i < 10; ++i) std::memcpy(h.data() + kLayerOffsets[i], init_layers[i], kLayerSizes[i] * sizeof(float));
    bool ok = cudaMemcpy(t->theta, h.data(), kNumParams * sizeof(float), cudaMemcpyHostToDevice) == cudaSuccess &&
              cudaMemcpy(t->z0, latent, kLatent * sizeof(float), cudaMemcpyHostToDevice) == cudaSuccess &&
              cudaMemset(t->m, 0, kNumParams * sizeof(float)) == cudaSuccess &&
              cudaMemset(t->v, 0, kNumParams * sizeof(float)) == cudaSuccess &&
              cudaMemset(t->dev_err, 0, sizeof(int)) == cudaSuccess &&
              cudaFuncSetAttribute(fwd_hidden_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   static_cast<int>(kGemmSmem)) == cudaSuccess &&
              cudaFuncSetAttribute(bwd_weight_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   static_cast<int>(kGemmSmem)) == cudaSuccess &&
              cudaFuncSetAttribute(bwd_input_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   static_cast<int>(kGemmSmem)) == cudaSuccess;
    if (!ok) {
        std::snprintf(g_train_err, sizeof(g_train_err), "initialisation failed: %s",
                      cudaGetErrorString(cudaGetLastError()));
        mppi_train_destroy(t);
        return MPPI_E_CUDA;
    }
    TrainBufs& T = t->T;
    T.theta = t->theta;
    T.grad = t->grad;
    T.partial = t->partial;
    T.opart = t->opart;
    T.l1part = t->l1part;
    T.b1p = t->b1p;
    T.z0 = t->z0;
    T.loss = t->loss;
    T.err = t->dev_err;
    T.beta = cfg->softplus_beta;
    T.lam_e = cfg->eikonal_weight;
    // training and held-out points from two Philox keys
    const uint32_t k0 = static_cast<uint32_t>(cfg->seed), k1 = static_cast<uint32_t>(cfg->seed >> 32);
    sample_kernel<<<(cfg->n_points + 255) / 256, 256, 0, t->stream>>>(
        cfg->n_points, k0, k1, cfg->near_surface_fraction, cfg->near_surface_sigma, cfg->cube_half,
        cfg->gate_inner_half, cfg->gate_outer_half, cfg->gate_half_depth, t->data);
    sample_kernel<<<(cfg->n_holdout + 255) / 256, 256, 0, t->stream>>>(
        cfg->n_holdout, k0 ^ 0x9E3779B9u, k1 ^ 0x7F4A7C15u, cfg->near_surface_fraction, cfg->near_surface_sigma,
        cfg->cube_half, cfg->gate_inner_half, cfg->gate_outer_half, cfg->gate_half_depth, t->holdout);
    if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(t->stream) != cudaSuccess) {
        std::snprintf(g_train_err, sizeof(g_train_err), "point sampling failed");
        mppi_train_destroy(t);
        return MPPI_E_CUDA;
    }
    *out = t;
    return MPPI_OK;
}

int mppi_train_set_lr(mppi_trainer* t, float lr) {
    if (!t) return tfail(nullptr, MPPI_E_INVALID, "trainer is NULL");
    if (!(lr > 0.f) || !std::isfinite(lr)) return tfail(t, MPPI_E_INVALID, "lr must be finite and > 0");
    t->cfg.lr = lr;
    return MPPI_OK;
}

int mppi_train_set_gemm_precision(mppi_trainer* t, int precision) {
    if (!t) return tfail(nullptr, MPPI_E_INVALID, "trainer is NULL");
    if (precision != MPPI_TRAIN_GEMM_FP32 && precision != MPPI_TRAIN_GEMM_BF16)
        return tfail(t, MPPI_E_INVALID, "unknown GEMM precision %d", precision);
    if (precision == MPPI_TRAIN_GEMM_BF16) {
        int dev = 0, major = 0, minor = 0;
        TRY(t, cudaGetDevice(&dev));
        cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev);
        cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev);
        if (major != 10 || minor != 3)
            return tfail(t, MPPI_E_UNSUPPORTED, "BF16 tensor-core GEMMs need an sm_103 device (found sm_%d%d)", major,
                         minor);
        TRY(t, configure_tc_train());
    }
    t->gemm = precision;
    return MPPI_OK;
}

int mppi_train_step(mppi_trainer* t, int n_steps, float* last_loss) {
    if (!t || n_steps < 0) return tfail(t, MPPI_E_INVALID, "bad arguments");
    const mppi_train_config& c = t->cfg;
    const int per_epoch = c.n_points / c.batch;
    for (int i = 0; i < n_steps; ++i) {
        bind_batch(t, t->data + static_cast<size_t>(t->step % per_epoch) * c.batch, c.batch);
        const bool tc = t->gemm == MPPI_TRAIN_GEMM_BF16;
        int rc = forward(t, tc);
        if (rc == MPPI_OK) rc = backward(t, tc);
        if (rc != MPPI_OK) return rc;
        ++t->step;
        const float c1 = 1.f - std::pow(c.beta1, static_cast<float>(t->step));
        const float c2 = 1.f - std::pow(c.beta2, static_cast<float>(t->step));
        adam_kernel<<<(kNumParams + 255) / 256, 256, 0, t->stream>>>(t->theta, t->grad, t->m, t->v, kNumParams, c.lr,
                                                                     c.beta1, c.beta2, c.eps, c1, c2);
        TRY(t, cudaGetLastError());
    }
    if (last_loss) {
        TRY(t, cudaMemcpyAsync(last_loss, t->loss_mean, sizeof(float), cudaMemcpyDeviceToHost, t->stream));
    }
    TRY(t, cudaStreamSynchronize(t->stream));
    return check_device_error(t);
}

int mppi_train_loss_grads(mppi_trainer* t, const float* points, int n, float* loss, float* grads) {
    if (!t || !points || n < kTileRows || n % kTileRows != 0 || n > t->cfg.batch)
        return tfail(t, MPPI_E_INVALID, "n must be a multiple of 128 and at most the batch size");
    TRY(t, cudaMemcpyAsync(t->batch_pts, points, static_cast<size_t>(n) * sizeof(float4), cudaMemcpyHostToDevice,
                           t->stream));
    bind_batch(t, t->batch_pts, n);
    const bool tc = t->gemm == MPPI_TRAIN_GEMM_BF16;
    int rc = forward(t, tc);
    if (rc == MPPI_OK) rc = backward(t, tc);
    if (rc != MPPI_OK) return rc;
    if (loss) TRY(t, cudaMemcpyAsync(loss, t->loss_mean, sizeof(float), cudaMemcpyDeviceToHost, t->stream));
    if (grads) TRY(t, cudaMemcpyAsync(grads, t->grad, kNumParams * sizeof(float), cudaMemcpyDeviceToHost, t->stream));
    TRY(t, cudaStreamSynchronize(t->stream));
    return check_device_error(t);
}

int mppi_train_get_weights(mppi_trainer* t, float* const* layers_out) {
    if (!t || !layers_out) return tfail(t, MPPI_E_INVALID, "NULL argument");
    std::vector<float> h(kNumParams);
    TRY(t, cudaStreamSynchronize(t->stream));
    TRY(t, cudaMemcpy(h.data(), t->theta, kNumParams * sizeof(float), cudaMemcpyDeviceToHost));
    for (int i = 0; i < 10; ++i) {
        if (!layers_out[i]) return tfail(t, MPPI_E_INVALID, "output pointer %d is NULL", i);
        std::memcpy(layers_out[i], h.data() + kLayerOffsets[i], kLayerSizes[i] * sizeof(float));
    }
    return MPPI_OK;
}

int mppi_train_evaluate(mppi_trainer* t, float* mae, float* p99, float* max_err, float* near_p99) {
    if (!t) return tfail(nullptr, MPPI_E_INVALID, "NULL trainer");
    const int n = t->cfg.n_holdout;
    // the held-out set goes through the FP32 forward pass in batch-sized chunks (whatever the
    // training GEMMs' precision, the error is the learned weights' own)
    for (int p0 = 0; p0 < n; p0 += t->cfg.batch) {
        const int len = std::min(t->cfg.batch, n - p0);
        bind_batch(t, t->holdout + p0, len);
        int rc = forward(t, false);
        if (rc != MPPI_OK) return rc;
        eval_output_kernel<<<(len + 7) / 8, 256, 0, t->stream>>>(t->T, t->errs + p0);
        TRY(t, cudaGetLastError());
    }
    std::vector<float> e(n);
    std::vector<float4> p(n);
    TRY(t, cudaMemcpyAsync(e.data(), t->errs, n * sizeof(float), cudaMemcpyDeviceToHost, t->stream));
    TRY(t, cudaMemcpyAsync(p.data(), t->holdout, n * sizeof(float4), cudaMemcpyDeviceToHost, t->stream));
    TRY(t, cudaStreamSynchronize(t->stream));
    double sum = 0.0;
    std::vector<float> near;
    for (int i = 0; i < n; ++i) {
        sum += e[i];
        if (std::fabs(p[i].w) < 0.3f) near.push_back(e[i]);
    }
    std::vector<float> all = e;
    const size_t k99 = static_cast<size_t>(0.99 * (all.size() - 1));
    std::nth_element(all.begin(), all.begin() + static_cast<long>(k99), all.end());
    if (mae) *mae = static_cast<float>(sum / n);
    if (p99) *p99 = all[k99];
    if (max_err) *max_err = *std::max_element(e.begin(), e.end());
    if (near_p99) {
        if (near.empty()) {
            *near_p99 = 0.f;
        } else {
            const size_t kn = static_cast<size_t>(0.99 * (near.size() - 1));
            std::nth_element(near.begin(), near.begin() + static_cast<long>(kn), near.end());
            *near_p99 = near[kn];
        }
    }
    return MPPI_OK;
}

int mppi_train_read_points(mppi_trainer* t, int which, float* out, size_t n_floats) {
    if (!t || !out) return tfail(t, MPPI_E_INVALID, "NULL argument");
    const size_t n = which == 0 ? t->cfg.n_points : t->cfg.n_holdout;
    if (n_floats < 4 * n) return tfail(t, MPPI_E_INVALID, "needs %zu floats", 4 * n);
    TRY(t, cudaMemcpy(out, which == 0 ? t->data : t->holdout, n * sizeof(float4), cudaMemcpyDeviceToHost));
    return MPPI_OK;
}

int mppi_train_num_params(void) { return kNumParams; }

}  // extern "C"
