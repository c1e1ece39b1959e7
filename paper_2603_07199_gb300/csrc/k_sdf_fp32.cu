// (c) Gate-SDF MLP at every rollout state, FP32 on the CUDA cores: the plain
// FP32 path.  One CTA takes a tile of 128 rollouts at one horizon step, runs
// the whole MLP for every gate with register-blocked FP32 GEMMs through
// shared memory, keeps the minimum over gates and folds the stage hinge of
// that minimum s(p) into per-rollout partial sums of the collision cost (s(p)
// itself is stored only for diagnostics).
#include "kernels.h"

namespace mppi {

namespace {

constexpr int kThreads = 256;
constexpr int kLdA = kTileRows + 4;     // activations stored feature-major: act[feature][row]
constexpr int kMaxPoint = 3 + 6 * 6;    // point features with the most positional-encoding levels

// sp(x) = max(x, 0) + log1p(exp(-beta |x|)) / beta, accurate FP32 library calls
__device__ __forceinline__ float softplus_acc(float x, float beta, float inv_beta) {
    return fmaxf(x, 0.f) + log1pf(expf(-beta * fabsf(x))) * inv_beta;
}

// rows / columns of the 8 x 8 register tile of thread (tr, tn): two 4-wide
// strips 64 apart, so 16 threads read 256 contiguous bytes per shared load
__device__ __forceinline__ int strip(int t, int i) { return (i < 4) ? t * 4 + i : 64 + t * 4 + (i - 4); }

template <bool kPE>
__global__ void __launch_bounds__(kThreads, 1) sdf_mlp_fp32_kernel(StepParams P, StepBuffers B, MlpWeights W) {
    extern __shared__ __align__(16) float smem[];
    float* act = smem;                              // [128][kLdA]
    float* wt = act + kHidden * kLdA;               // [128 in][128 out]
    float* sW1 = wt + kHidden * kHidden;            // [NP][128]  W1[:, 0:NP] transposed (NP point features)
    float* sB1 = sW1 + kMaxPoint * kHidden;         // [G][128]   per-gate first-layer bias
    float* sBias = sB1 + kMaxGates * kHidden;       // [3][128]   b2, b3, b4
    float* sW5 = sBias + 3 * kHidden;               // [128]
    float* sPg = sW5 + kHidden;                     // [NP][128]  point features of the tile's rows
    float* sMin = sPg + kMaxPoint * kTileRows;      // [128]      min over gates
    float* sPose = sMin + kTileRows;                // [G][8]

    const int tid = threadIdx.x;
    const int G = P.G;
    const int NP = kPE ? 3 + 6 * P.pe : 3;          // point features: p and its positional encoding
    for (int i = tid; i < NP * kHidden; i += kThreads) {
        const int j = i / kHidden, n = i - j * kHidden;
        sW1[i] = W.W1[n * (NP + kLatent) + j];
    }
    for (int i = tid; i < 3 * kHidden; i += kThreads) {
        const int j = i / kHidden, n = i - j * kHidden;
        sBias[i] = W.b[j][n];
    }
    for (int i = tid; i < G * kHidden; i += kThreads) sB1[i] = B.b1p[i];
    for (int i = tid; i < kHidden; i += kThreads) sW5[i] = W.w5[i];
    for (int i = tid; i < G * 8; i += kThreads) sPose[i] = B.poses[i];
    __syncthreads();
    pdl_trigger();
    pdl_wait();

    const float beta = P.beta, inv_beta = 1.0f / P.beta;
    const int tn = tid & 15, tr = tid >> 4;
    // gates queried: all (min over gates), or the target gate only (the paper's form)
    int g_lo = 0, g_hi = G;
    if (P.paper) {
        Vec3 n;
        const int t = target_gate(sPose, G, v3(B.state[0], B.state[1], B.state[2]), &n);
        g_lo = t < 0 ? 0 : t;
        g_hi = t < 0 ? 0 : t + 1;
    }
    // tile = 128 consecutive rollout states of the [K][H] position array
    const int n_rows = P.K * P.H;
    const int n_items = (n_rows + kTileRows - 1) / kTileRows;

    for (int item = blockIdx.x; item < n_items; item += gridDim.x) {
        if (tid < kTileRows) sMin[tid] = __int_as_float(0x7f800000);
        for (int g = g_lo; g < g_hi; ++g) {
            if (tid < kTileRows) {
                const float4 p = B.pos[min(item * kTileRows + tid, n_rows - 1)];
                const Vec3 pg = to_gate(sPose + 8 * g, v3(p.x, p.y, p.z));
                sPg[tid] = pg.x;
                sPg[kTileRows + tid] = pg.y;
                sPg[2 * kTileRows + tid] = pg.z;
                // positional encoding (Sec. III-B): sin, cos of 2^l pi p per level
                for (int l = 0; l < (kPE ? P.pe : 0); ++l) {
                    const float sc = static_cast<float>(1 << l);
                    float s0, c0, s1, c1, s2, c2;
                    sincospif(sc * pg.x, &s0, &c0);
                    sincospif(sc * pg.y, &s1, &c1);
                    sincospif(sc * pg.z, &s2, &c2);
                    float* f = sPg + (3 + 6 * l) * kTileRows + tid;
                    f[0] = s0; f[kTileRows] = s1; f[2 * kTileRows] = s2;
                    f[3 * kTileRows] = c0; f[4 * kTileRows] = c1; f[5 * kTileRows] = c2;
                }
            }
            __syncthreads();
            // layer 1: [p, z] -> 128, with the latent part folded into the per-gate bias
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const int r = strip(tr, i);
                const float x0 = sPg[r], x1 = sPg[kTileRows + r], x2 = sPg[2 * kTileRows + r];
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    const int n = strip(tn, j);
                    float a = sB1[g * kHidden + n] + sW1[n] * x0 + sW1[kHidden + n] * x1 + sW1[2 * kHidden + n] * x2;
                    if (kPE)
                        for (int f = 3; f < NP; ++f) a += sW1[f * kHidden + n] * sPg[f * kTileRows + r];
                    act[n * kLdA + r] = softplus_acc(a, beta, inv_beta);
                }
            }
            // layers 2..4: 128 x 128 GEMMs; the last one is followed by the output dot
            for (int l = 0; l < 3; ++l) {
                const float4* src = reinterpret_cast<const float4*>(W.Wt[l]);
                float4* dst = reinterpret_cast<float4*>(wt);
                __syncthreads();
                for (int i = tid; i < kHidden * kHidden / 4; i += kThreads) dst[i] = __ldg(src + i);
                __syncthreads();
                float acc[8][8];
#pragma unroll
                for (int i = 0; i < 8; ++i)
#pragma unroll
                    for (int j = 0; j < 8; ++j) acc[i][j] = 0.f;
#pragma unroll 4
                for (int kk = 0; kk < kHidden; ++kk) {
                    const float4 a0 = *reinterpret_cast<const float4*>(act + kk * kLdA + tr * 4);
                    const float4 a1 = *reinterpret_cast<const float4*>(act + kk * kLdA + 64 + tr * 4);
                    const float4 b0 = *reinterpret_cast<const float4*>(wt + kk * kHidden + tn * 4);
                    const float4 b1 = *reinterpret_cast<const float4*>(wt + kk * kHidden + 64 + tn * 4);
                    const float av[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
                    const float bv[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
                    for (int i = 0; i < 8; ++i)
#pragma unroll
                        for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
                }
                __syncthreads();
                if (l < 2) {
#pragma unroll
                    for (int j = 0; j < 8; ++j) {
                        const int n = strip(tn, j);
                        const float bn = sBias[l * kHidden + n];
                        float4 lo, hi;
                        lo.x = softplus_acc(acc[0][j] + bn, beta, inv_beta);
                        lo.y = softplus_acc(acc[1][j] + bn, beta, inv_beta);
                        lo.z = softplus_acc(acc[2][j] + bn, beta, inv_beta);
                        lo.w = softplus_acc(acc[3][j] + bn, beta, inv_beta);
                        hi.x = softplus_acc(acc[4][j] + bn, beta, inv_beta);
                        hi.y = softplus_acc(acc[5][j] + bn, beta, inv_beta);
                        hi.z = softplus_acc(acc[6][j] + bn, beta, inv_beta);
                        hi.w = softplus_acc(acc[7][j] + bn, beta, inv_beta);
                        *reinterpret_cast<float4*>(act + n * kLdA + tr * 4) = lo;
                        *reinterpret_cast<float4*>(act + n * kLdA + 64 + tr * 4) = hi;
                    }
                } else {
                    // s_r = w5 . sp(h4_r + b4) + b5, reduced over the 16 column threads
#pragma unroll
                    for (int i = 0; i < 8; ++i) {
                        float part = 0.f;
#pragma unroll
                        for (int j = 0; j < 8; ++j) {
                            const int n = strip(tn, j);
                            part = fmaf(sW5[n], softplus_acc(acc[i][j] + sBias[2 * kHidden + n], beta, inv_beta),
                                        part);
                        }
                        part += __shfl_xor_sync(0xffffffffu, part, 1);
                        part += __shfl_xor_sync(0xffffffffu, part, 2);
                        part += __shfl_xor_sync(0xffffffffu, part, 4);
                        part += __shfl_xor_sync(0xffffffffu, part, 8);
                        if (tn == 0) {
                            const int r = strip(tr, i);
                            sMin[r] = fminf(sMin[r], part + W.b5);
                        }
                    }
                }
            }
        }
        __syncthreads();
        // collision-cost fold (Eq. 8-10): stage hinge of every row, summed per rollout over the tile
        const int row0 = item * kTileRows;
        if (tid < kTileRows) {
            const int r = row0 + tid;
            if (P.store_sdf && r < n_rows) B.sdf[r] = sMin[tid];
            fold_warp(r < n_rows ? stage_hinge(sMin[tid], P.d_safe, P.paper) : 0.f, r, n_rows, P.H, tid & 31, B.colp);
        }
        __syncthreads();
    }
}

constexpr size_t kSmemBytes = sizeof(float) * (kHidden * kLdA + kHidden * kHidden + kMaxPoint * kHidden +
                                                kMaxGates * kHidden + 3 * kHidden + kHidden + kMaxPoint * kTileRows +
                                                kTileRows + kMaxGates * 8);

}  // namespace

cudaError_t configure_sdf_mlp_fp32() {
    cudaError_t e = cudaFuncSetAttribute(sdf_mlp_fp32_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(kSmemBytes));
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(sdf_mlp_fp32_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 static_cast<int>(kSmemBytes));
    return e;
}

cudaError_t launch_sdf_mlp_fp32(const StepParams& P, const StepBuffers& B, const MlpWeights& W, int num_sms,
                                cudaStream_t s) {
    const int n_items = (P.K * P.H + kTileRows - 1) / kTileRows;
    const int grid = n_items < num_sms ? n_items : num_sms;
    if (P.pe > 0)
        return launch_dependent(P.pdl != 0, sdf_mlp_fp32_kernel<true>, dim3(grid), dim3(kThreads), kSmemBytes, s, P, B,
                                W);
    return launch_dependent(P.pdl != 0, sdf_mlp_fp32_kernel<false>, dim3(grid), dim3(kThreads), kSmemBytes, s, P, B, W);
}

}  // namespace mppi
