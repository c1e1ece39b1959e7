// (c) Gate-SDF MLP at every rollout state on the Blackwell tensor cores.
//
// Work item = one tile of 128 rollouts at one horizon step; for every gate the
// tile runs the chain
//   layer 1 (3 inputs + per-gate bias, FMA)  -> softplus -> BF16 A tile (smem)
//   3 x [tcgen05.mma 128x128x128 BF16 -> FP32 in TMEM] -> TMEM load -> bias,
//        softplus -> BF16 A tile (layers 2, 3) or the FP32 output dot (layer 4)
// and keeps the running minimum over gates in a register; the item ends by
// storing that minimum s(p) for the 128 states of the tile.
//
// CTA = 3 epilogue warpgroups (one tile chain each, own A tile and own
// 128-column TMEM accumulator) + 1 MMA warp whose lane 0 issues the MMAs of
// whichever warpgroup has its A tile ready.  W2..W4 (BF16, 96 KB) stay in
// shared memory for the life of the persistent CTA.  Every wait is bounded.
//
// Activations are carried in log2 units: with c = beta log2(e) and y = c x,
//   sp_beta(x) = (ln 2 / beta) h(y),   h(y) = log2(1 + 2^y) = max(y, 0) + log2(1 + 2^-|y|),
// and c (ln 2 / beta) = 1, so the hidden weights are used unchanged while the
// first layer and the hidden biases are scaled by c and the output weights by
// ln 2 / beta.  h is evaluated with one hardware exp2 and a quartic in
// e = 2^-|y| (see log2_1p_poly), in packed f32x2 arithmetic.
#include "kernels.h"
#include "tc.cuh"

namespace mppi {

namespace {

constexpr int kEpiWarpgroups = 3;
constexpr int kThreads = kEpiWarpgroups * 128 + 32;
constexpr int kMmaWarp = kEpiWarpgroups * 4;
constexpr uint32_t kTileBytes = kHidden * kHidden * 2;     // one 128 x 128 BF16 operand
constexpr uint32_t kTmemCols = 512;
constexpr uint32_t kIdesc = tc::idesc_bf16_f32(128, 128);

struct __align__(16) TcShared {
    uint8_t w[3][kTileBytes];                 // W2, W3, W4 (B operands, N = out, K = in)
    uint8_t a[kEpiWarpgroups][kTileBytes];    // activation tiles (A operands, M = rows, K = features)
    float w1[3][kHidden];                     // W1[:, 0:3] transposed
    float b1[kMaxGates][kHidden];             // per-gate first-layer bias
    float bias[3][kHidden];                   // b2, b3, b4
    float w5[kHidden];
    float pose[kMaxGates][8];
    uint64_t act_full[kEpiWarpgroups];        // epilogue -> MMA: A tile written
    uint64_t acc_full[kEpiWarpgroups];        // MMA -> epilogue: accumulator ready
    uint32_t tmem_base;
    int abort_flag;
};

// ---------------------------------------------------------------- packed f32x2 helpers
__device__ __forceinline__ uint64_t pk(float lo, float hi) {
    uint64_t r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ float2 upk(uint64_t v) {
    float2 r;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(r.x), "=f"(r.y) : "l"(v));
    return r;
}
__device__ __forceinline__ uint64_t fma2(uint64_t a, uint64_t b, uint64_t c) {
    uint64_t r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
    return r;
}
__device__ __forceinline__ uint64_t add2(uint64_t a, uint64_t b) {
    uint64_t r;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ uint64_t mul2(uint64_t a, uint64_t b) {
    uint64_t r;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}

// log2(1 + e) for e in [0, 1] as e (c1 + e (c2 + e (c3 + e c4))) with c1 = 1 / ln 2
// exact and c2..c4 a weighted least-squares (near-minimax) fit made for this
// kernel: max abs error 2.1e-4, relative error 1.4e-4 as e -> 0 (below the
// BF16 rounding of the activations it feeds).
constexpr float kL1 = 1.4426950408889634f;
constexpr float kL2 = -0.69991479f;
constexpr float kL3 = 0.35777588f;
constexpr float kL4 = -0.10076641f;

// Two activations at once: h(y) = max(y, 0) + log2(1 + 2^-|y|) for y = acc + bias.
__device__ __forceinline__ uint32_t softplus2_log2_bf16(float a0, float a1, uint64_t bias2) {
    const float2 y = upk(add2(pk(a0, a1), bias2));
    const uint64_t e = pk(tc::ex2_approx(-fabsf(y.x)), tc::ex2_approx(-fabsf(y.y)));
    uint64_t p = fma2(e, pk(kL4, kL4), pk(kL3, kL3));
    p = fma2(e, p, pk(kL2, kL2));
    p = fma2(e, p, pk(kL1, kL1));
    const uint64_t g = mul2(e, p);
    const float2 h = upk(add2(pk(fmaxf(y.x, 0.f), fmaxf(y.y, 0.f)), g));
    return tc::pack_bf16x2(h.x, h.y);
}
__device__ __forceinline__ float softplus_log2(float y) {
    const float e = tc::ex2_approx(-fabsf(y));
    return fmaxf(y, 0.f) + e * fmaf(e, fmaf(e, fmaf(e, kL4, kL3), kL2), kL1);
}

__device__ __forceinline__ int items_of_slot(int slot, int nslots, int n_items) {
    return slot < n_items ? (n_items - slot + nslots - 1) / nslots : 0;
}

__global__ void __launch_bounds__(kThreads, 1) sdf_mlp_bf16_kernel(StepParams P, StepBuffers B, MlpWeights W) {
    extern __shared__ uint8_t smem_raw[];
    TcShared& S = *reinterpret_cast<TcShared*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    const int tid = threadIdx.x;
    const int warp = tid >> 5, lane = tid & 31;
    const int K = P.K, G = P.G;

    // ---- set-up: TMEM, barriers, resident weights
    if (warp == kMmaWarp) {
        tc::tmem_alloc(tc::smem_u32(&S.tmem_base), kTmemCols);
        tc::tmem_relinquish();
    }
    if (tid == 0) {
        for (int i = 0; i < kEpiWarpgroups; ++i) {
            tc::mbar_init(tc::smem_u32(&S.act_full[i]), 1);
            tc::mbar_init(tc::smem_u32(&S.acc_full[i]), 1);
        }
        S.abort_flag = 0;
        tc::mbar_fence_init();
    }
    for (int l = 0; l < 3; ++l) {
        const uint4* src = reinterpret_cast<const uint4*>(W.Wbf[l]);
        uint4* dst = reinterpret_cast<uint4*>(S.w[l]);
        for (int i = tid; i < int(kTileBytes / 16); i += kThreads) dst[i] = __ldg(src + i);
    }
    const float cl2 = P.beta * 1.4426950408889634f;          // beta log2(e)
    for (int i = tid; i < 3 * kHidden; i += kThreads) {
        const int j = i / kHidden, n = i - j * kHidden;
        S.w1[j][n] = cl2 * W.W1[n * (3 + kLatent) + j];
        S.bias[j][n] = cl2 * W.b[j][n];
    }
    for (int i = tid; i < G * kHidden; i += kThreads) S.b1[i / kHidden][i % kHidden] = cl2 * B.b1p[i];
    for (int i = tid; i < kHidden; i += kThreads) S.w5[i] = (0.69314718055994531f / P.beta) * W.w5[i];
    for (int i = tid; i < G * 8; i += kThreads) S.pose[i / 8][i % 8] = B.poses[i];
    tc::fence_proxy_async_smem();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem_base = S.tmem_base;

    const int n_kb = (K + kTileRows - 1) / kTileRows;
    const int n_items = P.H * n_kb;
    const int nslots = gridDim.x * kEpiWarpgroups;
    volatile int* abort_flag = &S.abort_flag;

    if (warp == kMmaWarp) {
        // ---------------------------------------------------------- MMA issuer
        if (lane == 0) {
            int nreq[kEpiWarpgroups], issued[kEpiWarpgroups];
            uint32_t phase[kEpiWarpgroups];
            uint64_t adesc[kEpiWarpgroups], bdesc[3];
            for (int i = 0; i < kEpiWarpgroups; ++i) {
                nreq[i] = items_of_slot(blockIdx.x * kEpiWarpgroups + i, nslots, n_items) * G * 3;
                issued[i] = 0;
                phase[i] = 0;
                adesc[i] = tc::smem_desc(tc::smem_u32(S.a[i]), 128, 2048);
            }
            for (int l = 0; l < 3; ++l) bdesc[l] = tc::smem_desc(tc::smem_u32(S.w[l]), 128, 2048);
            uint64_t t0 = tc::global_timer();
            int spins = 0;
            while (true) {
                bool pending = false, progressed = false;
                for (int i = 0; i < kEpiWarpgroups; ++i) {
                    if (issued[i] >= nreq[i]) continue;
                    pending = true;
                    if (!tc::mbar_try_wait(tc::smem_u32(&S.act_full[i]), phase[i])) continue;
                    phase[i] ^= 1u;
                    tc::fence_after_sync();
                    const int l = issued[i] % 3;
                    const uint32_t d = tmem_base + static_cast<uint32_t>(i * kHidden);
#pragma unroll
                    for (int s = 0; s < kHidden / 16; ++s)   // K = 16 per instruction: 256 B along K
                        tc::mma_bf16(d, adesc[i] + static_cast<uint64_t>(s * 16), bdesc[l] + static_cast<uint64_t>(s * 16),
                                     kIdesc, s > 0 ? 1u : 0u);
                    tc::mma_commit(tc::smem_u32(&S.acc_full[i]));
                    ++issued[i];
                    progressed = true;
                }
                if (!pending) break;
                if (progressed) {
                    t0 = tc::global_timer();
                    spins = 0;
                } else if (++spins >= 64) {
                    spins = 0;
                    if (*abort_flag) break;
                    if (tc::global_timer() - t0 > tc::kWaitLimitNs) {
                        *abort_flag = 1;
                        atomicExch(B.err, kDevErrTimeout);
                        break;
                    }
                }
            }
            // on abort: let the MMAs already issued finish before TMEM is released
            for (int i = 0; i < kEpiWarpgroups; ++i) {
                if (issued[i] > 0) {
                    int dummy = 0;
                    tc::mbar_wait_bounded(tc::smem_u32(&S.acc_full[i]), static_cast<uint32_t>((issued[i] - 1) & 1),
                                          &dummy, B.err, kDevErrTimeout);
                }
            }
        }
        __syncwarp();
    } else {
        // ---------------------------------------------------------- epilogue warpgroups
        const int wg = warp >> 2;
        const int row = (warp & 3) * 32 + lane;                       // TMEM lane == tile row
        const uint32_t a_base = tc::smem_u32(S.a[wg]);
        const uint32_t t_row = tmem_base + (static_cast<uint32_t>((warp & 3) * 32) << 16) +
                               static_cast<uint32_t>(wg * kHidden);
        const uint32_t act_bar = tc::smem_u32(&S.act_full[wg]);
        const uint32_t acc_bar = tc::smem_u32(&S.acc_full[wg]);
        uint32_t acc_phase = 0;
        bool ok = true;

        for (int item = blockIdx.x * kEpiWarpgroups + wg; item < n_items && ok; item += nslots) {
            const int h = item / n_kb, kb = item - h * n_kb;
            const int k = kb * kTileRows + row;
            const float4 p = B.pos[h * K + min(k, K - 1)];
            float smin = __int_as_float(0x7f800000);
            for (int g = 0; g < G && ok; ++g) {
                // layer 1: a_c = b1'_g[c] + W1[c, 0:3] . p_g  -> softplus -> BF16 row of the A tile
                const Vec3 pg = to_gate(S.pose[g], v3(p.x, p.y, p.z));
                const uint64_t px = pk(pg.x, pg.x), py = pk(pg.y, pg.y), pz = pk(pg.z, pg.z);
#pragma unroll 2
                for (int c = 0; c < kHidden; c += 8) {
                    uint32_t o[4];
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        const int n = c + 2 * j;
                        uint64_t a = fma2(pk(S.w1[0][n], S.w1[0][n + 1]), px,
                                          pk(S.b1[g][n], S.b1[g][n + 1]));
                        a = fma2(pk(S.w1[1][n], S.w1[1][n + 1]), py, a);
                        a = fma2(pk(S.w1[2][n], S.w1[2][n + 1]), pz, a);
                        const float2 af = upk(a);
                        o[j] = softplus2_log2_bf16(af.x, af.y, pk(0.f, 0.f));
                    }
                    tc::st_shared_v4(a_base + tc::operand_offset_bytes(row, c), o[0], o[1], o[2], o[3]);
                }
                tc::fence_proxy_async_smem();
                tc::named_barrier(1 + wg, 128);
                if ((warp & 3) == 0 && lane == 0) tc::mbar_arrive(act_bar);

                float s = W.b5;
                for (int l = 0; l < 3; ++l) {
                    // every thread of the warpgroup agrees on the outcome before going on, so a
                    // timeout seen by one thread cannot strand the others at a named barrier
                    const bool got = tc::mbar_wait_bounded(acc_bar, acc_phase, abort_flag, B.err, kDevErrTimeout);
                    if (!tc::named_barrier_and(1 + wg, 128, got)) {
                        ok = false;
                        break;
                    }
                    acc_phase ^= 1u;
                    tc::fence_after_sync();
                    for (int ch = 0; ch < kHidden; ch += 32) {
                        uint32_t v[32];
                        tc::tmem_ld_32x32b_x32(t_row + static_cast<uint32_t>(ch), v);
                        tc::tmem_wait_ld();
                        if (l < 2) {
#pragma unroll
                            for (int j = 0; j < 32; j += 8) {
                                const float4 b0 = *reinterpret_cast<const float4*>(&S.bias[l][ch + j]);
                                const float4 b1 = *reinterpret_cast<const float4*>(&S.bias[l][ch + j + 4]);
                                tc::st_shared_v4(
                                    a_base + tc::operand_offset_bytes(row, ch + j),
                                    softplus2_log2_bf16(__uint_as_float(v[j]), __uint_as_float(v[j + 1]), pk(b0.x, b0.y)),
                                    softplus2_log2_bf16(__uint_as_float(v[j + 2]), __uint_as_float(v[j + 3]), pk(b0.z, b0.w)),
                                    softplus2_log2_bf16(__uint_as_float(v[j + 4]), __uint_as_float(v[j + 5]), pk(b1.x, b1.y)),
                                    softplus2_log2_bf16(__uint_as_float(v[j + 6]), __uint_as_float(v[j + 7]), pk(b1.z, b1.w)));
                            }
                        } else {
#pragma unroll
                            for (int j = 0; j < 32; ++j)
                                s = fmaf(S.w5[ch + j], softplus_log2(__uint_as_float(v[j]) + S.bias[2][ch + j]), s);
                        }
                    }
                    tc::fence_before_sync();
                    if (l < 2) {
                        tc::fence_proxy_async_smem();
                        tc::named_barrier(1 + wg, 128);
                        if ((warp & 3) == 0 && lane == 0) tc::mbar_arrive(act_bar);
                    } else {
                        // the accumulator is free again once every thread of the warpgroup has read it;
                        // the next request (next gate or item) is only posted after the next A tile is
                        // written and the warpgroup barrier has passed
                    }
                }
                smin = fminf(smin, s);
            }
            if (ok && k < K) B.sdf[h * K + k] = smin;
        }
    }

    tc::fence_before_sync();
    __syncthreads();
    if (warp == kMmaWarp) {
        tc::fence_after_sync();
        tc::tmem_dealloc(tmem_base, kTmemCols);
    }
}

// ---------------------------------------------------------------------------- self-test
// One 128 x 128 x 128 tile: A, B row-major BF16 in global -> operand layout in
// shared memory -> 8 tcgen05.mma -> TMEM -> D row-major FP32.
__global__ void __launch_bounds__(128, 1) tc_selftest_kernel(const uint16_t* __restrict__ A,
                                                             const uint16_t* __restrict__ Bm, float* __restrict__ D,
                                                             int* err) {
    extern __shared__ uint8_t st_raw[];
    uint8_t* sa = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(st_raw) + 1023) & ~uintptr_t(1023));
    uint8_t* sb = sa + kTileBytes;
    __shared__ uint64_t bar;
    __shared__ uint32_t tbase;
    __shared__ int abort_flag;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (warp == 0) {
        tc::tmem_alloc(tc::smem_u32(&tbase), 128);
        tc::tmem_relinquish();
    }
    if (tid == 0) {
        tc::mbar_init(tc::smem_u32(&bar), 1);
        abort_flag = 0;
        tc::mbar_fence_init();
    }
    // thread r copies row r of A and of B (16 chunks of 8 BF16 each)
    for (int c = 0; c < kHidden; c += 8) {
        const uint4 va = *reinterpret_cast<const uint4*>(A + tid * kHidden + c);
        const uint4 vb = *reinterpret_cast<const uint4*>(Bm + tid * kHidden + c);
        tc::st_shared_v4(tc::smem_u32(sa) + tc::operand_offset_bytes(tid, c), va.x, va.y, va.z, va.w);
        tc::st_shared_v4(tc::smem_u32(sb) + tc::operand_offset_bytes(tid, c), vb.x, vb.y, vb.z, vb.w);
    }
    tc::fence_proxy_async_smem();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t t = tbase;
    if (tid == 0) {
        const uint64_t ad = tc::smem_desc(tc::smem_u32(sa), 128, 2048);
        const uint64_t bd = tc::smem_desc(tc::smem_u32(sb), 128, 2048);
        for (int s = 0; s < kHidden / 16; ++s)
            tc::mma_bf16(t, ad + static_cast<uint64_t>(s * 16), bd + static_cast<uint64_t>(s * 16), kIdesc,
                         s > 0 ? 1u : 0u);
        tc::mma_commit(tc::smem_u32(&bar));
    }
    __syncwarp();
    const bool ok = tc::mbar_wait_bounded(tc::smem_u32(&bar), 0, &abort_flag, err, kDevErrTimeout);
    tc::fence_after_sync();
    if (ok) {
        const int row = warp * 32 + lane;
        for (int ch = 0; ch < kHidden; ch += 32) {
            uint32_t v[32];
            tc::tmem_ld_32x32b_x32(t + (static_cast<uint32_t>(warp * 32) << 16) + static_cast<uint32_t>(ch), v);
            tc::tmem_wait_ld();
            for (int j = 0; j < 32; ++j) D[row * kHidden + ch + j] = __uint_as_float(v[j]);
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) {
        tc::fence_after_sync();
        tc::tmem_dealloc(t, 128);
    }
}

constexpr size_t kSmemBytes = sizeof(TcShared) + 1024;

}  // namespace

cudaError_t configure_sdf_mlp_bf16() {
    return cudaFuncSetAttribute(sdf_mlp_bf16_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                static_cast<int>(kSmemBytes));
}

cudaError_t launch_sdf_mlp_bf16(const StepParams& P, const StepBuffers& B, const MlpWeights& W, int num_sms,
                                cudaStream_t s) {
    const int n_items = P.H * ((P.K + kTileRows - 1) / kTileRows);
    const int want = (n_items + kEpiWarpgroups - 1) / kEpiWarpgroups;
    const int grid = want < num_sms ? want : num_sms;
    sdf_mlp_bf16_kernel<<<grid, kThreads, kSmemBytes, s>>>(P, B, W);
    return cudaGetLastError();
}

cudaError_t launch_tc_selftest(const uint16_t* A, const uint16_t* Bm, float* D, int* err, cudaStream_t s) {
    const int bytes = static_cast<int>(2 * kTileBytes + 1024);
    cudaError_t e = cudaFuncSetAttribute(tc_selftest_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e != cudaSuccess) return e;
    tc_selftest_kernel<<<1, 128, bytes, s>>>(A, Bm, D, err);
    return cudaGetLastError();
}

}  // namespace mppi
