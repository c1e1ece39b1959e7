// Step kernels around the SDF query: (a) noise, (b) rollouts, (d) cost ->
// weights -> update, receding-horizon plant step, per-gate first-layer bias.
#include "kernels.h"

namespace mppi {

namespace {

// ------------------------------------------------------------------ (a) noise
// One Philox4x32-10 block per (h, k) -> four normals -> delta u (Sec. IV-A, Eq. 5).
// Layout [h][k] so the rollout kernel's per-h reads are coalesced across k.
__global__ void __launch_bounds__(256) noise_kernel(StepParams P, const uint32_t* __restrict__ step,
                                                    float4* __restrict__ noise) {
    pdl_trigger();
    const int n = P.K * P.H;
    const uint32_t st = __ldg(step);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int h = i / P.K;
        const int k = i - h * P.K;
        noise[i] = noise_from_block(P, noise_block(P, k, h, st));
    }
}

__global__ void noise_words_kernel(StepParams P, const uint32_t* __restrict__ step, uint4* __restrict__ out) {
    const int n = P.K * P.H;
    const uint32_t st = __ldg(step);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int h = i / P.K;
        const int k = i - h * P.K;
        out[i] = noise_block(P, k, h, st);
    }
}

// ------------------------------------------------------------------ (b) rollouts
// One rollout per thread, state in registers, serial over the horizon.  Each
// step clips U*_h + delta, accumulates the control cost, integrates RK4 and
// stores the position as one float4 (coalesced across k).  In analytic mode
// the frame SDF of every gate and the collision hinge are evaluated here too.
constexpr int kPrefetch = 8;

__global__ void __launch_bounds__(64) rollout_kernel(StepParams P, StepBuffers B, int analytic) {
    extern __shared__ float4 sU[];                 // [H]
    __shared__ float sPose[kMaxGates * 8];
    pdl_trigger();
    pdl_wait();
    for (int i = threadIdx.x; i < P.H; i += blockDim.x) sU[i] = B.nominal[i];
    for (int i = threadIdx.x; i < P.G * 8; i += blockDim.x) sPose[i] = B.poses[i];
    __syncthreads();
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= P.K) return;

    const Vec3 p0 = v3(B.state[0], B.state[1], B.state[2]);
    Vec3 p = p0;
    Vec3 v = v3(B.state[3], B.state[4], B.state[5]);
    Quat q{B.state[6], B.state[7], B.state[8], B.state[9]};

    // target gate: the first gate whose plane the current position has not crossed
    int tgt = -1;
    Vec3 n_tgt = v3(0.f, 0.f, 0.f);
    for (int g = 0; g < P.G; ++g) {
        const float* ps = sPose + 8 * g;
        const Vec3 n = quat_x_axis(Quat{ps[3], ps[4], ps[5], ps[6]});
        const float side = n.x * (p0.x - ps[0]) + n.y * (p0.y - ps[1]) + n.z * (p0.z - ps[2]);
        if (tgt < 0 && side < 0.f) { tgt = g; n_tgt = n; }
        if (tgt < 0 && g == P.G - 1) { tgt = g; n_tgt = n; }
    }

    const float uh = P.mass * P.gravity;
    float jctl = 0.f, jcol = 0.f;
    const int K = P.K, H = P.H;
    // The noise of the next kPrefetch steps is loaded while the current ones are
    // integrated, so the load latency is not on the serial RK4 chain.
    float4 cur[kPrefetch], nxt[kPrefetch];
#pragma unroll
    for (int j = 0; j < kPrefetch; ++j) cur[j] = (j < H) ? __ldcs(B.noise + j * K + k) : make_float4(0.f, 0.f, 0.f, 0.f);
    for (int h0 = 0; h0 < H; h0 += kPrefetch) {
#pragma unroll
        for (int j = 0; j < kPrefetch; ++j) {
            const int hn = h0 + kPrefetch + j;
            nxt[j] = (hn < H) ? __ldcs(B.noise + hn * K + k) : make_float4(0.f, 0.f, 0.f, 0.f);
        }
#pragma unroll
        for (int j = 0; j < kPrefetch; ++j) {
            const int h = h0 + j;
            if (h < H) {
                const float4 d = cur[j];
                const float4 un = sU[h];
                const float4 u = clip_control(P, make_float4(un.x + d.x, un.y + d.y, un.z + d.z, un.w + d.w));
                const float e0 = u.x - uh;
                jctl += e0 * e0 + u.y * u.y + u.z * u.z + u.w * u.w;
                rk4_step(P, p, v, q, u.x, v3(u.y, u.z, u.w));
                B.pos[h * K + k] = make_float4(p.x, p.y, p.z, 0.f);
                if (analytic) {
                    float smin = __int_as_float(0x7f800000);
                    for (int g = 0; g < P.G; ++g) {
                        const Vec3 pg = to_gate(sPose + 8 * g, p);
                        smin = fminf(smin, frame_sdf(pg.x, pg.y, pg.z, P.a_in, P.a_out, P.half_depth));
                    }
                    jcol += hinge_sq(smin, P.d_safe);
                }
            }
        }
#pragma unroll
        for (int j = 0; j < kPrefetch; ++j) cur[j] = nxt[j];
    }
    const float jprog = (tgt >= 0) ? -(n_tgt.x * (p.x - p0.x) + n_tgt.y * (p.y - p0.y) + n_tgt.z * (p.z - p0.z))
                                   : 0.f;
    B.parts[k] = analytic ? P.w_col * jcol : 0.f;
    B.parts[K + k] = jprog;
    B.parts[2 * K + k] = P.w_u * jctl;
}

// ------------------------------------------------------------------ (d1) costs
// J_k = J_col + J_prog + J_ctl (MLP modes: J_col = w_col sum_h max(0, d_safe - s_h)^2
// over the stored SDF values, in order of h).  Each block also leaves the
// partial (m_b, s_b) = (min_{k in b} J_k, sum_{k in b} exp(-(J_k - m_b) / lambda)),
// from which rho = min J and eta = sum exp(-(J - rho) / lambda) of Eq. 5 follow
// without another pass (online softmax).  Fixed reduction order: reruns are
// bit-identical.
constexpr int kCostThreads = 128;

__device__ __forceinline__ float warp_min(float x) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x = fminf(x, __shfl_xor_sync(0xffffffffu, x, o));
    return x;
}
__device__ __forceinline__ float warp_sum(float x) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    return x;
}

__global__ void __launch_bounds__(kCostThreads) cost_kernel(StepParams P, StepBuffers B, int mlp) {
    __shared__ float sh[kCostThreads / 32];
    const int K = P.K;
    const int k = blockIdx.x * kCostThreads + threadIdx.x;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    pdl_trigger();
    pdl_wait();
    float J = __int_as_float(0x7f800000);
    if (k < K) {
        float jcol;
        if (mlp) {
            float acc = 0.f;
#pragma unroll 10
            for (int h = 0; h < P.H; ++h) acc += hinge_sq(__ldcs(B.sdf + h * K + k), P.d_safe);
            jcol = P.w_col * acc;
            B.parts[k] = jcol;
        } else {
            jcol = B.parts[k];
        }
        J = jcol + B.parts[K + k] + B.parts[2 * K + k];
        B.J[k] = J;
    }
    float m = warp_min(J);
    if (lane == 0) sh[wid] = m;
    __syncthreads();
    m = sh[0];
#pragma unroll
    for (int i = 1; i < kCostThreads / 32; ++i) m = fminf(m, sh[i]);
    __syncthreads();
    const float e = (k < K) ? expf(-(J - m) / P.lam) : 0.f;
    float s = warp_sum(e);
    if (lane == 0) sh[wid] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        float t = sh[0];
#pragma unroll
        for (int i = 1; i < kCostThreads / 32; ++i) t += sh[i];
        B.red[2 * blockIdx.x] = m;
        B.red[2 * blockIdx.x + 1] = t;
    }
}

// ------------------------------------------------------------------ (d2) weights, update, receding horizon
// Every block first combines the cost blocks' partials into rho and eta (same
// fixed order in every block), then block h forms w_k = exp(-(J_k - rho) / lambda) / eta
// and U*_new[h] = sum_k w_k clip(U*_h + delta_{k,h}) (Eq. 5) with a fixed-order
// tree; block 0 also stores w.  The last block to finish applies U*_new[0] to
// the device-resident state with one RK4 step, writes the shifted warm start
// and bumps the step counter.
constexpr int kUpdThreads = 512;

__global__ void __launch_bounds__(kUpdThreads) update_plant_kernel(StepParams P, StepBuffers B) {
    __shared__ float4 sh[kUpdThreads / 32];
    __shared__ float s_rho, s_eta;
    __shared__ int is_last;
    pdl_wait();
    const int h = blockIdx.x;
    const int K = P.K;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int nb = (K + kCostThreads - 1) / kCostThreads;
    if (wid == 0) {
        float m = __int_as_float(0x7f800000);
        for (int b = lane; b < nb; b += 32) m = fminf(m, B.red[2 * b]);
        const float rho = warp_min(m);
        float s = 0.f;
        for (int b = lane; b < nb; b += 32) s += B.red[2 * b + 1] * expf(-(B.red[2 * b] - rho) / P.lam);
        const float eta = warp_sum(s);
        if (lane == 0) {
            s_rho = rho;
            s_eta = eta;
        }
    }
    __syncthreads();
    const float rho = s_rho, eta = s_eta;
    const float4 un = B.nominal[h];
    float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll 4
    for (int k = threadIdx.x; k < K; k += kUpdThreads) {
        const float w = expf(-(B.J[k] - rho) / P.lam) / eta;
        if (h == 0) B.w[k] = w;
        const float4 d = __ldcs(B.noise + h * K + k);
        const float4 u = clip_control(P, make_float4(un.x + d.x, un.y + d.y, un.z + d.z, un.w + d.w));
        acc.x = fmaf(w, u.x, acc.x);
        acc.y = fmaf(w, u.y, acc.y);
        acc.z = fmaf(w, u.z, acc.z);
        acc.w = fmaf(w, u.w, acc.w);
    }
    acc.x = warp_sum(acc.x);
    acc.y = warp_sum(acc.y);
    acc.z = warp_sum(acc.z);
    acc.w = warp_sum(acc.w);
    if (lane == 0) sh[wid] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        float4 t = sh[0];
        for (int i = 1; i < kUpdThreads / 32; ++i) {
            t.x += sh[i].x; t.y += sh[i].y; t.z += sh[i].z; t.w += sh[i].w;
        }
        B.unew[h] = t;
        if (h == 0) {
            B.stats[0] = rho;
            B.stats[1] = eta;
        }
        __threadfence();
        const unsigned tk = atomicAdd(&B.tickets[1], 1u);
        is_last = (tk == gridDim.x - 1);
    }
    __syncthreads();
    if (!is_last) return;
    __threadfence();

    const float uh = P.mass * P.gravity;
    for (int i = threadIdx.x; i < P.H; i += kUpdThreads) {
        B.nominal[i] = (i + 1 < P.H) ? __ldcg(&B.unew[i + 1]) : make_float4(uh, 0.f, 0.f, 0.f);
    }
    if (threadIdx.x == 0) {
        const float4 u0 = __ldcg(&B.unew[0]);
        float* s = B.state;
        Vec3 p = v3(s[0], s[1], s[2]);
        Vec3 v = v3(s[3], s[4], s[5]);
        Quat q{s[6], s[7], s[8], s[9]};
        rk4_step(P, p, v, q, u0.x, v3(u0.y, u0.z, u0.w));
        s[0] = p.x; s[1] = p.y; s[2] = p.z;
        s[3] = v.x; s[4] = v.y; s[5] = v.z;
        s[6] = q.w; s[7] = q.x; s[8] = q.y; s[9] = q.z;
        s[10] = u0.y; s[11] = u0.z; s[12] = u0.w;
        const uint32_t lo = B.step[0] + 1u;
        B.step[0] = lo;
        if (lo == 0u) B.step[1] += 1u;
        B.tickets[1] = 0u;
    }
}

// ------------------------------------------------------------------ per-gate first-layer bias
// The Gate-SDF decoder's first layer sees [p, z]; z is fixed per gate, so its
// part W1[:, 3:] z + b1 is computed once per gate instead of once per query.
__global__ void first_layer_bias_kernel(const float* __restrict__ W1, const float* __restrict__ b1,
                                        const float* __restrict__ lat, int G, float* __restrict__ b1p) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= G * kHidden) return;
    const int g = i / kHidden, c = i - g * kHidden;
    const float* wr = W1 + c * (3 + kLatent) + 3;
    const float* z = lat + g * kLatent;
    float acc = 0.f;
    for (int j = 0; j < kLatent; ++j) acc = fmaf(wr[j], z[j], acc);
    b1p[i] = b1[c] + acc;
}

}  // namespace

cudaError_t launch_noise(const StepParams& P, const StepBuffers& B, cudaStream_t s) {
    const int n = P.K * P.H;
    const int blocks = (n + 255) / 256;
    noise_kernel<<<blocks, 256, 0, s>>>(P, B.step, B.noise);
    return cudaGetLastError();
}

cudaError_t launch_noise_words(const StepParams& P, const StepBuffers& B, uint4* out, cudaStream_t s) {
    const int n = P.K * P.H;
    noise_words_kernel<<<(n + 255) / 256, 256, 0, s>>>(P, B.step, out);
    return cudaGetLastError();
}

cudaError_t launch_rollout(const StepParams& P, const StepBuffers& B, int analytic, cudaStream_t s) {
    const int threads = 64;
    return launch_dependent(P.pdl != 0, rollout_kernel, dim3((P.K + threads - 1) / threads), dim3(threads),
                            P.H * sizeof(float4), s, P, B, analytic);
}

cudaError_t launch_cost_weights(const StepParams& P, const StepBuffers& B, int mlp, cudaStream_t s) {
    return launch_dependent(P.pdl != 0, cost_kernel, dim3((P.K + kCostThreads - 1) / kCostThreads), dim3(kCostThreads), 0, s,
                            P, B, mlp);
}

cudaError_t launch_update_plant(const StepParams& P, const StepBuffers& B, cudaStream_t s) {
    return launch_dependent(P.pdl != 0, update_plant_kernel, dim3(P.H), dim3(kUpdThreads), 0, s, P, B);
}

cudaError_t launch_first_layer_bias(const float* W1, const float* b1, const float* latents, int G, float* b1p,
                                    cudaStream_t s) {
    if (G <= 0) return cudaSuccess;
    const int n = G * kHidden;
    first_layer_bias_kernel<<<(n + 127) / 128, 128, 0, s>>>(W1, b1, latents, G, b1p);
    return cudaGetLastError();
}

}  // namespace mppi
