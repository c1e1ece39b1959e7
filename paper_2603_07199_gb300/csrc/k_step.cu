// Step kernels around the SDF query: (a) + (b) noise and rollouts, (d) costs ->
// softmax weights -> update -> receding-horizon plant step, and the per-gate
// first-layer bias.
#include "kernels.h"

namespace mppi {

namespace {

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
// Shuffles within segments of W consecutive lanes (W = 32: the whole warp); src and the
// lane index of the scans count from the segment's first lane.
template <int W>
__device__ __forceinline__ Quat shfl_up(const Quat& q, int d) {
    return Quat{__shfl_up_sync(0xffffffffu, q.w, d, W), __shfl_up_sync(0xffffffffu, q.x, d, W),
                __shfl_up_sync(0xffffffffu, q.y, d, W), __shfl_up_sync(0xffffffffu, q.z, d, W)};
}
template <int W>
__device__ __forceinline__ Vec3 shfl_up(const Vec3& v, int d) {
    return v3(__shfl_up_sync(0xffffffffu, v.x, d, W), __shfl_up_sync(0xffffffffu, v.y, d, W),
              __shfl_up_sync(0xffffffffu, v.z, d, W));
}
template <int W>
__device__ __forceinline__ Quat shfl_idx(const Quat& q, int src) {
    return Quat{__shfl_sync(0xffffffffu, q.w, src, W), __shfl_sync(0xffffffffu, q.x, src, W),
                __shfl_sync(0xffffffffu, q.y, src, W), __shfl_sync(0xffffffffu, q.z, src, W)};
}
template <int W>
__device__ __forceinline__ Vec3 shfl_idx(const Vec3& v, int src) {
    return v3(__shfl_sync(0xffffffffu, v.x, src, W), __shfl_sync(0xffffffffu, v.y, src, W),
              __shfl_sync(0xffffffffu, v.z, src, W));
}
// Sum over a segment of W lanes (every lane of the segment gets it).
template <int W>
__device__ __forceinline__ float seg_sum(float x) {
#pragma unroll
    for (int o = W / 2; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    return x;
}
// Inclusive prefix sum over the lanes of a segment (Hillis-Steele).
template <int W>
__device__ __forceinline__ Vec3 seg_scan_add(Vec3 x, int sub) {
#pragma unroll
    for (int d = 1; d < W; d <<= 1) {
        const Vec3 t = shfl_up<W>(x, d);
        if (sub >= d) x = v3(t.x + x.x, t.y + x.y, t.z + x.z);
    }
    return x;
}
// Inclusive ordered product x_0 (x) x_1 (x) ... (x) x_sub over a segment: at every round the
// partial product of the earlier lanes multiplies from the left.
template <int W>
__device__ __forceinline__ Quat seg_scan_qmul(Quat x, int sub) {
#pragma unroll
    for (int d = 1; d < W; d <<= 1) {
        const Quat t = shfl_up<W>(x, d);
        if (sub >= d) x = qmul(t, x);
    }
    return x;
}

__global__ void noise_words_kernel(StepParams P, const uint32_t* __restrict__ step, uint4* __restrict__ out) {
    const int n = P.K * P.H;
    const uint32_t st = __ldg(step);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int k = i / P.H;
        const int h = i - k * P.H;
        out[i] = noise_block(P, k, h, st);
    }
}

// ------------------------------------------------------------------ (a) + (b) noise and rollouts
// One segment of kLanes lanes per rollout (32 / kLanes rollouts per warp); the horizon runs
// across the segment's lanes in chunks of kLanes x kSteps steps, lane l of the segment owning
// the kSteps consecutive steps h = c0 + kSteps l + j.  For each of its steps a lane draws the noise
// (Philox4x32-10 block (k, h, step, drone) -> four normals -> delta u,
// Sec. IV-A, Eq. 5), stores it, clips U*_h + delta and adds the control cost.
// With the body rate held over a step (dw/dt = 0) the RK4 attitude update is
// q_{h+1} = normalise(q_h (x) M_h), M_h = (a_n, b_n w_h) with a_n, b_n the
// polynomials in |w_h| dt of rk4_step, so q_{h+1} = q_h (x) N_h with the unit
// N_h = M_h / |M_h|: the attitude at the start of every lane's segment is an
// ordered prefix product of state-independent factors (a warp scan).  Each lane
// then walks its segment: stage accelerations of every step, the velocity
// offsets V_j = sum_{i<j} dv_i and position offsets L_j relative to the
// segment's start, with
//   v_{h+1} = v_h + dt/6 (a1 + 2 a2 + 2 a3 + a4),  p_{h+1} = p_h + dt v_h + dt^2/6 (a1 + a2 + a3),
// so p after j + 1 steps of the lane's steps = p_s + (j + 1) dt v_s + L_j.  Two more
// scans give every lane's v_s and p_s.  The serial chain of H dependent RK4 steps becomes
// log2(kLanes) shuffle rounds per chunk; with 16 lanes x 4 steps a warp serves two rollouts,
// so the scans' rounds are shared and fewer lanes idle at H = 50 than with one 32-lane
// rollout per warp (17 % fewer warp instructions at K = 4096, H = 50; the launch picks the
// form).  Stores: one float4 per step, contiguous across the rollout's lanes in the [K][H]
// arrays.  In analytic mode the frame SDF of every gate and the collision hinge are
// evaluated at every p_{h+1}.
constexpr int kRollWarps = 4;

// The body of one block (block = the block's index among this controller's rollout blocks;
// sU: H floats4 and sPose: kMaxGates x 8 floats of shared memory); the per-controller kernel
// and the batched serving kernel both run it.
template <int kLanes, int kSteps>
__device__ __forceinline__ void rollout_body(const StepParams& P, const StepBuffers& B, int analytic, int block,
                                             float4* sU, float* sPose) {
    static_assert(kLanes == 16 || kLanes == 32, "a rollout's lanes are a half warp or a warp");
    pdl_trigger();
    pdl_wait();
    for (int i = threadIdx.x; i < P.H; i += blockDim.x) sU[i] = B.nominal[i];
    for (int i = threadIdx.x; i < P.G * 8; i += blockDim.x) sPose[i] = B.poses[i];
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int sub = lane & (kLanes - 1);          // lane within the rollout's segment
    const int k_first = (block * kRollWarps + (threadIdx.x >> 5)) * (32 / kLanes);
    if (k_first >= P.K) return;                    // whole warps only
    // a segment past the last rollout (odd K) mirrors the last one and stores nothing
    const bool valid = k_first + lane / kLanes < P.K;
    const int k = valid ? k_first + lane / kLanes : P.K - 1;
    const int K = P.K, H = P.H;
    const uint32_t st = B.step[0];

    const Vec3 p0 = v3(B.state[0], B.state[1], B.state[2]);
    Vec3 pc = p0;                                  // p, v, q at the start of the chunk
    Vec3 vc = v3(B.state[3], B.state[4], B.state[5]);
    Quat qc{B.state[6], B.state[7], B.state[8], B.state[9]};

    // target gate: the first gate whose plane the current position has not crossed; its
    // centre is the waypoint of the paper's cost form
    Vec3 n_tgt;
    const int tgt = target_gate(sPose, P.G, p0, &n_tgt);
    const float* pose_t = sPose + 8 * (tgt < 0 ? 0 : tgt);
    const Vec3 wp = v3(pose_t[0], pose_t[1], pose_t[2]);

    const float uh = P.u_hover;
    const float dt = P.dt;
    const float c3 = dt * dt * (1.f / 6.f), c6 = dt * (1.f / 6.f);
    const float b2 = 0.25f * dt;
    const float inv_m = 1.f / P.mass;
    float jctl = 0.f, jcol = 0.f, jvis = 0.f;
    float4* noise_k = B.noise + static_cast<size_t>(k) * H;
    float4* pos_k = B.pos + static_cast<size_t>(k) * H;
    for (int c0 = 0; c0 < H; c0 += kLanes * kSteps) {
        const int h0 = c0 + kSteps * sub;
        // pass A: noise, clipped controls, control cost, the segment's attitude increment
        float4 u[kSteps];
        Quat N[kSteps];
        Quat seg{1.f, 0.f, 0.f, 0.f};
        int nact = 0;
#pragma unroll
        for (int j = 0; j < kSteps; ++j) {
            const int h = h0 + j;
            u[j] = make_float4(uh, 0.f, 0.f, 0.f);       // steps past H: no rotation, no increments
            if (h < H) {
                const float4 d = noise_from_block(P, noise_block(P, k, h, st));
                if (valid) noise_k[h] = d;
                const float4 un = sU[h];
                u[j] = clip_control(P, make_float4(un.x + d.x, un.y + d.y, un.z + d.z, un.w + d.w));
                const float e0 = u[j].x - uh;
                jctl += e0 * e0 + u[j].y * u[j].y + u[j].z * u[j].z + u[j].w * u[j].w;
                ++nact;
            }
            const float d2 = dt * dt * (u[j].y * u[j].y + u[j].z * u[j].z + u[j].w * u[j].w);
            const float an = 1.f - d2 * 0.125f + d2 * d2 * (1.f / 384.f);
            const float bn = dt * (0.5f - d2 * (1.f / 48.f));
            N[j] = qnormalize(Quat{an, bn * u[j].y, bn * u[j].z, bn * u[j].w});
            seg = (j == 0) ? N[0] : qmul(seg, N[j]);
        }
        const Quat S = seg_scan_qmul<kLanes>(seg, sub);
        Quat E = shfl_up<kLanes>(S, 1);
        if (sub == 0) E = Quat{1.f, 0.f, 0.f, 0.f};
        // attitude at the segment's start (the first step uses the state's attitude as given,
        // as the sequential form does)
        Quat q = (h0 == 0) ? qc : qnormalize(qmul(qc, E));

        // pass B: stage accelerations; velocity and position offsets within the segment
        Vec3 L[kSteps];
        Quat Qa[kSteps];                                 // attitude after each step (paper form)
        Vec3 V = v3(0.f, 0.f, 0.f);
        Vec3 Lacc = v3(0.f, 0.f, 0.f);
#pragma unroll
        for (int j = 0; j < kSteps; ++j) {
            const bool act = h0 + j < H;
            const float tm = u[j].x * inv_m;
            const float d2 = dt * dt * (u[j].y * u[j].y + u[j].z * u[j].z + u[j].w * u[j].w);
            const Quat wq{-q.x * u[j].y - q.y * u[j].z - q.z * u[j].w,
                          q.w * u[j].y + q.y * u[j].w - q.z * u[j].z,
                          q.w * u[j].z - q.x * u[j].w + q.z * u[j].y,
                          q.w * u[j].w + q.x * u[j].z - q.y * u[j].y};
            const float a3 = 1.f - d2 * (1.f / 16.f);
            const float a4 = 1.f - d2 * 0.125f;
            const float b4 = dt * (0.5f - d2 * (1.f / 32.f));
            const Quat q2{q.w + b2 * wq.w, q.x + b2 * wq.x, q.y + b2 * wq.y, q.z + b2 * wq.z};
            const Quat q3{a3 * q.w + b2 * wq.w, a3 * q.x + b2 * wq.x, a3 * q.y + b2 * wq.y, a3 * q.z + b2 * wq.z};
            const Quat q4{a4 * q.w + b4 * wq.w, a4 * q.x + b4 * wq.x, a4 * q.y + b4 * wq.y, a4 * q.z + b4 * wq.z};
            const Vec3 z1 = body_z(q), z2 = body_z(q2), z3 = body_z(q3), z4 = body_z(q4);
            const Vec3 s3 = v3(z1.x + z2.x + z3.x, z1.y + z2.y + z3.y, z1.z + z2.z + z3.z);
            const Vec3 s6 = v3(z1.x + 2.f * (z2.x + z3.x) + z4.x, z1.y + 2.f * (z2.y + z3.y) + z4.y,
                               z1.z + 2.f * (z2.z + z3.z) + z4.z);
            if (act) {
                // p offset after this step: previous offset + dt V_j + dt^2/6 (a1 + a2 + a3)
                Lacc = v3(Lacc.x + dt * V.x + c3 * (tm * s3.x), Lacc.y + dt * V.y + c3 * (tm * s3.y),
                          Lacc.z + dt * V.z + c3 * (tm * s3.z - 3.f * P.gravity));
                V = v3(V.x + c6 * (tm * s6.x), V.y + c6 * (tm * s6.y), V.z + (c6 * (tm * s6.z) - dt * P.gravity));
            }
            L[j] = Lacc;
            if (P.paper || j + 1 < kSteps) q = qnormalize(qmul(q, N[j]));
            Qa[j] = q;
        }
        // segment start velocities and positions: exclusive scans of the segments' totals
        const Vec3 Sv = seg_scan_add<kLanes>(V, sub);
        Vec3 ev = shfl_up<kLanes>(Sv, 1);
        if (sub == 0) ev = v3(0.f, 0.f, 0.f);
        const Vec3 vs = v3(vc.x + ev.x, vc.y + ev.y, vc.z + ev.z);
        const float tn = dt * static_cast<float>(nact);
        const Vec3 dP = v3(tn * vs.x + Lacc.x, tn * vs.y + Lacc.y, tn * vs.z + Lacc.z);
        const Vec3 Sp = seg_scan_add<kLanes>(dP, sub);
        Vec3 ep = shfl_up<kLanes>(Sp, 1);
        if (sub == 0) ep = v3(0.f, 0.f, 0.f);
        const Vec3 ps = v3(pc.x + ep.x, pc.y + ep.y, pc.z + ep.z);

        // pass C: positions p_{h+1} = p_s + (j + 1) dt v_s + L_j
#pragma unroll
        for (int j = 0; j < kSteps; ++j) {
            const int h = h0 + j;
            if (h < H) {
                const float tj = dt * static_cast<float>(j + 1);
                const Vec3 p = v3(ps.x + tj * vs.x + L[j].x, ps.y + tj * vs.y + L[j].y, ps.z + tj * vs.z + L[j].z);
                if (valid) pos_k[h] = make_float4(p.x, p.y, p.z, 0.f);
                if (P.paper) {
                    if (tgt >= 0) {
                        jvis += misalignment(Qa[j], p, wp);
                        if (analytic) jcol += fmaxf(P.d_safe - guide_sdf(to_gate(pose_t, p), P.a_in, P.tan_alpha), 0.f);
                    }
                } else if (analytic) {
                    float smin = __int_as_float(0x7f800000);
                    for (int g = 0; g < P.G; ++g) {
                        const Vec3 pg = to_gate(sPose + 8 * g, p);
                        smin = fminf(smin, frame_sdf(pg.x, pg.y, pg.z, P.a_in, P.a_out, P.half_depth));
                    }
                    jcol += hinge_sq(smin, P.d_safe);
                }
            }
        }
        // state at the end of the chunk
        const Vec3 pe = shfl_idx<kLanes>(Sp, kLanes - 1);
        pc = v3(pc.x + pe.x, pc.y + pe.y, pc.z + pe.z);
        const Vec3 sv = shfl_idx<kLanes>(Sv, kLanes - 1);
        vc = v3(vc.x + sv.x, vc.y + sv.y, vc.z + sv.z);
        qc = qnormalize(qmul(qc, shfl_idx<kLanes>(S, kLanes - 1)));
    }
    jctl = seg_sum<kLanes>(jctl);
    jcol = seg_sum<kLanes>(jcol);
    jvis = seg_sum<kLanes>(jvis);
    if (sub == 0 && valid) {
        if (P.paper) {
            // Eq. 6 telescoped: sum_k |p_{k+1} - wp|^2 - |p_k - wp|^2 = |p_H - wp|^2 - |p_0 - wp|^2
            const float dHx = pc.x - wp.x, dHy = pc.y - wp.y, dHz = pc.z - wp.z;
            const float d0x = p0.x - wp.x, d0y = p0.y - wp.y, d0z = p0.z - wp.z;
            const float jgate = (tgt >= 0) ? (dHx * dHx + dHy * dHy + dHz * dHz) - (d0x * d0x + d0y * d0y + d0z * d0z)
                                           : 0.f;
            B.parts[k] = analytic ? P.q_sdf * jcol : 0.f;
            B.parts[K + k] = P.q_gate * jgate;
            B.parts[2 * K + k] = P.q_vis * jvis;
        } else {
            const float jprog =
                (tgt >= 0) ? -(n_tgt.x * (pc.x - p0.x) + n_tgt.y * (pc.y - p0.y) + n_tgt.z * (pc.z - p0.z)) : 0.f;
            B.parts[k] = analytic ? P.w_col * jcol : 0.f;
            B.parts[K + k] = jprog;
            B.parts[2 * K + k] = P.w_u * jctl;
        }
    }
}

template <int kLanes, int kSteps>
__global__ void __launch_bounds__(kRollWarps * 32) rollout_kernel(StepParams P, StepBuffers B, int analytic) {
    extern __shared__ float4 sU[];                 // [H]
    __shared__ float sPose[kMaxGates * 8];
    rollout_body<kLanes, kSteps>(P, B, analytic, blockIdx.x, sU, sPose);
}

// ------------------------------------------------------------------ (a) + (b) rotor-thrust-rate model
// The paper's command (Sec. IV-A): the four rotor-thrust rates, the body rate following from
// the rotors' torques (rk4_rotor).  The body rate now has dynamics of its own, so the attitude
// is no longer a product of state-independent factors: each rollout is integrated by one
// thread, sequentially over the horizon.  A block (4 warps) owns 32 rollouts: warp 0 integrates
// them (one lane each) while warps 1-3 draw the noise of the next kRotorChunk steps (the same
// Philox blocks as the thrust / body-rate model, scaled by sigma_tdot) into the [K][H] noise
// array, from which warp 0 reads it after the block's barrier; the draws are off the
// integration's serial chain.  Positions are stored in the [K][H] array.
constexpr int kRotorThreads = 128;
constexpr int kRotorRollouts = 32;               // rollouts per block (warp 0's lanes)
constexpr int kRotorChunk = 16;                  // horizon steps drawn ahead per block barrier
static_assert(kRotorThreads == kRollWarps * 32, "the batched rollout kernel runs the rotor body in its 128-thread blocks");

// the noise of rollouts [k0, k0 + 32) x steps [h0, h0 + n), drawn by `nthreads` threads from t0
__device__ __forceinline__ void rotor_draw(const StepParams& P, const StepBuffers& B, int k0, int h0, int n,
                                           uint32_t st, int t, int nthreads) {
    for (int i = t; i < kRotorRollouts * n; i += nthreads) {
        const int r = i / n, h = h0 + (i - r * n);
        const int k = k0 + r;
        if (k < P.K) B.noise[static_cast<size_t>(k) * P.H + h] = noise_from_block(P, noise_block(P, k, h, st));
    }
}

__device__ __forceinline__ void rotor_body(const StepParams& P, const StepBuffers& B, int analytic, int block,
                                           float4* sU, float* sPose) {
    pdl_trigger();
    pdl_wait();
    for (int i = threadIdx.x; i < P.H; i += blockDim.x) sU[i] = B.nominal[i];
    for (int i = threadIdx.x; i < P.G * 8; i += blockDim.x) sPose[i] = B.poses[i];
    const int K = P.K, H = P.H;
    const int k0 = block * kRotorRollouts;
    const uint32_t st = B.step[0];
    // the first chunk's noise, drawn by the whole block
    rotor_draw(P, B, k0, 0, min(kRotorChunk, H), st, threadIdx.x, blockDim.x);
    __syncthreads();
    const bool integrator = threadIdx.x < 32;
    const int k = k0 + static_cast<int>(threadIdx.x);
    const bool valid = integrator && k < K;
    const float* s0 = B.state;
    const Vec3 p0 = v3(s0[0], s0[1], s0[2]);
    Vec3 p = p0, v = v3(s0[3], s0[4], s0[5]), w = v3(s0[10], s0[11], s0[12]);
    Quat q{s0[6], s0[7], s0[8], s0[9]};
    float T[4] = {s0[13], s0[14], s0[15], s0[16]};
    Vec3 n_tgt;
    const int tgt = target_gate(sPose, P.G, p0, &n_tgt);
    const float* pose_t = sPose + 8 * (tgt < 0 ? 0 : tgt);
    const Vec3 wp = v3(pose_t[0], pose_t[1], pose_t[2]);
    float jctl = 0.f, jcol = 0.f, jvis = 0.f;
    const float4* noise_k = B.noise + static_cast<size_t>(valid ? k : 0) * H;
    float4* pos_k = B.pos + static_cast<size_t>(valid ? k : 0) * H;
    for (int h0 = 0; h0 < H; h0 += kRotorChunk) {
        const int n = min(kRotorChunk, H - h0);
        if (!integrator) {
            // warps 1-3: the next chunk's noise while warp 0 integrates this one
            if (h0 + n < H)
                rotor_draw(P, B, k0, h0 + n, min(kRotorChunk, H - h0 - n), st, threadIdx.x - 32, blockDim.x - 32);
        } else if (valid) {
            float4 d = noise_k[h0];
            for (int j = 0; j < n; ++j) {
                const int h = h0 + j;
                const float4 d_next = (j + 1 < n) ? noise_k[h + 1] : d;   // loaded while this step runs
                const float4 un = sU[h];
                const float4 u = clip_control(P, make_float4(un.x + d.x, un.y + d.y, un.z + d.z, un.w + d.w));
                const float e0 = u.x - P.u_hover;
                jctl += e0 * e0 + u.y * u.y + u.z * u.z + u.w * u.w;
                rk4_rotor(P, p, v, q, w, T, u);
                pos_k[h] = make_float4(p.x, p.y, p.z, 0.f);
                if (P.paper) {
                    if (tgt >= 0) {
                        jvis += misalignment(q, p, wp);
                        if (analytic) jcol += fmaxf(P.d_safe - guide_sdf(to_gate(pose_t, p), P.a_in, P.tan_alpha), 0.f);
                    }
                } else if (analytic) {
                    float smin = __int_as_float(0x7f800000);
                    for (int g = 0; g < P.G; ++g) {
                        const Vec3 pg = to_gate(sPose + 8 * g, p);
                        smin = fminf(smin, frame_sdf(pg.x, pg.y, pg.z, P.a_in, P.a_out, P.half_depth));
                    }
                    jcol += hinge_sq(smin, P.d_safe);
                }
                d = d_next;
            }
        }
        __syncthreads();
    }
    if (!valid) return;
    if (P.paper) {
        const float dHx = p.x - wp.x, dHy = p.y - wp.y, dHz = p.z - wp.z;
        const float d0x = p0.x - wp.x, d0y = p0.y - wp.y, d0z = p0.z - wp.z;
        const float jgate = (tgt >= 0) ? (dHx * dHx + dHy * dHy + dHz * dHz) - (d0x * d0x + d0y * d0y + d0z * d0z) : 0.f;
        B.parts[k] = analytic ? P.q_sdf * jcol : 0.f;
        B.parts[K + k] = P.q_gate * jgate;
        B.parts[2 * K + k] = P.q_vis * jvis;
    } else {
        const float jprog =
            (tgt >= 0) ? -(n_tgt.x * (p.x - p0.x) + n_tgt.y * (p.y - p0.y) + n_tgt.z * (p.z - p0.z)) : 0.f;
        B.parts[k] = analytic ? P.w_col * jcol : 0.f;
        B.parts[K + k] = jprog;
        B.parts[2 * K + k] = P.w_u * jctl;
    }
}

__global__ void __launch_bounds__(kRotorThreads) rollout_rotor_kernel(StepParams P, StepBuffers B, int analytic) {
    extern __shared__ float4 sU[];                 // [H]
    __shared__ float sPose[kMaxGates * 8];
    rotor_body(P, B, analytic, blockIdx.x, sU, sPose);
}

// ------------------------------------------------------------------ (d) costs, weights, update, receding horizon
// Block b owns R consecutive rollouts (R a multiple of 32, at most kCuMaxBlocks blocks):
//  1. J_k = J_col + J_prog + J_ctl (MLP modes: J_col = w_col sum_h max(0, d_safe - s_h)^2,
//     or Q_sdf sum_h max(0, d_safe - s_h) in the paper's form, from the per-tile partial sums
//     the SDF kernel folded), rho_b = min of the block's J_k,
//     e_k = exp(-(J_k - rho_b) / lambda), eta_b = sum of the block's e_k;
//  2. S_b[h] = sum_{k in b} e_k clip(U*_h + delta_{k,h});
//  3. grid barrier (the kernel is a cooperative launch, so all its blocks are resident; an
//     arrival counter with release / acquire ordering);
//  4. every block forms rho = min_b rho_b, F_b = exp(-(rho_b - rho) / lambda) and
//     eta = sum_b F_b eta_b from the same data in the same order (bit-identical in every
//     block), writes its own weights w_k = e_k F_b / eta (Eq. 5 with max subtraction) and
//     U*_new[h] = sum_b (F_b / eta) S_b[h] for its share of the horizon, written in place
//     as the shifted warm start; the block owning h = 0 applies U*_new[0] to the
//     device-resident state with one RK4 step and bumps the step counter.
// Every reduction runs in a fixed order: reruns are bit-identical.  Loads are issued in
// explicit batches so each phase waits for memory about once.  When the caller passed
// device buffers for U*_new, w and J, the kernel writes them too.
constexpr int kCuThreads = 256;
constexpr int kCuWarps = kCuThreads / 32;
constexpr int kCuMaxBlocks = 128;
constexpr uint64_t kGridWaitLimitNs = 2000000000ull;  // bound of the grid barrier's wait


constexpr int kCuHChunk = 64;                      // horizon steps per pass of the weighted sums
constexpr int kCuBatch = 4;                        // rollouts per warp whose loads are in flight together

__device__ __forceinline__ float4 f4_fma(float a, float4 x, float4 y) {
    return make_float4(fmaf(a, x.x, y.x), fmaf(a, x.y, y.y), fmaf(a, x.z, y.z), fmaf(a, x.w, y.w));
}

// Shared scratch of the update kernels (besides R floats of dynamic shared memory).
struct UpdShared {
    float4 red[kCuWarps][kCuHChunk];
    float warp[kCuWarps];
    float F[kCuMaxBlocks];
    float rho, eta;
    int flag;
};

// Phases 1 and 2 of update block `block` of a controller (R rollouts from k0 = block R; sE: R
// floats of shared memory): J_k, e_k (into B.w), the block statistics B.bstat[block] and the
// partial sums B.upart[block][h].  The per-controller kernel and the batched serving kernel
// both run it.
__device__ __forceinline__ void update_local(const StepParams& P, const StepBuffers& B, int mlp, int R, int block,
                                             float* sE, UpdShared& U) {
    float4 (&sRed)[kCuWarps][kCuHChunk] = U.red;
    float* sWarp = U.warp;
    const float4* __restrict__ noise = B.noise;
    const float* parts_in = B.parts;             // also written below (J_col of the MLP modes)
    const int K = P.K, H = P.H;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int k0 = block * R;
    const int nk = min(K, k0 + R) - k0;
    const float inv_lam = 1.f / P.lam;
    const float inf = __int_as_float(0x7f800000);

    // the noise rows of this warp's first kCuBatch rollouts (first kCuHChunk steps) are
    // loaded now; their latency overlaps the cost phase
    float4 pre_a[kCuBatch], pre_b[kCuBatch];
#pragma unroll
    for (int u = 0; u < kCuBatch; ++u) {
        const int i = wid + u * kCuWarps;
        const float4* nrow = noise + static_cast<size_t>(k0 + (i < nk ? i : 0)) * H;
        pre_a[u] = (i < nk && lane < H) ? __ldcs(nrow + lane) : make_float4(0.f, 0.f, 0.f, 0.f);
        pre_b[u] = (i < nk && lane + 32 < H) ? __ldcs(nrow + 32 + lane) : make_float4(0.f, 0.f, 0.f, 0.f);
    }

    // 1. costs: one thread per rollout.  MLP modes: J_col = w_col (or Q_sdf) times the sum of the
    //    rollout's per-segment partial sums of the stage hinge, which the SDF kernel folded in its
    //    epilogue (fold_warp), added in segment order
    float mloc = inf;
    const int n_colp = col_slots(H);
    for (int i = threadIdx.x; i < nk; i += kCuThreads) {
        const int k = k0 + i;
        float jcol;
        if (mlp) {
            const int n = ((k * H + H - 1) >> 5) - ((k * H) >> 5) + 1;     // the rollout's 32-row segments
            const float* cp = B.colp + static_cast<size_t>(k) * n_colp;
            float a = __ldcs(cp);
            for (int j = 1; j < n; ++j) a += __ldcs(cp + j);
            jcol = (P.paper ? P.q_sdf : P.w_col) * a;
            B.parts[k] = jcol;
        } else {
            jcol = parts_in[k];
        }
        const float J = jcol + parts_in[K + k] + parts_in[2 * K + k];
        sE[i] = J;
        mloc = fminf(mloc, J);
    }
    mloc = warp_min(mloc);
    if (lane == 0) sWarp[wid] = mloc;
    __syncthreads();
    if (threadIdx.x == 0) {
        float m = sWarp[0];
#pragma unroll
        for (int i = 1; i < kCuWarps; ++i) m = fminf(m, sWarp[i]);
        U.rho = m;
    }
    __syncthreads();
    const float rho_b = U.rho;
    float eloc = 0.f;
    for (int i = threadIdx.x; i < nk; i += kCuThreads) {
        const float J = sE[i];
        const float e = expf(-(J - rho_b) * inv_lam);
        B.J[k0 + i] = J;
        if (B.out_J) B.out_J[k0 + i] = J;
        B.w[k0 + i] = e;                           // scaled to w_k by the last combiner
        sE[i] = e;
        eloc += e;
    }
    eloc = warp_sum(eloc);
    if (lane == 0) sWarp[wid] = eloc;
    __syncthreads();
    if (threadIdx.x == 0) {
        float e = sWarp[0];
#pragma unroll
        for (int i = 1; i < kCuWarps; ++i) e += sWarp[i];
        B.bstat[block] = make_float2(rho_b, e);
    }

    // 2. e-weighted sums of the rolled-out (clipped) controls, kCuHChunk horizon steps per pass
    for (int c0 = 0; c0 < H; c0 += kCuHChunk) {
        const int ha = c0 + lane, hb = c0 + 32 + lane;
        const bool va = ha < H, vb = hb < H;
        const float4 una = B.nominal[min(ha, H - 1)];
        const float4 unb = B.nominal[min(hb, H - 1)];
        float4 aa = make_float4(0.f, 0.f, 0.f, 0.f), ab = aa;
        for (int i0 = wid; i0 < nk; i0 += kCuWarps * kCuBatch) {
            float4 da[kCuBatch], db[kCuBatch];
            float e[kCuBatch];
            const bool first = (c0 == 0 && i0 == wid);
#pragma unroll
            for (int u = 0; u < kCuBatch; ++u) {
                const int i = i0 + u * kCuWarps;
                const bool v = i < nk;
                const float4* nrow = noise + static_cast<size_t>(k0 + (v ? i : 0)) * H;
                e[u] = v ? sE[i] : 0.f;
                if (first) {
                    da[u] = pre_a[u];
                    db[u] = pre_b[u];
                } else {
                    da[u] = (v && va) ? __ldcs(nrow + ha) : make_float4(0.f, 0.f, 0.f, 0.f);
                    db[u] = (v && vb) ? __ldcs(nrow + hb) : make_float4(0.f, 0.f, 0.f, 0.f);
                }
            }
#pragma unroll
            for (int u = 0; u < kCuBatch; ++u) {
                aa = f4_fma(e[u], clip_control(P, make_float4(una.x + da[u].x, una.y + da[u].y, una.z + da[u].z,
                                                             una.w + da[u].w)), aa);
                ab = f4_fma(e[u], clip_control(P, make_float4(unb.x + db[u].x, unb.y + db[u].y, unb.z + db[u].z,
                                                             unb.w + db[u].w)), ab);
            }
        }
        sRed[wid][lane] = aa;
        sRed[wid][32 + lane] = ab;
        __syncthreads();
        if (threadIdx.x < kCuHChunk && c0 + threadIdx.x < H) {
            float4 t = sRed[0][threadIdx.x];
#pragma unroll
            for (int i = 1; i < kCuWarps; ++i) {
                const float4 o = sRed[i][threadIdx.x];
                t.x += o.x; t.y += o.y; t.z += o.z; t.w += o.w;
            }
            B.upart[static_cast<size_t>(block) * H + c0 + threadIdx.x] = t;
        }
        __syncthreads();
    }
}

// Phase 4: rho = min_b rho_b, F_b = exp(-(rho_b - rho) / lambda), eta = sum_b F_b eta_b from the
// nb blocks' statistics (warp 0, the same data in the same order wherever it runs), then the
// weights w_k = e_k F_b / eta of the rollouts of blocks [b_lo, b_hi) and U*_new[h] = sum_b
// (F_b / eta) S_b[h] for h = h0, h0 + hs, ..., written in place as the shifted warm start; the
// caller that covers h = 0 also applies U*_new[0] to the device-resident state with one RK4 step
// and bumps the step counter.
__device__ __forceinline__ void update_combine(const StepParams& P, const StepBuffers& B, int nb, int R, int b_lo,
                                               int b_hi, int h0, int hs, UpdShared& U) {
    float* sF = U.F;
    const int K = P.K, H = P.H;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const float inv_lam = 1.f / P.lam;
    const float inf = __int_as_float(0x7f800000);

    if (wid == 0) {
        float2 bs[kCuMaxBlocks / 32];
        float m = inf;
#pragma unroll
        for (int j = 0; j < kCuMaxBlocks / 32; ++j) {
            const int b = lane + 32 * j;
            bs[j] = (b < nb) ? __ldcg(&B.bstat[b]) : make_float2(inf, 0.f);
            m = fminf(m, bs[j].x);
        }
        const float rho = warp_min(m);
        float e = 0.f;
#pragma unroll
        for (int j = 0; j < kCuMaxBlocks / 32; ++j) {
            const int b = lane + 32 * j;
            const float f = (b < nb) ? expf(-(bs[j].x - rho) * inv_lam) : 0.f;
            if (b < nb) sF[b] = f;
            e += f * bs[j].y;
        }
        const float eta = warp_sum(e);
        if (lane == 0) {
            U.rho = rho;
            U.eta = eta;
        }
    }
    __syncthreads();
    const float eta = U.eta;
    // weights w_k = e_k F_b / eta of blocks [b_lo, b_hi) (e_k as update_local stored it in B.w)
    for (int b = b_lo; b < b_hi; ++b) {
        const int k0 = b * R;
        const int nk = min(K, k0 + R) - k0;
        const float fw = sF[b] / eta;
        for (int i = threadIdx.x; i < nk; i += kCuThreads) {
            const float wk = __ldcg(B.w + k0 + i) * fw;
            B.w[k0 + i] = wk;
            if (B.out_w) B.out_w[k0 + i] = wk;
        }
    }
    // U*_new[h] for h = h0, h0 + hs, ...: thread t < nb loads block t's partial; fixed-order
    // sums: xor shuffles within each warp, then the warps' sums in warp order
    float4* sU = reinterpret_cast<float4*>(U.red);
    const float uh = P.u_hover;
    for (int h = h0; h < H; h += hs) {
        float4 t = make_float4(0.f, 0.f, 0.f, 0.f);
        if (threadIdx.x < nb) {
            const float4 sb = __ldcg(B.upart + static_cast<size_t>(threadIdx.x) * H + h);
            const float f = sF[threadIdx.x] / eta;
            t = make_float4(f * sb.x, f * sb.y, f * sb.z, f * sb.w);
        }
        t.x = warp_sum(t.x);
        t.y = warp_sum(t.y);
        t.z = warp_sum(t.z);
        t.w = warp_sum(t.w);
        if (lane == 0) sU[wid] = t;
        __syncthreads();
        if (threadIdx.x == 0) {
            float4 u = sU[0];
#pragma unroll
            for (int i = 1; i < kCuWarps; ++i) {
                const float4 o = sU[i];
                u = make_float4(u.x + o.x, u.y + o.y, u.z + o.z, u.w + o.w);
            }
            B.unew[h] = u;
            if (B.out_U) B.out_U[h] = u;
            if (h >= 1) B.nominal[h - 1] = u;                     // the warm start, shifted by one
            if (h == H - 1) B.nominal[H - 1] = make_float4(uh, 0.f, 0.f, 0.f);
            if (h == 0) {
                // apply U*_new[0] to the device-resident state
                B.stats[0] = U.rho;
                B.stats[1] = eta;
                float* st = B.state;
                Vec3 p = v3(st[0], st[1], st[2]);
                Vec3 v = v3(st[3], st[4], st[5]);
                Quat q{st[6], st[7], st[8], st[9]};
                if (P.rotor) {
                    Vec3 w = v3(st[10], st[11], st[12]);
                    float T[4] = {st[13], st[14], st[15], st[16]};
                    rk4_rotor(P, p, v, q, w, T, u);
                    st[10] = w.x; st[11] = w.y; st[12] = w.z;
                    st[13] = T[0]; st[14] = T[1]; st[15] = T[2]; st[16] = T[3];
                } else {
                    rk4_step(P, p, v, q, u.x, v3(u.y, u.z, u.w));
                    st[10] = u.y; st[11] = u.z; st[12] = u.w;
                }
                st[0] = p.x; st[1] = p.y; st[2] = p.z;
                st[3] = v.x; st[4] = v.y; st[5] = v.z;
                st[6] = q.w; st[7] = q.x; st[8] = q.y; st[9] = q.z;
                const uint32_t lo = B.step[0] + 1u;
                B.step[0] = lo;
                if (lo == 0u) B.step[1] += 1u;
                // every earlier wait of this step has ended (every block's phases are done)
                if (B.err_out) *B.err_out = *reinterpret_cast<volatile int*>(B.err);
            }
        }
        __syncthreads();
    }
}

__global__ void __launch_bounds__(kCuThreads) cost_update_kernel(StepParams P, StepBuffers B, int mlp, int R) {
    extern __shared__ float sE[];                  // [R] J_k, then e_k
    __shared__ UpdShared U;
    pdl_wait();
    update_local(P, B, mlp, R, blockIdx.x, sE, U);
    // 3. grid barrier (cooperative launch: every block is resident; the wait is bounded).  The
    //    arrival counter (64 bits, ticket words 12-13) only grows: after the block's writes
    //    (the __syncthreads above), one thread adds 1 with release semantics; the launch's
    //    target is the next multiple of the grid size above the count it saw, and it polls
    //    with acquire loads.  A launch that timed out leaves the count off a multiple of the
    //    grid: the host zeroes the ticket words together with the error word.  Ticket word 31
    //    (0 unless set by mppi_debug_inject_timeout) moves the target that many grids further,
    //    so that every block's wait runs out: the test of the timeout path, with no fault.
    if (threadIdx.x == 0) {
        U.flag = grid_arrive_wait(reinterpret_cast<unsigned long long*>(B.tickets + 12), B.tickets[31], B.err,
                                   kGridWaitLimitNs)
                      ? 1
                      : 0;
    }
    __syncthreads();
    if (!U.flag) return;

    // 4. every block combines the blocks' statistics the same way, writes its own weights and its
    //    share of the horizon
    update_combine(P, B, gridDim.x, R, blockIdx.x, blockIdx.x + 1, blockIdx.x, gridDim.x, U);
}

// ------------------------------------------------------------------ per-gate first-layer bias
// The Gate-SDF decoder's first layer sees [PE(p), z]; z is fixed per gate, so its
// part W1[:, P:] z + b1 (P point features) is computed once per gate instead of once per query.
__global__ void first_layer_bias_kernel(const float* __restrict__ W1, const float* __restrict__ b1,
                                        const float* __restrict__ lat, int G, int n_point, float* __restrict__ b1p) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= G * kHidden) return;
    const int g = i / kHidden, c = i - g * kHidden;
    const float* wr = W1 + c * (n_point + kLatent) + n_point;
    const float* z = lat + g * kLatent;
    float acc = 0.f;
    for (int j = 0; j < kLatent; ++j) acc = fmaf(wr[j], z[j], acc);
    b1p[i] = b1[c] + acc;
}


// ------------------------------------------------------------------ batched serving step
// The index of the slot whose range [start, next start) holds x (starts ascending, slot 0 at 0).
template <typename Start>
__device__ __forceinline__ int find_slot(const BatchSlot* __restrict__ slots, int n, int x, Start start) {
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (start(slots[mid]) <= x) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// One block per controller: its state, gate poses and latents from the batch's input block into
// its buffers, and the first-layer bias of every gate (the arithmetic of first_layer_bias_kernel).
__global__ void __launch_bounds__(128) batch_prep_kernel(const BatchSlot* __restrict__ slots,
                                                         const float* __restrict__ in) {
    const BatchSlot& S = slots[blockIdx.x];
    const float* src = in + S.in_off;
    const int G = S.P.G;
    for (int i = threadIdx.x; i < S.state_floats; i += blockDim.x) S.B.state[i] = src[i];
    const float* poses = src + kBatchStateSlot;
    for (int i = threadIdx.x; i < G * 8; i += blockDim.x) S.B.poses[i] = poses[i];
    if (!S.mlp) return;
    const float* lat = poses + G * 8;
    for (int i = threadIdx.x; i < G * kLatent; i += blockDim.x) S.latents[i] = lat[i];
    for (int i = threadIdx.x; i < G * kHidden; i += blockDim.x) {
        const int g = i / kHidden, c = i - g * kHidden;
        const float* wr = S.W1 + c * (S.n_point + kLatent) + S.n_point;
        const float* z = lat + g * kLatent;
        float acc = 0.f;
        for (int j = 0; j < kLatent; ++j) acc = fmaf(wr[j], z[j], acc);
        S.B.b1p[i] = S.b1[c] + acc;
    }
}

// Rollout blocks of every controller of the batch (128 threads each): a block finds its
// controller and runs that controller's rollout form on its parameters and buffers.
__global__ void __launch_bounds__(kRollWarps * 32) rollout_batch_kernel(const BatchSlot* __restrict__ slots, int n) {
    extern __shared__ float4 sU[];                 // [max H]
    __shared__ float sPose[kMaxGates * 8];
    __shared__ StepParams sP;
    __shared__ StepBuffers sB;
    __shared__ int s_form, s_block, s_analytic;
    if (threadIdx.x == 0) {
        const int d = find_slot(slots, n, static_cast<int>(blockIdx.x), [](const BatchSlot& t) { return t.roll_block0; });
        sP = slots[d].P;
        sB = slots[d].B;
        s_form = slots[d].roll_form;
        s_block = static_cast<int>(blockIdx.x) - slots[d].roll_block0;
        s_analytic = slots[d].mlp ? 0 : 1;
    }
    __syncthreads();
    switch (s_form) {
        case 0: rollout_body<32, 2>(sP, sB, s_analytic, s_block, sU, sPose); break;
        case 1: rollout_body<16, 2>(sP, sB, s_analytic, s_block, sU, sPose); break;
        case 2: rollout_body<16, 4>(sP, sB, s_analytic, s_block, sU, sPose); break;
        default: rotor_body(sP, sB, s_analytic, s_block, sU, sPose); break;
    }
}

// Update blocks of every controller of the batch: phases 1 and 2 as in cost_update_kernel, then
// the last of a controller's blocks to finish (an arrival count on the controller's barrier
// counter, release / acquire) combines all of them with the same arithmetic, so no block waits
// for another and the launch needs no co-residency.
__global__ void __launch_bounds__(kCuThreads) cost_update_batch_kernel(const BatchSlot* __restrict__ slots, int n) {
    extern __shared__ float sE[];                  // [max R]
    __shared__ UpdShared U;
    __shared__ StepParams sP;
    __shared__ StepBuffers sB;
    __shared__ int s_block, s_R, s_nb, s_mlp;
    pdl_wait();
    if (threadIdx.x == 0) {
        const int d = find_slot(slots, n, static_cast<int>(blockIdx.x), [](const BatchSlot& t) { return t.upd_block0; });
        sP = slots[d].P;
        sB = slots[d].B;
        s_R = slots[d].upd_R;
        s_nb = (sP.K + s_R - 1) / s_R;
        s_block = static_cast<int>(blockIdx.x) - slots[d].upd_block0;
        s_mlp = slots[d].mlp;
    }
    __syncthreads();
    update_local(sP, sB, s_mlp, s_R, s_block, sE, U);
    if (threadIdx.x == 0) {
        __threadfence();
        const unsigned long long prev = atomicAdd(reinterpret_cast<unsigned long long*>(sB.tickets + 12), 1ull);
        U.flag = ((prev + 1ull) % static_cast<unsigned long long>(s_nb) == 0ull) ? 1 : 0;
    }
    __syncthreads();
    if (!U.flag) return;
    __threadfence();
    update_combine(sP, sB, s_nb, s_R, 0, s_nb, 0, 1, U);
}
}  // namespace

cudaError_t launch_noise_words(const StepParams& P, const StepBuffers& B, uint4* out, cudaStream_t s) {
    const int n = P.K * P.H;
    noise_words_kernel<<<(n + 255) / 256, 256, 0, s>>>(P, B.step, out);
    return cudaGetLastError();
}

cudaError_t launch_rollout(const StepParams& P, const StepBuffers& B, int analytic, cudaStream_t s) {
    // first kernel of the step: ordered after the previous step's last kernel by the stream
    if (P.rotor)
        return launch_dependent(false, rollout_rotor_kernel, dim3((P.K + kRotorRollouts - 1) / kRotorRollouts),
                                dim3(kRotorThreads), P.H * sizeof(float4), s, P, B, analytic);
    // two rollouts per warp (16 lanes x 4 steps, or x 2 when the horizon fits in 32), except for
    // a long horizon at small K: there a warp per rollout (32 lanes x 2 steps) keeps more warps
    // on each SM for the latency-bound scans (K = 4096, H = 50: the two forms are level; at
    // K = 16384, H = 64 the half-warp form is 7 % faster)
    const dim3 block(kRollWarps * 32);
    const size_t smem = P.H * sizeof(float4);
    if (P.H > 32 && P.K < 8192)
        return launch_dependent(false, rollout_kernel<32, 2>, dim3((P.K + kRollWarps - 1) / kRollWarps), block, smem, s,
                                P, B, analytic);
    const dim3 grid((P.K + 2 * kRollWarps - 1) / (2 * kRollWarps));
    if (P.H <= 32) return launch_dependent(false, rollout_kernel<16, 2>, grid, block, smem, s, P, B, analytic);
    return launch_dependent(false, rollout_kernel<16, 4>, grid, block, smem, s, P, B, analytic);
}

int update_rollouts_per_block(int K) {
    const int r = (K + kCuMaxBlocks - 1) / kCuMaxBlocks;
    const int r32 = ((r + 31) / 32) * 32;
    return r32 < 32 ? 32 : r32;
}

int update_blocks(int K) {
    const int R = update_rollouts_per_block(K);
    return (K + R - 1) / R;
}



cudaError_t configure_cost_update() {
    // R floats of dynamic shared memory: up to MPPI_MAX_K / kCuMaxBlocks
    const int bytes = static_cast<int>(sizeof(float) * update_rollouts_per_block(kMaxRollouts));
    cudaError_t e = cudaFuncSetAttribute(cost_update_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(cost_update_batch_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    // the batched rollout's H float4 of dynamic shared memory (up to MPPI_MAX_H)
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(rollout_batch_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 static_cast<int>(1024 * sizeof(float4)));
    return e;
}

cudaError_t launch_cost_update(const StepParams& P, const StepBuffers& B, int mlp, cudaStream_t s) {
    // a cooperative launch: the blocks meet at a grid barrier, so all of them must be resident
    const int R = update_rollouts_per_block(P.K);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((P.K + R - 1) / R);
    cfg.blockDim = dim3(kCuThreads);
    cfg.dynamicSmemBytes = sizeof(float) * R;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, cost_update_kernel, P, B, mlp, R);
}

int rollout_form(const StepParams& P) {
    if (P.rotor) return 3;
    if (P.H > 32 && P.K < 8192) return 0;
    return P.H <= 32 ? 1 : 2;
}

int rollout_batch_blocks(const StepParams& P) {
    switch (rollout_form(P)) {
        case 0: return (P.K + kRollWarps - 1) / kRollWarps;
        case 1:
        case 2: return (P.K + 2 * kRollWarps - 1) / (2 * kRollWarps);
        default: return (P.K + kRotorRollouts - 1) / kRotorRollouts;
    }
}

cudaError_t launch_batch_prep(const BatchSlot* slots, int n, const float* inputs, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    batch_prep_kernel<<<n, 128, 0, s>>>(slots, inputs);
    return cudaGetLastError();
}

cudaError_t launch_rollout_batch(const BatchSlot* slots, int n, int blocks, int max_h, cudaStream_t s) {
    if (n <= 0 || blocks <= 0) return cudaSuccess;
    rollout_batch_kernel<<<blocks, kRollWarps * 32, max_h * sizeof(float4), s>>>(slots, n);
    return cudaGetLastError();
}

cudaError_t launch_cost_update_batch(const BatchSlot* slots, int n, int blocks, int max_r, cudaStream_t s) {
    if (n <= 0 || blocks <= 0) return cudaSuccess;
    cost_update_batch_kernel<<<blocks, kCuThreads, max_r * sizeof(float), s>>>(slots, n);
    return cudaGetLastError();
}

cudaError_t launch_first_layer_bias(const float* W1, const float* b1, const float* latents, int G, int n_point,
                                    float* b1p, cudaStream_t s) {
    if (G <= 0) return cudaSuccess;
    const int n = G * kHidden;
    first_layer_bias_kernel<<<(n + 127) / 128, 128, 0, s>>>(W1, b1, latents, G, n_point, b1p);
    return cudaGetLastError();
}

}  // namespace mppi
