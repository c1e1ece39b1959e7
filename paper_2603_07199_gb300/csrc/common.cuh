// Device-side building blocks shared by the step kernels: launch parameters,
// Philox4x32-10, Box-Muller, quaternion kinematics, RK4 and the frame SDF.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace mppi {

constexpr int kHidden = 128;
constexpr int kLatent = 64;
constexpr int kMaxGates = 8;
constexpr int kTileRows = 128;       // SDF rows (rollout states) per tile
constexpr int kMaxRollouts = 1 << 20;

// device error word values
constexpr int kDevErrTimeout = 1;

// Columns of the layer-1 tensor-core GEMM: 0..8 the query point split [hi, lo, hi] (against
// [W_hi, W_hi, W_lo]), 9..15 zero, then one 8-column core-matrix chunk per positional-encoding
// level l: columns 16 + 8 l + (0..5) = sin(2^l pi p) (x, y, z), cos(2^l pi p) (x, y, z).
// K = 16 + 8 L rounded up to a multiple of 16 (16 .. 64).
__host__ __device__ inline int layer1_gemm_k(int pe_levels) {
    return pe_levels == 0 ? 16 : ((16 + 8 * pe_levels + 15) / 16) * 16;
}
__host__ __device__ inline int pe_column(int level, int t) { return 16 + 8 * level + t; }

// Scalars every step kernel needs, passed by value.
struct StepParams {
    int K, H, G;
    float dt, mass, gravity;
    float tmin, tmax, rmax;
    float sig_t, sig_r, lam;
    float w_col, d_safe, w_u;
    float a_in, a_out, half_depth;
    float beta;
    uint32_t key0, key1, drone;
    int pdl;               // host side: launch kernels as programmatic dependents
    int paper;             // cost form of Eq. 6-9 on the target gate (else the configured form)
    float q_gate, q_vis, q_sdf, tan_alpha;
    int rotor;             // rotor-thrust-rate model (17-number state) instead of thrust + body rates
    float u_hover;         // first control channel of the hover command (m g, or 0 for thrust rates)
    float arm_d, kappa, t_rotor_max;  // rotor offset l / sqrt(2), reaction torque per newton, thrust bound
    float3 J, inv_J;       // diagonal inertia and its reciprocal
    int pe;                // positional-encoding levels of the decoder's query point
    int store_sdf;         // the SDF kernels also store s(p) of every rollout state (diagnostics)
    int sdf_pair;          // host side: 16-bit SDF MLP kernel in its CTA-pair form (else one CTA per tile group set)
};

// Device buffers of one controller.
struct StepBuffers {
    float* state;          // 16 floats: 13-float true state (+pad)
    float4* nominal;       // [H] warm-start sequence U*
    uint32_t* step;        // [2] step counter (lo, hi)
    float* poses;          // [maxG][8] (t, q, pad)
    float* b1p;            // [maxG][128] per-gate first-layer bias W1[:,3:] z_g + b1
    float4* noise;         // [K][H] delta u (h fastest)
    float4* pos;           // [K][H] rollout positions p_1..p_H (x, y, z, 0)
    float* parts;          // [3][K] J_col, J_prog, J_ctl
    float* sdf;            // [K][H] min-over-gates SDF at every rollout state (MLP modes, diagnostics only)
    float* colp;           // [K][col_slots(H)] per-rollout partial sums of the stage hinge, one per SDF tile
    float* J;              // [K]
    float* w;              // [K]
    float4* unew;          // [H] updated sequence U*_new
    float4* upart;         // [update blocks][H] per-block sums of e_k U^k_h
    float2* bstat;         // [update blocks] per-block (min J, sum e_k)
    float4* out_U;         // optional caller device buffers written by the step (H x 4, K, K)
    float* out_w;
    float* out_J;
    int* err_out;          // optional: the step's last kernel copies *err here when it is done
    float* stats;          // [4] rho, eta of the last step
    unsigned* tickets;     // [32]: [12..13] the update kernel's 64-bit grid-barrier arrival count, [31] test skew
    int* err;              // [1] device error word
};

// ---------------------------------------------------------------- Philox4x32-10
// Salmon et al., SC'11: 10 rounds; multipliers on words 0 and 2; Weyl key bump.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r > 0) { k0 += 0x9E3779B9u; k1 += 0xBB67AE85u; }
        const uint32_t hi0 = __umulhi(0xD2511F53u, c.x);
        const uint32_t lo0 = 0xD2511F53u * c.x;
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z);
        const uint32_t lo1 = 0xCD9E8D57u * c.z;
        c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
    }
    return c;
}

// 32-bit word -> uniform in (0, 1): (x >> 8) + 1/2 on the 2^-24 grid (exact in FP32).
__device__ __forceinline__ float word_to_uniform(uint32_t x) {
    return (static_cast<float>(x >> 8) + 0.5f) * 5.9604644775390625e-08f;
}

// Box-Muller: (ua, ub) -> (r cos 2 pi ub, r sin 2 pi ub), r = sqrt(-2 ln ua).
__device__ __forceinline__ float2 box_muller(float ua, float ub) {
    const float r = sqrtf(-2.0f * logf(ua));
    float s, c;
    sincospif(2.0f * ub, &s, &c);
    return make_float2(r * c, r * s);
}

// The Philox block of rollout k, horizon step h.
__device__ __forceinline__ uint4 noise_block(const StepParams& P, int k, int h, uint32_t step_lo) {
    return philox4x32_10(make_uint4(static_cast<uint32_t>(k), static_cast<uint32_t>(h), step_lo, P.drone),
                         P.key0, P.key1);
}

// delta u = diag(sig_t, sig_r, sig_r, sig_r) n.
__device__ __forceinline__ float4 noise_from_block(const StepParams& P, uint4 w) {
    const float2 a = box_muller(word_to_uniform(w.x), word_to_uniform(w.y));
    const float2 b = box_muller(word_to_uniform(w.z), word_to_uniform(w.w));
    return make_float4(P.sig_t * a.x, P.sig_r * a.y, P.sig_r * b.x, P.sig_r * b.y);
}

__device__ __forceinline__ float4 clip_control(const StepParams& P, float4 u) {
    u.x = fminf(fmaxf(u.x, P.tmin), P.tmax);
    u.y = fminf(fmaxf(u.y, -P.rmax), P.rmax);
    u.z = fminf(fmaxf(u.z, -P.rmax), P.rmax);
    u.w = fminf(fmaxf(u.w, -P.rmax), P.rmax);
    return u;
}

// ---------------------------------------------------------------- rigid body
struct Quat { float w, x, y, z; };
struct Vec3 { float x, y, z; };

__device__ __forceinline__ Vec3 v3(float x, float y, float z) { return Vec3{x, y, z}; }

// Hamilton product a (x) b.
__device__ __forceinline__ Quat qmul(const Quat& a, const Quat& b) {
    return Quat{a.w * b.w - a.x * b.x - a.y * b.y - a.z * b.z,
                a.w * b.x + a.x * b.w + a.y * b.z - a.z * b.y,
                a.w * b.y - a.x * b.z + a.y * b.w + a.z * b.x,
                a.w * b.z + a.x * b.y - a.y * b.x + a.z * b.w};
}
__device__ __forceinline__ Quat qnormalize(const Quat& q) {
    const float inv = rsqrtf(q.w * q.w + q.x * q.x + q.y * q.y + q.z * q.z);
    return Quat{q.w * inv, q.x * inv, q.y * inv, q.z * inv};
}

// Rotate v by the conjugate of unit q (world -> body/gate frame): R(q)^T v.
__device__ __forceinline__ Vec3 rotate_inv(const Quat& q, const Vec3& v) {
    // R^T v with R the rotation matrix of q, written out
    const float ww = q.w * q.w, xx = q.x * q.x, yy = q.y * q.y, zz = q.z * q.z;
    const float xy = q.x * q.y, xz = q.x * q.z, yz = q.y * q.z;
    const float wx = q.w * q.x, wy = q.w * q.y, wz = q.w * q.z;
    const float r00 = ww + xx - yy - zz, r01 = 2.f * (xy - wz), r02 = 2.f * (xz + wy);
    const float r10 = 2.f * (xy + wz), r11 = ww - xx + yy - zz, r12 = 2.f * (yz - wx);
    const float r20 = 2.f * (xz - wy), r21 = 2.f * (yz + wx), r22 = ww - xx - yy + zz;
    return v3(r00 * v.x + r10 * v.y + r20 * v.z,
              r01 * v.x + r11 * v.y + r21 * v.z,
              r02 * v.x + r12 * v.y + r22 * v.z);
}

// First column of R(q): the gate normal.
__device__ __forceinline__ Vec3 quat_x_axis(const Quat& q) {
    return v3(q.w * q.w + q.x * q.x - q.y * q.y - q.z * q.z,
              2.f * (q.x * q.y + q.w * q.z),
              2.f * (q.x * q.z - q.w * q.y));
}

// One RK4 step of dp = v, dv = (T/m) R(q) e_z - g e_z, dq = q (x) (0, w) / 2,
// then renormalise q.  T, w held over the step.
//
// With w constant, q -> q (x) (0, w) is linear and squares to -|w|^2, so every
// RK4 stage quaternion is a q + b Wq (Wq = q (x) (0, w)) with a, b polynomials in
// |w|^2 dt^2, and the stage sums collapse (same RK4 polynomial as the four-stage
// form, written out):
//   q2 = q + dt/4 Wq,   q3 = (1 - dt^2 w2/16) q + dt/4 Wq,
//   q4 = (1 - dt^2 w2/8) q + (dt/2 - dt^3 w2/32) Wq,
//   q' = (1 - dt^2 w2/8 + dt^4 w2^2/384) q + (dt/2 - dt^3 w2/48) Wq,
//   p' = p + dt v + dt^2/6 (a1 + a2 + a3),  v' = v + dt/6 (a1 + 2 a2 + 2 a3 + a4),
// where a_s = (T/m) z(q_s) - g e_z and z(q) = R(q) e_z in the unit-quaternion form.
__device__ __forceinline__ Vec3 body_z(const Quat& a) {
    return v3(2.f * (a.x * a.z + a.w * a.y), 2.f * (a.y * a.z - a.w * a.x), 1.f - 2.f * (a.x * a.x + a.y * a.y));
}

__device__ __forceinline__ void rk4_step(const StepParams& P, Vec3& p, Vec3& v, Quat& q, float T, Vec3 w) {
    const float dt = P.dt;
    const float tm = T / P.mass;
    const Quat wq{-q.x * w.x - q.y * w.y - q.z * w.z,
                  q.w * w.x + q.y * w.z - q.z * w.y,
                  q.w * w.y - q.x * w.z + q.z * w.x,
                  q.w * w.z + q.x * w.y - q.y * w.x};
    const float w2 = w.x * w.x + w.y * w.y + w.z * w.z;
    const float d2 = dt * dt * w2;                       // (|w| dt)^2
    const float b2 = 0.25f * dt;
    const float a3 = 1.f - d2 * (1.f / 16.f);
    const float a4 = 1.f - d2 * 0.125f;
    const float b4 = dt * (0.5f - d2 * (1.f / 32.f));
    const float an = 1.f - d2 * 0.125f + d2 * d2 * (1.f / 384.f);
    const float bn = dt * (0.5f - d2 * (1.f / 48.f));
    const Quat q2{q.w + b2 * wq.w, q.x + b2 * wq.x, q.y + b2 * wq.y, q.z + b2 * wq.z};
    const Quat q3{a3 * q.w + b2 * wq.w, a3 * q.x + b2 * wq.x, a3 * q.y + b2 * wq.y, a3 * q.z + b2 * wq.z};
    const Quat q4{a4 * q.w + b4 * wq.w, a4 * q.x + b4 * wq.x, a4 * q.y + b4 * wq.y, a4 * q.z + b4 * wq.z};
    const Vec3 z1 = body_z(q), z2 = body_z(q2), z3 = body_z(q3), z4 = body_z(q4);
    const Vec3 s3 = v3(z1.x + z2.x + z3.x, z1.y + z2.y + z3.y, z1.z + z2.z + z3.z);
    const Vec3 s6 = v3(z1.x + 2.f * (z2.x + z3.x) + z4.x, z1.y + 2.f * (z2.y + z3.y) + z4.y,
                       z1.z + 2.f * (z2.z + z3.z) + z4.z);
    const float c3 = dt * dt * (1.f / 6.f);
    const float c6 = dt * (1.f / 6.f);
    p.x += dt * v.x + c3 * (tm * s3.x);
    p.y += dt * v.y + c3 * (tm * s3.y);
    p.z += dt * v.z + c3 * (tm * s3.z - 3.f * P.gravity);
    v.x += c6 * (tm * s6.x);
    v.y += c6 * (tm * s6.y);
    v.z += c6 * (tm * s6.z) - dt * P.gravity;
    Quat qn{an * q.w + bn * wq.w, an * q.x + bn * wq.x, an * q.y + bn * wq.y, an * q.z + bn * wq.z};
    const float inv = rsqrtf(qn.w * qn.w + qn.x * qn.x + qn.y * qn.y + qn.z * qn.z);
    q = Quat{qn.w * inv, qn.x * inv, qn.y * inv, qn.z * inv};
}

// ---------------------------------------------------------------- rotor-thrust-rate model
// State [p, v, q, w, T1..T4], command u = dT/dt (Sec. IV-A).  Rotor i sits at body
// d (1, -1), (-1, -1), (-1, 1), (1, 1) (X layout, d = arm / sqrt(2)) with reaction torque
// kappa (+1, -1, +1, -1) T_i about body z, so tau = (d (T3 + T4 - T1 - T2),
// d (T2 + T3 - T1 - T4), kappa (T1 + T3 - T2 - T4)) in 1-based rotor numbers, and
//   dv = (sum T / m) R(q) e_z - g e_z,  dq = q (x) (0, w) / 2,  dw = J^-1 (tau - w x J w),  dT = u.
struct RotorDeriv {
    Vec3 dv;
    Quat dq;
    Vec3 dw;
};

__device__ __forceinline__ RotorDeriv rotor_deriv(const StepParams& P, const Quat& q, const Vec3& w, float t0, float t1,
                                                  float t2, float t3) {
    RotorDeriv d;
    const float a = (t0 + t1 + t2 + t3) / P.mass;
    const Vec3 z = body_z(q);
    d.dv = v3(a * z.x, a * z.y, a * z.z - P.gravity);
    d.dq = Quat{-0.5f * (q.x * w.x + q.y * w.y + q.z * w.z), 0.5f * (q.w * w.x + q.y * w.z - q.z * w.y),
                0.5f * (q.w * w.y - q.x * w.z + q.z * w.x), 0.5f * (q.w * w.z + q.x * w.y - q.y * w.x)};
    const float tx = P.arm_d * ((t2 + t3) - (t0 + t1));
    const float ty = P.arm_d * ((t1 + t2) - (t0 + t3));
    const float tz = P.kappa * ((t0 + t2) - (t1 + t3));
    const Vec3 Jw = v3(P.J.x * w.x, P.J.y * w.y, P.J.z * w.z);
    d.dw = v3((tx - (w.y * Jw.z - w.z * Jw.y)) * P.inv_J.x, (ty - (w.z * Jw.x - w.x * Jw.z)) * P.inv_J.y,
              (tz - (w.x * Jw.y - w.y * Jw.x)) * P.inv_J.z);
    return d;
}

__device__ __forceinline__ Vec3 axpy(float a, const Vec3& x, const Vec3& y) {
    return v3(fmaf(a, x.x, y.x), fmaf(a, x.y, y.y), fmaf(a, x.z, y.z));
}
__device__ __forceinline__ Quat axpy(float a, const Quat& x, const Quat& y) {
    return Quat{fmaf(a, x.w, y.w), fmaf(a, x.x, y.x), fmaf(a, x.y, y.y), fmaf(a, x.z, y.z)};
}

// One classical RK4 step of the rotor model with u held; q renormalised, thrusts clamped to
// [0, t_rotor_max].  T: the four rotor thrusts, updated in place.
__device__ __forceinline__ void rk4_rotor(const StepParams& P, Vec3& p, Vec3& v, Quat& q, Vec3& w, float* T, float4 u) {
    const float dt = P.dt, h2 = 0.5f * dt;
    const float a0 = T[0] + h2 * u.x, a1 = T[1] + h2 * u.y, a2 = T[2] + h2 * u.z, a3 = T[3] + h2 * u.w;
    const RotorDeriv k1 = rotor_deriv(P, q, w, T[0], T[1], T[2], T[3]);
    const Vec3 v2 = axpy(h2, k1.dv, v);
    const RotorDeriv k2 = rotor_deriv(P, axpy(h2, k1.dq, q), axpy(h2, k1.dw, w), a0, a1, a2, a3);
    const Vec3 v3s = axpy(h2, k2.dv, v);
    const RotorDeriv k3 = rotor_deriv(P, axpy(h2, k2.dq, q), axpy(h2, k2.dw, w), a0, a1, a2, a3);
    const Vec3 v4 = axpy(dt, k3.dv, v);
    const RotorDeriv k4 = rotor_deriv(P, axpy(dt, k3.dq, q), axpy(dt, k3.dw, w), T[0] + dt * u.x, T[1] + dt * u.y,
                                      T[2] + dt * u.z, T[3] + dt * u.w);
    const float c = dt * (1.f / 6.f);
    p = v3(p.x + c * (v.x + 2.f * (v2.x + v3s.x) + v4.x), p.y + c * (v.y + 2.f * (v2.y + v3s.y) + v4.y),
           p.z + c * (v.z + 2.f * (v2.z + v3s.z) + v4.z));
    v = v3(v.x + c * (k1.dv.x + 2.f * (k2.dv.x + k3.dv.x) + k4.dv.x), v.y + c * (k1.dv.y + 2.f * (k2.dv.y + k3.dv.y) + k4.dv.y),
           v.z + c * (k1.dv.z + 2.f * (k2.dv.z + k3.dv.z) + k4.dv.z));
    const Quat qn{q.w + c * (k1.dq.w + 2.f * (k2.dq.w + k3.dq.w) + k4.dq.w), q.x + c * (k1.dq.x + 2.f * (k2.dq.x + k3.dq.x) + k4.dq.x),
                  q.y + c * (k1.dq.y + 2.f * (k2.dq.y + k3.dq.y) + k4.dq.y), q.z + c * (k1.dq.z + 2.f * (k2.dq.z + k3.dq.z) + k4.dq.z)};
    q = qnormalize(qn);
    w = v3(w.x + c * (k1.dw.x + 2.f * (k2.dw.x + k3.dw.x) + k4.dw.x), w.y + c * (k1.dw.y + 2.f * (k2.dw.y + k3.dw.y) + k4.dw.y),
           w.z + c * (k1.dw.z + 2.f * (k2.dw.z + k3.dw.z) + k4.dw.z));
    T[0] = fminf(fmaxf(T[0] + dt * u.x, 0.f), P.t_rotor_max);
    T[1] = fminf(fmaxf(T[1] + dt * u.y, 0.f), P.t_rotor_max);
    T[2] = fminf(fmaxf(T[2] + dt * u.z, 0.f), P.t_rotor_max);
    T[3] = fminf(fmaxf(T[3] + dt * u.w, 0.f), P.t_rotor_max);
}

// ---------------------------------------------------------------- programmatic dependent launch
// Wait until the preceding kernel in the stream has completed and its writes are
// visible (returns at once when the kernel was not launched as a dependent).
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
// Allow the next kernel in the stream to start launching (its prologue overlaps this kernel).
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// ---------------------------------------------------------------- grid barrier of a cooperative launch
__device__ __forceinline__ uint64_t global_timer_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
    return t;
}
// GPU-scope release add (returns the old value) and acquire load of a barrier's counter
__device__ __forceinline__ unsigned long long atom_add_release_gpu(unsigned long long* p, unsigned long long v) {
    unsigned long long old;
    asm volatile("atom.release.gpu.global.add.u64 %0, [%1], %2;" : "=l"(old) : "l"(p), "l"(v) : "memory");
    return old;
}
__device__ __forceinline__ unsigned long long ld_acquire_gpu(const unsigned long long* p) {
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
// Thread 0's half of a grid barrier over a counter that only grows (call after a
// __syncthreads that follows the block's writes; broadcast the result through shared memory
// and a second __syncthreads): one release add, the target is the next multiple of the grid
// size (+ skew grids; 0 except in tests of the timeout path) above the count seen, acquire
// polls bounded by limit_ns.  Returns false when the wait gave up (after setting *err).  A
// launch that gave up leaves the count off a multiple of the grid: the host zeroes it.
__device__ __forceinline__ bool grid_arrive_wait(unsigned long long* ctr, unsigned long long skew, int* err,
                                                 uint64_t limit_ns) {
    const unsigned long long nbl = gridDim.x;
    const unsigned long long target = (atom_add_release_gpu(ctr, 1ull) / nbl + 1ull + skew) * nbl;
    if (ld_acquire_gpu(ctr) >= target) return true;
    const uint64_t t0 = global_timer_ns();
    while (ld_acquire_gpu(ctr) < target) {
        if (global_timer_ns() - t0 > limit_ns) {
            atomicExch(err, kDevErrTimeout);
            return false;
        }
    }
    return true;
}

// ---------------------------------------------------------------- gate frame SDF
// Exact signed distance to the square frame {|x| <= d, a_in <= max(|y|,|z|) <= a_out}.
// The frame is symmetric in x, y and z, so the query is folded into the first
// octant, where the solid is the union of the top bar [0,d]x[0,a_out]x[a_in,a_out]
// and the side post [0,d]x[a_in,a_out]x[0,a_in].
__device__ __forceinline__ float frame_sdf(float x, float y, float z, float a_in, float a_out, float d) {
    const float ax = fabsf(x), ay = fabsf(y), az = fabsf(z);
    const float r = fmaxf(ay, az);
    if (ax <= d && r <= a_out && r >= a_in) {
        const float ey = fmaxf(ay - a_in, 0.f), ez = fmaxf(az - a_in, 0.f);
        const float open = sqrtf(ey * ey + ez * ez);
        return -fminf(fminf(d - ax, a_out - r), open);
    }
    const float gx = fmaxf(ax - d, 0.f);
    // top bar: y in [0, a_out], z in [a_in, a_out]
    const float ty = fmaxf(ay - a_out, 0.f);
    const float tz = fmaxf(fmaxf(a_in - az, az - a_out), 0.f);
    // side post: y in [a_in, a_out], z in [0, a_in]
    const float sy = fmaxf(fmaxf(a_in - ay, ay - a_out), 0.f);
    const float sz = fmaxf(az - a_in, 0.f);
    const float dt2 = gx * gx + ty * ty + tz * tz;
    const float ds2 = gx * gx + sy * sy + sz * sz;
    return sqrtf(fminf(dt2, ds2));
}

// World point -> gate frame for pose (t, q) stored as 8 floats.
__device__ __forceinline__ Vec3 to_gate(const float* pose, Vec3 p) {
    const Quat q{pose[3], pose[4], pose[5], pose[6]};
    return rotate_inv(q, v3(p.x - pose[0], p.y - pose[1], p.z - pose[2]));
}

__device__ __forceinline__ float hinge_sq(float s, float d_safe) {
    const float e = fmaxf(d_safe - s, 0.f);
    return e * e;
}

// The collision / safety stage cost of one state: configured w_col-free form max(0, d - s)^2,
// or the paper's linear hinge max(0, d - s) (Eq. 8).
__device__ __forceinline__ float stage_hinge(float s, float d_safe, int paper) {
    const float e = fmaxf(d_safe - s, 0.f);
    return paper ? e : e * e;
}

// ---------------------------------------------------------------- collision-cost fold in the SDF kernels
// The SDF kernels fold the stage hinge of Eq. 8 over the horizon in their epilogue (Eq. 9-10:
// J_col of a rollout is a sum over its states) instead of storing s(p) for every state.  The
// rows of the [K][H] state array are folded 32 at a time (one row per lane of a warp): rollout
// k owns rows k H .. k H + H - 1, which touch the 32-row segments floor(k H / 32) ..
// floor((k H + H - 1) / 32), at most col_slots(H) of them; segment w writes the sum over its
// rows of rollout k to colp[k][w - floor(k H / 32)].  The cost kernel adds a rollout's slots in
// segment order, so every sum runs in a fixed order.
__host__ __device__ inline int col_slots(int H) { return (H + 30) / 32 + 1; }

// One warp, 32 consecutive rows r (one per lane, stage cost c, 0 for rows past the end): an
// inclusive scan that restarts at every rollout boundary; the last row of each run in the warp
// stores the run's sum.
__device__ __forceinline__ void fold_warp(float c, int r, int n_rows, int H, int lane, float* colp) {
    const unsigned full = 0xffffffffu;
    const int key = r / H;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const float t = __shfl_up_sync(full, c, d);
        const int kk = __shfl_up_sync(full, key, d);
        if (lane >= d && kk == key) c += t;
    }
    const int knext = __shfl_down_sync(full, key, 1);
    if ((lane == 31 || knext != key) && r < n_rows)
        colp[static_cast<size_t>(key) * col_slots(H) + ((r >> 5) - ((key * H) >> 5))] = c;
}

// Index of the first gate whose plane the position p has not crossed (n_g . (p - t_g) < 0),
// else the last gate; -1 without gates.  poses: [G][8] = (t, q, pad); n_out: its normal.
__device__ __forceinline__ int target_gate(const float* poses, int G, Vec3 p, Vec3* n_out) {
    for (int g = 0; g < G; ++g) {
        const float* ps = poses + 8 * g;
        const Vec3 n = quat_x_axis(Quat{ps[3], ps[4], ps[5], ps[6]});
        const float side = n.x * (p.x - ps[0]) + n.y * (p.y - ps[1]) + n.z * (p.z - ps[2]);
        if (side < 0.f || g == G - 1) {
            *n_out = n;
            return g;
        }
    }
    *n_out = v3(0.f, 0.f, 0.f);
    return -1;
}

// Eq. 2: guidance SDF c + |x| tan(alpha) - max(|y|, |z|) of a gate-frame point.
__device__ __forceinline__ float guide_sdf(Vec3 pg, float c, float tan_alpha) {
    return c + fabsf(pg.x) * tan_alpha - fmaxf(fabsf(pg.y), fabsf(pg.z));
}

// 1 - cos(psi - psi_gate) of Eq. 7 for attitude q at position p and waypoint wp: psi is the
// heading of the body x axis, (1 - 2 (y^2 + z^2), 2 (xy + wz)), psi_gate the bearing of
// wp - p in the horizontal plane; a zero vector has heading 0 (the atan2(0, 0) convention).
__device__ __forceinline__ float misalignment(const Quat& q, Vec3 p, Vec3 wp) {
    float hx = 1.f - 2.f * (q.y * q.y + q.z * q.z), hy = 2.f * (q.x * q.y + q.w * q.z);
    float lx = wp.x - p.x, ly = wp.y - p.y;
    float hn = hx * hx + hy * hy, ln = lx * lx + ly * ly;
    if (hn == 0.f) { hx = 1.f; hy = 0.f; hn = 1.f; }
    if (ln == 0.f) { lx = 1.f; ly = 0.f; ln = 1.f; }
    return 1.f - (hx * lx + hy * ly) * rsqrtf(hn * ln);
}

}  // namespace mppi
