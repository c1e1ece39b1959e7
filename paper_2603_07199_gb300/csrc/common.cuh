// Device-side building blocks shared by the step kernels: launch parameters,
// Philox4x32-10, Box-Muller, quaternion kinematics, RK4 and the frame SDF.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace mppi {

constexpr int kHidden = 128;
constexpr int kLatent = 64;
constexpr int kMaxGates = 8;
constexpr int kTileRows = 128;       // SDF rows (rollouts) per tile

// device error word values
constexpr int kDevErrTimeout = 1;

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
};

// Device buffers of one controller.
struct StepBuffers {
    float* state;          // 16 floats: 13-float true state (+pad)
    float4* nominal;       // [H] warm-start sequence U*
    uint32_t* step;        // [2] step counter (lo, hi)
    float* poses;          // [maxG][8] (t, q, pad)
    float* b1p;            // [maxG][128] per-gate first-layer bias W1[:,3:] z_g + b1
    float4* noise;         // [H][K] delta u
    float4* pos;           // [H][K] rollout positions (x, y, z, 0)
    float* parts;          // [3][K] J_col, J_prog, J_ctl
    float* sdf;            // [H][K] min-over-gates SDF at every rollout state (MLP modes)
    float* J;              // [K]
    float* w;              // [K]
    float4* unew;          // [H] updated sequence U*_new
    float* red;            // [2 * cost blocks] per-block (min J, sum exp) partials
    float* stats;          // [4] rho, eta of the last step
    unsigned* tickets;     // [4] last-block counters
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
__device__ __forceinline__ void rk4_step(const StepParams& P, Vec3& p, Vec3& v, Quat& q, float T, Vec3 w) {
    const float tm = T / P.mass;
    const float g = P.gravity;
    const float dt = P.dt, hdt = 0.5f * P.dt;
    // stage derivative helpers
    auto acc = [&](const Quat& a) -> Vec3 {
        return v3(tm * 2.f * (a.x * a.z + a.w * a.y),
                  tm * 2.f * (a.y * a.z - a.w * a.x),
                  tm * (1.f - 2.f * (a.x * a.x + a.y * a.y)) - g);
    };
    auto qdot = [&](const Quat& a) -> Quat {
        return Quat{0.5f * (-a.x * w.x - a.y * w.y - a.z * w.z),
                    0.5f * (a.w * w.x + a.y * w.z - a.z * w.y),
                    0.5f * (a.w * w.y - a.x * w.z + a.z * w.x),
                    0.5f * (a.w * w.z + a.x * w.y - a.y * w.x)};
    };
    auto qadd = [](const Quat& a, float s, const Quat& d) -> Quat {
        return Quat{a.w + s * d.w, a.x + s * d.x, a.y + s * d.y, a.z + s * d.z};
    };
    // k1
    const Vec3 dp1 = v;
    const Vec3 dv1 = acc(q);
    const Quat dq1 = qdot(q);
    // k2
    const Vec3 v2 = v3(v.x + hdt * dv1.x, v.y + hdt * dv1.y, v.z + hdt * dv1.z);
    const Quat q2 = qadd(q, hdt, dq1);
    const Vec3 dp2 = v2;
    const Vec3 dv2 = acc(q2);
    const Quat dq2 = qdot(q2);
    // k3
    const Vec3 v3s = v3(v.x + hdt * dv2.x, v.y + hdt * dv2.y, v.z + hdt * dv2.z);
    const Quat q3 = qadd(q, hdt, dq2);
    const Vec3 dp3 = v3s;
    const Vec3 dv3 = acc(q3);
    const Quat dq3 = qdot(q3);
    // k4
    const Vec3 v4 = v3(v.x + dt * dv3.x, v.y + dt * dv3.y, v.z + dt * dv3.z);
    const Quat q4 = qadd(q, dt, dq3);
    const Vec3 dp4 = v4;
    const Vec3 dv4 = acc(q4);
    const Quat dq4 = qdot(q4);
    const float s6 = dt / 6.f;
    p.x += s6 * (dp1.x + 2.f * dp2.x + 2.f * dp3.x + dp4.x);
    p.y += s6 * (dp1.y + 2.f * dp2.y + 2.f * dp3.y + dp4.y);
    p.z += s6 * (dp1.z + 2.f * dp2.z + 2.f * dp3.z + dp4.z);
    v.x += s6 * (dv1.x + 2.f * dv2.x + 2.f * dv3.x + dv4.x);
    v.y += s6 * (dv1.y + 2.f * dv2.y + 2.f * dv3.y + dv4.y);
    v.z += s6 * (dv1.z + 2.f * dv2.z + 2.f * dv3.z + dv4.z);
    Quat qn{q.w + s6 * (dq1.w + 2.f * dq2.w + 2.f * dq3.w + dq4.w),
            q.x + s6 * (dq1.x + 2.f * dq2.x + 2.f * dq3.x + dq4.x),
            q.y + s6 * (dq1.y + 2.f * dq2.y + 2.f * dq3.y + dq4.y),
            q.z + s6 * (dq1.z + 2.f * dq2.z + 2.f * dq3.z + dq4.z)};
    const float inv = 1.0f / sqrtf(qn.w * qn.w + qn.x * qn.x + qn.y * qn.y + qn.z * qn.z);
    q = Quat{qn.w * inv, qn.x * inv, qn.y * inv, qn.z * inv};
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

}  // namespace mppi
