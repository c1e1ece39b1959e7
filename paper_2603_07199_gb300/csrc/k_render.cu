// Depth images of the gate frames (the onboard observation of Sec. III-B) by exact
// ray casting, and the optional synthetic sensor noise of the denoising pre-training
// stage (I_noisy).
//
// Work split: a block owns a band of 8 rows of one view.  Its prologue turns every
// gate into per-view constants, 8 threads per gate: the 10 slab numerators of the
// frame's planes (plane offset minus the camera position, in the gate frame), the 3
// columns of the camera -> gate rotation, and the pixel box the frame can cover (the
// bounding box of its outer box's projected corners).  Each warp then takes rows of
// the band in 128-pixel segments (4 pixels per lane, so a warp stores 512
// contiguous bytes) and keeps, by one ballot, the gates whose box overlaps the
// segment, so a segment that sees no gate costs one store per pixel.  Per pixel and
// kept gate: the ray direction in the gate frame (3 FMA after a per-row part), three
// approximate reciprocals, and the first point of the solid along the ray:
//     solid on the ray = [enter, leave] (the outer box |x| <= d, |y|, |z| <= a_out)
//                        minus the open interval (h0, h1) where |y|, |z| < a_in,
// the first such point at t >= 0 being s = max(enter, 0), or h1 when s falls in
// the opening (when h1 <= leave), or none.
// Noise: one Philox block gives the dropout uniforms of 4 consecutive pixels (one
// word each) and, only where a pixel needs one, another block the Box-Muller pair of
// normals of 2 consecutive pixels.
#include <climits>
#include <cstdio>

#include "kernels.h"
#include "mppi.h"

namespace mppi {
namespace {

constexpr int kRtThreads = 256;
constexpr int kRtWarps = kRtThreads / 32;
constexpr int kRtPixPerLane = 4;
constexpr int kRtSegW = 32 * kRtPixPerLane;    // 128 pixels per warp item
constexpr int kRtBandRows = 8;                 // rows of one view per block (one per warp)
constexpr int kRtGateF4 = 5;                   // 19 constants (+1 pad) per gate as float4
constexpr uint32_t kNormalTag = 0xDE9750u;
constexpr uint32_t kDropoutTag = 0xDE9751u;

struct RenderParams {
    int W, H, n_views, n_gates, segs, bands;
    float fx, fy, inv_fx, inv_fy, cx, cy, max_range;
    float a_in, a_out, hd;           // frame geometry
    float noise_c, dropout;
    uint32_t key0, key1, frame;
};

struct Mat3 { float m[3][3]; };

// Rotation matrix of q = (w, x, y, z), normalised first.
__device__ __forceinline__ Mat3 quat_to_mat(float w, float x, float y, float z) {
    const float n = rsqrtf(w * w + x * x + y * y + z * z);
    w *= n; x *= n; y *= n; z *= n;
    Mat3 R;
    R.m[0][0] = 1.f - 2.f * (y * y + z * z); R.m[0][1] = 2.f * (x * y - w * z); R.m[0][2] = 2.f * (x * z + w * y);
    R.m[1][0] = 2.f * (x * y + w * z); R.m[1][1] = 1.f - 2.f * (x * x + z * z); R.m[1][2] = 2.f * (y * z - w * x);
    R.m[2][0] = 2.f * (x * z - w * y); R.m[2][1] = 2.f * (y * z + w * x); R.m[2][2] = 1.f - 2.f * (x * x + y * y);
    return R;
}

// Pixel bounds [lo, hi] (clamped to [0, n - 1], one pixel of margin) of the pixels whose
// slope (c - (i + 1/2)) / f lies in [s_lo, s_hi].
__device__ __forceinline__ int2 slope_pixels(float2 s, float c, float f, int n) {
    const float lo = fminf(fmaxf(floorf(c - 0.5f - s.y * f) - 1.f, 0.f), static_cast<float>(n - 1));
    const float hi = fminf(fmaxf(ceilf(c - 0.5f - s.x * f) + 1.f, 0.f), static_cast<float>(n - 1));
    return make_int2(static_cast<int>(lo), static_cast<int>(hi));
}

// 1 / x to about 1 ulp (PTX rcp.approx.ftz.f32: +-0 -> +-inf, subnormal inputs flushed to 0).
__device__ __forceinline__ float rcp_approx(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// First ray parameter t >= 0 of the frame solid on the ray with gate-frame direction d;
// num = {-d - ox, d - ox, -a_out - oy, a_out - oy, -a_in - oy, a_in - oy, (same for z)}.
__device__ __forceinline__ float ray_frame(const float* num, float dx, float dy, float dz) {
    const float ix = rcp_approx(dx), iy = rcp_approx(dy), iz = rcp_approx(dz);
    const float x0 = num[0] * ix, x1 = num[1] * ix;
    const float yo0 = num[2] * iy, yo1 = num[3] * iy, yi0 = num[4] * iy, yi1 = num[5] * iy;
    const float zo0 = num[6] * iz, zo1 = num[7] * iz, zi0 = num[8] * iz, zi1 = num[9] * iz;
    const float enter = fmaxf(fminf(x0, x1), fmaxf(fminf(yo0, yo1), fminf(zo0, zo1)));
    const float leave = fminf(fmaxf(x0, x1), fminf(fmaxf(yo0, yo1), fmaxf(zo0, zo1)));
    const float h0 = fmaxf(fminf(yi0, yi1), fminf(zi0, zi1));
    const float h1 = fminf(fmaxf(yi0, yi1), fmaxf(zi0, zi1));
    float s = fmaxf(enter, 0.f);
    if (s > h0 && s < h1) s = h1;
    return s <= leave ? s : __int_as_float(0x7f800000);
}

__device__ __forceinline__ uint32_t pick_word(const uint4& w, uint32_t i) {
    return i == 0 ? w.x : (i == 1 ? w.y : (i == 2 ? w.z : w.w));
}

template <bool kVec>
__global__ void __launch_bounds__(kRtThreads) render_depth_kernel(RenderParams P, const float* __restrict__ cams,
                                                                  const float* __restrict__ gates,
                                                                  float* __restrict__ depth) {
    __shared__ float4 s_gate[MPPI_MAX_RENDER_GATES][kRtGateF4];
    __shared__ int4 s_box[MPPI_MAX_RENDER_GATES];   // (u_lo, u_hi, v_lo, v_hi) of each gate's pixels
    const int view = blockIdx.x / P.bands;
    const int band = blockIdx.x - view * P.bands;
    const int v_begin = band * kRtBandRows;
    const int v_end = min(v_begin + kRtBandRows, P.H);
    // a consumer launched as a programmatic dependent (the depth encoder) may start launching
    // now; it waits for this grid to complete before it reads the depths
    pdl_trigger();

    // ---- prologue: the per-view constants of every gate, 8 threads per gate (thread k of a
    // gate projects corner k of its outer box; the 8 reduce the bounds by shuffles)
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int base = warp * 32; base < 8 * P.n_gates; base += kRtThreads) {
        const int t = base + lane;
        const int g = min(t >> 3, P.n_gates - 1);   // lanes past the last gate repeat it, unused
        const int k = t & 7;
        const float* cp = cams + static_cast<size_t>(view) * 7;
        const Mat3 Rc = quat_to_mat(cp[3], cp[4], cp[5], cp[6]);
        const float* gp = gates + g * 7;
        const Mat3 Rg = quat_to_mat(gp[3], gp[4], gp[5], gp[6]);
        const float dtx = gp[0] - cp[0], dty = gp[1] - cp[1], dtz = gp[2] - cp[2];
        // gate centre in the camera frame: c = Rc^T (t_g - t_c)
        const float ccx = Rc.m[0][0] * dtx + Rc.m[1][0] * dty + Rc.m[2][0] * dtz;
        const float ccy = Rc.m[0][1] * dtx + Rc.m[1][1] * dty + Rc.m[2][1] * dtz;
        const float ccz = Rc.m[0][2] * dtx + Rc.m[1][2] * dty + Rc.m[2][2] * dtz;
        // camera -> gate rotation M = Rg^T Rc
        float M[3][3];
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int j = 0; j < 3; ++j)
                M[i][j] = Rg.m[0][i] * Rc.m[0][j] + Rg.m[1][i] * Rc.m[1][j] + Rg.m[2][i] * Rc.m[2][j];
        // pixels the frame can cover: the bounding box of the projections of the 8 corners of its
        // outer box (a point of the box is a convex combination of the corners, so its slopes
        // y / x and z / x lie between theirs when every corner is ahead of the camera); none
        // when the box lies behind the camera or beyond max_range, all when it straddles x ~ 0.
        // Corner k in the camera frame: M^T p_k + c (M^T = Rc^T Rg).
        const float px = (k & 1) ? P.hd : -P.hd, py = (k & 2) ? P.a_out : -P.a_out, pz = (k & 4) ? P.a_out : -P.a_out;
        const float qx = M[0][0] * px + M[1][0] * py + M[2][0] * pz + ccx;
        const float qy = M[0][1] * px + M[1][1] * py + M[2][1] * pz + ccy;
        const float qz = M[0][2] * px + M[1][2] * py + M[2][2] * pz + ccz;
        float xmin = qx, xmax = qx, amin = __fdividef(qy, qx), amax = amin, bmin = __fdividef(qz, qx), bmax = bmin;
#pragma unroll
        for (int o = 1; o < 8; o <<= 1) {
            xmin = fminf(xmin, __shfl_xor_sync(0xffffffffu, xmin, o));
            xmax = fmaxf(xmax, __shfl_xor_sync(0xffffffffu, xmax, o));
            amin = fminf(amin, __shfl_xor_sync(0xffffffffu, amin, o));
            amax = fmaxf(amax, __shfl_xor_sync(0xffffffffu, amax, o));
            bmin = fminf(bmin, __shfl_xor_sync(0xffffffffu, bmin, o));
            bmax = fmaxf(bmax, __shfl_xor_sync(0xffffffffu, bmax, o));
        }
        if (k == 0 && t < 8 * P.n_gates) {
            // camera origin in the gate frame: o = Rg^T (t_c - t_g)
            const float ox = -(Rg.m[0][0] * dtx + Rg.m[1][0] * dty + Rg.m[2][0] * dtz);
            const float oy = -(Rg.m[0][1] * dtx + Rg.m[1][1] * dty + Rg.m[2][1] * dtz);
            const float oz = -(Rg.m[0][2] * dtx + Rg.m[1][2] * dty + Rg.m[2][2] * dtz);
            s_gate[g][0] = make_float4(-P.hd - ox, P.hd - ox, -P.a_out - oy, P.a_out - oy);
            s_gate[g][1] = make_float4(-P.a_in - oy, P.a_in - oy, -P.a_out - oz, P.a_out - oz);
            s_gate[g][2] = make_float4(-P.a_in - oz, P.a_in - oz, M[0][0], M[1][0]);
            s_gate[g][3] = make_float4(M[2][0], M[0][1], M[1][1], M[2][1]);
            s_gate[g][4] = make_float4(M[0][2], M[1][2], M[2][2], 0.f);
            int4 box = make_int4(0, P.W - 1, 0, P.H - 1);
            if (xmax < 0.f || xmin > P.max_range) {
                box = make_int4(1, 0, 1, 0);
            } else if (xmin > 1e-2f) {
                const int2 bu = slope_pixels(make_float2(amin, amax), P.cx, P.fx, P.W);
                const int2 bv = slope_pixels(make_float2(bmin, bmax), P.cy, P.fy, P.H);
                box = make_int4(bu.x, bu.y, bv.x, bv.y);
            }
            s_box[g] = box;
        }
    }
    __syncthreads();

    const bool noisy = P.noise_c > 0.f || P.dropout > 0.f;
    for (int v = v_begin + warp; v < v_end; v += kRtWarps) {
        const float b = (P.cy - (static_cast<float>(v) + 0.5f)) * P.inv_fy;
        // gates whose pixel box covers this row (warp-uniform mask; lane g tests gate g)
        unsigned long long row_gates = 0ull;
        for (int g0 = 0; g0 < P.n_gates; g0 += 32) {
            const int g = g0 + lane;
            const bool k = g < P.n_gates && s_box[g].z <= v && v <= s_box[g].w;
            row_gates |= static_cast<unsigned long long>(__ballot_sync(0xffffffffu, k)) << g0;
        }
        for (int u0 = 0; u0 < P.W; u0 += kRtSegW) {
            const int ub = u0 + lane * kRtPixPerLane;
            float z[kRtPixPerLane];
#pragma unroll
            for (int j = 0; j < kRtPixPerLane; ++j) z[j] = __int_as_float(0x7f800000);
            unsigned long long keep = 0ull;
            if (row_gates) {
                for (int g0 = 0; g0 < P.n_gates; g0 += 32) {
                    const int g = g0 + lane;
                    const bool k = g < P.n_gates && ((row_gates >> g) & 1ull) && s_box[g].x <= u0 + kRtSegW - 1 &&
                                   s_box[g].y >= u0;
                    keep |= static_cast<unsigned long long>(__ballot_sync(0xffffffffu, k)) << g0;
                }
            }
            if (keep) {
                float a[kRtPixPerLane];
#pragma unroll
                for (int j = 0; j < kRtPixPerLane; ++j) a[j] = (P.cx - (static_cast<float>(ub + j) + 0.5f)) * P.inv_fx;
                do {
                    const int i = __ffsll(static_cast<long long>(keep)) - 1;
                    keep &= keep - 1ull;
                    float num[10];
                    const float4 g0 = s_gate[i][0], g1 = s_gate[i][1], g2 = s_gate[i][2], g3 = s_gate[i][3],
                                 g4 = s_gate[i][4];
                    num[0] = g0.x; num[1] = g0.y; num[2] = g0.z; num[3] = g0.w;
                    num[4] = g1.x; num[5] = g1.y; num[6] = g1.z; num[7] = g1.w;
                    num[8] = g2.x; num[9] = g2.y;
                    // gate-frame direction M (1, a, b): the row part e = M e_x + b M e_z, then + a M e_y
                    const float ex = fmaf(b, g4.x, g2.z), ey = fmaf(b, g4.y, g2.w), ez = fmaf(b, g4.z, g3.x);
#pragma unroll
                    for (int j = 0; j < kRtPixPerLane; ++j)
                        z[j] = fminf(z[j], ray_frame(num, fmaf(a[j], g3.y, ex), fmaf(a[j], g3.z, ey),
                                                     fmaf(a[j], g3.w, ez)));
                } while (keep);
            }
            if (ub >= P.W) continue;
#pragma unroll
            for (int j = 0; j < kRtPixPerLane; ++j) z[j] = z[j] <= P.max_range ? z[j] : P.max_range;
            if (noisy) {
                const uint32_t pix0 = static_cast<uint32_t>(v) * static_cast<uint32_t>(P.W) + static_cast<uint32_t>(ub);
                uint32_t cur_q = 0xffffffffu, cur_pair = 0xffffffffu;
                uint4 dw = make_uint4(0u, 0u, 0u, 0u);
                float2 nn = make_float2(0.f, 0.f);
#pragma unroll
                for (int j = 0; j < kRtPixPerLane; ++j) {
                    const uint32_t pix = pix0 + j;
                    if (P.dropout > 0.f) {
                        if ((pix >> 2) != cur_q) {
                            cur_q = pix >> 2;
                            dw = philox4x32_10(make_uint4(cur_q, static_cast<uint32_t>(view), P.frame, kDropoutTag),
                                               P.key0, P.key1);
                        }
                        if (word_to_uniform(pick_word(dw, pix & 3u)) < P.dropout) {
                            z[j] = 0.f;
                            continue;
                        }
                    }
                    if (P.noise_c > 0.f && z[j] < P.max_range) {
                        if ((pix >> 1) != cur_pair) {
                            cur_pair = pix >> 1;
                            const uint4 w = philox4x32_10(
                                make_uint4(cur_pair, static_cast<uint32_t>(view), P.frame, kNormalTag), P.key0, P.key1);
                            nn = box_muller(word_to_uniform(w.x), word_to_uniform(w.y));
                        }
                        const float n = (pix & 1u) ? nn.y : nn.x;
                        z[j] = fminf(fmaxf(fmaf(P.noise_c * z[j] * z[j], n, z[j]), 0.f), P.max_range);
                    }
                }
            }
            float* row = depth + (static_cast<size_t>(view) * P.H + v) * P.W;
            if (kVec) {
                if constexpr (kRtPixPerLane % 4 == 0) {
#pragma unroll
                    for (int j = 0; j < kRtPixPerLane; j += 4)
                        __stcs(reinterpret_cast<float4*>(row + ub + j), make_float4(z[j], z[j + 1], z[j + 2], z[j + 3]));
                } else if constexpr (kRtPixPerLane == 2) {
                    __stcs(reinterpret_cast<float2*>(row + ub), make_float2(z[0], z[1]));
                } else {
                    __stcs(row + ub, z[0]);
                }
            } else {
#pragma unroll
                for (int j = 0; j < kRtPixPerLane; ++j)
                    if (ub + j < P.W) __stcs(row + ub + j, z[j]);
            }
        }
    }
}

// Training queries of the SDF supervision: camera-frame points of image i and the exact SDF
// of the nearest frame there (Philox blocks A, B of (point, image, frame, tag); see the header).
constexpr uint32_t kQueryTagA = 0x5DF0Au;
constexpr uint32_t kQueryTagB = 0x5DF0Bu;

__global__ void __launch_bounds__(128) sample_queries_kernel(RenderParams P, const float* __restrict__ cams,
                                                             const float* __restrict__ gates, int n_points,
                                                             float near_frac, float* __restrict__ points,
                                                             float* __restrict__ labels) {
    const long long e = static_cast<long long>(blockIdx.x) * 128 + threadIdx.x;
    if (e >= static_cast<long long>(P.n_views) * n_points) return;
    const int i = static_cast<int>(e / n_points), j = static_cast<int>(e - static_cast<long long>(i) * n_points);
    const float* cp = cams + static_cast<size_t>(i) * 7;
    const Mat3 Rc = quat_to_mat(cp[3], cp[4], cp[5], cp[6]);
    const uint4 A = philox4x32_10(make_uint4(static_cast<uint32_t>(j), static_cast<uint32_t>(i), P.frame, kQueryTagA),
                                  P.key0, P.key1);
    const uint4 Bw = philox4x32_10(make_uint4(static_cast<uint32_t>(j), static_cast<uint32_t>(i), P.frame, kQueryTagB),
                                   P.key0, P.key1);
    float px, py, pz;                                  // camera frame
    if (word_to_uniform(A.w) < near_frac && P.n_gates > 0) {
        const int g = static_cast<int>((static_cast<unsigned long long>(A.x >> 8) * P.n_gates) >> 24);
        const float* gp = gates + g * 7;
        const Mat3 Rg = quat_to_mat(gp[3], gp[4], gp[5], gp[6]);
        const float hx = P.hd + 0.3f, hy = P.a_out + 0.3f;
        const float qx = (2.f * word_to_uniform(Bw.x) - 1.f) * hx;
        const float qy = (2.f * word_to_uniform(Bw.y) - 1.f) * hy;
        const float qz = (2.f * word_to_uniform(Bw.z) - 1.f) * hy;
        // world = Rg q + t_g; camera = Rc^T (world - t_c)
        const float wx = Rg.m[0][0] * qx + Rg.m[0][1] * qy + Rg.m[0][2] * qz + gp[0] - cp[0];
        const float wy = Rg.m[1][0] * qx + Rg.m[1][1] * qy + Rg.m[1][2] * qz + gp[1] - cp[1];
        const float wz = Rg.m[2][0] * qx + Rg.m[2][1] * qy + Rg.m[2][2] * qz + gp[2] - cp[2];
        px = Rc.m[0][0] * wx + Rc.m[1][0] * wy + Rc.m[2][0] * wz;
        py = Rc.m[0][1] * wx + Rc.m[1][1] * wy + Rc.m[2][1] * wz;
        pz = Rc.m[0][2] * wx + Rc.m[1][2] * wy + Rc.m[2][2] * wz;
    } else {
        px = 0.2f + word_to_uniform(A.y) * (P.max_range - 0.2f);
        py = -(static_cast<float>(P.W) * word_to_uniform(A.z) - P.cx) * px * P.inv_fx;
        pz = -(static_cast<float>(P.H) * word_to_uniform(Bw.w) - P.cy) * px * P.inv_fy;
    }
    // label: the nearest frame's exact SDF at world = Rc p + t_c
    const float wx = Rc.m[0][0] * px + Rc.m[0][1] * py + Rc.m[0][2] * pz + cp[0];
    const float wy = Rc.m[1][0] * px + Rc.m[1][1] * py + Rc.m[1][2] * pz + cp[1];
    const float wz = Rc.m[2][0] * px + Rc.m[2][1] * py + Rc.m[2][2] * pz + cp[2];
    float best = __int_as_float(0x7f800000);
    for (int g = 0; g < P.n_gates; ++g) {
        const float* gp = gates + g * 7;
        const Mat3 Rg = quat_to_mat(gp[3], gp[4], gp[5], gp[6]);
        const float dx = wx - gp[0], dy = wy - gp[1], dz = wz - gp[2];
        const float gx = Rg.m[0][0] * dx + Rg.m[1][0] * dy + Rg.m[2][0] * dz;
        const float gy = Rg.m[0][1] * dx + Rg.m[1][1] * dy + Rg.m[2][1] * dz;
        const float gz = Rg.m[0][2] * dx + Rg.m[1][2] * dy + Rg.m[2][2] * dz;
        best = fminf(best, frame_sdf(gx, gy, gz, P.a_in, P.a_out, P.hd));
    }
    points[e * 3 + 0] = px;
    points[e * 3 + 1] = py;
    points[e * 3 + 2] = pz;
    labels[e] = best;
}

int render_fail(const char* msg, int code = MPPI_E_INVALID, cudaError_t e = cudaSuccess) {
    char buf[256];
    if (e != cudaSuccess)
        snprintf(buf, sizeof(buf), "mppi_render_depth: %s: %s", msg, cudaGetErrorString(e));
    else
        snprintf(buf, sizeof(buf), "mppi_render_depth: %s", msg);
    set_thread_error(buf);
    return code;
}

bool finite_positive(float x) { return x > 0.f && x <= 3.0e38f; }

}  // namespace
}  // namespace mppi

extern "C" void mppi_depth_camera_default(mppi_depth_camera* cam) {
    if (!cam) return;
    *cam = mppi_depth_camera{};
    cam->width = 640;
    cam->height = 480;
    cam->fx = cam->fy = 385.f;
    cam->cx = 320.f;
    cam->cy = 240.f;
    cam->max_range = 10.f;
    cam->gate_inner_half = 0.5f;
    cam->gate_outer_half = 0.75f;
    cam->gate_half_depth = 0.1f;
}

extern "C" int mppi_render_depth(const mppi_depth_camera* cam, int n_views, const float* d_cam_poses, int n_gates,
                                 const float* d_gate_poses, float* d_depth, void* stream) {
    using namespace mppi;
    if (!cam) return render_fail("NULL camera");
    if (cam->width < 1 || cam->width > MPPI_MAX_IMAGE_SIDE || cam->height < 1 || cam->height > MPPI_MAX_IMAGE_SIDE)
        return render_fail("width or height out of [1, MPPI_MAX_IMAGE_SIDE]");
    if (n_views < 0 || n_views > (1 << 24)) return render_fail("n_views out of [0, 2^24]");
    if (n_gates < 0 || n_gates > MPPI_MAX_RENDER_GATES) return render_fail("n_gates out of [0, MPPI_MAX_RENDER_GATES]");
    if (!finite_positive(cam->fx) || !finite_positive(cam->fy) || !finite_positive(cam->max_range))
        return render_fail("fx, fy and max_range must be finite and > 0");
    if (!(cam->cx >= -1e30f && cam->cx <= 1e30f) || !(cam->cy >= -1e30f && cam->cy <= 1e30f))
        return render_fail("cx, cy must be finite");
    if (!finite_positive(cam->gate_inner_half) || !(cam->gate_outer_half > cam->gate_inner_half) ||
        !finite_positive(cam->gate_outer_half) || !finite_positive(cam->gate_half_depth))
        return render_fail("frame geometry needs 0 < gate_inner_half < gate_outer_half and gate_half_depth > 0");
    if (!(cam->noise_depth_coeff >= 0.f && cam->noise_depth_coeff <= 1e30f) ||
        !(cam->dropout >= 0.f && cam->dropout <= 1.f))
        return render_fail("noise_depth_coeff must be finite and >= 0, dropout in [0, 1]");
    if (cam->reserved != 0) return render_fail("reserved must be 0");
    if (n_views == 0) return MPPI_OK;
    if (!d_cam_poses || !d_depth || (n_gates > 0 && !d_gate_poses)) return render_fail("NULL pose or output pointer");

    RenderParams P{};
    P.W = cam->width;
    P.H = cam->height;
    P.n_views = n_views;
    P.n_gates = n_gates;
    P.segs = (P.W + kRtSegW - 1) / kRtSegW;
    P.bands = (P.H + kRtBandRows - 1) / kRtBandRows;
    if (static_cast<long long>(P.bands) * n_views > INT_MAX)
        return render_fail("n_views x row bands of an image exceeds the grid limit");
    P.fx = cam->fx;
    P.fy = cam->fy;
    P.inv_fx = 1.f / cam->fx;
    P.inv_fy = 1.f / cam->fy;
    P.cx = cam->cx;
    P.cy = cam->cy;
    P.max_range = cam->max_range;
    P.a_in = cam->gate_inner_half;
    P.a_out = cam->gate_outer_half;
    P.hd = cam->gate_half_depth;
    P.noise_c = cam->noise_depth_coeff;
    P.dropout = cam->dropout;
    P.key0 = static_cast<uint32_t>(cam->seed);
    P.key1 = static_cast<uint32_t>(cam->seed >> 32);
    P.frame = cam->frame;

    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const dim3 grid(static_cast<unsigned>(P.bands * n_views));
    const int vec_px = kRtPixPerLane % 4 == 0 ? 4 : kRtPixPerLane;
    const bool vec = (P.W % kRtPixPerLane == 0) && (reinterpret_cast<uintptr_t>(d_depth) % (4 * vec_px) == 0);
    if (vec)
        render_depth_kernel<true><<<grid, kRtThreads, 0, s>>>(P, d_cam_poses, d_gate_poses, d_depth);
    else
        render_depth_kernel<false><<<grid, kRtThreads, 0, s>>>(P, d_cam_poses, d_gate_poses, d_depth);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return render_fail("launch failed", MPPI_E_CUDA, e);
    return MPPI_OK;
}

extern "C" int mppi_sample_sdf_queries(const mppi_depth_camera* cam, int n_views, const float* d_cam_poses,
                                       int n_gates, const float* d_gate_poses, int n_points, float near_frac,
                                       float* d_points, float* d_labels, void* stream) {
    using namespace mppi;
    if (!cam) return render_fail("NULL camera");
    if (cam->width < 1 || cam->height < 1 || !finite_positive(cam->fx) || !finite_positive(cam->fy) ||
        !finite_positive(cam->max_range) || !(cam->max_range > 0.2f))
        return render_fail("camera size, focal lengths or max_range (> 0.2 m) out of range");
    if (!finite_positive(cam->gate_inner_half) || !(cam->gate_outer_half > cam->gate_inner_half) ||
        !finite_positive(cam->gate_half_depth))
        return render_fail("frame geometry needs 0 < gate_inner_half < gate_outer_half and gate_half_depth > 0");
    if (n_views < 0 || n_views > (1 << 24) || n_points < 1 || n_points > (1 << 20) ||
        static_cast<long long>(n_views) * n_points > (1LL << 31))
        return render_fail("n_views in [0, 2^24], n_points in [1, 2^20], n_views x n_points <= 2^31");
    if (n_gates < 1 || n_gates > MPPI_MAX_RENDER_GATES) return render_fail("n_gates out of [1, MPPI_MAX_RENDER_GATES]");
    if (!(near_frac >= 0.f && near_frac <= 1.f)) return render_fail("near_frac out of [0, 1]");
    if (n_views == 0) return MPPI_OK;
    if (!d_cam_poses || !d_gate_poses || !d_points || !d_labels) return render_fail("NULL pointer");
    RenderParams P{};
    P.W = cam->width;
    P.H = cam->height;
    P.n_views = n_views;
    P.n_gates = n_gates;
    P.inv_fx = 1.f / cam->fx;
    P.inv_fy = 1.f / cam->fy;
    P.cx = cam->cx;
    P.cy = cam->cy;
    P.max_range = cam->max_range;
    P.a_in = cam->gate_inner_half;
    P.a_out = cam->gate_outer_half;
    P.hd = cam->gate_half_depth;
    P.key0 = static_cast<uint32_t>(cam->seed);
    P.key1 = static_cast<uint32_t>(cam->seed >> 32);
    P.frame = cam->frame;
    const long long total = static_cast<long long>(n_views) * n_points;
    sample_queries_kernel<<<static_cast<unsigned>((total + 127) / 128), 128, 0, static_cast<cudaStream_t>(stream)>>>(
        P, d_cam_poses, d_gate_poses, n_points, near_frac, d_points, d_labels);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return render_fail("launch failed", MPPI_E_CUDA, e);
    return MPPI_OK;
}
