// Depth images of the gate frames (the onboard observation of Sec. III-B) by exact
// ray casting, one thread per 4 consecutive pixels of a row, and the optional
// synthetic sensor noise of the denoising pre-training stage (I_noisy).
//
// Work split: a block renders a 128 x 8 pixel tile of one view (a warp per row,
// 4 pixels per lane, so each warp stores 512 contiguous bytes).  Its prologue
// turns every gate into 19 per-view constants -- the 10 slab numerators of the
// frame's planes (plane offset minus the camera position, in the gate frame)
// and the 3 columns of the camera -> gate rotation -- and keeps only the gates
// whose bounding sphere meets the tile's view frustum (a conservative cull:
// every plane of the frustum must pass within the sphere's radius), so a tile
// that sees no gate costs one store per pixel.  Per pixel and kept gate: the
// ray direction in the gate frame (3 FMA after a per-row part), three IEEE
// reciprocals, and the first point of the solid along the ray:
//     solid on the ray = [enter, leave] (the outer box |x| <= d, |y|, |z| <= a_out)
//                        minus the open interval (h0, h1) where |y|, |z| < a_in,
// the first such point at t >= 0 being s = max(enter, 0), or h1 when s falls in
// the opening (when h1 <= leave), or none.
#include <climits>
#include <cstdio>

#include "kernels.h"
#include "mppi.h"

namespace mppi {
namespace {

constexpr int kRtThreads = 256;
constexpr int kRtPixPerLane = 4;
constexpr int kRtTileW = 32 * kRtPixPerLane;   // 128 pixels
constexpr int kRtTileH = kRtThreads / 32;      // 8 rows
constexpr int kRtGateF4 = 5;                   // 19 constants (+1 pad) per gate as float4
constexpr uint32_t kDepthNoiseTag = 0xDE9750u;

struct RenderParams {
    int W, H, n_views, n_gates, tiles_x, tiles_per_view;
    float fx, fy, cx, cy, max_range;
    float a_in, a_out, hd, radius;   // frame geometry; bounding-sphere radius of a frame
    float noise_c, dropout;
    uint32_t key0, key1, frame;
    int noise;                       // 1: apply the sensor noise
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

// Does the sphere (centre c in the camera frame, radius r) meet the frustum of rays
// (1, a, b) t, t >= 0, a in [a_lo, a_hi], b in [b_lo, b_hi], before depth max_range?
__device__ __forceinline__ bool sphere_in_frustum(float cx, float cy, float cz, float r, float a_lo, float a_hi,
                                                  float b_lo, float b_hi, float max_range) {
    if (cx < -r || cx - r > max_range) return false;
    if (cy - a_hi * cx > r * sqrtf(1.f + a_hi * a_hi)) return false;
    if (a_lo * cx - cy > r * sqrtf(1.f + a_lo * a_lo)) return false;
    if (cz - b_hi * cx > r * sqrtf(1.f + b_hi * b_hi)) return false;
    if (b_lo * cx - cz > r * sqrtf(1.f + b_lo * b_lo)) return false;
    return true;
}

// First ray parameter t >= 0 of the frame solid on the ray with gate-frame direction d;
// num = {-d - ox, d - ox, -a_out - oy, a_out - oy, -a_in - oy, a_in - oy, (same for z)}.
__device__ __forceinline__ float ray_frame(const float* num, float dx, float dy, float dz) {
    const float ix = __frcp_rn(dx), iy = __frcp_rn(dy), iz = __frcp_rn(dz);
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

template <bool kVec>
__global__ void __launch_bounds__(kRtThreads) render_depth_kernel(RenderParams P, const float* __restrict__ cams,
                                                                  const float* __restrict__ gates,
                                                                  float* __restrict__ depth) {
    __shared__ float4 s_gate[MPPI_MAX_RENDER_GATES][kRtGateF4];
    __shared__ int s_n;
    const int view = blockIdx.x / P.tiles_per_view;
    const int tile = blockIdx.x - view * P.tiles_per_view;
    const int ty = tile / P.tiles_x, tx = tile - ty * P.tiles_x;
    const int u0 = tx * kRtTileW, v0 = ty * kRtTileH;
    if (threadIdx.x == 0) s_n = 0;
    __syncthreads();

    // ---- prologue: per-gate constants of this view, culled against the tile's frustum
    const float* cp = cams + static_cast<size_t>(view) * 7;
    if (threadIdx.x < P.n_gates) {
        const Mat3 Rc = quat_to_mat(cp[3], cp[4], cp[5], cp[6]);
        const float* gp = gates + threadIdx.x * 7;
        const Mat3 Rg = quat_to_mat(gp[3], gp[4], gp[5], gp[6]);
        const float dtx = gp[0] - cp[0], dty = gp[1] - cp[1], dtz = gp[2] - cp[2];
        // gate centre in the camera frame: Rc^T (t_g - t_c)
        const float ccx = Rc.m[0][0] * dtx + Rc.m[1][0] * dty + Rc.m[2][0] * dtz;
        const float ccy = Rc.m[0][1] * dtx + Rc.m[1][1] * dty + Rc.m[2][1] * dtz;
        const float ccz = Rc.m[0][2] * dtx + Rc.m[1][2] * dty + Rc.m[2][2] * dtz;
        const float a_hi = (P.cx - (static_cast<float>(u0) + 0.5f)) / P.fx;
        const float a_lo = (P.cx - (static_cast<float>(u0 + kRtTileW - 1) + 0.5f)) / P.fx;
        const float b_hi = (P.cy - (static_cast<float>(v0) + 0.5f)) / P.fy;
        const float b_lo = (P.cy - (static_cast<float>(v0 + kRtTileH - 1) + 0.5f)) / P.fy;
        if (sphere_in_frustum(ccx, ccy, ccz, P.radius, a_lo, a_hi, b_lo, b_hi, P.max_range)) {
            // camera origin in the gate frame: o = Rg^T (t_c - t_g); camera -> gate rotation M = Rg^T Rc
            const float ox = -(Rg.m[0][0] * dtx + Rg.m[1][0] * dty + Rg.m[2][0] * dtz);
            const float oy = -(Rg.m[0][1] * dtx + Rg.m[1][1] * dty + Rg.m[2][1] * dtz);
            const float oz = -(Rg.m[0][2] * dtx + Rg.m[1][2] * dty + Rg.m[2][2] * dtz);
            float M[3][3];
#pragma unroll
            for (int i = 0; i < 3; ++i)
#pragma unroll
                for (int j = 0; j < 3; ++j)
                    M[i][j] = Rg.m[0][i] * Rc.m[0][j] + Rg.m[1][i] * Rc.m[1][j] + Rg.m[2][i] * Rc.m[2][j];
            const int slot = atomicAdd(&s_n, 1);
            s_gate[slot][0] = make_float4(-P.hd - ox, P.hd - ox, -P.a_out - oy, P.a_out - oy);
            s_gate[slot][1] = make_float4(-P.a_in - oy, P.a_in - oy, -P.a_out - oz, P.a_out - oz);
            s_gate[slot][2] = make_float4(-P.a_in - oz, P.a_in - oz, M[0][0], M[1][0]);
            s_gate[slot][3] = make_float4(M[2][0], M[0][1], M[1][1], M[2][1]);
            s_gate[slot][4] = make_float4(M[0][2], M[1][2], M[2][2], 0.f);
        }
    }
    __syncthreads();

    const int lane = threadIdx.x & 31, v = v0 + (threadIdx.x >> 5);
    if (v >= P.H) return;
    const int ub = u0 + lane * kRtPixPerLane;
    if (ub >= P.W) return;
    const float b = -((static_cast<float>(v) + 0.5f) - P.cy) / P.fy;
    float a[kRtPixPerLane], best[kRtPixPerLane];
#pragma unroll
    for (int j = 0; j < kRtPixPerLane; ++j) {
        a[j] = -((static_cast<float>(ub + j) + 0.5f) - P.cx) / P.fx;
        best[j] = __int_as_float(0x7f800000);
    }
    const int n_keep = s_n;
    for (int i = 0; i < n_keep; ++i) {
        float num[10];
        const float4 g0 = s_gate[i][0], g1 = s_gate[i][1], g2 = s_gate[i][2], g3 = s_gate[i][3], g4 = s_gate[i][4];
        num[0] = g0.x; num[1] = g0.y; num[2] = g0.z; num[3] = g0.w;
        num[4] = g1.x; num[5] = g1.y; num[6] = g1.z; num[7] = g1.w;
        num[8] = g2.x; num[9] = g2.y;
        // gate-frame direction M (1, a, b): the row part e = M e_x + b M e_z, then + a M e_y
        const float ex = fmaf(b, g4.x, g2.z), ey = fmaf(b, g4.y, g2.w), ez = fmaf(b, g4.z, g3.x);
#pragma unroll
        for (int j = 0; j < kRtPixPerLane; ++j)
            best[j] = fminf(best[j], ray_frame(num, fmaf(a[j], g3.y, ex), fmaf(a[j], g3.z, ey), fmaf(a[j], g3.w, ez)));
    }

    float out[kRtPixPerLane];
#pragma unroll
    for (int j = 0; j < kRtPixPerLane; ++j) {
        float z = best[j] <= P.max_range ? best[j] : P.max_range;
        if (P.noise) {
            const uint32_t pix = static_cast<uint32_t>(v) * static_cast<uint32_t>(P.W) + static_cast<uint32_t>(ub + j);
            const uint4 w = philox4x32_10(make_uint4(pix, static_cast<uint32_t>(view), P.frame, kDepthNoiseTag),
                                          P.key0, P.key1);
            if (word_to_uniform(w.z) < P.dropout) {
                z = 0.f;
            } else if (z < P.max_range) {
                const float n = box_muller(word_to_uniform(w.x), word_to_uniform(w.y)).x;
                z = fminf(fmaxf(fmaf(P.noise_c * z * z, n, z), 0.f), P.max_range);
            }
        }
        out[j] = z;
    }
    float* row = depth + (static_cast<size_t>(view) * P.H + v) * P.W;
    if (kVec) {
        __stcs(reinterpret_cast<float4*>(row + ub), make_float4(out[0], out[1], out[2], out[3]));
    } else {
#pragma unroll
        for (int j = 0; j < kRtPixPerLane; ++j)
            if (ub + j < P.W) __stcs(row + ub + j, out[j]);
    }
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
    P.tiles_x = (P.W + kRtTileW - 1) / kRtTileW;
    P.tiles_per_view = P.tiles_x * ((P.H + kRtTileH - 1) / kRtTileH);
    if (static_cast<long long>(P.tiles_per_view) * n_views > INT_MAX)
        return render_fail("n_views x tiles of an image exceeds the grid limit");
    P.fx = cam->fx;
    P.fy = cam->fy;
    P.cx = cam->cx;
    P.cy = cam->cy;
    P.max_range = cam->max_range;
    P.a_in = cam->gate_inner_half;
    P.a_out = cam->gate_outer_half;
    P.hd = cam->gate_half_depth;
    // bounding sphere of the frame, widened so that FP32 rounding in the cull never drops a gate
    P.radius = sqrtf(2.f * P.a_out * P.a_out + P.hd * P.hd) * 1.001f + 1e-3f;
    P.noise_c = cam->noise_depth_coeff;
    P.dropout = cam->dropout;
    P.key0 = static_cast<uint32_t>(cam->seed);
    P.key1 = static_cast<uint32_t>(cam->seed >> 32);
    P.frame = cam->frame;
    P.noise = (cam->noise_depth_coeff > 0.f || cam->dropout > 0.f) ? 1 : 0;

    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const dim3 grid(static_cast<unsigned>(P.tiles_per_view * n_views));
    const bool vec = (P.W % 4 == 0) && (reinterpret_cast<uintptr_t>(d_depth) % 16 == 0);
    if (vec)
        render_depth_kernel<true><<<grid, kRtThreads, 0, s>>>(P, d_cam_poses, d_gate_poses, d_depth);
    else
        render_depth_kernel<false><<<grid, kRtThreads, 0, s>>>(P, d_cam_poses, d_gate_poses, d_depth);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return render_fail("launch failed", MPPI_E_CUDA, e);
    return MPPI_OK;
}
