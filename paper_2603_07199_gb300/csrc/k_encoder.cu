// Depth encoder E_theta (Sec. III-B): depth images -> latent codes z, in the convolutional
// reading stated in include/mppi.h (4 stride-2 3x3 convolutions with ReLU, mean pool,
// linear head), for batches of images.
//
// Each convolution is a GEMM over (ci, ky, kx) with the input gathered on the fly
// (implicit im2col): all-channel x (4096 / CO)-pixel block tiles, 16-deep chunks staged
// in shared memory, 4 x 4 outputs per thread, and the reduction split over the blocks of
// a thread-block cluster, summed through distributed shared memory, when a layer has too
// few tiles to fill the GPU (small batches, deep layers).  Layers are programmatic dependent
// launches: a layer's grid launches while the previous one drains and waits for its output.
// Activations are NCHW in device memory (L2-resident at these sizes); the first
// layer scales the depths by 1 / max_range as it reads them.  The head (mean over
// pixels, 64 x 64 matrix) is one block per image.
#include <algorithm>
#include <cstdarg>
#include <cstdio>
#include <new>
#include <vector>

#include <cooperative_groups.h>

#include "encoder_internal.h"
#include "kernels.h"
#include "mppi.h"

namespace cg = cooperative_groups;

namespace mppi {
namespace {

constexpr int kEncLayers = 4;
constexpr int kEncChannels[kEncLayers] = {16, 32, 64, 64};
constexpr int kConvThreads = 256;
constexpr int kBK = 16;               // reduction (ci, ky, kx) per staged chunk
constexpr int kTile = 4096;           // CO x BN outputs per block tile (BN = 4096 / CO pixels)
constexpr int kMaxSplit = 8;          // portable cluster size
constexpr int kHeadThreads = 256;
constexpr int kLatent = MPPI_LATENT_DIM;

// One 3x3 stride-2 convolution as a GEMM  Y[co][p] = sum_k W[co][k] X[k][p]  over
// k = (ci, ky, kx) and p = (image, i, j).  A block computes all CO channels of
// BN = 4096 / CO consecutive output pixels, staging 16-deep chunks of W (transposed,
// [k][co]) and of the gathered input X ([k][p], zero outside the image) in shared
// memory; a thread accumulates 4 channels x 4 pixels (two 16-byte shared loads per 16
// FMA).  When a layer has too few tiles to fill the GPU, the reduction is split over
// the S blocks of a thread-block cluster (grid z): each block leaves its partial tile in
// its shared memory and, after a cluster barrier, every block sums a 1 / S share of the
// tile over the S partials (in rank order, through distributed shared memory), adds the
// bias, applies the ReLU and stores it.
template <int CI, int CO, bool kScaleInput>
__global__ void __launch_bounds__(kConvThreads) conv3x3s2_gemm_kernel(const float* __restrict__ x, int n_img, int H,
                                                                      int W, int Ho, int Wo,
                                                                      const float* __restrict__ wt,
                                                                      const float* __restrict__ bias, float scale,
                                                                      int chunks_per_slice, float* __restrict__ y) {
    constexpr int K = 9 * CI;
    constexpr int kChunks = (K + kBK - 1) / kBK;
    constexpr int kTco = CO / 4;                 // threads along channels
    constexpr int kTpx = kConvThreads / kTco;    // threads along pixels
    constexpr int BN = 4 * kTpx;                 // pixels per tile
    constexpr int kGR = kBK * BN / kConvThreads; // gathered rows per thread per chunk
    constexpr int kRS = kConvThreads / BN;       // their row stride
    static_assert(CO * BN == kTile, "tile");
    __shared__ __align__(16) float As[kBK][CO];
    __shared__ __align__(16) float Bs[kBK][BN];
    __shared__ __align__(16) float Cs[kTile];    // this block's partial tile [co][px] (split only)
    const int tpx = threadIdx.x % kTpx, tco = threadIdx.x / kTpx;
    const int hw = Ho * Wo;
    const long long P = static_cast<long long>(n_img) * hw;
    const long long p0 = static_cast<long long>(blockIdx.x) * BN;
    const int c_begin = blockIdx.z * chunks_per_slice;
    const int c_end = min(c_begin + chunks_per_slice, kChunks);
    float acc[4][4];
#pragma unroll
    for (int m = 0; m < 4; ++m)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[m][q] = 0.f;
    // this thread gathers pixel pp = tid % BN of the tile for rows kk = tid / BN + kRS r of each
    // chunk: its pixel is fixed, and (ci, tap) of each row advance by kBK per chunk
    const int pp = threadIdx.x % BN;
    const int kk0 = threadIdx.x / BN;
    const long long pg = p0 + pp;
    const bool pix_live = pg < P;
    int ii = 0, jj = 0;
    const float* xp = x;
    if (pix_live) {
        const int n = static_cast<int>(pg / hw);
        const int rem = static_cast<int>(pg - static_cast<long long>(n) * hw);
        ii = 2 * (rem / Wo);
        jj = 2 * (rem - (rem / Wo) * Wo);
        xp = x + static_cast<size_t>(n) * CI * H * W;
    }
    int ci_r[kGR], t_r[kGR];
#pragma unroll
    for (int r = 0; r < kGR; ++r) {
        const int k = c_begin * kBK + kk0 + kRS * r;
        ci_r[r] = k / 9;
        t_r[r] = k - 9 * (k / 9);
    }
    // software pipeline: the chunk after the current one is loaded into registers while the
    // current one is multiplied out of shared memory
    constexpr int kAR = CO * kBK / kConvThreads;           // weights staged per thread per chunk
    float a_reg[kAR], b_reg[kGR];
    auto load_chunk = [&](int ch) {
        const int k0 = ch * kBK;
#pragma unroll
        for (int r = 0; r < kAR; ++r) {
            const int e = threadIdx.x + r * kConvThreads;
            const int co = e / kBK, kk = e - co * kBK;
            a_reg[r] = (k0 + kk < K) ? __ldg(wt + co * K + k0 + kk) : 0.f;
        }
#pragma unroll
        for (int r = 0; r < kGR; ++r) {
            const int t = t_r[r];
            const int dy = ((t * 11) >> 5) - 1;              // t / 3 - 1 for t in [0, 9)
            const int dx = t - 3 * (dy + 1) - 1;
            const int yy = ii + dy, xx = jj + dx;
            float v = 0.f;
            if (pix_live && ci_r[r] < CI && yy >= 0 && yy < H && xx >= 0 && xx < W) {
                v = __ldg(xp + (static_cast<size_t>(ci_r[r]) * H + yy) * W + xx);
                if (kScaleInput) v *= scale;
            }
            b_reg[r] = v;
            // next chunk: k += 16 = 9 + 7
            t_r[r] += 7;
            ci_r[r] += 1;
            if (t_r[r] >= 9) {
                t_r[r] -= 9;
                ci_r[r] += 1;
            }
        }
    };
    // programmatic dependent launch: let the next layer's grid start launching, and wait for
    // the previous kernel's output (a no-op when launched without the attribute)
    pdl_trigger();
    pdl_wait();
    if (c_begin < c_end) load_chunk(c_begin);
    for (int ch = c_begin; ch < c_end; ++ch) {
        __syncthreads();
#pragma unroll
        for (int r = 0; r < kAR; ++r) {
            const int e = threadIdx.x + r * kConvThreads;
            As[e - (e / kBK) * kBK][e / kBK] = a_reg[r];
        }
#pragma unroll
        for (int r = 0; r < kGR; ++r) Bs[kk0 + kRS * r][pp] = b_reg[r];
        __syncthreads();
        if (ch + 1 < c_end) load_chunk(ch + 1);
#pragma unroll
        for (int kk = 0; kk < kBK; ++kk) {
            const float4 a = *reinterpret_cast<const float4*>(&As[kk][tco * 4]);
            const float4 b = *reinterpret_cast<const float4*>(&Bs[kk][tpx * 4]);
            const float av[4] = {a.x, a.y, a.z, a.w};
#pragma unroll
            for (int m = 0; m < 4; ++m) {
                acc[m][0] = fmaf(av[m], b.x, acc[m][0]);
                acc[m][1] = fmaf(av[m], b.y, acc[m][1]);
                acc[m][2] = fmaf(av[m], b.z, acc[m][2]);
                acc[m][3] = fmaf(av[m], b.w, acc[m][3]);
            }
        }
    }
    if (gridDim.z == 1) {
        // the 4 pixels of a thread are consecutive; with hw % 4 == 0 they lie in one image
        // and start on a 16-byte boundary of each channel plane
        const long long pq = p0 + tpx * 4;
        if (pq >= P) return;
        const int n = static_cast<int>(pq / hw);
        const int rem = static_cast<int>(pq - static_cast<long long>(n) * hw);
#pragma unroll
        for (int m = 0; m < 4; ++m) {
            const int co = tco * 4 + m;
            const float bb = bias[co];
            if ((hw & 3) == 0) {
                *reinterpret_cast<float4*>(y + (static_cast<size_t>(n) * CO + co) * hw + rem) =
                    make_float4(fmaxf(acc[m][0] + bb, 0.f), fmaxf(acc[m][1] + bb, 0.f), fmaxf(acc[m][2] + bb, 0.f),
                                fmaxf(acc[m][3] + bb, 0.f));
            } else {
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const long long p = pq + q;
                    if (p >= P) break;
                    const int nq = static_cast<int>(p / hw);
                    const int rq = static_cast<int>(p - static_cast<long long>(nq) * hw);
                    y[(static_cast<size_t>(nq) * CO + co) * hw + rq] = fmaxf(acc[m][q] + bb, 0.f);
                }
            }
        }
        return;
    }
    // ---- split reduction over the cluster (the S blocks of this tile)
#pragma unroll
    for (int m = 0; m < 4; ++m)
        *reinterpret_cast<float4*>(&Cs[(tco * 4 + m) * BN + tpx * 4]) =
            make_float4(acc[m][0], acc[m][1], acc[m][2], acc[m][3]);
    cg::cluster_group cluster = cg::this_cluster();
    cluster.sync();
    const int S = static_cast<int>(cluster.num_blocks());
    const int rank = static_cast<int>(cluster.block_rank());
    for (int e = rank * kConvThreads + threadIdx.x; e < kTile; e += S * kConvThreads) {
        float sum = 0.f;
        for (int q = 0; q < S; ++q) sum += cluster.map_shared_rank(Cs, q)[e];
        const int co = e / BN, pxi = e - co * BN;
        const long long p = p0 + pxi;
        if (p < P) {
            const int n = static_cast<int>(p / hw);
            const int rem = static_cast<int>(p - static_cast<long long>(n) * hw);
            y[(static_cast<size_t>(n) * CO + co) * hw + rem] = fmaxf(sum + bias[co], 0.f);
        }
    }
    cluster.sync();   // keep every block's partial tile alive until all shares are read
}

// z[n] = W5 mean_pixels(x4[n]) + b5, one block per image: W5 staged in shared memory; 4
// threads per channel sum interleaved pixels with 4 partial sums each; one thread per output.
__global__ void __launch_bounds__(kHeadThreads) encoder_head_kernel(const float* __restrict__ x4, int hw,
                                                                    const float* __restrict__ W5,
                                                                    const float* __restrict__ b5,
                                                                    float* __restrict__ z) {
    constexpr int kParts = kHeadThreads / kLatent;
    __shared__ float w_s[kLatent][kLatent + 1];
    __shared__ float part[kParts][kLatent];
    __shared__ float m[kLatent];
    const int n = blockIdx.x, c = threadIdx.x % kLatent, q = threadIdx.x / kLatent;
    for (int e = threadIdx.x; e < kLatent * kLatent; e += kHeadThreads) w_s[e / kLatent][e % kLatent] = W5[e];
    pdl_wait();
    const float* xc = x4 + (static_cast<size_t>(n) * kLatent + c) * hw;
    float s0 = 0.f, s1 = 0.f, s2 = 0.f, s3 = 0.f;
    int k = q;
    for (; k + 3 * kParts < hw; k += 4 * kParts) {
        s0 += xc[k];
        s1 += xc[k + kParts];
        s2 += xc[k + 2 * kParts];
        s3 += xc[k + 3 * kParts];
    }
    for (; k < hw; k += kParts) s0 += xc[k];
    part[q][c] = (s0 + s1) + (s2 + s3);
    __syncthreads();
    if (q == 0) {
        float t = 0.f;
#pragma unroll
        for (int r = 0; r < kParts; ++r) t += part[r][c];
        m[c] = t / static_cast<float>(hw);
    }
    __syncthreads();
    if (q == 0) {
        float acc = b5[c];
#pragma unroll 16
        for (int kk = 0; kk < kLatent; ++kk) acc = fmaf(w_s[c][kk], m[kk], acc);
        z[static_cast<size_t>(n) * kLatent + c] = acc;
    }
}

thread_local char g_enc_err[512] = "";

}  // namespace
}  // namespace mppi

namespace {

int efail(mppi_encoder* e, int code, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    std::snprintf(e ? e->err : mppi::g_enc_err, 512, "%s", buf);
    return code;
}

void encoder_free(mppi_encoder* e) {
    for (int l = 0; l < 4; ++l) {
        cudaFree(e->wt[l]);
        cudaFree(e->bias[l]);
        cudaFree(e->act[l]);
        cudaFree(e->wpack[l]);
        cudaFree(e->dgpack[l]);
    }
    cudaFree(e->W5);
    cudaFree(e->b5);
    cudaFree(e->d_err);
}

// Split the reduction so that a layer with few output tiles still puts about two blocks on
// every SM (at most kMaxSplit slices, at least one chunk each).
int conv_split(const mppi_encoder* e, long long tiles, int chunks) {
    const long long want = (2LL * e->n_sms + tiles - 1) / tiles;
    return static_cast<int>(std::max(1LL, std::min<long long>({want, static_cast<long long>(mppi::kMaxSplit),
                                                               static_cast<long long>(chunks)})));
}

template <int CI, int CO, bool kScale>
cudaError_t launch_conv(const mppi_encoder* e, int l, int n, const float* x, float scale, float* y) {
    constexpr int kChunks = (9 * CI + mppi::kBK - 1) / mppi::kBK;
    constexpr int BN = mppi::kTile / CO;
    const long long P = static_cast<long long>(n) * e->h[l + 1] * e->w[l + 1];
    const long long tiles = (P + BN - 1) / BN;
    int split = conv_split(e, tiles, kChunks);
    const int cps = (kChunks + split - 1) / split;
    split = (kChunks + cps - 1) / cps;                     // no empty slice
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(static_cast<unsigned>(tiles), 1, split);
    cfg.blockDim = dim3(mppi::kConvThreads);
    cfg.stream = e->stream;
    cudaLaunchAttribute attr[2];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    attr[1].id = cudaLaunchAttributeClusterDimension;
    attr[1].val.clusterDim.x = 1;
    attr[1].val.clusterDim.y = 1;
    attr[1].val.clusterDim.z = split;
    cfg.attrs = attr;
    cfg.numAttrs = split > 1 ? 2 : 1;
    return cudaLaunchKernelEx(&cfg, mppi::conv3x3s2_gemm_kernel<CI, CO, kScale>, x, n, e->h[l], e->w[l], e->h[l + 1],
                              e->w[l + 1], static_cast<const float*>(e->wt[l]), static_cast<const float*>(e->bias[l]),
                              scale, cps, y);
}

}  // namespace

extern "C" int mppi_encoder_create(int height, int width, int max_images, const float* const* layers, int n_arrays,
                                   void* stream, mppi_encoder** out) {
    using namespace mppi;
    if (!out) return efail(nullptr, MPPI_E_INVALID, "mppi_encoder_create: NULL out");
    *out = nullptr;
    if (height < 1 || height > MPPI_MAX_IMAGE_SIDE || width < 1 || width > MPPI_MAX_IMAGE_SIDE)
        return efail(nullptr, MPPI_E_INVALID, "mppi_encoder_create: height, width out of [1, MPPI_MAX_IMAGE_SIDE]");
    if (max_images < 1 || max_images > 65535)
        return efail(nullptr, MPPI_E_INVALID, "mppi_encoder_create: max_images out of [1, 65535]");
    if (!layers || n_arrays != 2 * MPPI_ENCODER_LAYERS)
        return efail(nullptr, MPPI_E_INVALID, "mppi_encoder_create: expected %d weight arrays", 2 * MPPI_ENCODER_LAYERS);
    for (int i = 0; i < n_arrays; ++i)
        if (!layers[i]) return efail(nullptr, MPPI_E_INVALID, "mppi_encoder_create: weight array %d is NULL", i);
    mppi_encoder* e = new (std::nothrow) mppi_encoder();
    if (!e) return efail(nullptr, MPPI_E_OOM, "mppi_encoder_create: host allocation failed");
    e->H = height;
    e->W = width;
    e->max_images = max_images;
    e->stream = static_cast<cudaStream_t>(stream);
    e->h[0] = height;
    e->w[0] = width;
    for (int l = 0; l < 4; ++l) {
        e->h[l + 1] = (e->h[l] + 1) / 2;
        e->w[l + 1] = (e->w[l] + 1) / 2;
    }
    auto alloc = [&](float** p, size_t n) { return cudaMalloc(p, n * sizeof(float)) == cudaSuccess; };
    bool ok = true;
    int ci = 1;
    for (int l = 0; l < 4 && ok; ++l) {
        const int co = kEncChannels[l];
        ok = alloc(&e->wt[l], static_cast<size_t>(ci) * 9 * co) && alloc(&e->bias[l], co) &&
             alloc(&e->act[l], static_cast<size_t>(max_images) * co * e->h[l + 1] * e->w[l + 1]);
        if (!ok) break;
        ok = cudaMemcpy(e->wt[l], layers[2 * l], static_cast<size_t>(ci) * 9 * co * sizeof(float),
                        cudaMemcpyHostToDevice) == cudaSuccess &&
             cudaMemcpy(e->bias[l], layers[2 * l + 1], co * sizeof(float), cudaMemcpyHostToDevice) == cudaSuccess;
        ci = co;
    }
    {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&e->n_sms, cudaDevAttrMultiProcessorCount, dev);
        if (e->n_sms < 1) e->n_sms = 1;
    }
    constexpr int kZ = MPPI_LATENT_DIM;
    ok = ok && cudaMalloc(&e->d_err, sizeof(int)) == cudaSuccess && cudaMemset(e->d_err, 0, sizeof(int)) == cudaSuccess &&
         configure_conv_tc() == cudaSuccess;
    for (int l = 0; l < 4 && ok; ++l) ok = cudaMalloc(&e->wpack[l], conv_tc_packed_bytes(l)) == cudaSuccess;
    for (int l = 1; l < 4 && ok; ++l) ok = cudaMalloc(&e->dgpack[l], conv_dgrad_tc_packed_bytes(l)) == cudaSuccess;
    ok = ok && pack_conv_tc_weights(e->wt, e->wpack, e->dgpack, e->stream) == cudaSuccess &&
         cudaStreamSynchronize(e->stream) == cudaSuccess;
    ok = ok && alloc(&e->W5, kZ * kZ) && alloc(&e->b5, kZ) &&
         cudaMemcpy(e->W5, layers[8], kZ * kZ * sizeof(float), cudaMemcpyHostToDevice) == cudaSuccess &&
         cudaMemcpy(e->b5, layers[9], kZ * sizeof(float), cudaMemcpyHostToDevice) == cudaSuccess;
    if (!ok) {
        const cudaError_t ce = cudaGetLastError();
        encoder_free(e);
        delete e;
        return efail(nullptr, ce == cudaErrorMemoryAllocation ? MPPI_E_OOM : MPPI_E_CUDA,
                     "mppi_encoder_create: device allocation or copy failed: %s", cudaGetErrorString(ce));
    }
    *out = e;
    return MPPI_OK;
}

extern "C" void mppi_encoder_destroy(mppi_encoder* e) {
    if (!e) return;
    cudaStreamSynchronize(e->stream);
    encoder_free(e);
    delete e;
}

extern "C" const char* mppi_encoder_last_error(const mppi_encoder* e) { return e ? e->err : mppi::g_enc_err; }

extern "C" int mppi_encode_depth(mppi_encoder* e, int n_images, const float* d_depth, float max_range,
                                 float* d_latents) {
    if (!e) return efail(nullptr, MPPI_E_INVALID, "mppi_encode_depth: NULL encoder");
    if (n_images < 0 || n_images > e->max_images)
        return efail(e, MPPI_E_INVALID, "mppi_encode_depth: n_images out of [0, max_images = %d]", e->max_images);
    if (!(max_range > 0.f && max_range <= 3.0e38f)) return efail(e, MPPI_E_INVALID, "mppi_encode_depth: max_range must be > 0");
    if (n_images == 0) return MPPI_OK;
    if (!d_depth || !d_latents) return efail(e, MPPI_E_INVALID, "mppi_encode_depth: NULL pointer");
    cudaError_t ce = cudaSuccess;
    if (e->conv_path == MPPI_ENC_CONV_TC) {
        const float* in = d_depth;
        for (int l = 0; l < 4 && ce == cudaSuccess; ++l) {
            ce = mppi::launch_conv_tc(l, in, n_images, e->h[l], e->w[l], e->h[l + 1], e->w[l + 1], e->wpack[l],
                                      e->bias[l], l == 0 ? 1.f / max_range : 1.f, e->act[l], e->d_err,
                                      l == 0 ? e->inject_timeout : 0, e->stream);
            in = e->act[l];
        }
        e->inject_timeout = 0;
    } else {
        ce = launch_conv<1, 16, true>(e, 0, n_images, d_depth, 1.f / max_range, e->act[0]);
        if (ce == cudaSuccess) ce = launch_conv<16, 32, false>(e, 1, n_images, e->act[0], 1.f, e->act[1]);
        if (ce == cudaSuccess) ce = launch_conv<32, 64, false>(e, 2, n_images, e->act[1], 1.f, e->act[2]);
        if (ce == cudaSuccess) ce = launch_conv<64, 64, false>(e, 3, n_images, e->act[2], 1.f, e->act[3]);
    }
    if (ce == cudaSuccess) {
        ce = mppi::launch_dependent(true, mppi::encoder_head_kernel, dim3(n_images), dim3(mppi::kHeadThreads), 0,
                                    e->stream, static_cast<const float*>(e->act[3]), e->h[4] * e->w[4],
                                    static_cast<const float*>(e->W5), static_cast<const float*>(e->b5), d_latents);
    }
    if (ce != cudaSuccess) return efail(e, MPPI_E_CUDA, "mppi_encode_depth: launch failed: %s", cudaGetErrorString(ce));
    return MPPI_OK;
}

extern "C" int mppi_encoder_set_conv_path(mppi_encoder* e, int path) {
    if (!e) return efail(nullptr, MPPI_E_INVALID, "mppi_encoder_set_conv_path: NULL encoder");
    if (path != MPPI_ENC_CONV_FP32 && path != MPPI_ENC_CONV_TC)
        return efail(e, MPPI_E_INVALID, "mppi_encoder_set_conv_path: unknown path %d", path);
    e->conv_path = path;
    return MPPI_OK;
}

extern "C" int mppi_encoder_check(mppi_encoder* e) {
    if (!e) return efail(nullptr, MPPI_E_INVALID, "mppi_encoder_check: NULL encoder");
    int word = 0;
    cudaError_t ce = cudaMemcpyAsync(&word, e->d_err, sizeof(int), cudaMemcpyDeviceToHost, e->stream);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(e->stream);
    if (ce != cudaSuccess) return efail(e, MPPI_E_CUDA, "mppi_encoder_check: %s", cudaGetErrorString(ce));
    if (word != 0) {
        ce = cudaMemsetAsync(e->d_err, 0, sizeof(int), e->stream);
        if (ce == cudaSuccess) ce = cudaStreamSynchronize(e->stream);
        if (ce != cudaSuccess) return efail(e, MPPI_E_CUDA, "mppi_encoder_check: %s", cudaGetErrorString(ce));
        return efail(e, MPPI_E_TIMEOUT, "a tensor-core convolution gave up waiting for its MMAs (device error word %d)",
                     word);
    }
    return MPPI_OK;
}

extern "C" int mppi_encoder_debug_inject_timeout(mppi_encoder* e) {
    if (!e) return efail(nullptr, MPPI_E_INVALID, "mppi_encoder_debug_inject_timeout: NULL encoder");
    if (e->conv_path != MPPI_ENC_CONV_TC)
        return efail(e, MPPI_E_INVALID, "mppi_encoder_debug_inject_timeout: the FP32 convolutions have no device waits");
    e->inject_timeout = 1;
    return MPPI_OK;
}
