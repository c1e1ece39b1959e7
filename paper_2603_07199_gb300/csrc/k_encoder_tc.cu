// Depth-encoder convolutions (Sec. III-B, the convolutional reading of E_theta stated in
// include/mppi.h) on the Blackwell tensor cores: the forward pass (conv3x3s2_tc_kernel), the
// weight gradients (conv_wgrad_tc_kernel) and the input gradients (conv_dgrad_tc_kernel) of the
// encoder's training.  Every contraction runs as tcgen05.mma kind::f16 on BF16 operand splits:
// each FP32 value v is stored as v_hi = bf16(v) and v_lo = bf16(v - v_hi), and per 16-deep slice
// one thread issues the three products A_hi B_hi + A_hi B_lo + A_lo B_hi into an FP32 TMEM
// accumulator (the dropped A_lo B_lo and the split's own rounding are ~2^-16 of each product:
// the accuracy of the FP32 path's reading of the encoder).  Operands are K-major, no swizzle,
// in 8 x 16-byte core matrices (stage_offset).
//
// Forward: Y[p][co] = sum_k X[p][k] W'[co][k] over the output pixels p = (image, i, j) and the
// reduction index k = t CI + ci, tap-major (t = 3 ky + kx), so that for CI >= 8 every 8
// consecutive k share one tap: X[p][k] = x[ci][2i + ky - 1][2j + kx - 1] (zero outside the image)
// is gathered on the fly from the NCHW input at one precomputed offset per tap, W'[co][k] =
// W[co][ci][ky][kx] comes from the weights' packed hi / lo stages (pack_conv_weights_kernel,
// refreshed whenever the weights change) by one bulk copy per CTA.  A CTA owns 128 consecutive
// output pixels (M = 128, one TMEM lane each) and all CO channels (N = CO); two threads share
// each pixel row, each gathering half of a stage's KS columns; two stage buffers, the next
// stage's loads in flight while the current one is stored and its MMAs issued and committed to
// the buffer's mbarrier.  Layers with few output tiles split their stages over the kSplit CTAs
// of a thread-block cluster, whose partial accumulators meet through distributed shared memory
// in rank order.  The epilogue adds the bias, applies the ReLU and writes NCHW FP32 (the
// activations the head and the trainer read); a warp's stores of one channel are 32 consecutive
// pixels.
//
// Every wait is bounded (tc::kWaitLimitNs of %globaltimer): on timeout a kernel sets
// *err = kDevErrTimeout, lets its issued MMAs and copies finish, still takes part in every
// cluster barrier, frees TMEM and returns.
#include <cooperative_groups.h>

#include "encoder_internal.h"
#include "kernels.h"
#include "mppi.h"
#include "tc.cuh"

namespace cg = cooperative_groups;

namespace mppi {
namespace {

constexpr int kEtThreads = 256;   // two threads per tile row: thread t -> row t % 128, half t / 128
constexpr int kEtRows = 128;      // output pixels per CTA (M)

template <int CI, int CO, int kSplit>
struct ConvTcShape {
    static constexpr int K = 9 * CI;                          // reduction length
    static constexpr int Kp = (K + 15) / 16 * 16;             // padded to whole MMA slices
    static constexpr int KS = (Kp % 48 == 0) ? 48 : 16;       // reduction columns per stage
    static constexpr int kStages = Kp / KS;
    static constexpr int kStagesPerCta = kStages / kSplit;
    static constexpr int kHalfCols = KS / 2;                  // columns a thread gathers per stage
    static constexpr uint32_t kAHalf = kEtRows * KS * 2;      // one BF16 half of the X stage
    static constexpr uint32_t kBHalf = CO * KS * 2;           // one BF16 half of the W stage
    static constexpr uint32_t kBuf = 2 * kAHalf;              // X_hi, X_lo of one stage
    static constexpr uint32_t kBStage = 2 * kBHalf;           // W_hi, W_lo of one stage (packed layout)
    static constexpr uint32_t kBBytes = kStagesPerCta * kBStage;  // the CTA's weights, resident
    static constexpr uint32_t kHead = 1024;                   // barriers, TMEM base, flag, bias
    static constexpr uint32_t kSmem = kHead + 2 * kBuf + kBBytes;
    static constexpr uint32_t kTmemCols = CO <= 32 ? 32 : CO; // a power of two >= 32
    static constexpr uint32_t kSbo = KS * 16;                 // bytes between 8-row groups
    static constexpr int kBChunks = CO * KS / 8;              // 8-column weight chunks per stage
    static_assert(CO % 16 == 0 && CO <= 256, "N of an M = 128 MMA");
    static_assert(CO * 4 + 64 <= kHead, "bias area");
    static_assert(kStages % kSplit == 0, "whole stages per CTA of a split");
    static_assert(CI % 8 == 0 || CI == 1, "8-column chunks of one tap, or the single-channel layer");
    static_assert(kHalfCols % 8 == 0, "whole chunks per thread");
    static_assert(kSplit == 1 || CO * kEtRows * 4 <= 2 * kBuf, "partial tile fits the X buffers");
    static_assert(kBBytes % 16 == 0 && kBBytes < (1u << 20), "one bulk copy, within an mbarrier's tx count");
};

// Packed weights of one layer: for every stage, W'_hi then W'_lo ([CO][KS] BF16 in the operand
// layout of stage_offset), so that the kSplit CTAs' stage ranges are contiguous byte ranges.
template <int CI, int CO>
constexpr size_t packed_bytes() {
    return static_cast<size_t>(ConvTcShape<CI, CO, 1>::kStages) * ConvTcShape<CI, CO, 1>::kBStage;
}

// Byte offset of (row, col) in a [rows][KS] K-major operand stage (8 x 8 core matrices of
// 128 contiguous bytes: LBO 128 B along K, SBO 16 KS B along rows).  col a multiple of 8.
template <int KS>
__device__ __forceinline__ uint32_t stage_offset(int row, int col) {
    return static_cast<uint32_t>((row >> 3) * (KS * 16) + (col >> 3) * 128 + (row & 7) * 16);
}

// Eight FP32 values -> their BF16 hi halves and lo remainders, stored as one 16-byte core
// matrix row each.
__device__ __forceinline__ void store_split8(uint32_t hi_addr, uint32_t lo_addr, const float* v) {
    uint32_t h[4], l[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        h[q] = tc::pack_bf16x2(v[2 * q], v[2 * q + 1]);
        const float r0 = v[2 * q] - __uint_as_float(h[q] << 16);
        const float r1 = v[2 * q + 1] - __uint_as_float(h[q] & 0xFFFF0000u);
        l[q] = tc::pack_bf16x2(r0, r1);
    }
    tc::st_shared_v4(hi_addr, h[0], h[1], h[2], h[3]);
    tc::st_shared_v4(lo_addr, l[0], l[1], l[2], l[3]);
}

// 32 lanes x 8 consecutive 32-bit columns (thread i: lane i, columns [col, col + 8)).
__device__ __forceinline__ void tmem_ld_32x32b_x8(uint32_t taddr, uint32_t (&r)[8]) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                 : "r"(taddr));
}

// The tap's entry of a 9-entry register table (t < 9 at run time; a select chain keeps the table
// in registers).
__device__ __forceinline__ int tap_pick(const int (&tab)[9], int t) {
    int r = tab[8];
#pragma unroll
    for (int q = 7; q >= 0; --q) r = (t == q) ? tab[q] : r;
    return r;
}

// One bulk (non-tensor) copy global -> this CTA's shared memory, completing on an mbarrier that
// expects its bytes (addresses 16-byte aligned, size a multiple of 16).
__device__ __forceinline__ void bulk_load(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 ::"r"(dst), "l"(src), "r"(bytes), "r"(bar)
                 : "memory");
}

// W'[co][k] = W[co][ci][t] for k = t CI + ci (tap-major), split into BF16 hi / lo in the packed
// layout; one thread per 8-column chunk (stage, co, c8).
template <int CI, int CO>
__global__ void __launch_bounds__(256) pack_conv_weights_kernel(const float* __restrict__ wt, uint8_t* __restrict__ out) {
    using S = ConvTcShape<CI, CO, 1>;
    constexpr int KS = S::KS;
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= S::kStages * S::kBChunks) return;
    const int s = e / S::kBChunks, r = e - s * S::kBChunks;
    const int co = r / (KS / 8), c = (r - co * (KS / 8)) * 8;
    float v[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        const int k = s * KS + c + q;
        const int t = k / CI, ci = k - t * CI;
        v[q] = (k < S::K) ? wt[(static_cast<size_t>(co) * CI + ci) * 9 + t] : 0.f;
    }
    uint32_t h[4], l[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        h[q] = tc::pack_bf16x2(v[2 * q], v[2 * q + 1]);
        l[q] = tc::pack_bf16x2(v[2 * q] - __uint_as_float(h[q] << 16), v[2 * q + 1] - __uint_as_float(h[q] & 0xFFFF0000u));
    }
    uint8_t* st = out + static_cast<size_t>(s) * S::kBStage + stage_offset<KS>(co, c);
    *reinterpret_cast<uint4*>(st) = make_uint4(h[0], h[1], h[2], h[3]);
    *reinterpret_cast<uint4*>(st + S::kBHalf) = make_uint4(l[0], l[1], l[2], l[3]);
}

template <int CI, int CO, bool kScale, int kSplit>
__global__ void __launch_bounds__(kEtThreads) conv3x3s2_tc_kernel(const float* __restrict__ x, int n_img, int H,
                                                                  int W, int Ho, int Wo,
                                                                  const uint8_t* __restrict__ wpack,
                                                                  const float* __restrict__ bias, float scale,
                                                                  float* __restrict__ y, int* err, int inject) {
    using S = ConvTcShape<CI, CO, kSplit>;
    constexpr int KS = S::KS;
    extern __shared__ __align__(1024) uint8_t smem[];
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem);                 // [2] MMAs done with X buffer
    uint64_t* bar_w = reinterpret_cast<uint64_t*>(smem + 32);          // the weights have arrived
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(smem + 16);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(smem + 20);
    float* bias_s = reinterpret_cast<float*>(smem + 64);
    const int tid = threadIdx.x, warp = tid >> 5;
    const int row = tid & (kEtRows - 1), half = tid >> 7;

    if (warp == 0) {
        tc::tmem_alloc(tc::smem_u32(tmem_slot), S::kTmemCols);
        tc::tmem_relinquish();
    }
    if (tid == 0) {
        tc::mbar_init(tc::smem_u32(&bar[0]), 1);
        tc::mbar_init(tc::smem_u32(&bar[1]), 1);
        tc::mbar_init(tc::smem_u32(bar_w), 1);
        *abort_flag = 0;
        tc::mbar_fence_init();
    }
    // the weights may have been written by the preceding kernel (an optimiser step and the
    // repacking after it), the input by the previous layer: every global read comes after the wait
    pdl_trigger();
    pdl_wait();
    const uint32_t bres = tc::smem_u32(smem + S::kHead + 2 * S::kBuf);
    if (tid == 0)   // this CTA's stage range of the packed weights, one bulk copy
        bulk_load(bres, wpack + static_cast<size_t>(blockIdx.z) * S::kBBytes, S::kBBytes, tc::smem_u32(bar_w));
    for (int i = tid; i < CO; i += kEtThreads) bias_s[i] = bias[i];
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = *tmem_slot;

    // this thread's output pixel and the input offset and validity of each of its nine taps
    const int hw = Ho * Wo;
    const long long P = static_cast<long long>(n_img) * hw;
    const long long p = static_cast<long long>(blockIdx.x) * kEtRows + row;
    const bool live = p < P;
    int n = 0, rem = 0;
    int toff[9];
    uint32_t tvalid = 0;
    {
        int iy0 = 0, ix0 = 0;
        if (live) {
            n = static_cast<int>(p / hw);
            rem = static_cast<int>(p - static_cast<long long>(n) * hw);
            iy0 = 2 * (rem / Wo) - 1;
            ix0 = 2 * (rem - (rem / Wo) * Wo) - 1;
        }
#pragma unroll
        for (int t = 0; t < 9; ++t) {
            const int yy = iy0 + t / 3, xx = ix0 + t % 3;
            const bool v = live && yy >= 0 && yy < H && xx >= 0 && xx < W;
            toff[t] = v ? yy * W + xx : 0;
            tvalid |= (v ? 1u : 0u) << t;
        }
    }
    const float* xn = x + static_cast<size_t>(n) * CI * H * W;
    const size_t plane = static_cast<size_t>(H) * W;
    const uint32_t buf0 = tc::smem_u32(smem + S::kHead);
    constexpr uint32_t kIdesc = tc::idesc_bf16_f32(kEtRows, CO);
    const int s_begin = static_cast<int>(blockIdx.z) * S::kStagesPerCta;

    // this thread's half of its row for stage s (inputs, tap-major k)
    auto gather = [&](int s, float (&a)[S::kHalfCols]) {
#pragma unroll
        for (int c8 = 0; c8 < S::kHalfCols; c8 += 8) {
            const int k0 = s * KS + half * S::kHalfCols + c8;
            if constexpr (CI % 8 == 0) {
                const int t = k0 / CI, ci0 = k0 - t * CI;        // one tap, 8 consecutive channels
                const bool v = (tvalid >> t) & 1u;
                const float* src = xn + static_cast<size_t>(ci0) * plane + tap_pick(toff, t);
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    float val = v ? __ldg(src + static_cast<size_t>(q) * plane) : 0.f;
                    if (kScale) val *= scale;
                    a[c8 + q] = val;
                }
            } else {
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    const int t = k0 + q;                          // CI = 1: k is the tap
                    float val = (t < 9 && ((tvalid >> t) & 1u)) ? __ldg(xn + tap_pick(toff, t)) : 0.f;
                    if (kScale) val *= scale;
                    a[c8 + q] = val;
                }
            }
        }
    };

    bool ok = true;
    int last_commit = -1;   // thread 0: local stage of its last commit
    float a_next[S::kHalfCols];
    gather(s_begin, a_next);
#pragma unroll 1
    for (int sl = 0; sl < S::kStagesPerCta; ++sl) {
        const uint32_t buf = buf0 + static_cast<uint32_t>(sl & 1) * S::kBuf;
        float a[S::kHalfCols];
#pragma unroll
        for (int c = 0; c < S::kHalfCols; ++c) a[c] = a_next[c];
        // the next stage's loads are in flight while this one is stored and issued
        if (sl + 1 < S::kStagesPerCta) gather(s_begin + sl + 1, a_next);
        // the MMAs two stages back must be done with this buffer
        if (sl >= 2) ok = tc::mbar_wait_bounded(tc::smem_u32(&bar[sl & 1]), static_cast<uint32_t>(((sl - 2) >> 1) & 1),
                                                abort_flag, err, kDevErrTimeout);
        if (!__syncthreads_and(ok)) {
            ok = false;
            break;
        }
#pragma unroll
        for (int c8 = 0; c8 < S::kHalfCols; c8 += 8) {
            const uint32_t off = stage_offset<KS>(row, half * S::kHalfCols + c8);
            store_split8(buf + off, buf + S::kAHalf + off, a + c8);
        }
        tc::fence_proxy_async_smem();
        tc::fence_before_sync();
        __syncthreads();
        if (tid == 0) {
            tc::fence_after_sync();
            // the weights' bulk copy must have landed before the first MMA reads them (a test hook
            // waits for a phase that never completes instead, so that the bounded wait runs out)
            const bool go = sl > 0 || tc::mbar_wait_bounded(tc::smem_u32(bar_w), inject ? 1u : 0u, abort_flag, err,
                                                            kDevErrTimeout);
            if (!go) ok = false;   // every thread sees the flag it set at its next wait
            if (go) {
                const uint32_t wb = bres + static_cast<uint32_t>(sl) * S::kBStage;
#pragma unroll
                for (int j = 0; j < KS / 16; ++j) {
                    const uint32_t dj = static_cast<uint32_t>(256 * j);
                    const uint64_t ahi = tc::smem_desc(buf + dj, 128, S::kSbo);
                    const uint64_t alo = tc::smem_desc(buf + S::kAHalf + dj, 128, S::kSbo);
                    const uint64_t bhi = tc::smem_desc(wb + dj, 128, S::kSbo);
                    const uint64_t blo = tc::smem_desc(wb + S::kBHalf + dj, 128, S::kSbo);
                    tc::mma_bf16(tmem, ahi, bhi, kIdesc, (sl > 0 || j > 0) ? 1u : 0u);
                    tc::mma_bf16(tmem, ahi, blo, kIdesc, 1u);
                    tc::mma_bf16(tmem, alo, bhi, kIdesc, 1u);
                }
                tc::mma_commit(tc::smem_u32(&bar[sl & 1]));
                last_commit = sl;
            }
        }
    }
    // the last stage's commit covers every MMA issued before it
    constexpr int kLast = S::kStagesPerCta - 1;
    if (ok) ok = tc::mbar_wait_bounded(tc::smem_u32(&bar[kLast & 1]), static_cast<uint32_t>((kLast >> 1) & 1),
                                       abort_flag, err, kDevErrTimeout);
    ok = __syncthreads_and(ok);
    if (!ok && tid == 0) {
        // give up: let the MMAs already issued and the weights' copy finish before TMEM and
        // shared memory are reused
        int dummy = 0;
        if (last_commit >= 0)
            tc::mbar_wait_bounded(tc::smem_u32(&bar[last_commit & 1]), static_cast<uint32_t>((last_commit >> 1) & 1),
                                  &dummy, err, kDevErrTimeout);
        tc::mbar_wait_bounded(tc::smem_u32(bar_w), 0u, &dummy, err, kDevErrTimeout);
    }
    tc::fence_after_sync();
    // this thread's accumulator columns: TMEM lanes of warp % 4, columns [half CO / 2, + CO / 2)
    const uint32_t lane_addr = tmem + (static_cast<uint32_t>((warp & 3) * 32) << 16);
    constexpr int kHalfCo = CO / 2;
    if constexpr (kSplit == 1) {
        if (ok) {
            float* yo = y + static_cast<size_t>(n) * CO * hw + rem;
#pragma unroll
            for (int c0 = half * kHalfCo; c0 < (half + 1) * kHalfCo; c0 += 8) {
                uint32_t v[8];
                tmem_ld_32x32b_x8(lane_addr + static_cast<uint32_t>(c0), v);
                tc::tmem_wait_ld();
                if (live) {
#pragma unroll
                    for (int q = 0; q < 8; ++q)
                        yo[static_cast<size_t>(c0 + q) * hw] = fmaxf(__uint_as_float(v[q]) + bias_s[c0 + q], 0.f);
                }
            }
        }
    } else {
        // partial tile [co][row] in this CTA's operand buffers (all its MMAs are done)
        float* part = reinterpret_cast<float*>(smem + S::kHead);
#pragma unroll
        for (int c0 = half * kHalfCo; c0 < (half + 1) * kHalfCo; c0 += 8) {
            uint32_t v[8];
            tmem_ld_32x32b_x8(lane_addr + static_cast<uint32_t>(c0), v);
            tc::tmem_wait_ld();
#pragma unroll
            for (int q = 0; q < 8; ++q) part[(c0 + q) * kEtRows + row] = ok ? __uint_as_float(v[q]) : 0.f;
        }
        cg::cluster_group cluster = cg::this_cluster();
        cluster.sync();
        const int rank = static_cast<int>(cluster.block_rank());
        for (int e = rank * kEtThreads + tid; e < CO * kEtRows; e += kSplit * kEtThreads) {
            float sum = 0.f;
#pragma unroll
            for (int q = 0; q < kSplit; ++q) sum += cluster.map_shared_rank(part, q)[e];
            const int co = e / kEtRows, r = e - co * kEtRows;
            const long long pe = static_cast<long long>(blockIdx.x) * kEtRows + r;
            if (pe < P) {
                const int ne = static_cast<int>(pe / hw);
                const int re = static_cast<int>(pe - static_cast<long long>(ne) * hw);
                y[(static_cast<size_t>(ne) * CO + co) * hw + re] = fmaxf(sum + bias_s[co], 0.f);
            }
        }
        cluster.sync();   // keep every block's partial tile alive until all shares are read
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) {
        tc::fence_after_sync();
        tc::tmem_dealloc(tmem, S::kTmemCols);
    }
}

// ---------------------------------------------------------------- weight gradients
// Partial sums over a slice of output pixels of the weight gradient of one convolution as the
// GEMM  D[k][co] = sum_p X[p][k] delta[p][co]  (M = 128 rows of k = ci 9 + t, the weights' own
// order, with the ones row k = 9 CI giving the bias gradient; N = CO; the reduction over pixels
// p in stages of kWgStage), both operands K-major (pixels contiguous): row k of the X stage holds
// X[p][k] for the stage's 64 pixels (gathered from the NCHW input of the layer), row co of the
// delta stage delta[n][co][i][j] of the same pixels.  The same BF16 hi/lo split and three
// products as the forward pass, two stage buffers, one commit per stage.  Each CTA writes its
// slice's partial D to ws[slice][co][k] (k < 9 CI + 1); the caller sums the slices in order.
constexpr int kWgStage = 64;   // pixels per stage
constexpr int kWgRows = 128;   // k rows per CTA (M)

template <int CI, int CO>
struct WgradShape {
    static constexpr int K1 = 9 * CI + 1;
    static constexpr uint32_t kXHalf = kWgRows * kWgStage * 2;
    static constexpr uint32_t kDHalf = CO * kWgStage * 2;
    static constexpr uint32_t kBuf = 2 * kXHalf + 2 * kDHalf;
    static constexpr uint32_t kHead = 1024;
    static constexpr uint32_t kSmem = kHead + 2 * kBuf;
    static constexpr uint32_t kTmemCols = CO <= 32 ? 32 : CO;
    static constexpr uint32_t kSbo = kWgStage * 16;
    static constexpr int kXTasks = kWgRows * kWgStage / 8 / kEtThreads;       // 8-pixel chunks per thread
    static constexpr int kDTasks = (CO * kWgStage / 8 + kEtThreads - 1) / kEtThreads;
    static_assert(kXTasks * kEtThreads * 8 == kWgRows * kWgStage, "whole X chunks per thread");
};

// Flat output pixel p -> (image n, row i, column j) of an Ho x Wo output; advanced one pixel at a
// time without divisions.
struct PixCursor {
    int n, i, j;
    __device__ __forceinline__ void start(long long p, int hw, int Wo) {
        n = static_cast<int>(p / hw);
        const int rem = static_cast<int>(p - static_cast<long long>(n) * hw);
        i = rem / Wo;
        j = rem - i * Wo;
    }
    __device__ __forceinline__ void next(int Ho, int Wo) {
        if (++j == Wo) {
            j = 0;
            if (++i == Ho) {
                i = 0;
                ++n;
            }
        }
    }
};

template <int CI, int CO, bool kScale>
__global__ void __launch_bounds__(kEtThreads) conv_wgrad_tc_kernel(const float* __restrict__ x,
                                                                   const float* __restrict__ delta, int n_img, int H,
                                                                   int W, int Ho, int Wo, float scale,
                                                                   int stages_per_slice, float* __restrict__ ws,
                                                                   int* err) {
    using S = WgradShape<CI, CO>;
    extern __shared__ __align__(1024) uint8_t smem[];
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem);
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(smem + 16);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(smem + 20);
    const int tid = threadIdx.x, warp = tid >> 5;
    if (warp == 0) {
        tc::tmem_alloc(tc::smem_u32(tmem_slot), S::kTmemCols);
        tc::tmem_relinquish();
    }
    if (tid == 0) {
        tc::mbar_init(tc::smem_u32(&bar[0]), 1);
        tc::mbar_init(tc::smem_u32(&bar[1]), 1);
        *abort_flag = 0;
        tc::mbar_fence_init();
    }
    pdl_trigger();
    pdl_wait();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = *tmem_slot;
    const int hw = Ho * Wo;
    const long long P = static_cast<long long>(n_img) * hw;
    const long long n_stages = (P + kWgStage - 1) / kWgStage;
    const long long s_begin = static_cast<long long>(blockIdx.y) * stages_per_slice;
    const int n_local = static_cast<int>(max(0LL, min(static_cast<long long>(stages_per_slice), n_stages - s_begin)));
    const int k_base = blockIdx.x * kWgRows;
    const size_t plane = static_cast<size_t>(H) * W;
    const uint32_t buf0 = tc::smem_u32(smem + S::kHead);
    constexpr uint32_t kIdesc = tc::idesc_bf16_f32(kWgRows, CO);

    // X chunks: task -> row r (8 consecutive rows per quarter warp), 8-pixel chunk c; delta chunks:
    // task -> row co, 8-pixel chunk c (a quarter warp: eight rows of one chunk)
    auto gather = [&](int sl, float (&xv)[S::kXTasks][8], float (&dv)[S::kDTasks][8]) {
        const long long p0 = (s_begin + sl) * kWgStage;
#pragma unroll
        for (int u = 0; u < S::kXTasks; ++u) {
            const int task = tid + u * kEtThreads;
            const int r = (task & 7) + 8 * ((task >> 3) & 15), c = task >> 7;
            const int k = k_base + r;
            const int ci = k / 9, t = k - 9 * (k / 9);
            const int ky = t / 3, kx = t - 3 * (t / 3);
            PixCursor pc;
            pc.start(p0 + 8 * c, hw, Wo);
            if (k < 9 * CI && pc.j + 8 <= Wo && p0 + 8 * c + 7 < P) {
                // the chunk's eight pixels lie in one output row: one input row, columns 2 apart
                const int yy = 2 * pc.i + ky - 1, xx0 = 2 * pc.j + kx - 1;
                const bool row_ok = yy >= 0 && yy < H;
                const float* src = x + (static_cast<size_t>(pc.n) * CI + ci) * plane + static_cast<size_t>(row_ok ? yy : 0) * W;
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    const int xx = xx0 + 2 * q;
                    float v = 0.f;
                    if (row_ok && xx >= 0 && xx < W) {
                        v = __ldg(src + xx);
                        if (kScale) v *= scale;
                    }
                    xv[u][q] = v;
                }
            } else {
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    const bool live = p0 + 8 * c + q < P;
                    float v = 0.f;
                    if (live && k < 9 * CI) {
                        const int yy = 2 * pc.i + ky - 1, xx = 2 * pc.j + kx - 1;
                        if (yy >= 0 && yy < H && xx >= 0 && xx < W) {
                            v = __ldg(x + (static_cast<size_t>(pc.n) * CI + ci) * plane + static_cast<size_t>(yy) * W + xx);
                            if (kScale) v *= scale;
                        }
                    } else if (live && k == 9 * CI) {
                        v = 1.f;
                    }
                    xv[u][q] = v;
                    pc.next(Ho, Wo);
                }
            }
        }
#pragma unroll
        for (int u = 0; u < S::kDTasks; ++u) {
            const int task = tid + u * kEtThreads;
            const int co = (task & 7) + 8 * ((task >> 3) % (CO / 8)), c = task / CO;
            PixCursor pc;
            pc.start(p0 + 8 * c, hw, Wo);
            if (task < CO * kWgStage / 8 && pc.j + 8 <= Wo && p0 + 8 * c + 7 < P) {
                // eight consecutive pixels of one output row: contiguous
                const float* src = delta + (static_cast<size_t>(pc.n) * CO + co) * hw + pc.i * Wo + pc.j;
#pragma unroll
                for (int q = 0; q < 8; ++q) dv[u][q] = __ldg(src + q);
            } else {
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    float v = 0.f;
                    if (task < CO * kWgStage / 8 && p0 + 8 * c + q < P)
                        v = __ldg(delta + (static_cast<size_t>(pc.n) * CO + co) * hw + pc.i * Wo + pc.j);
                    dv[u][q] = v;
                    pc.next(Ho, Wo);
                }
            }
        }
    };

    bool ok = true;
    int last_commit = -1;
    float xn_[S::kXTasks][8], dn_[S::kDTasks][8];
    if (n_local > 0) gather(0, xn_, dn_);
#pragma unroll 1
    for (int sl = 0; sl < n_local; ++sl) {
        const uint32_t buf = buf0 + static_cast<uint32_t>(sl & 1) * S::kBuf;
        float xv[S::kXTasks][8], dv[S::kDTasks][8];
#pragma unroll
        for (int u = 0; u < S::kXTasks; ++u)
#pragma unroll
            for (int q = 0; q < 8; ++q) xv[u][q] = xn_[u][q];
#pragma unroll
        for (int u = 0; u < S::kDTasks; ++u)
#pragma unroll
            for (int q = 0; q < 8; ++q) dv[u][q] = dn_[u][q];
        // the next stage's loads are in flight while this one is stored and issued
        if (sl + 1 < n_local) gather(sl + 1, xn_, dn_);
        if (sl >= 2) ok = tc::mbar_wait_bounded(tc::smem_u32(&bar[sl & 1]), static_cast<uint32_t>(((sl - 2) >> 1) & 1),
                                                abort_flag, err, kDevErrTimeout);
        if (!__syncthreads_and(ok)) {
            ok = false;
            break;
        }
#pragma unroll
        for (int u = 0; u < S::kXTasks; ++u) {
            const int task = tid + u * kEtThreads;
            const int r = (task & 7) + 8 * ((task >> 3) & 15), c = task >> 7;
            const uint32_t off = stage_offset<kWgStage>(r, 8 * c);
            store_split8(buf + off, buf + S::kXHalf + off, xv[u]);
        }
#pragma unroll
        for (int u = 0; u < S::kDTasks; ++u) {
            const int task = tid + u * kEtThreads;
            if (task < CO * kWgStage / 8) {
                const int co = (task & 7) + 8 * ((task >> 3) % (CO / 8)), c = task / CO;
                const uint32_t off = stage_offset<kWgStage>(co, 8 * c);
                store_split8(buf + 2 * S::kXHalf + off, buf + 2 * S::kXHalf + S::kDHalf + off, dv[u]);
            }
        }
        tc::fence_proxy_async_smem();
        tc::fence_before_sync();
        __syncthreads();
        if (tid == 0) {
            tc::fence_after_sync();
#pragma unroll
            for (int j = 0; j < kWgStage / 16; ++j) {
                const uint32_t dj = static_cast<uint32_t>(256 * j);
                const uint64_t ahi = tc::smem_desc(buf + dj, 128, S::kSbo);
                const uint64_t alo = tc::smem_desc(buf + S::kXHalf + dj, 128, S::kSbo);
                const uint64_t bhi = tc::smem_desc(buf + 2 * S::kXHalf + dj, 128, S::kSbo);
                const uint64_t blo = tc::smem_desc(buf + 2 * S::kXHalf + S::kDHalf + dj, 128, S::kSbo);
                tc::mma_bf16(tmem, ahi, bhi, kIdesc, (sl > 0 || j > 0) ? 1u : 0u);
                tc::mma_bf16(tmem, ahi, blo, kIdesc, 1u);
                tc::mma_bf16(tmem, alo, bhi, kIdesc, 1u);
            }
            tc::mma_commit(tc::smem_u32(&bar[sl & 1]));
            last_commit = sl;
        }
    }
    const int last = n_local - 1;
    if (ok && last >= 0)
        ok = tc::mbar_wait_bounded(tc::smem_u32(&bar[last & 1]), static_cast<uint32_t>((last >> 1) & 1), abort_flag,
                                   err, kDevErrTimeout);
    ok = __syncthreads_and(ok);
    if (!ok && tid == 0 && last_commit >= 0) {
        int dummy = 0;
        tc::mbar_wait_bounded(tc::smem_u32(&bar[last_commit & 1]), static_cast<uint32_t>((last_commit >> 1) & 1),
                              &dummy, err, kDevErrTimeout);
    }
    tc::fence_after_sync();
    {
        const int row = tid & (kWgRows - 1), half = tid >> 7;
        const int k = k_base + row;
        const uint32_t lane_addr = tmem + (static_cast<uint32_t>((warp & 3) * 32) << 16);
        constexpr int kHalfCo = CO / 2;
#pragma unroll
        for (int c0 = half * kHalfCo; c0 < (half + 1) * kHalfCo; c0 += 8) {
            uint32_t v[8];
            tmem_ld_32x32b_x8(lane_addr + static_cast<uint32_t>(c0), v);
            tc::tmem_wait_ld();
            if (k < S::K1) {
#pragma unroll
                for (int q = 0; q < 8; ++q)
                    ws[(static_cast<size_t>(blockIdx.y) * CO + c0 + q) * S::K1 + k] =
                        (ok && n_local > 0) ? __uint_as_float(v[q]) : 0.f;
            }
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) {
        tc::fence_after_sync();
        tc::tmem_dealloc(tmem, S::kTmemCols);
    }
}

// ---------------------------------------------------------------- input gradients
// The gradient at the input of a convolution (ReLU mask of that input applied),
//   delta_in[n][ci][y][x] = [x_in > 0] sum_{co, (ky, kx)} W[co][ci][ky][kx] delta[n][co][i][j],
// over the windows (i, j) = ((y + 1 - ky) / 2, (x + 1 - kx) / 2) that read pixel (y, x).  The
// taps that can reach (y, x) depend only on its parity class (y mod 2, x mod 2): ky = 1 for even
// y, ky in {0, 2} for odd y (kx likewise), so each class is one GEMM  D[q][ci] = sum_k A[q][k]
// B[ci][k]  over its pixels q (M = 128 per CTA, blockIdx.y = class), N = CI, and k = tap_index CO
// + co (1, 2 or 4 taps): A[q][k] = delta at the tap's window (zero outside the output), B the
// class's weights, packed per class (pack_dgrad_weights_kernel) and loaded by one bulk copy.
// Stages of 32 columns, two threads per row, the same BF16 hi/lo split and three products.
constexpr int kDgStage = 32;

template <int CI, int CO>
struct DgradShape {
    static constexpr uint32_t kAHalf = kEtRows * kDgStage * 2;
    static constexpr uint32_t kBuf = 2 * kAHalf;
    static constexpr uint32_t kBHalf = CI * kDgStage * 2;
    static constexpr uint32_t kBStage = 2 * kBHalf;
    static constexpr int kMaxStages = 4 * CO / kDgStage;      // the class with four taps
    static constexpr uint32_t kHead = 1024;
    static constexpr uint32_t kSmem = kHead + 2 * kBuf + kMaxStages * kBStage;
    static constexpr uint32_t kTmemCols = CI <= 32 ? 32 : CI;
    static constexpr uint32_t kSbo = kDgStage * 16;
    static_assert(CO % kDgStage == 0 && CI % 16 == 0, "whole stages per tap, N a multiple of 16");
    __host__ __device__ static constexpr int stages(int cls) { return (1 + (cls >> 1)) * (1 + (cls & 1)) * CO / kDgStage; }
    __host__ __device__ static constexpr size_t class_offset(int cls) {
        size_t o = 0;
        for (int c = 0; c < cls; ++c) o += static_cast<size_t>(stages(c)) * kBStage;
        return o;
    }
};

// (ky, kx) of tap index t of parity class cls: ky = 1 for even rows, {0, 2} for odd ones.
__device__ __forceinline__ void class_tap(int cls, int t, int& ky, int& kx) {
    const int py = cls >> 1, px = cls & 1;
    const int nkx = 1 + px;
    const int a = t / nkx, b = t - a * nkx;
    ky = py ? 2 * a : 1;
    kx = px ? 2 * b : 1;
}

template <int CI, int CO>
__global__ void __launch_bounds__(256) pack_dgrad_weights_kernel(const float* __restrict__ wt, uint8_t* __restrict__ out) {
    using S = DgradShape<CI, CO>;
    constexpr int kChunks = CI * kDgStage / 8;                 // per stage
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    int cls = 0, rem = e;
    while (cls < 4 && rem >= S::stages(cls) * kChunks) {
        rem -= S::stages(cls) * kChunks;
        ++cls;
    }
    if (cls >= 4) return;
    const int s = rem / kChunks, r = rem - s * kChunks;
    const int ci = r / (kDgStage / 8), c = (r - ci * (kDgStage / 8)) * 8;
    const int k0 = s * kDgStage + c;
    const int t = k0 / CO, co0 = k0 - t * CO;
    int ky, kx;
    class_tap(cls, t, ky, kx);
    float v[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) v[q] = wt[((static_cast<size_t>(co0 + q) * CI + ci) * 3 + ky) * 3 + kx];
    uint32_t h[4], l[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        h[q] = tc::pack_bf16x2(v[2 * q], v[2 * q + 1]);
        l[q] = tc::pack_bf16x2(v[2 * q] - __uint_as_float(h[q] << 16), v[2 * q + 1] - __uint_as_float(h[q] & 0xFFFF0000u));
    }
    uint8_t* st = out + S::class_offset(cls) + static_cast<size_t>(s) * S::kBStage + stage_offset<kDgStage>(ci, c);
    *reinterpret_cast<uint4*>(st) = make_uint4(h[0], h[1], h[2], h[3]);
    *reinterpret_cast<uint4*>(st + S::kBHalf) = make_uint4(l[0], l[1], l[2], l[3]);
}

template <int CI, int CO>
__global__ void __launch_bounds__(kEtThreads) conv_dgrad_tc_kernel(const float* __restrict__ delta,
                                                                   const uint8_t* __restrict__ wpack,
                                                                   const float* __restrict__ x_in, int n_img, int H,
                                                                   int W, int Ho, int Wo,
                                                                   float* __restrict__ delta_in, int* err) {
    using S = DgradShape<CI, CO>;
    const int cls = blockIdx.y, py = cls >> 1, px = cls & 1;
    const int ny = (H - py + 1) / 2, nx = (W - px + 1) / 2;
    const long long count = static_cast<long long>(n_img) * ny * nx;
    if (static_cast<long long>(blockIdx.x) * kEtRows >= count) return;   // the class has fewer tiles
    extern __shared__ __align__(1024) uint8_t smem[];
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem);
    uint64_t* bar_w = reinterpret_cast<uint64_t*>(smem + 32);
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(smem + 16);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(smem + 20);
    const int tid = threadIdx.x, warp = tid >> 5;
    const int row = tid & (kEtRows - 1), half = tid >> 7;
    if (warp == 0) {
        tc::tmem_alloc(tc::smem_u32(tmem_slot), S::kTmemCols);
        tc::tmem_relinquish();
    }
    if (tid == 0) {
        tc::mbar_init(tc::smem_u32(&bar[0]), 1);
        tc::mbar_init(tc::smem_u32(&bar[1]), 1);
        tc::mbar_init(tc::smem_u32(bar_w), 1);
        *abort_flag = 0;
        tc::mbar_fence_init();
    }
    pdl_trigger();
    pdl_wait();
    const int n_st = S::stages(cls);
    const uint32_t bres = tc::smem_u32(smem + S::kHead + 2 * S::kBuf);
    if (tid == 0)
        bulk_load(bres, wpack + S::class_offset(cls), static_cast<uint32_t>(n_st) * S::kBStage, tc::smem_u32(bar_w));
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = *tmem_slot;

    // this thread's pixel of the class
    const long long f = static_cast<long long>(blockIdx.x) * kEtRows + row;
    const bool live = f < count;
    int n = 0, y = 0, x = 0;
    if (live) {
        n = static_cast<int>(f / (static_cast<long long>(ny) * nx));
        const int r = static_cast<int>(f - static_cast<long long>(n) * ny * nx);
        y = 2 * (r / nx) + py;
        x = 2 * (r - (r / nx) * nx) + px;
    }
    const size_t hwo = static_cast<size_t>(Ho) * Wo;
    const float* dn = delta + static_cast<size_t>(n) * CO * hwo;
    const uint32_t buf0 = tc::smem_u32(smem + S::kHead);
    constexpr uint32_t kIdesc = tc::idesc_bf16_f32(kEtRows, CI);
    constexpr int kHalfCols = kDgStage / 2;

    auto gather = [&](int s, float (&a)[kHalfCols]) {
        const int k0 = s * kDgStage + half * kHalfCols;
        const int t = k0 / CO, co0 = k0 - t * CO;
        int ky, kx;
        class_tap(cls, t, ky, kx);
        const int i = (y + 1 - ky) >> 1, j = (x + 1 - kx) >> 1;
        const bool v = live && i < Ho && j < Wo;
        const float* src = dn + static_cast<size_t>(co0) * hwo + static_cast<size_t>(i) * Wo + j;
#pragma unroll
        for (int q = 0; q < kHalfCols; ++q) a[q] = v ? __ldg(src + static_cast<size_t>(q) * hwo) : 0.f;
    };

    bool ok = true;
    int last_commit = -1;
    float a_next[kHalfCols];
    gather(0, a_next);
#pragma unroll 1
    for (int sl = 0; sl < n_st; ++sl) {
        const uint32_t buf = buf0 + static_cast<uint32_t>(sl & 1) * S::kBuf;
        float a[kHalfCols];
#pragma unroll
        for (int c = 0; c < kHalfCols; ++c) a[c] = a_next[c];
        if (sl + 1 < n_st) gather(sl + 1, a_next);
        if (sl >= 2) ok = tc::mbar_wait_bounded(tc::smem_u32(&bar[sl & 1]), static_cast<uint32_t>(((sl - 2) >> 1) & 1),
                                                abort_flag, err, kDevErrTimeout);
        if (!__syncthreads_and(ok)) {
            ok = false;
            break;
        }
#pragma unroll
        for (int c8 = 0; c8 < kHalfCols; c8 += 8) {
            const uint32_t off = stage_offset<kDgStage>(row, half * kHalfCols + c8);
            store_split8(buf + off, buf + S::kAHalf + off, a + c8);
        }
        tc::fence_proxy_async_smem();
        tc::fence_before_sync();
        __syncthreads();
        if (tid == 0) {
            tc::fence_after_sync();
            const bool go = sl > 0 || tc::mbar_wait_bounded(tc::smem_u32(bar_w), 0u, abort_flag, err, kDevErrTimeout);
            if (!go) ok = false;
            if (go) {
                const uint32_t wb = bres + static_cast<uint32_t>(sl) * S::kBStage;
#pragma unroll
                for (int jj = 0; jj < kDgStage / 16; ++jj) {
                    const uint32_t dj = static_cast<uint32_t>(256 * jj);
                    const uint64_t ahi = tc::smem_desc(buf + dj, 128, S::kSbo);
                    const uint64_t alo = tc::smem_desc(buf + S::kAHalf + dj, 128, S::kSbo);
                    const uint64_t bhi = tc::smem_desc(wb + dj, 128, S::kSbo);
                    const uint64_t blo = tc::smem_desc(wb + S::kBHalf + dj, 128, S::kSbo);
                    tc::mma_bf16(tmem, ahi, bhi, kIdesc, (sl > 0 || jj > 0) ? 1u : 0u);
                    tc::mma_bf16(tmem, ahi, blo, kIdesc, 1u);
                    tc::mma_bf16(tmem, alo, bhi, kIdesc, 1u);
                }
                tc::mma_commit(tc::smem_u32(&bar[sl & 1]));
                last_commit = sl;
            }
        }
    }
    const int last = n_st - 1;
    if (ok) ok = tc::mbar_wait_bounded(tc::smem_u32(&bar[last & 1]), static_cast<uint32_t>((last >> 1) & 1), abort_flag,
                                       err, kDevErrTimeout);
    ok = __syncthreads_and(ok);
    if (!ok && tid == 0) {
        int dummy = 0;
        if (last_commit >= 0)
            tc::mbar_wait_bounded(tc::smem_u32(&bar[last_commit & 1]), static_cast<uint32_t>((last_commit >> 1) & 1),
                                  &dummy, err, kDevErrTimeout);
        tc::mbar_wait_bounded(tc::smem_u32(bar_w), 0u, &dummy, err, kDevErrTimeout);
    }
    tc::fence_after_sync();
    if (ok) {
        const uint32_t lane_addr = tmem + (static_cast<uint32_t>((warp & 3) * 32) << 16);
        constexpr int kHalfCi = CI / 2;
        const size_t hw = static_cast<size_t>(H) * W;
        const size_t o0 = static_cast<size_t>(n) * CI * hw + static_cast<size_t>(y) * W + x;
#pragma unroll
        for (int c0 = half * kHalfCi; c0 < (half + 1) * kHalfCi; c0 += 8) {
            uint32_t v[8];
            tmem_ld_32x32b_x8(lane_addr + static_cast<uint32_t>(c0), v);
            tc::tmem_wait_ld();
            if (live) {
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    const size_t o = o0 + static_cast<size_t>(c0 + q) * hw;
                    delta_in[o] = __ldg(x_in + o) > 0.f ? __uint_as_float(v[q]) : 0.f;
                }
            }
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) {
        tc::fence_after_sync();
        tc::tmem_dealloc(tmem, S::kTmemCols);
    }
}

template <int CI, int CO, bool kScale, int kSplit>
cudaError_t configure_one() {
    return cudaFuncSetAttribute(conv3x3s2_tc_kernel<CI, CO, kScale, kSplit>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize,
                                static_cast<int>(ConvTcShape<CI, CO, kSplit>::kSmem));
}

template <int CI, int CO, bool kScale, int kSplit>
cudaError_t launch_one(const float* x, int n_img, int H, int W, int Ho, int Wo, const uint8_t* wt, const float* b,
                       float scale, float* y, int* err, int inject, cudaStream_t s) {
    const long long P = static_cast<long long>(n_img) * Ho * Wo;
    const long long tiles = (P + kEtRows - 1) / kEtRows;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(static_cast<unsigned>(tiles), 1, kSplit);
    cfg.blockDim = dim3(kEtThreads);
    cfg.dynamicSmemBytes = ConvTcShape<CI, CO, kSplit>::kSmem;
    cfg.stream = s;
    cudaLaunchAttribute attr[2];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    attr[1].id = cudaLaunchAttributeClusterDimension;
    attr[1].val.clusterDim.x = 1;
    attr[1].val.clusterDim.y = 1;
    attr[1].val.clusterDim.z = kSplit;
    cfg.attrs = attr;
    cfg.numAttrs = kSplit > 1 ? 2 : 1;
    return cudaLaunchKernelEx(&cfg, conv3x3s2_tc_kernel<CI, CO, kScale, kSplit>, x, n_img, H, W, Ho, Wo, wt, b, scale,
                              y, err, inject);
}

// reduction split of each layer: the deep layers with few output tiles use a cluster
constexpr int kSplit2 = 2;   // 32 -> 64 channels: 6 stages, 3 per CTA
constexpr int kSplit3 = 4;   // 64 -> 64 channels: 12 stages, 3 per CTA

}  // namespace

template <int CI, int CO, bool kScale>
cudaError_t configure_wgrad() {
    return cudaFuncSetAttribute(conv_wgrad_tc_kernel<CI, CO, kScale>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                static_cast<int>(WgradShape<CI, CO>::kSmem));
}

template <int CI, int CO, bool kScale>
cudaError_t wgrad_one(const float* x, const float* delta, int n_img, int H, int W, int Ho, int Wo, float scale,
                      int slices, int stages_per_slice, float* ws, int* err, cudaStream_t s) {
    const int k_tiles = (WgradShape<CI, CO>::K1 + kWgRows - 1) / kWgRows;
    return launch_dependent(true, conv_wgrad_tc_kernel<CI, CO, kScale>, dim3(k_tiles, slices), dim3(kEtThreads),
                            WgradShape<CI, CO>::kSmem, s, x, delta, n_img, H, W, Ho, Wo, scale, stages_per_slice, ws,
                            err);
}

template <int CI, int CO>
cudaError_t configure_dgrad() {
    return cudaFuncSetAttribute(conv_dgrad_tc_kernel<CI, CO>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                static_cast<int>(DgradShape<CI, CO>::kSmem));
}

template <int CI, int CO>
cudaError_t dgrad_one(const float* delta, const uint8_t* wpack, const float* x_in, int n_img, int H, int W, int Ho,
                      int Wo, float* delta_in, int* err, cudaStream_t s) {
    // the most tiles of a class: the one with the even rows and columns
    const long long most = static_cast<long long>(n_img) * ((H + 1) / 2) * ((W + 1) / 2);
    const unsigned tiles = static_cast<unsigned>((most + kEtRows - 1) / kEtRows);
    return launch_dependent(true, conv_dgrad_tc_kernel<CI, CO>, dim3(tiles, 4), dim3(kEtThreads),
                            DgradShape<CI, CO>::kSmem, s, delta, wpack, x_in, n_img, H, W, Ho, Wo, delta_in, err);
}

template <int CI, int CO>
cudaError_t pack_dgrad_one(const float* wt, uint8_t* out, cudaStream_t s) {
    using S = DgradShape<CI, CO>;
    int n = 0;
    for (int c = 0; c < 4; ++c) n += S::stages(c) * CI * kDgStage / 8;
    pack_dgrad_weights_kernel<CI, CO><<<(n + 255) / 256, 256, 0, s>>>(wt, out);
    return cudaGetLastError();
}

cudaError_t configure_conv_tc() {
    cudaError_t e = configure_dgrad<16, 32>();
    if (e == cudaSuccess) e = configure_dgrad<32, 64>();
    if (e == cudaSuccess) e = configure_dgrad<64, 64>();
    if (e == cudaSuccess) e = configure_wgrad<1, 16, true>();
    if (e == cudaSuccess) e = configure_wgrad<16, 32, false>();
    if (e == cudaSuccess) e = configure_wgrad<32, 64, false>();
    if (e == cudaSuccess) e = configure_wgrad<64, 64, false>();
    if (e == cudaSuccess) e = configure_one<1, 16, true, 1>();
    if (e == cudaSuccess) e = configure_one<16, 32, false, 1>();
    if (e == cudaSuccess) e = configure_one<32, 64, false, kSplit2>();
    if (e == cudaSuccess) e = configure_one<64, 64, false, kSplit3>();
    return e;
}

cudaError_t launch_conv_tc(int layer, const float* x, int n_img, int H, int W, int Ho, int Wo, const uint8_t* wt,
                           const float* b, float scale, float* y, int* err, int inject, cudaStream_t s) {
    switch (layer) {
        case 0: return launch_one<1, 16, true, 1>(x, n_img, H, W, Ho, Wo, wt, b, scale, y, err, inject, s);
        case 1: return launch_one<16, 32, false, 1>(x, n_img, H, W, Ho, Wo, wt, b, scale, y, err, inject, s);
        case 2: return launch_one<32, 64, false, kSplit2>(x, n_img, H, W, Ho, Wo, wt, b, scale, y, err, inject, s);
        case 3: return launch_one<64, 64, false, kSplit3>(x, n_img, H, W, Ho, Wo, wt, b, scale, y, err, inject, s);
        default: return cudaErrorInvalidValue;
    }
}

int conv_wgrad_tc_stage_pixels() { return kWgStage; }
int conv_wgrad_tc_k_tiles(int layer) {
    static constexpr int kCin[4] = {1, 16, 32, 64};
    return (9 * kCin[layer] + 1 + kWgRows - 1) / kWgRows;
}

cudaError_t launch_conv_wgrad_tc(int layer, const float* x, const float* delta, int n_img, int H, int W, int Ho, int Wo,
                                 float scale, int slices, int stages_per_slice, float* ws, int* err, cudaStream_t s) {
    switch (layer) {
        case 0: return wgrad_one<1, 16, true>(x, delta, n_img, H, W, Ho, Wo, scale, slices, stages_per_slice, ws, err, s);
        case 1: return wgrad_one<16, 32, false>(x, delta, n_img, H, W, Ho, Wo, scale, slices, stages_per_slice, ws, err, s);
        case 2: return wgrad_one<32, 64, false>(x, delta, n_img, H, W, Ho, Wo, scale, slices, stages_per_slice, ws, err, s);
        case 3: return wgrad_one<64, 64, false>(x, delta, n_img, H, W, Ho, Wo, scale, slices, stages_per_slice, ws, err, s);
        default: return cudaErrorInvalidValue;
    }
}

size_t conv_dgrad_tc_packed_bytes(int layer) {
    switch (layer) {
        case 1: return DgradShape<16, 32>::class_offset(4);
        case 2: return DgradShape<32, 64>::class_offset(4);
        case 3: return DgradShape<64, 64>::class_offset(4);
        default: return 0;
    }
}

cudaError_t launch_conv_dgrad_tc(int layer, const float* delta, const uint8_t* wpack, const float* x_in, int n_img,
                                 int H, int W, int Ho, int Wo, float* delta_in, int* err, cudaStream_t s) {
    switch (layer) {
        case 1: return dgrad_one<16, 32>(delta, wpack, x_in, n_img, H, W, Ho, Wo, delta_in, err, s);
        case 2: return dgrad_one<32, 64>(delta, wpack, x_in, n_img, H, W, Ho, Wo, delta_in, err, s);
        case 3: return dgrad_one<64, 64>(delta, wpack, x_in, n_img, H, W, Ho, Wo, delta_in, err, s);
        default: return cudaErrorInvalidValue;
    }
}

size_t conv_tc_packed_bytes(int layer) {
    switch (layer) {
        case 0: return packed_bytes<1, 16>();
        case 1: return packed_bytes<16, 32>();
        case 2: return packed_bytes<32, 64>();
        case 3: return packed_bytes<64, 64>();
        default: return 0;
    }
}

template <int CI, int CO>
cudaError_t pack_one(const float* wt, uint8_t* out, cudaStream_t s) {
    using S = ConvTcShape<CI, CO, 1>;
    const int n = S::kStages * S::kBChunks;
    pack_conv_weights_kernel<CI, CO><<<(n + 255) / 256, 256, 0, s>>>(wt, out);
    return cudaGetLastError();
}

cudaError_t pack_conv_tc_weights(const float* const* wt, uint8_t* const* out, uint8_t* const* out_dgrad,
                                 cudaStream_t s) {
    cudaError_t e = pack_one<1, 16>(wt[0], out[0], s);
    if (e == cudaSuccess) e = pack_one<16, 32>(wt[1], out[1], s);
    if (e == cudaSuccess) e = pack_one<32, 64>(wt[2], out[2], s);
    if (e == cudaSuccess) e = pack_one<64, 64>(wt[3], out[3], s);
    if (e == cudaSuccess) e = pack_dgrad_one<16, 32>(wt[1], out_dgrad[1], s);
    if (e == cudaSuccess) e = pack_dgrad_one<32, 64>(wt[2], out_dgrad[2], s);
    if (e == cudaSuccess) e = pack_dgrad_one<64, 64>(wt[3], out_dgrad[3], s);
    return e;
}

}  // namespace mppi
