// Distillation trainer: the hidden layers' GEMMs on the 5th-generation tensor
// cores (tcgen05.mma kind::f16 with BF16 operands, FP32 accumulators in TMEM).
// Master weights, activations and adjoints stay FP32 in HBM; operands are
// rounded to BF16 while they are staged into shared memory (the no-swizzle
// core-matrix layouts of tc.cuh).  Per hidden layer l in {2, 3, 4} and
// 128-point tile (the Gate-SDF MLP of Sec. III-B, Eq. 3, with the input
// gradient carried in forward mode and the loss differentiated in reverse
// mode, as the FP32 kernels do):
//   forward        A_l = X_0 W^T + b,  AT_l^j = X_j W^T         four TMEM accumulators
//   input grads    dX_s = D_s W, then through layer l-1's activation
//   weight grads   dW_l = sum_s D_s^T X_s over the CTA's tiles   one TMEM accumulator
// X_s are the layer's four input streams (values and three tangents), D_s the
// adjoints of its outputs.  One thread issues the MMAs; every wait is bounded
// (tc::kWaitLimitNs) and reports through the device error word.
#include <cstdint>

#include "tc.cuh"
#include "train_internal.cuh"

namespace mppi {
namespace train {
namespace {

constexpr int kThreads = 512;                               // 16 warps
// epilogue: warp w reads TMEM lanes 32 (w mod 4) .. + 31 (the rule of tcgen05.ld) and the
// 32 columns 32 (w / 4) .. + 31 of each accumulator
constexpr int kEpiCols = kH / (kThreads / 128);
static_assert(kEpiCols == 32, "the epilogue assumes one 32-column slice per warp");
constexpr uint32_t kOpBytes = kH * kH * 2;                  // one 128 x 128 BF16 operand
constexpr uint32_t kIdesc = tc::idesc_bf16_f32(128, 128);
constexpr int kKSlices = kH / 16;                           // K = 16 per kind::f16 MMA

struct StreamShared {               // forward and input-gradient kernels
    uint8_t x[4][kOpBytes];         // A operands: the tile's four streams
    uint8_t w[kOpBytes];            // B operand: W (forward) or W^T (input gradients)
    float bias[kH];
    uint64_t bar;
    uint32_t tmem_base;
    int abort_flag;
};

// Weight gradients: units of kWPts points (the GEMM's K), four streams per unit, kWBufs
// buffers.  Operands are MN-major 128 x kWPts BF16: core matrices of 8 points x 8 features
// (each point's 8 features one 16-byte row), LBO = 128 B between core matrices adjacent in K,
// SBO = kWSbo between core matrices adjacent in the feature dimension.
constexpr int kWPts = 32;
constexpr int kWBufs = 3;
constexpr uint32_t kWOpBytes = kH * kWPts * 2;
constexpr uint32_t kWSbo = (kWPts / 8) * 128;
// kind::f16 with A and B MN-major (instruction-descriptor bits 15 and 16)
constexpr uint32_t kIdescMN = tc::idesc_bf16_f32(128, 128) | (1u << 15) | (1u << 16);

__device__ __forceinline__ uint32_t mn_offset_bytes(int feature, int point) {
    return static_cast<uint32_t>((feature >> 3) * kWSbo + (point >> 3) * 128 + (point & 7) * 16 + (feature & 7) * 2);
}

struct WeightShared {
    uint8_t d[kWBufs][4][kWOpBytes];   // A operands D_s  (M = o, K = points)
    uint8_t x[kWBufs][4][kWOpBytes];   // B operands X_s  (N = i, K = points)
    float db[kThreads][8];
    uint64_t bar[kWBufs];
    uint32_t tmem_base;
    int abort_flag;
};

constexpr size_t kStreamSmem = sizeof(StreamShared) + 1024;
constexpr size_t kWeightSmem = sizeof(WeightShared) + 1024;
static_assert(kStreamSmem <= 227 * 1024 && kWeightSmem <= 227 * 1024, "shared memory exceeds a CTA's 227 KB");

template <typename S>
__device__ __forceinline__ S& shared_block() {
    extern __shared__ uint8_t raw[];
    return *reinterpret_cast<S*>((reinterpret_cast<uintptr_t>(raw) + 1023) & ~uintptr_t(1023));
}

__device__ __forceinline__ void load8(const float* p, float (&v)[8]) {
    const float4 a = __ldg(reinterpret_cast<const float4*>(p));
    const float4 b = __ldg(reinterpret_cast<const float4*>(p) + 1);
    v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
    v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
}

// Eight values -> one 16-byte core-matrix row of BF16 (element 0 at the lowest address).
__device__ __forceinline__ void st_bf16x8(uint32_t addr, const float (&v)[8]) {
    tc::st_shared_v4(addr, tc::pack_bf16x2(v[0], v[1]), tc::pack_bf16x2(v[2], v[3]), tc::pack_bf16x2(v[4], v[5]),
                     tc::pack_bf16x2(v[6], v[7]));
}

__device__ __forceinline__ void sync_for_mma() {
    tc::fence_proxy_async_smem();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
}

// Epilogue transpose through shared memory (the operand buffers, free once the tile's MMAs
// completed): tcgen05.ld gives thread i TMEM lane (row) i, while whole-row global accesses want
// the eight lanes of a quarter warp on one row.  Per warp a 32 x 32 FP32 block with a 36-float
// row pitch: the 16-byte row writes of eight consecutive rows, and the 16-byte reads of one
// row by eight lanes, each fall on eight distinct bank quadruples.
constexpr int kScrLd = 36;
constexpr int kScrFloats = 32 * kScrLd;

__device__ __forceinline__ void ld_shared_v4(uint32_t addr, float (&v)[4]) {
    asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];"
                 : "=f"(v[0]), "=f"(v[1]), "=f"(v[2]), "=f"(v[3])
                 : "r"(addr)
                 : "memory");
}

// TMEM columns [col, col + 32) of this warp's 32 lanes -> the warp's scratch block (row = lane).
__device__ __forceinline__ void tmem_to_scratch(uint32_t taddr, uint32_t scr, int lane) {
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        uint32_t v[16];
        tc::tmem_ld_32x32b_x16(taddr + static_cast<uint32_t>(16 * h), v);
        tc::tmem_wait_ld();
        tc::reg_fence16(v);
#pragma unroll
        for (int j = 0; j < 16; j += 4)
            tc::st_shared_v4(scr + static_cast<uint32_t>((lane * kScrLd + 16 * h + j) * 4), v[j], v[j + 1], v[j + 2],
                             v[j + 3]);
    }
    __syncwarp();
}

// Work item it in [0, 2048) of a row-major [128][128] source -> (row, 8-column chunk).  The
// eight lanes of a quarter warp take eight consecutive rows of one chunk, so their 16-byte
// shared-memory stores fill one contiguous 128-byte core matrix (no bank conflicts), and a
// warp reads 128 contiguous bytes of each of 8 rows.
__device__ __forceinline__ int item_row(int it) { return (it >> 7) * 8 + (it & 7); }
__device__ __forceinline__ int item_col(int it) { return ((it >> 3) & 15) * 8; }

__device__ __forceinline__ void setup(uint32_t* tmem_slot, uint64_t* bars, int n_bars, int* abort_flag, uint32_t cols,
                                      int tid) {
    if (tid < 32) {
        tc::tmem_alloc(tc::smem_u32(tmem_slot), cols);
        tc::tmem_relinquish();
    }
    if (tid == 0) {
        for (int i = 0; i < n_bars; ++i) tc::mbar_init(tc::smem_u32(bars + i), 1);
        *abort_flag = 0;
        tc::mbar_fence_init();
    }
}

__device__ __forceinline__ void teardown(uint32_t tmem, uint32_t cols, int tid) {
    tc::fence_before_sync();
    __syncthreads();
    if (tid < 32) {
        tc::fence_after_sync();
        tc::tmem_dealloc(tmem, cols);
    }
}

// The four streams' 128 x 128 MMAs of one tile: accumulator s = TMEM columns [128 s, 128 s + 128).
__device__ __forceinline__ void issue_streams(uint32_t tmem, const StreamShared& S, uint32_t bar) {
    const uint64_t bd = tc::smem_desc(tc::smem_u32(S.w), 128, 2048);
#pragma unroll 1
    for (int s = 0; s < 4; ++s) {
        const uint64_t ad = tc::smem_desc(tc::smem_u32(S.x[s]), 128, 2048);
#pragma unroll
        for (int kk = 0; kk < kKSlices; ++kk)
            tc::mma_bf16(tmem + static_cast<uint32_t>(s * kH), ad + static_cast<uint64_t>(kk * 16),
                         bd + static_cast<uint64_t>(kk * 16), kIdesc, kk > 0 ? 1u : 0u);
    }
    tc::mma_commit(bar);
}

// ------------------------------------------------------------------ forward
// A_l = X_0 W_l^T + b_l,  AT_l^j = X_j W_l^T  (X_s = stream s of layer l-1's output).
__global__ void __launch_bounds__(kThreads, 1) fwd_hidden_tc_kernel(TrainBufs T, int l) {
    StreamShared& S = shared_block<StreamShared>();
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int lower = l - 1;
    setup(&S.tmem_base, &S.bar, 1, &S.abort_flag, 512, tid);
    // B operand W_l [n][k], K-major as stored
    const float* W = T.theta + offW(l);
    for (int it = tid; it < kH * kH / 8; it += kThreads) {
        const int n = item_row(it), k0 = item_col(it);
        float v[8];
        load8(W + n * kH + k0, v);
        st_bf16x8(tc::smem_u32(S.w) + tc::operand_offset_bytes(n, k0), v);
    }
    for (int i = tid; i < kH; i += kThreads) S.bias[i] = T.theta[offB(l) + i];
    sync_for_mma();
    const uint32_t tmem = S.tmem_base, bar = tc::smem_u32(&S.bar);
    const uint32_t xs = tc::smem_u32(S.x[0]);
    const int wq = warp & 3, col0 = (warp >> 2) * kEpiCols;
    const uint32_t lane_addr = tmem + (static_cast<uint32_t>(wq * 32) << 16);
    const size_t plane = static_cast<size_t>(T.B) * kH;
    const int n_tiles = T.B / kTileRows;
    uint32_t phase = 0;
    bool pending = false;
    for (int tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
        const int p0 = tile * kTileRows;
        // stage the four streams: sp(A), sp'(A) t_j (t_j = the tangent of layer l-1, W1[:, j] below layer 2)
#pragma unroll 1
        for (int it = tid; it < kTileRows * kH / 8; it += kThreads) {
            const int r = item_row(it), k0 = item_col(it);
            const size_t off = static_cast<size_t>(p0 + r) * kH + k0;
            float a[8], t[3][8];                 // every load of the item in flight at once
            load8(T.A[lower] + off, a);
            if (lower == 1) {
#pragma unroll
                for (int s = 1; s < 4; ++s)
#pragma unroll
                    for (int j = 0; j < 8; ++j) t[s - 1][j] = __ldg(T.theta + oW1 + (k0 + j) * kIn + (s - 1));
            } else {
#pragma unroll
                for (int s = 1; s < 4; ++s) load8(T.AT[lower] + static_cast<size_t>(s - 1) * plane + off, t[s - 1]);
            }
            float v[8], sg[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                v[j] = sp_beta(a[j], T.beta);
                sg[j] = sig_beta(a[j], T.beta);
            }
            const uint32_t dst = xs + tc::operand_offset_bytes(r, k0);
            st_bf16x8(dst, v);
#pragma unroll
            for (int s = 1; s < 4; ++s) {
#pragma unroll
                for (int j = 0; j < 8; ++j) v[j] = sg[j] * t[s - 1][j];
                st_bf16x8(dst + static_cast<uint32_t>(s) * kOpBytes, v);
            }
        }
        sync_for_mma();
        if (tid == 0) issue_streams(tmem, S, bar);
        __syncwarp();
        pending = true;
        const bool ok = tc::mbar_wait_bounded(bar, phase, &S.abort_flag, T.err, kDevErrTimeout);
        if (!__syncthreads_and(ok)) break;
        pending = false;
        phase ^= 1u;
        tc::fence_after_sync();
        // epilogue: this warp's 32 rows x 32 columns of each accumulator, transposed through its
        // scratch block; lane reads row 4 i + lane / 8, columns 4 (lane mod 8) .. + 3
        {
            const uint32_t scr = xs + static_cast<uint32_t>(warp * kScrFloats * 4);
            const int rq = lane >> 3, cc = (lane & 7) * 4;
#pragma unroll 1
            for (int s = 0; s < 4; ++s) {
                tmem_to_scratch(lane_addr + static_cast<uint32_t>(s * kH + col0), scr, lane);
                float* dst = (s == 0 ? T.A[l] : T.AT[l] + static_cast<size_t>(s - 1) * plane) +
                             static_cast<size_t>(p0 + wq * 32) * kH + col0 + cc;
                float bq[4] = {0.f, 0.f, 0.f, 0.f};
                if (s == 0) {
#pragma unroll
                    for (int q = 0; q < 4; ++q) bq[q] = S.bias[col0 + cc + q];
                }
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    const int rr = 4 * i + rq;
                    float o[4];
                    ld_shared_v4(scr + static_cast<uint32_t>((rr * kScrLd + cc) * 4), o);
                    *reinterpret_cast<float4*>(dst + static_cast<size_t>(rr) * kH) =
                        make_float4(o[0] + bq[0], o[1] + bq[1], o[2] + bq[2], o[3] + bq[3]);
                }
                __syncwarp();
            }
        }
        // the next tile's staging overwrites the scratch blocks
        __syncthreads();
        // the next tile's MMAs overwrite TMEM only after the barrier that ends its staging
        tc::fence_before_sync();
    }
    if (pending && tid == 0) {
        int dummy = 0;                       // let issued MMAs finish before TMEM is released
        tc::mbar_wait_bounded(bar, phase, &dummy, T.err, kDevErrTimeout);
    }
    teardown(tmem, 512, tid);
}

// ------------------------------------------------------------------ input gradients
// dX_s = D_s W_l (D_0 = dA_l, D_j = dAT_l^j), then through the activation of layer l-1:
//   dA_{l-1} = dX_0 sp'(A) + sum_j dX_j t_j sp''(A),   dAT_{l-1}^j = dX_j sp'(A).
__global__ void __launch_bounds__(kThreads, 1) bwd_input_tc_kernel(TrainBufs T, int l) {
    StreamShared& S = shared_block<StreamShared>();
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int lower = l - 1;
    setup(&S.tmem_base, &S.bar, 1, &S.abort_flag, 512, tid);
    // B operand W_l^T: row i holds W_l[o][i] over o (K = o)
    const float* W = T.theta + offW(l);
    for (int it = tid; it < kH * kH / 8; it += kThreads) {
        const int i = it & (kH - 1), o0 = (it >> 7) * 8;
        float v[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) v[j] = __ldg(W + (o0 + j) * kH + i);
        st_bf16x8(tc::smem_u32(S.w) + tc::operand_offset_bytes(i, o0), v);
    }
    sync_for_mma();
    const uint32_t tmem = S.tmem_base, bar = tc::smem_u32(&S.bar);
    const uint32_t xs = tc::smem_u32(S.x[0]);
    const int wq = warp & 3;
    const uint32_t lane_addr = tmem + (static_cast<uint32_t>(wq * 32) << 16);
    const size_t plane = static_cast<size_t>(T.B) * kH;
    const float beta = T.beta;
    const int n_tiles = T.B / kTileRows;
    uint32_t phase = 0;
    bool pending = false;
    for (int tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
        const int p0 = tile * kTileRows;
        for (int it = tid; it < kTileRows * kH / 8; it += kThreads) {
            const int r = item_row(it), k0 = item_col(it);
            const size_t off = static_cast<size_t>(p0 + r) * kH + k0;
            const uint32_t dst = xs + tc::operand_offset_bytes(r, k0);
            float v[4][8];
            load8(T.dA[l] + off, v[0]);
#pragma unroll
            for (int s = 1; s < 4; ++s) load8(T.dAT[l] + static_cast<size_t>(s - 1) * plane + off, v[s]);
#pragma unroll
            for (int s = 0; s < 4; ++s) st_bf16x8(dst + static_cast<uint32_t>(s) * kOpBytes, v[s]);
        }
        sync_for_mma();
        if (tid == 0) issue_streams(tmem, S, bar);
        __syncwarp();
        pending = true;
        const bool ok = tc::mbar_wait_bounded(bar, phase, &S.abort_flag, T.err, kDevErrTimeout);
        if (!__syncthreads_and(ok)) break;
        pending = false;
        phase ^= 1u;
        tc::fence_after_sync();
        // epilogue: this warp's 32 rows x 32 columns, each stream's dX transposed through the
        // warp's scratch block, so that A, AT of layer l-1 are read and dA, dAT written by whole
        // rows; lane holds rows 4 i + lane / 8 (i < 8), columns 4 (lane mod 8) .. + 3
        {
            const uint32_t scr = xs + static_cast<uint32_t>(warp * kScrFloats * 4);
            const int rq = lane >> 3, cc = (lane & 7) * 4;
            const int col0 = (warp >> 2) * kEpiCols;
            const size_t base = static_cast<size_t>(p0 + wq * 32) * kH + col0 + cc;
            float sg[8][4], tot[8][4];
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const float4 a = __ldg(reinterpret_cast<const float4*>(
                    T.A[lower] + base + static_cast<size_t>(4 * i + rq) * kH));
                sg[i][0] = sig_beta(a.x, beta);
                sg[i][1] = sig_beta(a.y, beta);
                sg[i][2] = sig_beta(a.z, beta);
                sg[i][3] = sig_beta(a.w, beta);
            }
            tmem_to_scratch(lane_addr + static_cast<uint32_t>(col0), scr, lane);
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                float d[4];
                ld_shared_v4(scr + static_cast<uint32_t>(((4 * i + rq) * kScrLd + cc) * 4), d);
#pragma unroll
                for (int q = 0; q < 4; ++q) tot[i][q] = d[q] * sg[i][q];
            }
            __syncwarp();
#pragma unroll 1
            for (int s = 1; s < 4; ++s) {
                tmem_to_scratch(lane_addr + static_cast<uint32_t>(s * kH + col0), scr, lane);
                float w1[4];
                if (lower == 1) {
#pragma unroll
                    for (int q = 0; q < 4; ++q) w1[q] = __ldg(T.theta + oW1 + (col0 + cc + q) * kIn + (s - 1));
                }
                const size_t so = static_cast<size_t>(s - 1) * plane + base;
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    const size_t ro = so + static_cast<size_t>(4 * i + rq) * kH;
                    float t[4];
                    if (lower == 1) {
#pragma unroll
                        for (int q = 0; q < 4; ++q) t[q] = w1[q];
                    } else {
                        const float4 t4 = __ldg(reinterpret_cast<const float4*>(T.AT[lower] + ro));
                        t[0] = t4.x; t[1] = t4.y; t[2] = t4.z; t[3] = t4.w;
                    }
                    float d[4], o[4];
                    ld_shared_v4(scr + static_cast<uint32_t>(((4 * i + rq) * kScrLd + cc) * 4), d);
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const float g = sg[i][q];
                        tot[i][q] = fmaf(d[q] * t[q], beta * g * (1.f - g), tot[i][q]);
                        o[q] = d[q] * g;
                    }
                    *reinterpret_cast<float4*>(T.dAT[lower] + ro) = make_float4(o[0], o[1], o[2], o[3]);
                }
                __syncwarp();
            }
#pragma unroll
            for (int i = 0; i < 8; ++i)
                *reinterpret_cast<float4*>(T.dA[lower] + base + static_cast<size_t>(4 * i + rq) * kH) =
                    make_float4(tot[i][0], tot[i][1], tot[i][2], tot[i][3]);
        }
        // the next tile's staging overwrites the scratch blocks
        __syncthreads();
        tc::fence_before_sync();
    }
    if (pending && tid == 0) {
        int dummy = 0;
        tc::mbar_wait_bounded(bar, phase, &dummy, T.err, kDevErrTimeout);
    }
    teardown(tmem, 512, tid);
}

// ------------------------------------------------------------------ weight gradients
// dW_l[o][i] = sum_pt sum_s D_s[pt][o] X_s[pt][i], accumulated in one TMEM accumulator over the
// CTA's units of 32 points (all four streams per unit), db_l[o] = sum_pt dA_l[pt][o] in FP32.
// Both operands are MN-major (o, resp. i, contiguous in 16-byte core-matrix rows; K = the
// points), so they are staged straight from the row-major [pt][feature] activations with
// 16-byte loads, and the layer-below activation (sp, sp') is evaluated once for all streams.
// Units rotate through kWBufs operand buffers, so staging overlaps the MMAs.
__global__ void __launch_bounds__(kThreads, 1) bwd_weight_tc_kernel(TrainBufs T, int l) {
    WeightShared& S = shared_block<WeightShared>();
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int lower = l - 1;
    setup(&S.tmem_base, S.bar, kWBufs, &S.abort_flag, 128, tid);
    sync_for_mma();
    const uint32_t tmem = S.tmem_base;
    const size_t plane = static_cast<size_t>(T.B) * kH;
    const int n_tiles = T.B / kTileRows;
    const int my_tiles = blockIdx.x < n_tiles ? (n_tiles - 1 - static_cast<int>(blockIdx.x)) / gridDim.x + 1 : 0;
    constexpr int kUnitsPerTile = kTileRows / kWPts;
    const int n_units = kUnitsPerTile * my_tiles;
    const int c0 = ((tid >> 3) & 15) * 8;             // this thread's 8 features (the same in every unit)
    float db8[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    bool ok = true;
    int last = -1;                                      // last unit whose MMAs were issued
    for (int u = 0; u < n_units; ++u) {
        const int b = u % kWBufs;
        if (u >= kWBufs) {                              // buffer b is free once unit u - kWBufs's MMAs completed
            const bool w = tc::mbar_wait_bounded(tc::smem_u32(&S.bar[b]),
                                                 static_cast<uint32_t>((u / kWBufs - 1) & 1), &S.abort_flag, T.err,
                                                 kDevErrTimeout);
            if (!__syncthreads_and(w)) {
                ok = false;
                break;
            }
        }
        const int tile = static_cast<int>(blockIdx.x) + static_cast<int>(gridDim.x) * (u / kUnitsPerTile);
        const int p0 = tile * kTileRows + (u % kUnitsPerTile) * kWPts;
        const uint32_t dbuf = tc::smem_u32(S.d[b][0]), xbuf = tc::smem_u32(S.x[b][0]);
#pragma unroll 1
        for (int it = tid; it < kWPts * kH / 8; it += kThreads) {
            const int r = (it >> 7) * 8 + (it & 7);     // point within the unit (K)
            const size_t off = static_cast<size_t>(p0 + r) * kH + c0;
            float a[8], d[4][8], t[3][8];
            load8(T.A[lower] + off, a);
            load8(T.dA[l] + off, d[0]);
#pragma unroll
            for (int s = 1; s < 4; ++s) load8(T.dAT[l] + static_cast<size_t>(s - 1) * plane + off, d[s]);
            if (lower == 1) {
#pragma unroll
                for (int s = 1; s < 4; ++s)
#pragma unroll
                    for (int j = 0; j < 8; ++j) t[s - 1][j] = __ldg(T.theta + oW1 + (c0 + j) * kIn + (s - 1));
            } else {
#pragma unroll
                for (int s = 1; s < 4; ++s) load8(T.AT[lower] + static_cast<size_t>(s - 1) * plane + off, t[s - 1]);
            }
            const uint32_t mo = mn_offset_bytes(c0, r);
            float x[8], sg[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                x[j] = sp_beta(a[j], T.beta);
                sg[j] = sig_beta(a[j], T.beta);
                db8[j] += d[0][j];
            }
            st_bf16x8(xbuf + mo, x);
            st_bf16x8(dbuf + mo, d[0]);
#pragma unroll
            for (int s = 1; s < 4; ++s) {
#pragma unroll
                for (int j = 0; j < 8; ++j) x[j] = sg[j] * t[s - 1][j];
                st_bf16x8(xbuf + static_cast<uint32_t>(s) * kWOpBytes + mo, x);
                st_bf16x8(dbuf + static_cast<uint32_t>(s) * kWOpBytes + mo, d[s]);
            }
        }
        sync_for_mma();
        if (tid == 0) {
#pragma unroll
            for (int s = 0; s < 4; ++s) {
                const uint64_t ad = tc::smem_desc(dbuf + static_cast<uint32_t>(s) * kWOpBytes, 128, kWSbo);
                const uint64_t bd = tc::smem_desc(xbuf + static_cast<uint32_t>(s) * kWOpBytes, 128, kWSbo);
#pragma unroll
                for (int kk = 0; kk < kWPts / 16; ++kk)
                    tc::mma_bf16(tmem, ad + static_cast<uint64_t>(kk * 16), bd + static_cast<uint64_t>(kk * 16),
                                 kIdescMN, (u > 0 || s > 0 || kk > 0) ? 1u : 0u);
            }
            tc::mma_commit(tc::smem_u32(&S.bar[b]));
        }
        __syncwarp();
        last = u;
    }
    if (ok && last >= 0) {                              // the last commit covers every earlier MMA
        const bool w = tc::mbar_wait_bounded(tc::smem_u32(&S.bar[last % kWBufs]),
                                             static_cast<uint32_t>((last / kWBufs) & 1), &S.abort_flag, T.err,
                                             kDevErrTimeout);
        ok = __syncthreads_and(w);
        if (ok) last = -1;
    }
    float* part = T.partial + static_cast<size_t>(blockIdx.x) * kNumParams;
    if (ok) {
        tc::fence_after_sync();
        const int wq = warp & 3, r = wq * 32 + lane;
        const uint32_t lane_addr = tmem + (static_cast<uint32_t>(wq * 32) << 16);
        {
            const int col0 = (warp >> 2) * kEpiCols;
            uint32_t v[32];
            if (n_units > 0) {
                tc::tmem_ld_32x32b_x32(lane_addr + static_cast<uint32_t>(col0), v);
                tc::tmem_wait_ld();
                tc::reg_fence32(v);
            } else {
#pragma unroll
                for (int j = 0; j < 32; ++j) v[j] = 0u;
            }
            float* dst = part + offW(l) + r * kH + col0;
#pragma unroll
            for (int j = 0; j < 32; ++j) dst[j] = __uint_as_float(v[j]);
        }
#pragma unroll
        for (int j = 0; j < 8; ++j) S.db[tid][j] = db8[j];
        __syncthreads();
        if (tid < kH) {
            // the threads that staged feature tid: (tid / 8) * 8 + q + 128 h, fixed order
            const int cb = (tid >> 3) * 8, e = tid & 7;
            float acc = 0.f;
#pragma unroll
            for (int h = 0; h < kThreads / 128; ++h)
#pragma unroll
                for (int q = 0; q < 8; ++q) acc += S.db[cb + q + 128 * h][e];
            part[offB(l) + tid] = acc;
        }
    }
    if (last >= 0 && tid == 0) {
        int dummy = 0;
        tc::mbar_wait_bounded(tc::smem_u32(&S.bar[last % kWBufs]), static_cast<uint32_t>((last / kWBufs) & 1), &dummy,
                              T.err, kDevErrTimeout);
    }
    teardown(tmem, 128, tid);
}

}  // namespace

cudaError_t configure_tc_train() {
    cudaError_t e = cudaFuncSetAttribute(fwd_hidden_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(kStreamSmem));
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(bwd_input_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 static_cast<int>(kStreamSmem));
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(bwd_weight_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 static_cast<int>(kWeightSmem));
    return e;
}

cudaError_t launch_fwd_hidden_tc(const TrainBufs& T, int l, int grid, cudaStream_t s) {
    fwd_hidden_tc_kernel<<<grid, kThreads, kStreamSmem, s>>>(T, l);
    return cudaGetLastError();
}

cudaError_t launch_bwd_input_tc(const TrainBufs& T, int l, int grid, cudaStream_t s) {
    bwd_input_tc_kernel<<<grid, kThreads, kStreamSmem, s>>>(T, l);
    return cudaGetLastError();
}

cudaError_t launch_bwd_weight_tc(const TrainBufs& T, int l, int grid, cudaStream_t s) {
    bwd_weight_tc_kernel<<<grid, kThreads, kWeightSmem, s>>>(T, l);
    return cudaGetLastError();
}

}  // namespace train
}  // namespace mppi
