// Launchers of the step kernels (host side, internal to the library).
#pragma once

#include <cuda_runtime.h>

#include <utility>

#include "common.cuh"

namespace mppi {

// Launch a kernel as a programmatic dependent of the preceding kernel in the
// stream: it may start while that kernel finishes; its griddepcontrol.wait
// (pdl_wait) orders its dependent reads.
template <typename... KArgs, typename... Args>
cudaError_t launch_dependent(bool pdl, void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                             Args&&... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = pdl ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

// raw Philox words for every (k, h), [K][H] (tests)
cudaError_t launch_noise_words(const StepParams& P, const StepBuffers& B, uint4* out, cudaStream_t s);
// (a) + (b) noise -> B.noise and rollouts -> B.pos, control / progress costs; with
// analytic != 0 the frame SDF cost is fused in
cudaError_t launch_rollout(const StepParams& P, const StepBuffers& B, int analytic, cudaStream_t s);
// (c) Gate-SDF MLP at every rollout state -> B.sdf (min over gates)
struct MlpWeights {
    const float* W1;        // [128][67]
    const float* Wt[3];     // W2..W4 transposed: [in][out], FP32
    const float* b[3];      // b2..b4
    const float* w5;        // [128]
    float b5;
    const uint16_t* Wbf[3]; // W2..W4 as BF16 in the tensor-core operand layout
    const uint16_t* Wh[3];  // W2..W4 as FP16 in the tensor-core operand layout
    const uint16_t* W1tc;   // layer-1 B operand [128][16] BF16: beta log2(e) W1[:, 0:3] as [hi, hi, lo, 0..]
    const uint8_t* W8[3];   // W2..W4 / (per-tensor weight scale) as E4M3 in the 8-bit operand layout
    float f8_dequant[3];    // weight scale x activation scale of each hidden GEMM (log2 units)
    float f8_inv_act[3];    // 1 / activation scale of the E4M3 inputs of the hidden GEMMs (log2 units)
};
// set the dynamic shared-memory limits (once per context, outside any stream capture)
cudaError_t configure_sdf_mlp_fp32();
cudaError_t configure_sdf_mlp_bf16();
cudaError_t launch_sdf_mlp_fp32(const StepParams& P, const StepBuffers& B, const MlpWeights& W, int num_sms,
                                cudaStream_t s);
cudaError_t launch_sdf_mlp_bf16(const StepParams& P, const StepBuffers& B, const MlpWeights& W, int num_sms,
                                cudaStream_t s);
cudaError_t launch_sdf_mlp_fp16(const StepParams& P, const StepBuffers& B, const MlpWeights& W, int num_sms,
                                cudaStream_t s);
cudaError_t launch_sdf_mlp_fp8(const StepParams& P, const StepBuffers& B, const MlpWeights& W, int num_sms,
                               cudaStream_t s);
// (d) costs -> weights -> weighted update -> plant step + shift (one kernel)
cudaError_t launch_cost_update(const StepParams& P, const StepBuffers& B, int mlp, cudaStream_t s);
cudaError_t configure_cost_update();
// blocks of the update kernel for K rollouts (sizes B.upart and B.bstat)
int update_blocks(int K);
// per-gate first-layer bias b1'_g = W1[:, 3:67] z_g + b1
cudaError_t launch_first_layer_bias(const float* W1, const float* b1, const float* latents, int G, int n_point,
                                    float* b1p, cudaStream_t s);
// tensor-core self-test (one 128x128x128 tile)
cudaError_t launch_tc_selftest(const uint16_t* A, const uint16_t* B, float* D, int* err, cudaStream_t s);

// ---------------------------------------------------------------- batched serving step
// One controller of a batched serving step (device memory): its parameters and buffers, where
// its inputs sit in the batch's input block and where its blocks and tiles start in the
// batched launches.  Every controller's results equal those of its own step (same kernels'
// arithmetic, same reduction orders).
constexpr int kBatchStateSlot = 24;    // floats reserved for a state in the batch's input block
struct BatchSlot {
    StepParams P;
    StepBuffers B;             // with the controller's output and error pointers set
    const float* W1;           // first-layer weights [128][n_point + 64] (MLP modes)
    const float* b1;           // [128]
    float* latents;            // the controller's latent buffer [max_gates][64]
    int n_point;               // point features of the first layer (3 + 6 pe_levels)
    int state_floats;          // 13 or 17
    int in_off;                // floats: state (kBatchStateSlot), then G x 8 poses, then G x 64 latents
    int roll_form;             // 0: 32 lanes x 2 steps, 1: 16 x 2, 2: 16 x 4, 3: rotor model
    int roll_block0;           // first block in the batched rollout launch
    int tile0;                 // first tile in the batched SDF launch
    int upd_block0;            // first block in the batched update launch
    int upd_R;                 // rollouts per update block
    int mlp;                   // SDF from the MLP (else analytic, folded into the rollout)
};
// Rollout form launch_rollout uses for P (0..3 as BatchSlot::roll_form) and the blocks of 128
// threads a batched launch gives it.
int rollout_form(const StepParams& P);
int rollout_batch_blocks(const StepParams& P);
// rollouts per update block for K rollouts (the per-controller update kernel's partition)
int update_rollouts_per_block(int K);
// The batched launches, all on one stream: inputs (state, gates, latents, first-layer biases)
// of every controller, rollouts, SDF (MLP modes; every controller shares the weights W and
// the softplus sharpness / encoding levels of P0) and costs / update / plant step.
cudaError_t launch_batch_prep(const BatchSlot* slots, int n, const float* inputs, cudaStream_t s);
cudaError_t launch_rollout_batch(const BatchSlot* slots, int n, int blocks, int max_h, cudaStream_t s);
cudaError_t launch_cost_update_batch(const BatchSlot* slots, int n, int blocks, int max_r, cudaStream_t s);
// pairs: run the CTA-pair form (only where sdf_batch_pairs_available); every controller's tiles
// then start at an even tile (tile0 even, its tile count rounded up to even) and tiles is even.
cudaError_t launch_sdf_batch(int sdf_mode, bool pairs, const BatchSlot* slots, int n, int tiles, const StepParams& P0,
                             const MlpWeights& W, int* err, int num_sms, cudaStream_t s);
// Whether this mode's batched SDF launch can run in the CTA-pair form (BF16 / FP16, after the
// kernels were configured on a device that holds the form's clusters).
bool sdf_batch_pairs_available(int sdf_mode);

// Store a message in the calling thread's error slot (read by mppi_last_error(NULL)).
void set_thread_error(const char* msg);
// Host helpers: BF16 / FP16 (round to nearest even) of a float.
uint16_t float_to_bf16(float f);
uint16_t float_to_f16(float f);
// Host helper: offset (in elements) of (row, k) in a 128 x k1 16-bit operand of 8 x 16-byte core
// matrices: LBO 128 B along K, SBO k1 / 8 x 128 B between 8-row groups.
inline int tc_operand_k_offset(int row, int k, int k1) { return (row >> 3) * (k1 * 8) + (k >> 3) * 64 + (row & 7) * 8 + (k & 7); }
// Host helper: offset (in elements) of (row, k) in the 128 x 16 layer-1 operand (LBO 128 B, SBO 256 B).
inline int tc_operand16_offset(int row, int k) { return (row >> 3) * 128 + (k >> 3) * 64 + (row & 7) * 8 + (k & 7); }
// Host helper: byte offset of (row, k) in the 128 x 128 E4M3 operand layout (LBO 128 B, SBO 1024 B).
inline int tc_operand8_offset(int row, int k) { return (row >> 3) * 1024 + (k >> 4) * 128 + (row & 7) * 16 + (k & 15); }
// Host helper: offset (in elements) of (row, col) in the 128 x 128 tensor-core operand layout.
inline int tc_operand_offset(int row, int col) {
    return ((row >> 3) * 16 + (col >> 3)) * 64 + (row & 7) * 8 + (col & 7);
}

}  // namespace mppi
