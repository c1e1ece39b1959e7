/*
 * mppi.h -- C ABI of the GB300 MPPI + Gate-SDF control-step library.
 *
 * One control step of a sampling-based MPPI controller whose rollouts are
 * scored by a gate-shaped signed distance field (Vision-Guided MPPI with a
 * neural Gate-SDF, Sec. IV, Eq. 5-10):
 *
 *   (a) sample K Gaussian control-noise sequences over a horizon of H steps
 *       from a counter-based Philox4x32-10 generator (Sec. IV-A, Eq. 5);
 *   (b) roll out K quadrotor trajectories with RK4 (Sec. IV-A);
 *   (c) query the gate SDF -- the exact rectangular-frame SDF or the Gate-SDF
 *       MLP g_phi(z, p) (Sec. III-B, Fig. 2) -- at every rollout state and
 *       fold the safety, progress and control costs (Eq. 8-10);
 *   (d) turn the costs into softmax weights and the weighted control update
 *       (Eq. 5), apply the first action and shift the sequence (receding
 *       horizon, Sec. IV-A).
 *
 * Conventions for every call:
 *   - All floats are IEEE binary32, row-major, SI units.  A state is 13
 *     floats [p(3), v(3), q(4) = (w, x, y, z), w_body(3)] (MPPI_DYN_ROTOR: 17, the
 *     rotor thrusts T1..T4 appended); a control is 4 floats [collective thrust T (N),
 *     body rates wx, wy, wz (rad/s)] (MPPI_DYN_ROTOR: the rotor-thrust rates); a gate
 *     pose is 7 floats [t(3), q(4) (w, x, y, z) rotating gate -> world]; the
 *     gate plane is x = 0 of the gate frame and its normal is R(q) e_x.
 *   - The caller owns every pointer it passes.  The library never keeps a
 *     caller pointer after the call returns.
 *   - Return value: MPPI_OK (0) or a negative MPPI_E_* code; the message is
 *     available from mppi_last_error().  The library never aborts or traps.
 *   - A context is bound to the CUDA device that was current at
 *     mppi_create() and to one CUDA stream.  Calls on one context must not
 *     overlap (not thread-safe per context); distinct contexts are
 *     independent.
 */
#ifndef MPPI_GB300_H
#define MPPI_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---- */
#define MPPI_OK             0
#define MPPI_E_INVALID     -1   /* bad argument, NaN/Inf input, size out of range */
#define MPPI_E_OOM         -2   /* device or pinned host allocation failed */
#define MPPI_E_CUDA        -3   /* a CUDA runtime call failed (message has the CUDA error) */
#define MPPI_E_TIMEOUT     -4   /* a device-side bounded wait gave up; the context stays usable */
#define MPPI_E_NOT_READY   -5   /* weights or gates required by the SDF mode are not set */
#define MPPI_E_UNSUPPORTED -6   /* the device is not an sm_103 GPU or the mode is not built */
#define MPPI_E_ADMISSION   -7   /* a serving request can never fit in the device-memory budget */
#define MPPI_PENDING        1   /* mppi_server_poll: the request is queued or running */

/* ---- SDF evaluation modes (mppi_config.sdf_mode) ---- */
#define MPPI_SDF_ANALYTIC  0    /* exact signed distance to the rectangular gate frame */
#define MPPI_SDF_MLP_FP32  1    /* Gate-SDF MLP, FP32 on the CUDA cores (plain FP32 path) */
#define MPPI_SDF_MLP_BF16  2    /* Gate-SDF MLP, hidden GEMMs in BF16 on tcgen05, FP32 accumulate */
#define MPPI_SDF_MLP_FP16  3    /* Gate-SDF MLP, hidden GEMMs in FP16 on tcgen05, FP32 accumulate,
                                   activations packed f16x2 between layers */
#define MPPI_SDF_MLP_FP8   4    /* Gate-SDF MLP, hidden GEMMs in FP8 E4M3 on tcgen05 (per-tensor scales),
                                   FP32 accumulate */

/* Gate-SDF MLP shape: [p(3), z(MPPI_LATENT_DIM)] -> 4 x MPPI_HIDDEN softplus -> 1. */
#define MPPI_LATENT_DIM 64
#define MPPI_HIDDEN     128
#define MPPI_MLP_LAYERS 5       /* affine maps */
#define MPPI_MAX_GATES  8
#define MPPI_MAX_K      (1 << 20)
#define MPPI_MAX_H      1024

/*
 * Controller parameters.  mppi_config_default() fills the values of the
 * single-gate hover workload (K = 256, H = 20).
 *   K, H          rollouts and horizon steps (1 <= K <= MPPI_MAX_K, 1 <= H <= MPPI_MAX_H)
 *   max_gates     gate capacity of the context (1 .. MPPI_MAX_GATES)
 *   sdf_mode      MPPI_SDF_*
 *   dt, mass, gravity                 RK4 step (s), vehicle mass (kg), g (m/s^2)
 *   thrust_min/max, rate_max          control box: T in [min, max], |w_i| <= rate_max
 *   sigma_thrust, sigma_rate          noise standard deviations (Sigma = diag)
 *   lambda                            temperature of Eq. 5 (> 0)
 *   w_col, d_safe, w_u                cost weights: w_col max(0, d_safe - s)^2 per
 *                                     state, w_u |u - u_hover|^2 per control
 *   gate_inner_half, gate_outer_half, gate_half_depth   frame geometry (m)
 *   softplus_beta                     sharpness of the MLP's softplus
 *   seed, drone_id                    Philox key and the counter's 4th word
 *   cost_mode                         MPPI_COST_CONFIGURED (w_col, w_u and the progress
 *                                     along the target gate's normal) or MPPI_COST_PAPER
 *   q_gate, q_vis, q_sdf              weights of Eq. 9 (MPPI_COST_PAPER): waypoint progress
 *                                     (Eq. 6), perception alignment (Eq. 7) and the linear SDF
 *                                     hinge max(0, d_safe - s) (Eq. 8) on the target gate
 *   guide_tan_alpha                   tan of the cone angle of the guidance SDF (Eq. 2), the
 *                                     analytic SDF of MPPI_COST_PAPER
 *   dynamics_mode                     MPPI_DYN_CTBR (u = collective thrust + body rates, the
 *                                     body rate tracked ideally) or MPPI_DYN_ROTOR (u = the
 *                                     four rotor-thrust rates, Sec. IV-A; the state adds the
 *                                     rotor thrusts)
 *   tdot_max, rotor_thrust_max        MPPI_DYN_ROTOR bounds: |u_i| <= tdot_max (N/s), each rotor
 *                                     thrust clamped to [0, rotor_thrust_max] (N) after a step
 *   sigma_tdot                        MPPI_DYN_ROTOR noise standard deviation (N/s)
 *   arm_length, torque_coeff          X layout arm (m) and rotor reaction torque per newton (m)
 *   inertia_x, inertia_y, inertia_z   diagonal inertia (kg m^2)
 *   pe_levels                         positional-encoding levels L of the decoder's query point
 *                                     (Sec. III-B): the MLP sees [PE(p), z] with PE(p) = [p, then
 *                                     sin(2^l pi p), cos(2^l pi p) for l < L] (3 + 6 L numbers);
 *                                     0 .. MPPI_MAX_PE_LEVELS, 0 = the raw point
 */
typedef struct mppi_config {
    int32_t K;
    int32_t H;
    int32_t max_gates;
    int32_t sdf_mode;
    float dt, mass, gravity;
    float thrust_min, thrust_max, rate_max;
    float sigma_thrust, sigma_rate, lambda;
    float w_col, d_safe, w_u;
    float gate_inner_half, gate_outer_half, gate_half_depth;
    float softplus_beta;
    uint64_t seed;
    uint32_t drone_id;
    int32_t cost_mode;
    float q_gate, q_vis, q_sdf;
    float guide_tan_alpha;
    int32_t dynamics_mode;
    float tdot_max, rotor_thrust_max, sigma_tdot;
    float arm_length, torque_coeff;
    float inertia_x, inertia_y, inertia_z;
    int32_t pe_levels;
} mppi_config;

#define MPPI_MAX_PE_LEVELS 6

/* Dynamics models (mppi_config.dynamics_mode). */
#define MPPI_DYN_CTBR   0       /* state [p, v, q, w] (13); u = [T, wx, wy, wz], ideal body-rate tracking */
#define MPPI_DYN_ROTOR  1       /* state [p, v, q, w, T1..T4] (17); u = [dT1/dt .. dT4/dt], rigid body with
                                   the rotors' torques (X layout) */
#define MPPI_STATE_MAX  17

/* Number of floats of a state under cfg: 13 (MPPI_DYN_CTBR) or 17 (MPPI_DYN_ROTOR). */
int mppi_state_dim(const mppi_config* cfg);

/* Cost forms (mppi_config.cost_mode). */
#define MPPI_COST_CONFIGURED 0  /* w_col max(0, d_safe - s)^2 + progress along the target gate's normal
                                   + w_u |u - u_hover|^2; s = min over gates */
#define MPPI_COST_PAPER      1  /* Q_gate J_gate + Q_vis J_vis + Q_sdf J_sdf (Eq. 6-9) on the target gate */

typedef struct mppi_ctx mppi_ctx;

/* Fill *cfg with the defaults listed above. */
void mppi_config_default(mppi_config* cfg);

/*
 * Create a controller: the MPPI problem of Sec. IV-A (K sampled control
 * sequences over a horizon of H steps, Eq. 5) with its cost of Sec. IV-B
 * (Eq. 6-10) for one vehicle.  cuda_stream is a cudaStream_t (NULL: the library
 * creates and owns a non-blocking stream).  Allocates every device buffer the
 * step needs for (K, H, max_gates); later calls allocate nothing on the
 * device.  Initial state: hovering at the origin, nominal = H copies of
 * u_hover = (mass * gravity, 0, 0, 0) (the warm start of Sec. IV-A before any
 * step has run), step counter 0, no gates, no weights.
 * Errors: MPPI_E_INVALID (cfg), MPPI_E_UNSUPPORTED (device), MPPI_E_OOM, MPPI_E_CUDA.
 * On error *out is NULL (the message is in the thread's last-error slot,
 * readable with mppi_last_error(NULL)).
 */
int mppi_create(const mppi_config* cfg, void* cuda_stream, mppi_ctx** out);

/* Free the context and its device buffers (the controller of mppi_create, Sec. IV-A); waits for
 * its stream first.  NULL is ignored. */
void mppi_destroy(mppi_ctx* ctx);

/* Last error message of ctx (or of the calling thread's last failed create when ctx is NULL).  The
 * paper defines no error reporting; the string is owned by the library and valid until the next
 * call on ctx (or, for NULL, the next failing call of this thread). */
const char* mppi_last_error(const mppi_ctx* ctx);

/*
 * Set the gates in view (host pointers).  poses: n_gates x 7; latents:
 * n_gates x MPPI_LATENT_DIM (the per-gate latent code z of the Gate-SDF
 * decoder, Sec. III-B; may be NULL in MPPI_SDF_ANALYTIC mode).  0 <= n_gates
 * <= max_gates.  With no gates the collision and progress costs are zero.
 * Synchronous.
 */
int mppi_set_gates(mppi_ctx* ctx, int n_gates, const float* poses, const float* latents);

/*
 * Set the Gate-SDF MLP weights (host pointers, FP32): layers[2*i] is W_i
 * [out_i x in_i] row-major and layers[2*i+1] its bias [out_i], for the five
 * affine maps (3 + 6 pe_levels + 64) -> 128 -> 128 -> 128 -> 128 -> 1 (67 -> ... without
 * positional encoding; n_layers = 10 pointers).  The library keeps FP32 copies and the
 * BF16 / FP16 / E4M3 copies the tensor-core paths use, and precomputes the per-gate
 * first-layer bias W1[:, P:] z_g + b1 (P = 3 + 6 pe_levels).  fp8_scales (MPPI_SDF_MLP_FP8 only; nullable): 3
 * per-tensor scales of the E4M3 activations entering the three hidden
 * 128 x 128 layers, in softplus-output units (an activation a is stored as
 * E4M3(a / scale), saturating at 448 scale); NULL selects 1/64.  The E4M3
 * weight scales are max|W| / 448 per tensor.  Synchronous.
 */
int mppi_set_sdf_weights(mppi_ctx* ctx, const float* const* layers, int n_layers, const float* fp8_scales);

/*
 * One control step, host buffers, synchronous.
 *   state        mppi_state_dim(cfg) floats, or NULL to continue from the device-resident state
 *                (advanced by the previous step's plant update)
 *   gate_poses   n_gates x 7, or NULL to keep the current gates
 *   latents      n_gates x 64, or NULL to keep the current latents
 *   nominal      H x 4 initial sequence U*, or NULL for the device-resident
 *                warm start (previous step's U* shifted by one)
 *   new_controls H x 4 out: the updated sequence U*_new of Eq. 5 (required)
 *   weights      K out: w_m of Eq. 5 (nullable)
 *   costs        K out: J_m (nullable)
 * After the update the library applies U*_new[0] to its device-resident
 * state with one RK4 step, stores U*_new shifted left by one (u_hover
 * appended) as the next warm start and increments the step counter that
 * keys the noise.
 * Errors: MPPI_E_INVALID (NaN/Inf in state, NULL new_controls),
 * MPPI_E_NOT_READY, MPPI_E_TIMEOUT, MPPI_E_CUDA.
 */
int mppi_step(mppi_ctx* ctx, const float* state, const float* gate_poses, const float* latents,
              const float* nominal, float* new_controls, float* weights, float* costs);

/*
 * Same as mppi_step with DEVICE pointers (same shapes, same NULL rules),
 * enqueued on the context's stream and returned without synchronising; the
 * outputs are valid once the stream has reached this point.  No host-side
 * NaN check.  d_new_controls must be 16-byte aligned (it is written as
 * float4); a misaligned or NULL d_new_controls returns MPPI_E_INVALID with
 * nothing enqueued.  Device-side timeouts are reported by the next
 * synchronous call (mppi_sync, mppi_step, mppi_get_*).
 */
int mppi_step_async(mppi_ctx* ctx, const float* d_state, const float* d_gate_poses, const float* d_latents,
                    const float* d_nominal, float* d_new_controls, float* d_weights, float* d_costs);

/* Wait for the context's stream and report any device-side error. */
int mppi_sync(mppi_ctx* ctx);

/* Read back the device-resident warm-start sequence (H x 4: the previous U*_new shifted by one,
 * u_hover appended -- the receding-horizon initialisation of Sec. IV-A) / the true state
 * (mppi_state_dim floats, after the plant step that applied U*_new[0]).  Synchronous. */
int mppi_get_nominal(mppi_ctx* ctx, float* out);
int mppi_get_state(mppi_ctx* ctx, float* out);

/* Overwrite the step counter that keys the Philox noise (the counter's 3rd word is its low 32 bits). */
int mppi_set_step_counter(mppi_ctx* ctx, uint64_t step);
uint64_t mppi_get_step_counter(const mppi_ctx* ctx);

/*
 * Copy one of the last step's intermediate buffers to host memory (tests and
 * diagnostics).  n is the number of floats the caller's buffer holds; it must
 * be at least the buffer's size.  Synchronous.
 *   MPPI_BUF_NOISE      K x H x 4  delta u, layout [k][h][4] (h fastest)
 *   MPPI_BUF_POSITIONS  K x H x 4  rollout positions p_1..p_H, [k][h][x,y,z,0]
 *   MPPI_BUF_COST_PARTS 3 x K      [J_col; J_prog; J_ctl] (MPPI_COST_PAPER: [Q_sdf J_sdf; Q_gate J_gate; Q_vis J_vis])
 *   MPPI_BUF_SDF        K x H      s(p_h) = min over gates of the SDF at every rollout state, [k][h] (MLP
 *                                  modes; written only while MPPI_DIAG_STORE_SDF is set, else MPPI_E_INVALID)
 *   MPPI_BUF_WEIGHTS    K
 *   MPPI_BUF_COSTS      K
 */
#define MPPI_BUF_NOISE       0
#define MPPI_BUF_POSITIONS   1
#define MPPI_BUF_COST_PARTS  2
#define MPPI_BUF_SDF         3
#define MPPI_BUF_WEIGHTS     4
#define MPPI_BUF_COSTS       5
int mppi_read_buffer(mppi_ctx* ctx, int which, float* host_out, size_t n);

/*
 * Diagnostics of the following steps (a bit mask; 0 = none, the default):
 *   MPPI_DIAG_STORE_SDF  the SDF kernel also stores s(p) of every rollout state for
 *                        MPPI_BUF_SDF (K x H floats written per step).  Without it the kernel
 *                        folds the safety cost of Eq. 8 over each rollout's states in its
 *                        epilogue (Eq. 9-10) and writes only K x (floor((H + 126) / 128) + 1)
 *                        partial sums; the step's results are bit-identical either way.
 *   MPPI_DIAG_SDF_SINGLE_CTA  the BF16 / FP16 SDF MLP kernel (without positional encoding) runs
 *                        in its single-CTA form (three tiles of 128 states in flight per SM, the
 *                        whole hidden weights in every CTA) instead of the default CTA-pair form
 *                        (clusters of two CTAs issuing 256-row tcgen05 MMAs, each CTA holding half
 *                        of every hidden weight matrix and four tiles in flight); for comparisons.
 * Errors: MPPI_E_INVALID (unknown bit).
 */
#define MPPI_DIAG_STORE_SDF 1
#define MPPI_DIAG_SDF_SINGLE_CTA 2
int mppi_set_diagnostics(mppi_ctx* ctx, int flags);

/*
 * Raw Philox4x32-10 words of the step's noise for the current step counter
 * (K x H x 4 uint32, [k][h][word]), produced by the same device function the
 * rollout kernel draws its noise with.  For bit-exact tests.  Synchronous.
 */
int mppi_read_noise_words(mppi_ctx* ctx, uint32_t* host_out, size_t n);

/*
 * Test hook for the failure path (no GPU fault is involved): the next step's update
 * kernel waits at its grid barrier for arrivals that never come, so every one of its
 * blocks gives up after its bounded wait (2 s of %globaltimer) and returns.  That step
 * reports MPPI_E_TIMEOUT (mppi_step, or mppi_sync after mppi_step_async); the device
 * error word and the barrier state are then reset and the context steps normally again.
 * The controls and warm start of the failed step are unspecified.  Synchronous.
 */
int mppi_debug_inject_timeout(mppi_ctx* ctx);

/*
 * Per-kernel timing of the last step run with timing enabled (milliseconds,
 * CUDA events on the context's stream).  mppi_set_timing(ctx, 1) makes each
 * following step record events around its kernels (this adds event records
 * to the stream); names[i] are static strings.  Returns the number of
 * entries written (<= cap) or a negative error.
 */
int mppi_set_timing(mppi_ctx* ctx, int enable);
int mppi_get_kernel_times(mppi_ctx* ctx, const char** names, float* ms, int cap);

/* Number of kernel launches one step makes in the context's current mode. */
int mppi_kernels_per_step(const mppi_ctx* ctx);

/*
 * Self-test of the tensor-core path: D = A * B^T for one 128 x 128 x 128
 * tile through the same shared-memory layout, tcgen05.mma and TMEM read-back
 * the BF16 SDF kernel uses.  d_A: 128 x 128 BF16 (row-major, rows = M),
 * d_B: 128 x 128 BF16 (row-major, rows = N, columns = K), d_D: 128 x 128 FP32
 * row-major; device pointers.  stream may be NULL (default stream).
 * Synchronous.  Returns MPPI_E_UNSUPPORTED off sm_103.
 */
int mppi_selftest_tc_gemm(const uint16_t* d_A, const uint16_t* d_B, float* d_D, void* stream);

/*
 * Allocation-free softmax weights and weighted control update, for costs the
 * caller computed elsewhere.  The paper has no counterpart: this entry point
 * exists for callers that cannot allocate device memory -- code that runs
 * inside a CUDA stream capture, real-time control loops that forbid allocation
 * after start-up (cudaMalloc can synchronise the device and take unbounded
 * time), and hosts whose device memory belongs to another allocator.  It
 * needs no context and calls no cudaMalloc, cudaFree or other allocating
 * routine.
 *   d_costs         K floats, the rollout costs J_m (device)
 *   d_noise         H x K x 4 floats, delta u in the layout [h][k][4] (the transpose of MPPI_BUF_NOISE) (device)
 *   d_nominal       H x 4 floats, the nominal sequence U* (device)
 *   K, H            1 <= K <= MPPI_NOALLOC_MAX_K, 1 <= H <= MPPI_MAX_H
 *   lambda          temperature (> 0); thrust_min <= thrust_max, rate_max >= 0:
 *                   the control box applied to U*_h + delta before weighting
 *   d_new_controls  H x 4 out: U*_new[h] = sum_k w_k clip(U*_h + delta_{k,h}) (device)
 *   d_weights       K out: w_k = exp(-(J_k - min J) / lambda) / sum (device, nullable)
 *   stream          cudaStream_t (NULL: the legacy default stream)
 * d_noise, d_nominal and d_new_controls must be 16-byte aligned (they are read and
 * written as float4); a misaligned pointer returns MPPI_E_INVALID with nothing enqueued.
 * Enqueues two kernels and returns; the outputs are valid once the stream
 * has reached them.  Scratch: a file-scope device array of 2 * 1024 floats
 * (8 KB) that every GPU which loads this library holds until the process
 * exits; it caps K at MPPI_NOALLOC_MAX_K.  The first call on each device looks
 * up the array's device address with that device current (cudaGetSymbolAddress);
 * make that first call before any stream capture.  Calls made outside a capture
 * look the address up again, so a device reset between calls is harmless; a call
 * inside a capture uses the address of the last call outside one.  Every call on a device
 * shares the array and each call overwrites what it uses (nothing needs to
 * start at zero), so calls whose kernels overlap on the GPU -- on different
 * streams, or from several host threads -- race and must not be issued.
 * Errors: MPPI_E_INVALID (NULL pointer, K or H out of range, bad lambda or
 * bounds; nothing is enqueued), MPPI_E_CUDA; the message is read with
 * mppi_last_error(NULL).
 */
#define MPPI_NOALLOC_MAX_K 131072
int mppi_softmax_update_noalloc(const float* d_costs, const float* d_noise, const float* d_nominal, int K, int H,
                                float lambda, float thrust_min, float thrust_max, float rate_max,
                                float* d_new_controls, float* d_weights, void* stream);

/* ======================================================================== vision front end: depth images
 * The onboard observation of Sec. III-B: a first-person depth image of the
 * gates, which the paper renders with a simulator (Sec. III-A, V) and from
 * which its encoder infers the latent z.  mppi_render_depth casts one ray per
 * pixel through a pinhole camera and returns the depth of the first point of
 * any gate frame on it (exact ray--frame intersection, no graphics API), for
 * many camera poses at once; optionally it adds the synthetic sensor noise of
 * the denoising pre-training stage (Sec. III-B, I_noisy).  Readings (the
 * paper gives neither a camera model nor its noise model):
 *   - camera frame x forward (optical axis), y left, z up; a camera pose is 7
 *     floats [t(3), q(4) (w, x, y, z) rotating camera -> world];
 *   - pixel (u, v), u to the right, v down, looks along
 *     (1, -(u + 1/2 - cx) / fx, -(v + 1/2 - cy) / fy); its depth is the
 *     optical-axis coordinate z of the first frame point on that ray (z >= 0),
 *     or max_range when there is none at or before max_range;
 *   - a gate frame is {|x| <= d, a_in <= max(|y|, |z|) <= a_out} in its gate
 *     frame (the solid of the analytic SDF);
 *   - noise: with p = v * width + u, the pixel's dropout uniform r is word
 *     (p mod 4) of the Philox4x32-10 block with key = seed and counter
 *     (p / 4, view, frame, 0xDE9751), and its normal n is the cosine (p even)
 *     or sine (p odd) Box-Muller normal of words 0, 1 of the block with
 *     counter (p / 2, view, frame, 0xDE9750) (uniforms and Box-Muller as in the
 *     control noise); the pixel reads 0 when r < dropout, else max_range when
 *     its clean depth is max_range, else clip(z + noise_depth_coeff z^2 n, 0,
 *     max_range).
 */
#define MPPI_MAX_IMAGE_SIDE   8192
#define MPPI_MAX_RENDER_GATES 64

typedef struct mppi_depth_camera {
    int32_t width, height;          /* pixels, 1 .. MPPI_MAX_IMAGE_SIDE each */
    float fx, fy, cx, cy;           /* pinhole intrinsics (pixels); fx, fy > 0 */
    float max_range;                /* m, > 0: depth of a pixel that sees no frame */
    float gate_inner_half, gate_outer_half, gate_half_depth;   /* frame geometry (m) */
    float noise_depth_coeff;        /* c of the noise sigma = c z^2 (1/m), >= 0; 0 = no Gaussian noise */
    float dropout;                  /* probability in [0, 1] that a pixel reads 0 */
    uint64_t seed;                  /* Philox key of the noise */
    uint32_t frame;                 /* Philox counter word 2 of the noise (e.g. an image index) */
    uint32_t reserved;              /* must be 0 */
} mppi_depth_camera;

/* Defaults: 640 x 480, fx = fy = 385, cx = 320, cy = 240 (a 80 x 64 degree field of view),
 * max_range 10 m, the 1.5 m / 1.0 m / 0.2 m frame, no noise, seed 0, frame 0. */
void mppi_depth_camera_default(mppi_depth_camera* cam);
/*
 * Render n_views depth images (device pointers, enqueued on stream):
 *   cam           camera intrinsics, range, frame geometry and noise (host struct)
 *   n_views       0 .. 2^24 camera poses
 *   d_cam_poses   n_views x 7 floats (device)
 *   n_gates       0 .. MPPI_MAX_RENDER_GATES gate poses (0: every pixel reads max_range,
 *                 or 0 where it drops out)
 *   d_gate_poses  n_gates x 7 floats (device; NULL when n_gates = 0)
 *   d_depth       n_views x height x width floats out (device), [view][v][u]
 *   stream        cudaStream_t (NULL: the legacy default stream)
 * Enqueues one kernel and returns.  Non-finite poses give unspecified (but
 * finite) depths.  Errors: MPPI_E_INVALID (NULL pointer, a size or parameter
 * out of range; nothing is enqueued), MPPI_E_CUDA; the message is read with
 * mppi_last_error(NULL).
 */
int mppi_render_depth(const mppi_depth_camera* cam, int n_views, const float* d_cam_poses, int n_gates,
                      const float* d_gate_poses, float* d_depth, void* stream);

/*
 * Training queries for the SDF supervision of the encoder (Sec. III-A samples points in
 * the camera frame and labels them with the analytic SDF): n_points camera-frame points per
 * view and the exact signed distance of the nearest gate frame at each.  For point j of
 * view i, Philox4x32-10 blocks A = (j, i, frame, 0x5DF0A) and B = (j, i, frame, 0x5DF0B)
 * with key = cam->seed (uniforms as in the control noise) give: when uA3 < near_frac, a
 * point near gate g = ((A0 >> 8) n_gates) >> 24, uniform in its frame's box grown by
 * 0.3 m ((2 uB0 - 1)(d + 0.3), (2 uB1 - 1)(a_out + 0.3), (2 uB2 - 1)(a_out + 0.3)) in the
 * gate frame; else a point of the view frustum at depth 0.2 + uA1 (max_range - 0.2) on
 * the ray through image position (width uA2, height uB3) (the pinhole camera of
 * mppi_render_depth, standing in for the depth camera of Sec. III-B and Sec. V).
 *   cam           intrinsics, max_range (> 0.2), frame geometry, seed and frame
 *   n_views       0 .. 2^24 camera poses (device, n_views x 7)
 *   n_gates       1 .. MPPI_MAX_RENDER_GATES gate poses (device, n_gates x 7)
 *   n_points      1 .. 2^20 points per view (n_views x n_points <= 2^31)
 *   d_points      n_views x n_points x 3 floats out (device), camera frame
 *   d_labels      n_views x n_points floats out (device)
 * One kernel on stream.  Errors: MPPI_E_INVALID, MPPI_E_CUDA (mppi_last_error(NULL)).
 */
int mppi_sample_sdf_queries(const mppi_depth_camera* cam, int n_views, const float* d_cam_poses, int n_gates,
                            const float* d_gate_poses, int n_points, float near_frac, float* d_points,
                            float* d_labels, void* stream);

/* ======================================================================== vision front end: depth encoder
 * The depth encoder E_theta of Sec. III-B, which maps the current depth image
 * to the latent code z once per control cycle (Sec. IV-B).  The paper gives
 * neither its architecture nor its weights; the reading built here is a small
 * convolutional encoder of an H x W depth image:
 *     x_0 = depth / max_range                               (1 channel)
 *     x_l = relu(conv3x3, stride 2, zero padding 1 (x_{l-1}))  l = 1..4,
 *           16, 32, 64, 64 channels, H_l = ceil(H_{l-1} / 2)
 *     z   = W_5 mean_{pixels}(x_4) + b_5                    (64 -> 64)
 * with out[co][i][j] = b[co] + sum_{ci,ky,kx} W[co][ci][ky][kx]
 * x[ci][2i+ky-1][2j+kx-1].  The weights are inputs (e.g. of a trained
 * encoder); the library does not train them.
 */
#define MPPI_ENCODER_LAYERS 5
typedef struct mppi_encoder mppi_encoder;
/*
 * Create an encoder for depth images of height x width pixels (1 ..
 * MPPI_MAX_IMAGE_SIDE) and batches of up to max_images (1 .. 65535) images:
 *   layers     n_arrays = 10 host arrays W1, b1, W2, b2, W3, b3, W4, b4, W5, b5:
 *              W_l [c_out][c_in][3][3] (c_in = 1, 16, 32, 64; c_out = 16, 32, 64, 64),
 *              b_l [c_out], W5 [64][64] row-major, b5 [64]; copied before the call returns
 *   stream     cudaStream_t the encoder's work goes to (NULL: the legacy default stream)
 *   *out       the encoder (NULL on error); it holds the weights and the
 *              activations of max_images images on the current device
 * Errors: MPPI_E_INVALID, MPPI_E_OOM, MPPI_E_CUDA; message from mppi_encoder_last_error(NULL).
 */
int mppi_encoder_create(int height, int width, int max_images, const float* const* layers, int n_arrays,
                        void* stream, mppi_encoder** out);
/* Wait for the encoder's stream and free it.  NULL is ignored. */
void mppi_encoder_destroy(mppi_encoder* enc);
/* Message of the encoder's last error (enc NULL: the calling thread's last failed create). */
const char* mppi_encoder_last_error(const mppi_encoder* enc);
/*
 * Enqueue the encoding of n_images (0 .. max_images) depth images:
 *   d_depth    n_images x height x width floats (device), e.g. from mppi_render_depth
 *   max_range  the depth scale (> 0): inputs are depth / max_range
 *   d_latents  n_images x 64 floats out (device)
 * Five kernels on the encoder's stream; calls on one encoder must not overlap.
 * Errors: MPPI_E_INVALID (nothing enqueued), MPPI_E_CUDA.
 */
int mppi_encode_depth(mppi_encoder* enc, int n_images, const float* d_depth, float max_range, float* d_latents);

/*
 * Convolution kernels of the encoder's four layers (the same arithmetic as above, Sec. III-B):
 *   MPPI_ENC_CONV_TC    (the default) tcgen05 tensor cores: each input and weight split into
 *                       a BF16 high part and a BF16 remainder, the three products hi.hi +
 *                       hi.lo + lo.hi accumulated in FP32 (each product within ~2^-16 of
 *                       its FP32 value); one CTA per 128 output pixels, no split reduction.
 *                       A bounded wait that gives up sets the encoder's error word
 *                       (mppi_encoder_check reports it).
 *   MPPI_ENC_CONV_FP32  FP32 implicit GEMMs on the CUDA cores.
 * Applies to later mppi_encode_depth calls and to the trainer's forward passes.
 * Errors: MPPI_E_INVALID (NULL encoder, unknown path).
 */
#define MPPI_ENC_CONV_FP32 0
#define MPPI_ENC_CONV_TC   1
int mppi_encoder_set_conv_path(mppi_encoder* enc, int path);
/*
 * Wait for the encoder's stream and read its device error word: MPPI_OK, or
 * MPPI_E_TIMEOUT when a tensor-core convolution gave up a bounded wait since the last
 * check (the word is cleared; the latents of that call are not valid).  MPPI_E_CUDA when
 * the stream itself failed.
 */
int mppi_encoder_check(mppi_encoder* enc);
/*
 * Test hook for the tensor-core convolutions' failure path (no GPU fault is involved): in the
 * next mppi_encode_depth, every CTA of the first convolution waits for a phase of its
 * weight-copy barrier that never completes, gives up after its bounded wait (2 s of
 * %globaltimer), sets the encoder's error word and returns; mppi_encoder_check then reports
 * MPPI_E_TIMEOUT once and the encoder works normally again.  The latents of that call are
 * unspecified.  Errors: MPPI_E_INVALID (NULL encoder, or the FP32 convolution path).
 */
int mppi_encoder_debug_inject_timeout(mppi_encoder* enc);

/*
 * Copy the encoder's current weights to host arrays (same 10 arrays and layouts as
 * mppi_encoder_create; a NULL entry is skipped).  Synchronous.
 */
int mppi_encoder_get_weights(mppi_encoder* enc, float* const* layers_out);

/* ======================================================================== vision front end: encoder training
 * Denoising training of the depth encoder: the reconstruction term of the first
 * (simulation) training stage of Sec. III-B.  The encoder reads noisy depth
 * images (e.g. mppi_render_depth with sensor noise); a depth decoder D_psi maps
 * each latent back to a coarse clean image; the L1 loss between the two is
 * minimised with Adam.  Readings (the paper gives neither D_psi nor its
 * resolution): the target is the clean image scaled by 1 / max_range and
 * averaged over 8 x 8 pixel blocks (edge blocks average the pixels they hold),
 * T = ceil(H / 8) x ceil(W / 8) values; D_psi is one affine map 64 -> T; the
 * loss is mean |D_psi(E(noisy)) - target| with d|r|/dr = sign(r) (0 at 0);
 * Adam beta1 = 0.9, beta2 = 0.999, eps = 1e-8, bias-corrected.  The SDF term
 * (below) runs through a frozen Gate-SDF decoder.  The trainer updates the encoder's weights in place, so
 * mppi_encode_depth uses the trained encoder; it uses the encoder's stream and
 * activations, so encoder calls must not overlap trainer calls.
 */
typedef struct mppi_encoder_trainer mppi_encoder_trainer;
/*
 * enc      the encoder to train (outlives the trainer); batch 1 .. its max_images
 * lr       Adam step size (> 0)
 * dec_W    T x 64 host floats (row-major), dec_b T host floats: D_psi's initial weights
 * Errors: MPPI_E_INVALID, MPPI_E_OOM, MPPI_E_CUDA; message from mppi_encoder_train_last_error(NULL).
 */
int mppi_encoder_train_create(mppi_encoder* enc, int batch, float lr, const float* dec_W, const float* dec_b,
                              mppi_encoder_trainer** out);
void mppi_encoder_train_destroy(mppi_encoder_trainer* trainer);
const char* mppi_encoder_train_last_error(const mppi_encoder_trainer* trainer);
/*
 * Loss and gradients of one batch without updating anything:
 *   n                 1 .. batch images
 *   d_noisy, d_clean  n x H x W floats each (device): encoder input and reconstruction source
 *   max_range         depth scale (> 0)
 *   loss              host float out (nullable): mean |r|
 *   grads_out         12 host arrays (nullable; NULL entries skipped): dL/dW1, dL/db1, ..,
 *                     dL/dW4, dL/db4, dL/dW5, dL/db5 (encoder layouts), dL/dW_D, dL/db_D
 * Synchronous when loss or grads_out is given; a synchronous call reports MPPI_E_TIMEOUT (its
 * results then unspecified) when a bounded wait of the tensor-core convolutions gave up.
 */
int mppi_encoder_train_loss_grads(mppi_encoder_trainer* trainer, int n, const float* d_noisy, const float* d_clean,
                                  float max_range, float* loss, float* const* grads_out);
/* One training step (loss and gradients of the batch, then Adam on all 12 tensors); loss as above. */
int mppi_encoder_train_step(mppi_encoder_trainer* trainer, int n, const float* d_noisy, const float* d_clean,
                            float max_range, float* loss);
/*
 * The SDF term of the same stage: L = lambda_recon L_recon + lambda_sdf mean
 * |g_phi(z_i, PE(p_ij)) - s_ij| over camera-frame query points p_ij of image i with exact SDF
 * labels s_ij (e.g. from mppi_sample_sdf_queries); the decoder's input is [PE(p), z] as in
 * mppi_set_sdf_weights with pe_levels, its activation softplus with softplus_beta.
 *   layers                10 host arrays W1 [128][3 + 6 pe_levels + 64], b1, W2..W4 [128][128],
 *                         b2..b4, w5 [1][128], b5 [1]: g_phi's initial weights (copied)
 *   max_points_per_image  32 .. 65536, a multiple of 32: the most query points a call may pass
 *   train_decoder         0: g_phi stays frozen (the paper's second stage); 1: g_phi trains with
 *                         the encoder and D_psi (its first stage), Adam on its 10 tensors too
 * Errors: MPPI_E_INVALID (bad argument, or a decoder already set), MPPI_E_OOM, MPPI_E_CUDA.
 */
int mppi_encoder_train_set_sdf(mppi_encoder_trainer* trainer, const float* const* layers, int pe_levels,
                               float softplus_beta, float lambda_recon, float lambda_sdf, int max_points_per_image,
                               int train_decoder);
/* g_phi's current weights (10 host arrays as in mppi_encoder_train_set_sdf; NULL entries skipped). */
int mppi_encoder_train_get_sdf_decoder(mppi_encoder_trainer* trainer, float* const* layers_out);
/*
 * As mppi_encoder_train_loss_grads / _step with the SDF term: d_points n x n_points x 3 and
 * d_labels n x n_points floats (device), n_points a multiple of 32 up to max_points_per_image;
 * losses (nullable, host [3]): the weighted total, the reconstruction mean |r| and the SDF mean
 * |r|; grads_out as before, followed, when g_phi trains, by its 10 gradients (22 arrays).
 * MPPI_E_NOT_READY before mppi_encoder_train_set_sdf.
 */
int mppi_encoder_train_loss_grads_sdf(mppi_encoder_trainer* trainer, int n, const float* d_noisy, const float* d_clean,
                                      float max_range, const float* d_points, const float* d_labels, int n_points,
                                      float* losses, float* const* grads_out);
int mppi_encoder_train_step_sdf(mppi_encoder_trainer* trainer, int n, const float* d_noisy, const float* d_clean,
                                float max_range, const float* d_points, const float* d_labels, int n_points,
                                float* losses);
/* D_psi's current weights (T x 64 and T host floats).  Synchronous. */
int mppi_encoder_train_get_decoder(mppi_encoder_trainer* trainer, float* W, float* b);

/* ======================================================================== learned part
 * Distillation of the exact gate-frame SDF (the frame of mppi_config's gate
 * geometry) into the Gate-SDF MLP (Sec. III-B trains the decoder with an L1
 * loss on the SDF; here the target is the exact frame SDF and an Eikonal
 * term regularises the input gradient):
 *     L = mean |s - s*| + eikonal_weight mean (|grad_p s| - 1)^2,
 * at one fixed latent z0, with Adam on FP32 master weights.  Training and
 * held-out points are sampled on the GPU from Philox: near_surface_fraction
 * of them a uniform point of the frame surface plus N(0, near_surface_sigma^2 I),
 * the rest uniform in [-cube_half, cube_half]^3 (gate frame).  The forward
 * pass carries the three input tangents next to the values; the backward pass
 * differentiates both (FP32, deterministic reductions).
 */
typedef struct mppi_trainer mppi_trainer;

typedef struct mppi_train_config {
    int32_t batch;                  /* points per step, a multiple of 128 (<= 2^20) */
    int32_t n_points;               /* training-set size, a multiple of batch (<= 2^26) */
    int32_t n_holdout;              /* held-out check points, a multiple of 128 (<= 2^22) */
    float lr, beta1, beta2, eps;    /* Adam */
    float eikonal_weight;
    float softplus_beta;
    float near_surface_fraction, near_surface_sigma, cube_half;
    float gate_inner_half, gate_outer_half, gate_half_depth;
    uint64_t seed;                  /* Philox key of the training set (the held-out set uses a derived key) */
} mppi_train_config;

/* Defaults: batch 65536, 2^21 points, 2^18 held out, lr 1e-3, (0.9, 0.999, 1e-8), Eikonal 0.1,
 * beta 100, 70 % near-surface with sigma 0.05 m, cube half-width 4 m, the 1.0 / 1.5 / 0.2 m gate. */
void mppi_train_config_default(mppi_train_config* cfg);
/*
 * Create a trainer from initial weights (10 host arrays as in
 * mppi_set_sdf_weights) and the latent z0 (64 floats); samples the training
 * and held-out sets on the device.  Synchronous.
 */
int mppi_train_create(const mppi_train_config* cfg, const float* const* init_layers, const float* latent,
                      mppi_trainer** out);
void mppi_train_destroy(mppi_trainer* trainer);
const char* mppi_train_last_error(const mppi_trainer* trainer);
/* Learning rate of the following steps (> 0, finite): a caller's schedule sets it between calls of
 * mppi_train_step.  Errors: MPPI_E_INVALID. */
int mppi_train_set_lr(mppi_trainer* trainer, float lr);
/*
 * Precision of the hidden layers' GEMMs (layers 2-4: forward values and
 * tangents, input and weight gradients) in mppi_train_step and
 * mppi_train_loss_grads.  MPPI_TRAIN_GEMM_FP32 (the default): FP32 on the CUDA
 * cores.  MPPI_TRAIN_GEMM_BF16: tcgen05 tensor cores with operands rounded to
 * BF16 and FP32 accumulation; weights, Adam state, activations and adjoints
 * stay FP32.  mppi_train_evaluate always runs the FP32 forward pass.  Errors:
 * MPPI_E_INVALID (unknown value), MPPI_E_UNSUPPORTED (BF16 on a device other
 * than sm_103), MPPI_E_CUDA.  A bounded device wait that gives up inside a
 * BF16 kernel makes the next mppi_train_step / mppi_train_loss_grads return
 * MPPI_E_TIMEOUT; the trainer stays usable.
 */
#define MPPI_TRAIN_GEMM_FP32 0
#define MPPI_TRAIN_GEMM_BF16 1
int mppi_train_set_gemm_precision(mppi_trainer* trainer, int precision);
/* Run n_steps Adam steps over consecutive batches of the training set; *last_loss (nullable) = last batch's loss. */
int mppi_train_step(mppi_trainer* trainer, int n_steps, float* last_loss);
/*
 * Loss and gradient of one explicit batch without updating (for checks):
 * points n x 4 host floats (x, y, z, target), n a multiple of 128 and <= batch;
 * grads receives mppi_train_num_params() floats in the order W1, b1, W2, b2,
 * W3, b3, W4, b4, w5, b5 (row-major).  Synchronous.
 */
int mppi_train_loss_grads(mppi_trainer* trainer, const float* points, int n, float* loss, float* grads);
/* Current weights into 10 host arrays (shapes of mppi_set_sdf_weights). */
int mppi_train_get_weights(mppi_trainer* trainer, float* const* layers_out);
/* Held-out error against the exact SDF, in metres: mean, p99, max, and p99 over points with |SDF| < 0.3 m. */
int mppi_train_evaluate(mppi_trainer* trainer, float* mae, float* p99, float* max_err, float* near_p99);
/* Copy the training (which = 0) or held-out (1) points, n x 4 floats (x, y, z, target). */
int mppi_train_read_points(mppi_trainer* trainer, int which, float* out, size_t n_floats);
/* Number of trainable parameters (the length of the gradient vector). */
int mppi_train_num_params(void);

/* ======================================================================== serving
 * Continuous batching of control steps from many drones (one request = one
 * control step of one drone).  The paper runs one MPPI controller per vehicle at a
 * fixed control rate (Sec. IV-A, Sec. V); serving many vehicles' controllers from
 * one GPU has no counterpart in the paper.  Each drone keeps a context on the
 * device: its warm-started nominal sequence, true state and Philox step counter
 * persist between its requests (the same chain as mppi_step), so a drone's results
 * do not depend on which other drones share the GPU.  Requests are admitted in
 * arrival order as soon as the drone has no request in flight, fewer than
 * max_inflight requests run and the drone's context fits in the device-memory
 * budget; the least recently used idle drone is evicted to host memory (its warm
 * start, state and counter are restored on its next request) when it does not.
 * Batched mode (batching = 1): every admissible queued request joins one batch,
 * launched as four kernels on a stream of the server's (inputs, one rollout launch
 * over all drones, one persistent tensor-core SDF launch whose tiles span all drones,
 * one update launch); up to four batches run at once on their own streams; each
 * drone's results agree with its own mppi_step's within the FP32 control tolerance.  Per-drone mode (batching = 0): each request is its
 * drone's captured step graph on the drone's own stream, and requests of different
 * drones overlap on the GPU.  All functions are thread-safe; a worker thread owned
 * by the server issues the GPU work.
 */
typedef struct mppi_server mppi_server;

typedef struct mppi_server_config {
    size_t hbm_budget_bytes;   /* device bytes the drone contexts may hold together; 0 = no limit */
    int32_t max_inflight;      /* requests on the device at once (1 .. 1024); in batched mode also the
                                  largest batch */
    int32_t sdf_mode;          /* MPPI_SDF_* used by every drone */
    int32_t batching;          /* 1: batched launches (every drone then shares softplus_beta and
                                  pe_levels); 0: one step graph per drone */
    int32_t sdf_single_cta;    /* 1 (default): BF16 / FP16 SDF kernels (batched or per drone) in their
                                  single-CTA form; 0: the CTA-pair form where it applies (see
                                  MPPI_DIAG_SDF_SINGLE_CTA).  With many drones' kernels in flight at
                                  once the single-CTA form measured faster: per-drone graphs 2.40e9
                                  vs 2.33e9 rollout-steps/s, batched 2.32e9 vs 2.26e9 (64 drones) */
} mppi_server_config;

typedef struct mppi_server_stats {
    uint64_t submitted, completed, queued, inflight;
    uint64_t evictions, restores;      /* drone contexts moved to host memory / brought back */
    size_t device_bytes, peak_device_bytes;
    uint64_t batches;                  /* batched mode: batches launched */
} mppi_server_stats;

/* Defaults: no budget, 16 requests in flight, FP16 tensor-core SDF, batched launches, single-CTA
 * SDF kernels. */
void mppi_server_config_default(mppi_server_config* cfg);
/* Create a server on the current device (starts its worker thread; batched mode also allocates four
 * pinned and four device batch blocks of max_inflight controllers each, and a stream for each).
 * *out is NULL on error:
 * MPPI_E_INVALID (cfg), MPPI_E_UNSUPPORTED (no device), MPPI_E_OOM. */
int mppi_server_create(const mppi_server_config* cfg, mppi_server** out);
/* Drain in-flight work, stop the worker and free every drone context.  NULL is ignored. */
void mppi_server_destroy(mppi_server* server);
/* Message of the server's last error (server NULL: the calling thread's last failed create); owned by
 * the server, valid until its next failing call. */
const char* mppi_server_last_error(const mppi_server* server);
/* Gate-SDF MLP weights (Sec. III-B, Fig. 2) for every drone (same arrays as mppi_set_sdf_weights); call
 * before the first request. */
int mppi_server_set_sdf_weights(mppi_server* server, const float* const* layers, int n_layers,
                                const float* fp8_scales);
/*
 * Queue one control step (Sec. IV-A, Eq. 5 and its receding-horizon update) of drone drone_id
 * (host buffers, copied before the call returns): cfg gives the drone's controller parameters
 * (K, H and max_gates must stay the same for a drone; the server's sdf_mode applies; in batched
 * mode softplus_beta and pe_levels must match the server's other drones), state
 * mppi_state_dim(cfg) floats, n_gates gate poses (n x 7) and latents (n x 64; NULL in analytic
 * mode).  *ticket identifies the request.  Returns at once.  Errors: MPPI_E_INVALID,
 * MPPI_E_NOT_READY (no weights set); MPPI_E_ADMISSION is reported through the ticket.
 */
int mppi_server_submit(mppi_server* server, int drone_id, const mppi_config* cfg, const float* state, int n_gates,
                       const float* poses, const float* latents, uint64_t* ticket);
/*
 * Result of one request (the new control sequence U*_new of Eq. 5).
 * Non-blocking: MPPI_PENDING while the request is queued or running; once it
 * is done, its status (MPPI_OK with new_controls = U*_new, H x 4, filled; or
 * the error of that request) and latency_us = submit-to-completion time in
 * microseconds (nullable).  A finished ticket is reported once.
 */
int mppi_server_poll(mppi_server* server, uint64_t ticket, float* new_controls, double* latency_us);
/*
 * Non-blocking: take any one finished request: MPPI_PENDING when none is
 * finished; otherwise *ticket, its status (as mppi_server_poll) and, for
 * MPPI_OK, new_controls (cap_floats floats available; H x 4 are written).
 */
int mppi_server_next_result(mppi_server* server, uint64_t* ticket, float* new_controls, size_t cap_floats,
                            double* latency_us);
/* Counters of the server (submitted, completed, queued, in flight, evictions, restores, device bytes,
 * batches launched; no counterpart in the paper). */
int mppi_server_get_stats(mppi_server* server, mppi_server_stats* out);

#ifdef __cplusplus
}
#endif

#endif /* MPPI_GB300_H */
