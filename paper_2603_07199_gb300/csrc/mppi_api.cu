// C ABI of the control-step library: context, device buffers, the step's
// launch sequence, host <-> device staging and diagnostics.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include <cuda_fp16.h>
#include <cuda_fp8.h>

#include "ctx_internal.h"
#include "kernels.h"
#include "mppi.h"

using namespace mppi;

namespace {
thread_local char g_thread_err[512] = "";
// floats reserved for the state in the device buffer and the host staging (>= MPPI_STATE_MAX)
constexpr int kStateSlot = 24;
}

struct mppi_ctx {
    mppi_config cfg{};
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int device = 0;
    int num_sms = 0;
    int n_gates = 0;
    bool have_weights = false;
    bool have_latents = false;
    bool timing = false;
    bool store_sdf = false;       // MPPI_DIAG_STORE_SDF
    bool sdf_single_cta = false;  // MPPI_DIAG_SDF_SINGLE_CTA
    uint64_t step_count = 0;
    char err[512] = "";

    StepBuffers B{};
    float* d_latents = nullptr;   // [maxG][64]
    // MLP weights
    float* d_W1 = nullptr;        // [128][67]
    float* d_b1 = nullptr;        // [128]
    float* d_Wt[3] = {nullptr, nullptr, nullptr};
    float* d_bias[3] = {nullptr, nullptr, nullptr};
    float* d_w5 = nullptr;
    uint16_t* d_Wbf[3] = {nullptr, nullptr, nullptr};
    uint16_t* d_Wh[3] = {nullptr, nullptr, nullptr};
    uint16_t* d_W1tc = nullptr;
    uint8_t* d_W8[3] = {nullptr, nullptr, nullptr};
    float f8_dequant[3] = {1.f, 1.f, 1.f};
    float f8_inv_act[3] = {1.f, 1.f, 1.f};
    float b5 = 0.f;
    // pinned staging
    float* h_in = nullptr;        // state(16) | nominal(H*4) | poses(maxG*8) | latents(maxG*64)
    float* h_out = nullptr;       // unew(H*4) | w(K) | J(K) | err(1)
    float* d_hout = nullptr;      // device address of h_out (the step writes its outputs there directly)
    // completion of the last step enqueued by the serving path
    cudaEvent_t done = nullptr;
    // the step's kernels as one CUDA graph, re-captured when a launch argument changes
    cudaGraphExec_t gexec = nullptr;          // the step's kernels
    cudaGraphExec_t gexec_state = nullptr;    // the same after a copy of the pinned state slot to B.state
    bool graph_dirty = true;
    // timing
    cudaEvent_t ev[8] = {};
    int n_ev = 0;
    const char* ev_names[8] = {};
    std::vector<void*> allocations;
};

namespace {

int fail(mppi_ctx* c, int code, const char* fmt, ...) {
    char* dst = c ? c->err : g_thread_err;
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(dst, 512, fmt, ap);
    va_end(ap);
    return code;
}

#define CUDA_TRY(ctx, expr)                                                                        \
    do {                                                                                           \
        cudaError_t e_ = (expr);                                                                   \
        if (e_ != cudaSuccess)                                                                     \
            return fail((ctx), MPPI_E_CUDA, "%s failed: %s", #expr, cudaGetErrorString(e_));      \
    } while (0)

template <typename T>
int dev_alloc(mppi_ctx* c, T** p, size_t count) {
    void* q = nullptr;
    cudaError_t e = cudaMalloc(&q, count * sizeof(T) > 0 ? count * sizeof(T) : 16);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(c, MPPI_E_OOM, "cudaMalloc(%zu bytes) failed: %s", count * sizeof(T), cudaGetErrorString(e));
    }
    c->allocations.push_back(q);
    *p = static_cast<T*>(q);
    return MPPI_OK;
}

StepParams make_params(const mppi_ctx* c) {
    const mppi_config& g = c->cfg;
    StepParams P{};
    P.K = g.K;
    P.H = g.H;
    P.G = c->n_gates;
    P.dt = g.dt;
    P.mass = g.mass;
    P.gravity = g.gravity;
    P.tmin = g.thrust_min;
    P.tmax = g.thrust_max;
    P.rmax = g.rate_max;
    P.sig_t = g.sigma_thrust;
    P.sig_r = g.sigma_rate;
    P.lam = g.lambda;
    P.w_col = g.w_col;
    P.d_safe = g.d_safe;
    P.w_u = g.w_u;
    P.a_in = g.gate_inner_half;
    P.a_out = g.gate_outer_half;
    P.half_depth = g.gate_half_depth;
    P.beta = g.softplus_beta;
    P.key0 = static_cast<uint32_t>(g.seed & 0xFFFFFFFFull);
    P.key1 = static_cast<uint32_t>(g.seed >> 32);
    P.drone = g.drone_id;
    P.paper = g.cost_mode == MPPI_COST_PAPER ? 1 : 0;
    P.q_gate = g.q_gate;
    P.q_vis = g.q_vis;
    P.q_sdf = g.q_sdf;
    P.tan_alpha = g.guide_tan_alpha;
    P.rotor = g.dynamics_mode == MPPI_DYN_ROTOR ? 1 : 0;
    P.u_hover = P.rotor ? 0.f : g.mass * g.gravity;
    if (P.rotor) {
        // the thrust-rate command: every channel in [-tdot_max, tdot_max], noise sigma_tdot
        P.tmin = -g.tdot_max;
        P.tmax = g.tdot_max;
        P.rmax = g.tdot_max;
        P.sig_t = g.sigma_tdot;
        P.sig_r = g.sigma_tdot;
    }
    P.arm_d = g.arm_length * 0.70710678f;
    P.kappa = g.torque_coeff;
    P.inv_J = make_float3(1.f / g.inertia_x, 1.f / g.inertia_y, 1.f / g.inertia_z);
    P.J = make_float3(g.inertia_x, g.inertia_y, g.inertia_z);
    P.t_rotor_max = g.rotor_thrust_max;
    P.pe = g.pe_levels;
    P.store_sdf = c->store_sdf ? 1 : 0;
    P.sdf_pair = c->sdf_single_cta ? 0 : 1;
    // per-kernel event timing measures kernels one after the other
    P.pdl = c->timing ? 0 : 1;
    return P;
}

int state_dim(const mppi_config& g) { return g.dynamics_mode == MPPI_DYN_ROTOR ? 17 : 13; }
// point features of the decoder's input (3 + 6 L) and the K of the layer-1 tensor-core GEMM
int point_features(const mppi_config& g) { return 3 + 6 * g.pe_levels; }
int layer1_k(const mppi_config& g) { return layer1_gemm_k(g.pe_levels); }

bool finite_all(const float* x, size_t n) {
    for (size_t i = 0; i < n; ++i)
        if (!std::isfinite(x[i])) return false;
    return true;
}

int check_config(const mppi_config* g) {
    if (!g) return fail(nullptr, MPPI_E_INVALID, "cfg is NULL");
    if (g->K < 1 || g->K > MPPI_MAX_K) return fail(nullptr, MPPI_E_INVALID, "K=%d out of [1, %d]", g->K, MPPI_MAX_K);
    if (g->H < 1 || g->H > MPPI_MAX_H) return fail(nullptr, MPPI_E_INVALID, "H=%d out of [1, %d]", g->H, MPPI_MAX_H);
    if (static_cast<long long>(g->K) * g->H > (1ll << 28))
        return fail(nullptr, MPPI_E_INVALID, "K*H=%lld exceeds 2^28", static_cast<long long>(g->K) * g->H);
    if (g->max_gates < 1 || g->max_gates > MPPI_MAX_GATES)
        return fail(nullptr, MPPI_E_INVALID, "max_gates=%d out of [1, %d]", g->max_gates, MPPI_MAX_GATES);
    if (g->sdf_mode < MPPI_SDF_ANALYTIC || g->sdf_mode > MPPI_SDF_MLP_FP8)
        return fail(nullptr, MPPI_E_UNSUPPORTED, "sdf_mode=%d is not built", g->sdf_mode);
    if (g->cost_mode != MPPI_COST_CONFIGURED && g->cost_mode != MPPI_COST_PAPER)
        return fail(nullptr, MPPI_E_INVALID, "cost_mode=%d is not one of MPPI_COST_*", g->cost_mode);
    if (g->pe_levels < 0 || g->pe_levels > MPPI_MAX_PE_LEVELS)
        return fail(nullptr, MPPI_E_INVALID, "pe_levels=%d out of [0, %d]", g->pe_levels, MPPI_MAX_PE_LEVELS);
    if (g->dynamics_mode != MPPI_DYN_CTBR && g->dynamics_mode != MPPI_DYN_ROTOR)
        return fail(nullptr, MPPI_E_INVALID, "dynamics_mode=%d is not one of MPPI_DYN_*", g->dynamics_mode);
    if (g->dynamics_mode == MPPI_DYN_ROTOR) {
        const float r[] = {g->tdot_max, g->rotor_thrust_max, g->sigma_tdot, g->arm_length, g->torque_coeff,
                           g->inertia_x, g->inertia_y, g->inertia_z};
        if (!finite_all(r, 8) || !(g->tdot_max >= 0.f) || !(g->rotor_thrust_max > 0.f) || g->sigma_tdot < 0.f ||
            !(g->arm_length > 0.f) || !(g->inertia_x > 0.f) || !(g->inertia_y > 0.f) || !(g->inertia_z > 0.f))
            return fail(nullptr, MPPI_E_INVALID, "rotor-model parameters");
    }
    const float f[] = {g->dt, g->mass, g->gravity, g->thrust_min, g->thrust_max, g->rate_max, g->sigma_thrust,
                       g->sigma_rate, g->lambda, g->w_col, g->d_safe, g->w_u, g->gate_inner_half,
                       g->gate_outer_half, g->gate_half_depth, g->softplus_beta, g->q_gate, g->q_vis, g->q_sdf,
                       g->guide_tan_alpha};
    if (!finite_all(f, sizeof(f) / sizeof(f[0]))) return fail(nullptr, MPPI_E_INVALID, "non-finite parameter");
    if (!(g->dt > 0.f) || !(g->mass > 0.f) || !(g->lambda > 0.f) || !(g->softplus_beta > 0.f))
        return fail(nullptr, MPPI_E_INVALID, "dt, mass, lambda and softplus_beta must be > 0");
    if (!(g->thrust_min <= g->thrust_max) || !(g->rate_max >= 0.f) || g->sigma_thrust < 0.f || g->sigma_rate < 0.f)
        return fail(nullptr, MPPI_E_INVALID, "inconsistent control bounds or negative sigma");
    if (!(g->gate_inner_half < g->gate_outer_half) || !(g->gate_half_depth > 0.f))
        return fail(nullptr, MPPI_E_INVALID, "gate geometry");
    return MPPI_OK;
}

int recompute_b1p(mppi_ctx* c) {
    if (!c->have_weights || !c->have_latents || c->n_gates == 0) return MPPI_OK;
    CUDA_TRY(c, launch_first_layer_bias(c->d_W1, c->d_b1, c->d_latents, c->n_gates, point_features(c->cfg), c->B.b1p,
                                        c->stream));
    return MPPI_OK;
}

bool is_mlp(const mppi_ctx* c) { return c->cfg.sdf_mode != MPPI_SDF_ANALYTIC; }

// Caller device buffers the step's last kernel writes U*_new, w and J into, and the slot
// it copies the device error word to (NULL: none).
void set_outputs(mppi_ctx* c, float4* U, float* w, float* J, int* err) {
    if (c->B.out_U != U || c->B.out_w != w || c->B.out_J != J || c->B.err_out != err) {
        c->B.out_U = U;
        c->B.out_w = w;
        c->B.out_J = J;
        c->B.err_out = err;
        c->graph_dirty = true;
    }
}

MlpWeights make_weights(const mppi_ctx* c) {
    MlpWeights W{};
    W.W1 = c->d_W1;
    for (int l = 0; l < 3; ++l) {
        W.Wt[l] = c->d_Wt[l];
        W.b[l] = c->d_bias[l];
        W.Wbf[l] = c->d_Wbf[l];
        W.Wh[l] = c->d_Wh[l];
    }
    W.w5 = c->d_w5;
    W.b5 = c->b5;
    W.W1tc = c->d_W1tc;
    for (int l = 0; l < 3; ++l) {
        W.W8[l] = c->d_W8[l];
        W.f8_dequant[l] = c->f8_dequant[l];
        W.f8_inv_act[l] = c->f8_inv_act[l];
    }
    return W;
}

void record(mppi_ctx* c, const char* name) {
    if (!c->timing || c->n_ev >= 8) return;
    // while the step is being captured, an external event node is what records the event at replay
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaStreamIsCapturing(c->stream, &cs);
    cudaEventRecordWithFlags(c->ev[c->n_ev], c->stream,
                             cs == cudaStreamCaptureStatusActive ? cudaEventRecordExternal : cudaEventRecordDefault);
    c->ev_names[c->n_ev] = name;
    ++c->n_ev;
}

// The kernels of one step, enqueued on the context's stream.
int enqueue_kernels(mppi_ctx* c) {
    const StepParams P = make_params(c);
    const bool mlp = is_mlp(c);
    c->n_ev = 0;
    record(c, "start");
    CUDA_TRY(c, launch_rollout(P, c->B, mlp ? 0 : 1, c->stream));
    record(c, "rollout");
    if (mlp) {
        const MlpWeights W = make_weights(c);
        if (c->cfg.sdf_mode == MPPI_SDF_MLP_FP32) {
            CUDA_TRY(c, launch_sdf_mlp_fp32(P, c->B, W, c->num_sms, c->stream));
            record(c, "sdf_mlp_fp32");
        } else if (c->cfg.sdf_mode == MPPI_SDF_MLP_BF16) {
            CUDA_TRY(c, launch_sdf_mlp_bf16(P, c->B, W, c->num_sms, c->stream));
            record(c, "sdf_mlp_bf16");
        } else if (c->cfg.sdf_mode == MPPI_SDF_MLP_FP16) {
            CUDA_TRY(c, launch_sdf_mlp_fp16(P, c->B, W, c->num_sms, c->stream));
            record(c, "sdf_mlp_fp16");
        } else {
            CUDA_TRY(c, launch_sdf_mlp_fp8(P, c->B, W, c->num_sms, c->stream));
            record(c, "sdf_mlp_fp8");
        }
    }
    CUDA_TRY(c, launch_cost_update(P, c->B, mlp ? 1 : 0, c->stream));
    record(c, "cost_update");
    return MPPI_OK;
}

// Launch the step: replay the captured graph -- with state_copy, the one whose first node
// copies the pinned state slot (h_in) to the device state, so that a step from a host state
// is one submission -- capturing it first when the launch arguments changed.  When the
// caller's stream is itself being captured, the copy and the kernels are enqueued directly
// into the caller's capture.
int launch_step(mppi_ctx* c, bool state_copy) {
    const size_t state_bytes = state_dim(c->cfg) * sizeof(float);
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    CUDA_TRY(c, cudaStreamIsCapturing(c->stream, &cs));
    if (cs != cudaStreamCaptureStatusNone) {
        if (state_copy)
            CUDA_TRY(c, cudaMemcpyAsync(c->B.state, c->h_in, state_bytes, cudaMemcpyHostToDevice, c->stream));
        return enqueue_kernels(c);
    }
    if (c->graph_dirty) {
        for (cudaGraphExec_t* e : {&c->gexec, &c->gexec_state}) {
            if (*e) cudaGraphExecDestroy(*e);
            *e = nullptr;
        }
        c->graph_dirty = false;
    }
    cudaGraphExec_t& exec = state_copy ? c->gexec_state : c->gexec;
    if (exec == nullptr) {
        CUDA_TRY(c, cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
        const cudaError_t ec = state_copy ? cudaMemcpyAsync(c->B.state, c->h_in, state_bytes,
                                                            cudaMemcpyHostToDevice, c->stream)
                                          : cudaSuccess;
        const int rc = ec == cudaSuccess ? enqueue_kernels(c) : MPPI_OK;
        cudaGraph_t g = nullptr;
        const cudaError_t e = cudaStreamEndCapture(c->stream, &g);
        if (ec != cudaSuccess || rc != MPPI_OK) {
            if (g) cudaGraphDestroy(g);
            return ec != cudaSuccess ? fail(c, MPPI_E_CUDA, "state copy capture failed: %s", cudaGetErrorString(ec))
                                     : rc;
        }
        if (e != cudaSuccess) return fail(c, MPPI_E_CUDA, "stream capture failed: %s", cudaGetErrorString(e));
        const cudaError_t ei = cudaGraphInstantiate(&exec, g, 0);
        cudaGraphDestroy(g);
        if (ei != cudaSuccess) {
            exec = nullptr;
            return fail(c, MPPI_E_CUDA, "graph instantiation failed: %s", cudaGetErrorString(ei));
        }
    }
    CUDA_TRY(c, cudaGraphLaunch(exec, c->stream));
    return MPPI_OK;
}

int check_ready(mppi_ctx* c) {
    if (is_mlp(c)) {
        if (!c->have_weights) return fail(c, MPPI_E_NOT_READY, "MLP SDF mode but no weights set");
        if (c->n_gates > 0 && !c->have_latents) return fail(c, MPPI_E_NOT_READY, "MLP SDF mode but no latents set");
    }
    return MPPI_OK;
}

// After a device-side timeout: clear the error word and the barrier counters (a timed-out
// grid barrier leaves its arrival count behind).
cudaError_t clear_device_error(mppi_ctx* c) {
    cudaError_t e = cudaMemsetAsync(c->B.err, 0, sizeof(int), c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->B.tickets, 0, 32 * sizeof(unsigned), c->stream);
    return e;
}

int read_err_word(mppi_ctx* c) {
    int e = 0;
    CUDA_TRY(c, cudaMemcpyAsync(&e, c->B.err, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    if (e != 0) {
        CUDA_TRY(c, clear_device_error(c));
        CUDA_TRY(c, cudaStreamSynchronize(c->stream));
        return fail(c, MPPI_E_TIMEOUT, "a device-side wait timed out (error word %d)", e);
    }
    return MPPI_OK;
}

}  // namespace

extern "C" {

void mppi_config_default(mppi_config* g) {
    if (!g) return;
    std::memset(g, 0, sizeof(*g));
    g->K = 256;
    g->H = 20;
    g->max_gates = 1;
    g->sdf_mode = MPPI_SDF_ANALYTIC;
    g->dt = 0.02f;
    g->mass = 0.8f;
    g->gravity = 9.81f;
    g->thrust_min = 0.f;
    g->thrust_max = 30.f;
    g->rate_max = 8.f;
    g->sigma_thrust = 2.f;
    g->sigma_rate = 1.5f;
    g->lambda = 0.1f;
    g->w_col = 100.f;
    g->d_safe = 0.3f;
    g->w_u = 1e-3f;
    g->gate_inner_half = 0.5f;
    g->gate_outer_half = 0.75f;
    g->gate_half_depth = 0.1f;
    g->softplus_beta = 100.f;
    g->seed = 0;
    g->drone_id = 0;
    g->cost_mode = MPPI_COST_CONFIGURED;
    g->q_gate = 1.f;
    g->q_vis = 1.f;
    g->q_sdf = 10.f;
    g->guide_tan_alpha = 0.57735027f;   // tan(30 deg)
    g->dynamics_mode = MPPI_DYN_CTBR;
    g->tdot_max = 10.f;
    g->rotor_thrust_max = 10.f;
    g->sigma_tdot = 5.f;
    g->arm_length = 0.15f;
    g->torque_coeff = 0.016f;
    g->inertia_x = 0.003f;
    g->inertia_y = 0.003f;
    g->inertia_z = 0.005f;
}

int mppi_state_dim(const mppi_config* g) { return g && g->dynamics_mode == MPPI_DYN_ROTOR ? 17 : 13; }

const char* mppi_last_error(const mppi_ctx* c) { return c ? c->err : g_thread_err; }

void mppi_destroy(mppi_ctx* c) {
    if (!c) return;
    cudaStreamSynchronize(c->stream);
    if (c->gexec) cudaGraphExecDestroy(c->gexec);
    if (c->gexec_state) cudaGraphExecDestroy(c->gexec_state);
    for (void* p : c->allocations) cudaFree(p);
    if (c->h_in) cudaFreeHost(c->h_in);
    if (c->h_out) cudaFreeHost(c->h_out);
    for (auto& e : c->ev)
        if (e) cudaEventDestroy(e);
    if (c->done) cudaEventDestroy(c->done);
    if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
    delete c;
}

int mppi_create(const mppi_config* cfg, void* cuda_stream, mppi_ctx** out) {
    if (!out) return fail(nullptr, MPPI_E_INVALID, "out is NULL");
    *out = nullptr;
    int rc = check_config(cfg);
    if (rc != MPPI_OK) return rc;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return fail(nullptr, MPPI_E_UNSUPPORTED, "no CUDA device");
    }
    int major = 0, minor = 0, sms = 0;
    cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev);
    cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (major != 10 || minor != 3)
        return fail(nullptr, MPPI_E_UNSUPPORTED, "device is sm_%d%d; this library is built for sm_103a only", major,
                    minor);

    mppi_ctx* c = new (std::nothrow) mppi_ctx();
    if (!c) return fail(nullptr, MPPI_E_OOM, "host allocation failed");
    c->cfg = *cfg;
    c->device = dev;
    c->num_sms = sms;
    if (configure_sdf_mlp_fp32() != cudaSuccess || configure_sdf_mlp_bf16() != cudaSuccess ||
        configure_cost_update() != cudaSuccess) {
        delete c;
        return fail(nullptr, MPPI_E_CUDA, "kernel attribute set-up failed: %s", cudaGetErrorString(cudaGetLastError()));
    }
    if (cuda_stream) {
        c->stream = static_cast<cudaStream_t>(cuda_stream);
    } else {
        if (cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess) {
            delete c;
            return fail(nullptr, MPPI_E_CUDA, "cudaStreamCreate failed");
        }
        c->own_stream = true;
    }
    const int K = cfg->K, H = cfg->H, MG = cfg->max_gates;
    const size_t KH = static_cast<size_t>(K) * H;
    const int nub = update_blocks(K);
    StepBuffers& B = c->B;
    rc = MPPI_OK;
    rc = rc ? rc : dev_alloc(c, &B.state, kStateSlot);
    rc = rc ? rc : dev_alloc(c, &B.nominal, H);
    rc = rc ? rc : dev_alloc(c, &B.step, 2);
    rc = rc ? rc : dev_alloc(c, &B.poses, static_cast<size_t>(MG) * 8);
    rc = rc ? rc : dev_alloc(c, &B.b1p, static_cast<size_t>(MG) * kHidden);
    rc = rc ? rc : dev_alloc(c, &B.noise, KH);
    rc = rc ? rc : dev_alloc(c, &B.pos, KH);
    rc = rc ? rc : dev_alloc(c, &B.parts, 3 * static_cast<size_t>(K));
    rc = rc ? rc : dev_alloc(c, &B.sdf, KH);
    rc = rc ? rc : dev_alloc(c, &B.colp, static_cast<size_t>(K) * col_slots(H));
    rc = rc ? rc : dev_alloc(c, &B.J, K);
    rc = rc ? rc : dev_alloc(c, &B.w, K);
    rc = rc ? rc : dev_alloc(c, &B.unew, H);
    rc = rc ? rc : dev_alloc(c, &B.upart, static_cast<size_t>(nub) * H);
    rc = rc ? rc : dev_alloc(c, &B.bstat, nub);
    rc = rc ? rc : dev_alloc(c, &B.stats, 4);
    rc = rc ? rc : dev_alloc(c, &B.tickets, 32);
    rc = rc ? rc : dev_alloc(c, &B.err, 1);
    rc = rc ? rc : dev_alloc(c, &c->d_latents, static_cast<size_t>(MG) * kLatent);
    rc = rc ? rc : dev_alloc(c, &c->d_W1, kHidden * (point_features(*cfg) + kLatent));
    rc = rc ? rc : dev_alloc(c, &c->d_b1, kHidden);
    for (int l = 0; l < 3; ++l) {
        rc = rc ? rc : dev_alloc(c, &c->d_Wt[l], kHidden * kHidden);
        rc = rc ? rc : dev_alloc(c, &c->d_bias[l], kHidden);
        rc = rc ? rc : dev_alloc(c, &c->d_Wbf[l], kHidden * kHidden);
        rc = rc ? rc : dev_alloc(c, &c->d_Wh[l], kHidden * kHidden);
        rc = rc ? rc : dev_alloc(c, &c->d_W8[l], kHidden * kHidden);
    }
    rc = rc ? rc : dev_alloc(c, &c->d_w5, kHidden);
    rc = rc ? rc : dev_alloc(c, &c->d_W1tc, kHidden * layer1_k(*cfg));
    if (rc != MPPI_OK) {
        std::snprintf(g_thread_err, sizeof(g_thread_err), "%s", c->err);
        mppi_destroy(c);
        return rc;
    }
    const size_t in_floats = kStateSlot + static_cast<size_t>(H) * 4 + MG * 8 + MG * kLatent;
    const size_t out_floats = static_cast<size_t>(H) * 4 + 2 * static_cast<size_t>(K) + 4;
    if (cudaMallocHost(&c->h_in, in_floats * sizeof(float)) != cudaSuccess ||
        cudaMallocHost(&c->h_out, out_floats * sizeof(float)) != cudaSuccess ||
        cudaHostGetDevicePointer(reinterpret_cast<void**>(&c->d_hout), c->h_out, 0) != cudaSuccess) {
        cudaGetLastError();
        std::snprintf(g_thread_err, sizeof(g_thread_err), "pinned host allocation failed");
        mppi_destroy(c);
        return MPPI_E_OOM;
    }
    if (cudaEventCreateWithFlags(&c->done, cudaEventDisableTiming) != cudaSuccess) {
        std::snprintf(g_thread_err, sizeof(g_thread_err), "cudaEventCreate failed");
        mppi_destroy(c);
        return MPPI_E_CUDA;
    }
    for (auto& e : c->ev) {
        if (cudaEventCreate(&e) != cudaSuccess) {
            std::snprintf(g_thread_err, sizeof(g_thread_err), "cudaEventCreate failed");
            mppi_destroy(c);
            return MPPI_E_CUDA;
        }
    }
    // initial state: hover at the origin; nominal: H copies of u_hover; counter 0
    // (rotor model: every rotor carrying m g / 4; nominal: zero thrust rates)
    float* st = c->h_in;
    std::memset(st, 0, kStateSlot * sizeof(float));
    st[6] = 1.f;
    const bool rotor = cfg->dynamics_mode == MPPI_DYN_ROTOR;
    if (rotor)
        for (int i = 0; i < 4; ++i) st[13 + i] = 0.25f * cfg->mass * cfg->gravity;
    float* nom = c->h_in + kStateSlot;
    for (int h = 0; h < H; ++h) {
        nom[4 * h + 0] = rotor ? 0.f : cfg->mass * cfg->gravity;
        nom[4 * h + 1] = nom[4 * h + 2] = nom[4 * h + 3] = 0.f;
    }
    bool ok = cudaMemcpyAsync(B.state, st, kStateSlot * sizeof(float), cudaMemcpyHostToDevice, c->stream) == cudaSuccess &&
              cudaMemcpyAsync(B.nominal, nom, H * sizeof(float4), cudaMemcpyHostToDevice, c->stream) == cudaSuccess &&
              cudaMemsetAsync(B.step, 0, 2 * sizeof(uint32_t), c->stream) == cudaSuccess &&
              cudaMemsetAsync(B.tickets, 0, 32 * sizeof(unsigned), c->stream) == cudaSuccess &&
              cudaMemsetAsync(B.err, 0, sizeof(int), c->stream) == cudaSuccess &&
              cudaMemsetAsync(B.poses, 0, MG * 8 * sizeof(float), c->stream) == cudaSuccess &&
              cudaStreamSynchronize(c->stream) == cudaSuccess;
    if (!ok) {
        std::snprintf(g_thread_err, sizeof(g_thread_err), "initialisation copies failed: %s",
                      cudaGetErrorString(cudaGetLastError()));
        mppi_destroy(c);
        return MPPI_E_CUDA;
    }
    *out = c;
    return MPPI_OK;
}

int mppi_set_gates(mppi_ctx* c, int n_gates, const float* poses, const float* latents) {
    if (!c) return fail(nullptr, MPPI_E_INVALID, "ctx is NULL");
    if (n_gates < 0 || n_gates > c->cfg.max_gates)
        return fail(c, MPPI_E_INVALID, "n_gates=%d out of [0, %d]", n_gates, c->cfg.max_gates);
    if (n_gates > 0 && !poses) return fail(c, MPPI_E_INVALID, "poses is NULL");
    if (n_gates > 0 && !finite_all(poses, static_cast<size_t>(n_gates) * 7))
        return fail(c, MPPI_E_INVALID, "non-finite gate pose");
    if (latents && !finite_all(latents, static_cast<size_t>(n_gates) * kLatent))
        return fail(c, MPPI_E_INVALID, "non-finite latent");
    float* hp = c->h_in + kStateSlot + c->cfg.H * 4;
    float* hl = hp + c->cfg.max_gates * 8;
    for (int g = 0; g < n_gates; ++g) {
        for (int i = 0; i < 7; ++i) hp[8 * g + i] = poses[7 * g + i];
        hp[8 * g + 7] = 0.f;
    }
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    if (c->n_gates != n_gates) c->graph_dirty = true;
    c->n_gates = n_gates;
    if (n_gates > 0)
        CUDA_TRY(c, cudaMemcpyAsync(c->B.poses, hp, n_gates * 8 * sizeof(float), cudaMemcpyHostToDevice, c->stream));
    if (latents && n_gates > 0) {
        std::memcpy(hl, latents, static_cast<size_t>(n_gates) * kLatent * sizeof(float));
        CUDA_TRY(c, cudaMemcpyAsync(c->d_latents, hl, n_gates * kLatent * sizeof(float), cudaMemcpyHostToDevice,
                                    c->stream));
        c->have_latents = true;
    } else if (!latents) {
        c->have_latents = (n_gates == 0);
    }
    int rc = recompute_b1p(c);
    if (rc != MPPI_OK) return rc;
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    return MPPI_OK;
}

int mppi_set_sdf_weights(mppi_ctx* c, const float* const* layers, int n_layers, const float* fp8_scales) {
    if (!c) return fail(nullptr, MPPI_E_INVALID, "ctx is NULL");
    if (!layers || n_layers != 2 * MPPI_MLP_LAYERS)
        return fail(c, MPPI_E_INVALID, "expected %d layer pointers (W, b for 5 affine maps)", 2 * MPPI_MLP_LAYERS);
    if (fp8_scales) {
        for (int i = 0; i < 3; ++i)
            if (!std::isfinite(fp8_scales[i]) || !(fp8_scales[i] > 0.f))
                return fail(c, MPPI_E_INVALID, "fp8_scales[%d] must be finite and > 0", i);
    }
    for (int i = 0; i < n_layers; ++i)
        if (!layers[i]) return fail(c, MPPI_E_INVALID, "layer pointer %d is NULL", i);
    const int pf = point_features(c->cfg);
    const int in1 = pf + kLatent;
    const size_t sizes[10] = {static_cast<size_t>(kHidden) * in1, kHidden, kHidden * kHidden, kHidden,
                              kHidden * kHidden, kHidden, kHidden * kHidden, kHidden, kHidden, 1};
    for (int i = 0; i < 10; ++i)
        if (!finite_all(layers[i], sizes[i])) return fail(c, MPPI_E_INVALID, "non-finite value in layer array %d", i);
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    CUDA_TRY(c, cudaMemcpy(c->d_W1, layers[0], sizes[0] * sizeof(float), cudaMemcpyHostToDevice));
    CUDA_TRY(c, cudaMemcpy(c->d_b1, layers[1], sizes[1] * sizeof(float), cudaMemcpyHostToDevice));
    std::vector<float> t(kHidden * kHidden);
    std::vector<uint16_t> bf(kHidden * kHidden), hf(kHidden * kHidden);
    std::vector<uint8_t> f8(kHidden * kHidden);
    const float cl2 = c->cfg.softplus_beta * 1.4426950408889634f;
    for (int l = 0; l < 3; ++l) {
        const float* Wl = layers[2 + 2 * l];
        // FP8: per-tensor weight scale max|W| / 448 (the E4M3 range); activation scale from
        // fp8_scales (softplus-output units, default 1/64), carried here in log2 units
        float wmax = 0.f;
        for (int i = 0; i < kHidden * kHidden; ++i) wmax = std::fmax(wmax, std::fabs(Wl[i]));
        const float sw = wmax > 0.f ? wmax / 448.f : 1.f;
        const float sa = cl2 * (fp8_scales ? fp8_scales[l] : (1.f / 64.f));
        c->f8_dequant[l] = sw * sa;
        c->f8_inv_act[l] = 1.f / sa;
        for (int n = 0; n < kHidden; ++n)
            for (int k = 0; k < kHidden; ++k)
                f8[tc_operand8_offset(n, k)] =
                    static_cast<uint8_t>(__nv_cvt_float_to_fp8(Wl[n * kHidden + k] / sw, __NV_SATFINITE, __NV_E4M3));
        for (int n = 0; n < kHidden; ++n)
            for (int k = 0; k < kHidden; ++k) {
                t[k * kHidden + n] = Wl[n * kHidden + k];
                bf[tc_operand_offset(n, k)] = float_to_bf16(Wl[n * kHidden + k]);
                hf[tc_operand_offset(n, k)] = float_to_f16(Wl[n * kHidden + k]);
            }
        CUDA_TRY(c, cudaMemcpy(c->d_Wt[l], t.data(), t.size() * sizeof(float), cudaMemcpyHostToDevice));
        CUDA_TRY(c, cudaMemcpy(c->d_Wbf[l], bf.data(), bf.size() * sizeof(uint16_t), cudaMemcpyHostToDevice));
        CUDA_TRY(c, cudaMemcpy(c->d_Wh[l], hf.data(), hf.size() * sizeof(uint16_t), cudaMemcpyHostToDevice));
        CUDA_TRY(c, cudaMemcpy(c->d_W8[l], f8.data(), f8.size(), cudaMemcpyHostToDevice));
        CUDA_TRY(c, cudaMemcpy(c->d_bias[l], layers[3 + 2 * l], kHidden * sizeof(float), cudaMemcpyHostToDevice));
    }
    CUDA_TRY(c, cudaMemcpy(c->d_w5, layers[8], kHidden * sizeof(float), cudaMemcpyHostToDevice));
    // layer-1 tensor-core operand, K = layer1_k columns of beta log2(e) W1: row n =
    // [hi(0..2), hi(0..2), lo(0..2) of the point columns, 0 x 7, then per PE level its six
    // columns in BF16 and 0 x 2] (layer1_gemm_k, pe_column)
    {
        const int k1 = layer1_k(c->cfg);
        std::vector<uint16_t> w1(static_cast<size_t>(kHidden) * k1, 0);
        for (int n = 0; n < kHidden; ++n) {
            for (int j = 0; j < 3; ++j) {
                const float ws = cl2 * layers[0][n * in1 + j];
                const uint16_t hi = float_to_bf16(ws);
                uint32_t hb = static_cast<uint32_t>(hi) << 16;
                float hf;
                std::memcpy(&hf, &hb, 4);
                const uint16_t lo = float_to_bf16(ws - hf);
                w1[tc_operand_k_offset(n, j, k1)] = hi;
                w1[tc_operand_k_offset(n, 3 + j, k1)] = hi;
                w1[tc_operand_k_offset(n, 6 + j, k1)] = lo;
            }
            for (int j = 3; j < pf; ++j)
                w1[tc_operand_k_offset(n, pe_column((j - 3) / 6, (j - 3) % 6), k1)] =
                    float_to_bf16(cl2 * layers[0][n * in1 + j]);
        }
        CUDA_TRY(c, cudaMemcpy(c->d_W1tc, w1.data(), w1.size() * sizeof(uint16_t), cudaMemcpyHostToDevice));
    }
    c->b5 = layers[9][0];
    c->graph_dirty = true;
    c->have_weights = true;
    int rc = recompute_b1p(c);
    if (rc != MPPI_OK) return rc;
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    return MPPI_OK;
}

int mppi_debug_inject_timeout(mppi_ctx* c) {
    if (!c) return fail(nullptr, MPPI_E_INVALID, "ctx is NULL");
    const unsigned one = 1u;
    CUDA_TRY(c, cudaMemcpyAsync(c->B.tickets + 31, &one, sizeof(unsigned), cudaMemcpyHostToDevice, c->stream));
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    return MPPI_OK;
}

int mppi_step(mppi_ctx* c, const float* state, const float* gate_poses, const float* latents, const float* nominal,
              float* new_controls, float* weights, float* costs) {
    if (!c) return fail(nullptr, MPPI_E_INVALID, "ctx is NULL");
    if (!new_controls) return fail(c, MPPI_E_INVALID, "new_controls is NULL");
    const int K = c->cfg.K, H = c->cfg.H;
    if (state && !finite_all(state, state_dim(c->cfg))) return fail(c, MPPI_E_INVALID, "non-finite state");
    if (nominal && !finite_all(nominal, static_cast<size_t>(H) * 4))
        return fail(c, MPPI_E_INVALID, "non-finite nominal");
    if (gate_poses || latents) {
        // gates change: same path as mppi_set_gates with the current count
        if (gate_poses) {
            int rc = mppi_set_gates(c, c->n_gates, gate_poses, latents);
            if (rc != MPPI_OK) return rc;
        } else {
            if (!finite_all(latents, static_cast<size_t>(c->n_gates) * kLatent))
                return fail(c, MPPI_E_INVALID, "non-finite latent");
            float* hl = c->h_in + kStateSlot + H * 4 + c->cfg.max_gates * 8;
            CUDA_TRY(c, cudaStreamSynchronize(c->stream));
            std::memcpy(hl, latents, static_cast<size_t>(c->n_gates) * kLatent * sizeof(float));
            if (c->n_gates > 0)
                CUDA_TRY(c, cudaMemcpyAsync(c->d_latents, hl, c->n_gates * kLatent * sizeof(float),
                                            cudaMemcpyHostToDevice, c->stream));
            c->have_latents = true;
            int rc = recompute_b1p(c);
            if (rc != MPPI_OK) return rc;
        }
    }
    int rc = check_ready(c);
    if (rc != MPPI_OK) return rc;
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));   // staging buffers are free
    if (state) std::memcpy(c->h_in, state, state_dim(c->cfg) * sizeof(float));   // copied by the step's graph
    if (nominal) {
        std::memcpy(c->h_in + kStateSlot, nominal, static_cast<size_t>(H) * 4 * sizeof(float));
        CUDA_TRY(c, cudaMemcpyAsync(c->B.nominal, c->h_in + kStateSlot, H * sizeof(float4), cudaMemcpyHostToDevice,
                                    c->stream));
    }
    // the step's last kernel writes U*_new (and w, J when asked for) straight into the
    // pinned staging buffer
    float* ho = c->h_out;
    float* dho = c->d_hout;
    // and the error word too: -1 stays if the step's last kernel did not finish its work
    volatile int* herr = reinterpret_cast<volatile int*>(ho + H * 4 + 2 * K);
    *herr = -1;
    set_outputs(c, reinterpret_cast<float4*>(dho), weights ? dho + H * 4 : nullptr, costs ? dho + H * 4 + K : nullptr,
                reinterpret_cast<int*>(dho + H * 4 + 2 * K));
    rc = launch_step(c, state != nullptr);
    if (rc != MPPI_OK) return rc;
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    ++c->step_count;
    if (*herr != 0) {
        CUDA_TRY(c, clear_device_error(c));
        CUDA_TRY(c, cudaStreamSynchronize(c->stream));
        return fail(c, MPPI_E_TIMEOUT, "a device-side wait timed out (error word %d)", *herr);
    }
    std::memcpy(new_controls, ho, static_cast<size_t>(H) * 4 * sizeof(float));
    if (weights) std::memcpy(weights, ho + H * 4, static_cast<size_t>(K) * sizeof(float));
    if (costs) std::memcpy(costs, ho + H * 4 + K, static_cast<size_t>(K) * sizeof(float));
    return MPPI_OK;
}

int mppi_step_async(mppi_ctx* c, const float* d_state, const float* d_gate_poses, const float* d_latents,
                    const float* d_nominal, float* d_new_controls, float* d_weights, float* d_costs) {
    if (!c) return fail(nullptr, MPPI_E_INVALID, "ctx is NULL");
    if (!d_new_controls) return fail(c, MPPI_E_INVALID, "d_new_controls is NULL");
    // the update kernel stores U*_new as float4: a misaligned buffer is refused before anything is enqueued
    if (reinterpret_cast<uintptr_t>(d_new_controls) % 16 != 0)
        return fail(c, MPPI_E_INVALID, "d_new_controls must be 16-byte aligned");
    const int H = c->cfg.H, G = c->n_gates;
    if (d_state)
        CUDA_TRY(c, cudaMemcpyAsync(c->B.state, d_state, state_dim(c->cfg) * sizeof(float), cudaMemcpyDeviceToDevice,
                                    c->stream));
    if (d_gate_poses && G > 0)
        CUDA_TRY(c, cudaMemcpy2DAsync(c->B.poses, 8 * sizeof(float), d_gate_poses, 7 * sizeof(float),
                                      7 * sizeof(float), G, cudaMemcpyDeviceToDevice, c->stream));
    if (d_latents && G > 0) {
        CUDA_TRY(c, cudaMemcpyAsync(c->d_latents, d_latents, G * kLatent * sizeof(float), cudaMemcpyDeviceToDevice,
                                    c->stream));
        c->have_latents = true;
        int rc = recompute_b1p(c);
        if (rc != MPPI_OK) return rc;
    }
    int rc = check_ready(c);
    if (rc != MPPI_OK) return rc;
    if (d_nominal)
        CUDA_TRY(c, cudaMemcpyAsync(c->B.nominal, d_nominal, H * sizeof(float4), cudaMemcpyDeviceToDevice, c->stream));
    // the step's last kernel writes the caller's buffers itself; a change of buffers is a
    // change of launch arguments (the step graph is captured again)
    set_outputs(c, reinterpret_cast<float4*>(d_new_controls), d_weights, d_costs, nullptr);
    rc = launch_step(c, false);
    if (rc != MPPI_OK) return rc;
    ++c->step_count;
    return MPPI_OK;
}

int mppi_sync(mppi_ctx* c) {
    if (!c) return fail(nullptr, MPPI_E_INVALID, "ctx is NULL");
    return read_err_word(c);
}

int mppi_get_nominal(mppi_ctx* c, float* out) {
    if (!c || !out) return fail(c, MPPI_E_INVALID, "NULL argument");
    CUDA_TRY(c, cudaMemcpyAsync(out, c->B.nominal, c->cfg.H * sizeof(float4), cudaMemcpyDeviceToHost, c->stream));
    return read_err_word(c);
}

int mppi_get_state(mppi_ctx* c, float* out) {
    if (!c || !out) return fail(c, MPPI_E_INVALID, "NULL argument");
    CUDA_TRY(c, cudaMemcpyAsync(out, c->B.state, state_dim(c->cfg) * sizeof(float), cudaMemcpyDeviceToHost, c->stream));
    return read_err_word(c);
}

int mppi_set_step_counter(mppi_ctx* c, uint64_t step) {
    if (!c) return fail(nullptr, MPPI_E_INVALID, "ctx is NULL");
    uint32_t* w = reinterpret_cast<uint32_t*>(c->h_in);
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    w[0] = static_cast<uint32_t>(step & 0xFFFFFFFFull);
    w[1] = static_cast<uint32_t>(step >> 32);
    CUDA_TRY(c, cudaMemcpyAsync(c->B.step, w, 2 * sizeof(uint32_t), cudaMemcpyHostToDevice, c->stream));
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    c->step_count = step;
    return MPPI_OK;
}

uint64_t mppi_get_step_counter(const mppi_ctx* c) { return c ? c->step_count : 0; }

int mppi_read_buffer(mppi_ctx* c, int which, float* host_out, size_t n) {
    if (!c || !host_out) return fail(c, MPPI_E_INVALID, "NULL argument");
    const size_t K = c->cfg.K, H = c->cfg.H;
    const void* src = nullptr;
    size_t count = 0;
    switch (which) {
        case MPPI_BUF_NOISE: src = c->B.noise; count = H * K * 4; break;
        case MPPI_BUF_POSITIONS: src = c->B.pos; count = H * K * 4; break;
        case MPPI_BUF_COST_PARTS: src = c->B.parts; count = 3 * K; break;
        case MPPI_BUF_SDF:
            if (!c->store_sdf)
                return fail(c, MPPI_E_INVALID, "MPPI_BUF_SDF is written only with MPPI_DIAG_STORE_SDF set");
            src = c->B.sdf;
            count = H * K;
            break;
        case MPPI_BUF_WEIGHTS: src = c->B.w; count = K; break;
        case MPPI_BUF_COSTS: src = c->B.J; count = K; break;
        default: return fail(c, MPPI_E_INVALID, "unknown buffer %d", which);
    }
    if (n < count) return fail(c, MPPI_E_INVALID, "buffer %d needs %zu floats, got %zu", which, count, n);
    CUDA_TRY(c, cudaMemcpyAsync(host_out, src, count * sizeof(float), cudaMemcpyDeviceToHost, c->stream));
    return read_err_word(c);
}

int mppi_read_noise_words(mppi_ctx* c, uint32_t* host_out, size_t n) {
    if (!c || !host_out) return fail(c, MPPI_E_INVALID, "NULL argument");
    const size_t count = static_cast<size_t>(c->cfg.K) * c->cfg.H * 4;
    if (n < count) return fail(c, MPPI_E_INVALID, "needs %zu words, got %zu", count, n);
    uint4* tmp = nullptr;
    CUDA_TRY(c, cudaMalloc(&tmp, count * sizeof(uint32_t)));
    const StepParams P = make_params(c);
    cudaError_t e = launch_noise_words(P, c->B, tmp, c->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(host_out, tmp, count * sizeof(uint32_t), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    cudaFree(tmp);
    if (e != cudaSuccess) return fail(c, MPPI_E_CUDA, "noise words: %s", cudaGetErrorString(e));
    return MPPI_OK;
}

int mppi_set_diagnostics(mppi_ctx* c, int flags) {
    if (!c) return fail(nullptr, MPPI_E_INVALID, "ctx is NULL");
    if (flags & ~(MPPI_DIAG_STORE_SDF | MPPI_DIAG_SDF_SINGLE_CTA))
        return fail(c, MPPI_E_INVALID, "unknown diagnostics flags 0x%x", flags);
    const bool store = (flags & MPPI_DIAG_STORE_SDF) != 0;
    const bool single = (flags & MPPI_DIAG_SDF_SINGLE_CTA) != 0;
    if (c->store_sdf != store || c->sdf_single_cta != single) c->graph_dirty = true;
    c->store_sdf = store;
    c->sdf_single_cta = single;
    return MPPI_OK;
}

int mppi_set_timing(mppi_ctx* c, int enable) {
    if (!c) return fail(nullptr, MPPI_E_INVALID, "ctx is NULL");
    if (c->timing != (enable != 0)) c->graph_dirty = true;
    c->timing = enable != 0;
    return MPPI_OK;
}

int mppi_get_kernel_times(mppi_ctx* c, const char** names, float* ms, int cap) {
    if (!c) return fail(nullptr, MPPI_E_INVALID, "ctx is NULL");
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    int n = 0;
    for (int i = 1; i < c->n_ev && n < cap; ++i, ++n) {
        float t = 0.f;
        CUDA_TRY(c, cudaEventElapsedTime(&t, c->ev[i - 1], c->ev[i]));
        if (names) names[n] = c->ev_names[i];
        if (ms) ms[n] = t;
    }
    return n;
}

int mppi_kernels_per_step(const mppi_ctx* c) {
    if (!c) return 0;
    return is_mlp(c) ? 3 : 2;
}

int mppi_selftest_tc_gemm(const uint16_t* d_A, const uint16_t* d_B, float* d_D, void* stream) {
    int dev = 0, major = 0, minor = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return fail(nullptr, MPPI_E_UNSUPPORTED, "no CUDA device");
    cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev);
    cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev);
    if (major != 10 || minor != 3) return fail(nullptr, MPPI_E_UNSUPPORTED, "device is sm_%d%d", major, minor);
    if (!d_A || !d_B || !d_D) return fail(nullptr, MPPI_E_INVALID, "NULL argument");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int* derr = nullptr;
    if (cudaMalloc(&derr, sizeof(int)) != cudaSuccess) return fail(nullptr, MPPI_E_OOM, "cudaMalloc failed");
    cudaError_t e = cudaMemsetAsync(derr, 0, sizeof(int), s);
    if (e == cudaSuccess) e = launch_tc_selftest(d_A, d_B, d_D, derr, s);
    int herr = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&herr, derr, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFree(derr);
    if (e != cudaSuccess) return fail(nullptr, MPPI_E_CUDA, "self-test: %s", cudaGetErrorString(e));
    if (herr != 0) return fail(nullptr, MPPI_E_TIMEOUT, "self-test wait timed out");
    return MPPI_OK;
}

}  // extern "C"

namespace mppi {
void set_thread_error(const char* msg) { std::snprintf(g_thread_err, sizeof(g_thread_err), "%s", msg); }

// ---------------------------------------------------------------- serving hooks
int ctx_enqueue_host_step(mppi_ctx* c, const float* state, int n_gates, const float* poses, const float* latents) {
    const int H = c->cfg.H;
    if (n_gates < 0 || n_gates > c->cfg.max_gates) return fail(c, MPPI_E_INVALID, "n_gates out of range");
    if (!finite_all(state, state_dim(c->cfg))) return fail(c, MPPI_E_INVALID, "non-finite state");
    if (n_gates > 0 && (!poses || !finite_all(poses, static_cast<size_t>(n_gates) * 7)))
        return fail(c, MPPI_E_INVALID, "bad gate poses");
    if (n_gates > 0 && is_mlp(c) && (!latents || !finite_all(latents, static_cast<size_t>(n_gates) * kLatent)))
        return fail(c, MPPI_E_INVALID, "bad latents");
    // the staging buffers are free: the caller has one request per context in flight
    float* hs = c->h_in;
    float* hp = c->h_in + kStateSlot + H * 4;
    float* hl = hp + c->cfg.max_gates * 8;
    std::memcpy(hs, state, state_dim(c->cfg) * sizeof(float));
    for (int g = 0; g < n_gates; ++g) {
        for (int i = 0; i < 7; ++i) hp[8 * g + i] = poses[7 * g + i];
        hp[8 * g + 7] = 0.f;
    }
    if (c->n_gates != n_gates) c->graph_dirty = true;
    c->n_gates = n_gates;
    if (n_gates > 0) {
        CUDA_TRY(c, cudaMemcpyAsync(c->B.poses, hp, n_gates * 8 * sizeof(float), cudaMemcpyHostToDevice, c->stream));
        if (latents) {
            std::memcpy(hl, latents, static_cast<size_t>(n_gates) * kLatent * sizeof(float));
            CUDA_TRY(c, cudaMemcpyAsync(c->d_latents, hl, n_gates * kLatent * sizeof(float), cudaMemcpyHostToDevice,
                                        c->stream));
            c->have_latents = true;
            int rc = recompute_b1p(c);
            if (rc != MPPI_OK) return rc;
        }
    }
    int rc = check_ready(c);
    if (rc != MPPI_OK) return rc;
    // U*_new and the error word straight into pinned staging (-1 stays if the step's last
    // kernel did not finish its work)
    *reinterpret_cast<volatile int*>(c->h_out + H * 4 + 2 * c->cfg.K) = -1;
    set_outputs(c, reinterpret_cast<float4*>(c->d_hout), nullptr, nullptr,
                reinterpret_cast<int*>(c->d_hout + H * 4 + 2 * c->cfg.K));
    rc = launch_step(c, true);                     // the graph copies the staged state first
    if (rc != MPPI_OK) return rc;
    CUDA_TRY(c, cudaEventRecord(c->done, c->stream));
    ++c->step_count;
    return MPPI_OK;
}

int ctx_batch_slot(mppi_ctx* c, const float* state, int n_gates, const float* poses, const float* latents,
                   BatchSlot* slot, float* in) {
    const int H = c->cfg.H, K = c->cfg.K;
    const bool mlp = is_mlp(c);
    if (n_gates < 0 || n_gates > c->cfg.max_gates) return fail(c, MPPI_E_INVALID, "n_gates out of range");
    if (!finite_all(state, state_dim(c->cfg))) return fail(c, MPPI_E_INVALID, "non-finite state");
    if (n_gates > 0 && (!poses || !finite_all(poses, static_cast<size_t>(n_gates) * 7)))
        return fail(c, MPPI_E_INVALID, "bad gate poses");
    if (n_gates > 0 && mlp && (!latents || !finite_all(latents, static_cast<size_t>(n_gates) * kLatent)))
        return fail(c, MPPI_E_INVALID, "bad latents");
    if (mlp && !c->have_weights) return fail(c, MPPI_E_NOT_READY, "MLP SDF mode but no weights set");
    if (c->n_gates != n_gates) c->graph_dirty = true;
    c->n_gates = n_gates;
    if (mlp && n_gates > 0) c->have_latents = true;
    // state, gate poses (7 + 1 pad each) and latents, as the batch's prep kernel reads them
    std::memset(in, 0, kBatchStateSlot * sizeof(float));
    std::memcpy(in, state, state_dim(c->cfg) * sizeof(float));
    float* hp = in + kBatchStateSlot;
    for (int g = 0; g < n_gates; ++g) {
        for (int i = 0; i < 7; ++i) hp[8 * g + i] = poses[7 * g + i];
        hp[8 * g + 7] = 0.f;
    }
    int used = kBatchStateSlot + 8 * n_gates;
    if (mlp) {
        std::memcpy(in + used, latents, static_cast<size_t>(n_gates) * kLatent * sizeof(float));
        used += kLatent * n_gates;
    }
    // U*_new and the error word straight into pinned staging (-1 stays if the step's last kernel
    // did not finish its work)
    *reinterpret_cast<volatile int*>(c->h_out + H * 4 + 2 * K) = -1;
    set_outputs(c, reinterpret_cast<float4*>(c->d_hout), nullptr, nullptr,
                reinterpret_cast<int*>(c->d_hout + H * 4 + 2 * K));
    slot->P = make_params(c);
    slot->P.pdl = 0;
    slot->B = c->B;
    slot->W1 = c->d_W1;
    slot->b1 = c->d_b1;
    slot->latents = c->d_latents;
    slot->n_point = point_features(c->cfg);
    slot->state_floats = state_dim(c->cfg);
    slot->mlp = mlp ? 1 : 0;
    return used;
}

void ctx_batch_launched(mppi_ctx* c) { ++c->step_count; }

int ctx_batch_result(mppi_ctx* c, float* new_controls) {
    const int H = c->cfg.H;
    const volatile int* herr = reinterpret_cast<const volatile int*>(c->h_out + H * 4 + 2 * c->cfg.K);
    if (*herr != 0) return fail(c, MPPI_E_TIMEOUT, "a device-side wait timed out (error word %d)", *herr);
    std::memcpy(new_controls, c->h_out, static_cast<size_t>(H) * 4 * sizeof(float));
    return MPPI_OK;
}

int ctx_clear_error(mppi_ctx* c) {
    CUDA_TRY(c, clear_device_error(c));
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    return MPPI_OK;
}

MlpWeights ctx_weights(const mppi_ctx* c) { return make_weights(c); }
StepParams ctx_params(const mppi_ctx* c) { return make_params(c); }
int ctx_num_sms(const mppi_ctx* c) { return c->num_sms; }

int ctx_poll_host_step(mppi_ctx* c, float* new_controls) {
    const cudaError_t q = cudaEventQuery(c->done);
    if (q == cudaErrorNotReady) return 1;
    if (q != cudaSuccess) return fail(c, MPPI_E_CUDA, "step failed: %s", cudaGetErrorString(q));
    const int H = c->cfg.H;
    const volatile int* herr = reinterpret_cast<const volatile int*>(c->h_out + H * 4 + 2 * c->cfg.K);
    if (*herr != 0) {
        CUDA_TRY(c, clear_device_error(c));
        return fail(c, MPPI_E_TIMEOUT, "a device-side wait timed out (error word %d)", *herr);
    }
    std::memcpy(new_controls, c->h_out, static_cast<size_t>(H) * 4 * sizeof(float));
    return MPPI_OK;
}

int ctx_save(mppi_ctx* c, float* nominal, float* state, uint64_t* step) {
    int rc = mppi_get_nominal(c, nominal);
    if (rc != MPPI_OK) return rc;
    rc = mppi_get_state(c, state);
    if (rc != MPPI_OK) return rc;
    *step = c->step_count;
    return MPPI_OK;
}

int ctx_restore(mppi_ctx* c, const float* nominal, const float* state, uint64_t step) {
    const int H = c->cfg.H;
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    std::memcpy(c->h_in, state, state_dim(c->cfg) * sizeof(float));
    std::memcpy(c->h_in + kStateSlot, nominal, static_cast<size_t>(H) * 4 * sizeof(float));
    CUDA_TRY(c, cudaMemcpyAsync(c->B.state, c->h_in, state_dim(c->cfg) * sizeof(float), cudaMemcpyHostToDevice,
                                c->stream));
    CUDA_TRY(c, cudaMemcpyAsync(c->B.nominal, c->h_in + kStateSlot, H * sizeof(float4), cudaMemcpyHostToDevice, c->stream));
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    return mppi_set_step_counter(c, step);
}

size_t ctx_device_bytes(const mppi_config& g) {
    const size_t K = g.K, H = g.H, MG = g.max_gates;
    const size_t nub = static_cast<size_t>(update_blocks(g.K));
    const size_t floats = 16 + 4 * H + 2 + MG * 8 + MG * kHidden + 4 * K * H * 2 + 3 * K + K * H +
                          K * static_cast<size_t>(col_slots(g.H)) + 2 * K + 4 * H + nub * (4 * H + 2) + 4 + 32 + 1 +
                          MG * kLatent;
    const size_t weights = sizeof(float) * (kHidden * (point_features(g) + kLatent) + kHidden +
                                            3 * (kHidden * kHidden + kHidden) + kHidden) +
                           3 * kHidden * kHidden * (2 + 2 + 1) + static_cast<size_t>(kHidden) * layer1_k(g) * 2;
    return floats * sizeof(float) + weights;
}

uint16_t float_to_bf16(float f) {
    uint32_t u;
    std::memcpy(&u, &f, 4);
    if ((u & 0x7F800000u) == 0x7F800000u) return static_cast<uint16_t>(u >> 16);   // inf / nan (inputs are finite)
    const uint32_t rounding = 0x7FFFu + ((u >> 16) & 1u);                           // round to nearest even
    return static_cast<uint16_t>((u + rounding) >> 16);
}
uint16_t float_to_f16(float f) { return __half_as_ushort(__float2half_rn(f)); }
}  // namespace mppi
