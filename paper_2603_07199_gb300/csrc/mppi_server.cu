// Serving engine: continuous batching of MPPI control steps from many drones.
//
// Each drone owns a controller context (device-resident warm start, true state
// and Philox step counter, its own stream and captured step graph), created on
// the drone's first request when the device-memory budget allows.  A worker
// thread admits queued requests in arrival order as soon as the drone is idle,
// an in-flight slot is free and the drone's context fits in the budget; when it
// does not fit, the least recently used idle drone is evicted (its warm start,
// state and counter go to host memory and come back on its next request).
// Batched mode (the default): the worker gathers every admissible queued request
// into one batch and launches it as four kernels on the server's stream -- the
// inputs of all drones, one rollout launch over all drones' rollouts, one
// persistent tensor-core SDF launch whose tiles span all drones, and one update
// launch whose per-drone combine is done by the last of the drone's blocks -- so
// that a batch of small solves fills the GPU like one large solve; up to four
// batches, each on its own stream, run at once.  Per-drone mode: each drone's step
// is its own captured graph on its own stream and requests of different drones
// overlap on the GPU.  Either way a drone's results are those of its own step
// (same kernels' arithmetic, per-drone noise counters, fixed-order reductions).
// Results are collected per ticket with their submit-to-completion latency.
#include <chrono>
#include <condition_variable>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <deque>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include "ctx_internal.h"
#include "kernels.h"
#include "mppi.h"

namespace {

using Clock = std::chrono::steady_clock;

struct Drone {
    mppi_config cfg{};
    mppi_ctx* ctx = nullptr;
    size_t bytes = 0;
    bool busy = false;
    uint64_t last_use = 0;
    bool saved = false;               // warm start held in host memory after an eviction
    std::vector<float> nominal;
    float state[MPPI_STATE_MAX] = {};
    uint64_t step = 0;
};

struct Request {
    uint64_t ticket = 0;
    int drone = 0;
    float state[MPPI_STATE_MAX] = {};
    int n_gates = 0;
    std::vector<float> poses, latents;
    Clock::time_point t_submit;
};

struct Inflight {
    uint64_t ticket;
    int drone;
    Clock::time_point t_submit;
};

struct Result {
    int status = MPPI_OK;
    std::vector<float> controls;
    double latency_us = 0.0;
};

// One batch buffer: pinned host block (slots, then packed inputs), its device copy, the
// batch's SDF error word (pinned, mapped) and completion event.
struct BatchBuf {
    cudaStream_t stream = nullptr;          // batches in different buffers overlap on the GPU
    char* h = nullptr;
    char* d = nullptr;
    int* h_err = nullptr;
    int* d_err = nullptr;
    cudaEvent_t done = nullptr;
    std::vector<Inflight> reqs;
    bool busy = false;
    bool pair_tiles = false;                // the batch's tile layout is for the pair form of the SDF kernel
};

constexpr int kBatchInFloats = mppi::kBatchStateSlot + MPPI_MAX_GATES * (8 + MPPI_LATENT_DIM);
constexpr int kBatchBufs = 4;             // batches in flight at once

}  // namespace

struct mppi_server {
    mppi_server_config cfg{};
    int device = 0;
    std::vector<std::vector<float>> layers;
    std::vector<float> fp8;
    bool have_weights = false;
    std::mutex mu;
    std::thread worker;
    bool stop = false;
    std::deque<Request> queue;
    std::unordered_map<int, Drone> drones;
    std::vector<Inflight> inflight;
    std::unordered_map<uint64_t, Result> results;
    uint64_t next_ticket = 1;
    uint64_t lru_clock = 0;
    size_t used_bytes = 0, peak_bytes = 0;
    uint64_t completed = 0, evictions = 0, restores = 0, admitted = 0;
    // batched mode
    BatchBuf buf[kBatchBufs];
    std::deque<int> order;                 // busy batch buffers, oldest first
    size_t slots_bytes = 0;
    float beta = 0.f;                      // softplus sharpness and encoding levels every drone shares
    int pe_levels = -1;
    uint64_t batches = 0;
    char err[512] = "";
};

namespace {

thread_local char g_server_err[512] = "";

int sfail(mppi_server* s, int code, const char* fmt, ...) {
    char* dst = s ? s->err : g_server_err;
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(dst, 512, fmt, ap);
    va_end(ap);
    return code;
}

// Make room for `need` bytes by evicting least recently used idle drones.
bool make_room(mppi_server* s, size_t need, int keep) {
    const size_t budget = s->cfg.hbm_budget_bytes;
    while (budget != 0 && s->used_bytes + need > budget) {
        Drone* victim = nullptr;
        for (auto& kv : s->drones) {
            Drone& d = kv.second;
            if (kv.first == keep || d.ctx == nullptr || d.busy) continue;
            if (victim == nullptr || d.last_use < victim->last_use) victim = &d;
        }
        if (victim == nullptr) return false;
        victim->nominal.assign(static_cast<size_t>(victim->cfg.H) * 4, 0.f);
        if (mppi::ctx_save(victim->ctx, victim->nominal.data(), victim->state, &victim->step) != MPPI_OK) return false;
        victim->saved = true;
        mppi_destroy(victim->ctx);
        victim->ctx = nullptr;
        s->used_bytes -= victim->bytes;
        ++s->evictions;
    }
    return true;
}

// Create (or restore) the drone's context.  Returns MPPI_OK, 1 when the budget
// cannot hold it right now, or an error.
int ensure_context(mppi_server* s, int id, Drone& d) {
    if (d.ctx) return MPPI_OK;
    const size_t need = mppi::ctx_device_bytes(d.cfg);
    if (s->cfg.hbm_budget_bytes != 0 && need > s->cfg.hbm_budget_bytes)
        return sfail(s, MPPI_E_ADMISSION, "drone %d needs %zu bytes, more than the whole budget", id, need);
    if (!make_room(s, need, id)) return 1;
    mppi_ctx* c = nullptr;
    int rc = mppi_create(&d.cfg, nullptr, &c);
    if (rc != MPPI_OK) return sfail(s, rc, "drone %d: %s", id, mppi_last_error(nullptr));
    if (s->cfg.sdf_single_cta) mppi_set_diagnostics(c, MPPI_DIAG_SDF_SINGLE_CTA);
    if (s->have_weights && d.cfg.sdf_mode != MPPI_SDF_ANALYTIC) {
        const float* ptrs[2 * MPPI_MLP_LAYERS];
        for (int i = 0; i < 2 * MPPI_MLP_LAYERS; ++i) ptrs[i] = s->layers[i].data();
        rc = mppi_set_sdf_weights(c, ptrs, 2 * MPPI_MLP_LAYERS, s->fp8.empty() ? nullptr : s->fp8.data());
        if (rc != MPPI_OK) {
            sfail(s, rc, "drone %d: %s", id, mppi_last_error(c));
            mppi_destroy(c);
            return rc;
        }
    }
    if (d.saved) {
        rc = mppi::ctx_restore(c, d.nominal.data(), d.state, d.step);
        if (rc != MPPI_OK) {
            sfail(s, rc, "drone %d restore: %s", id, mppi_last_error(c));
            mppi_destroy(c);
            return rc;
        }
        d.saved = false;
        ++s->restores;
    }
    d.ctx = c;
    d.bytes = need;
    s->used_bytes += need;
    if (s->used_bytes > s->peak_bytes) s->peak_bytes = s->used_bytes;
    return MPPI_OK;
}

void finish(mppi_server* s, const Inflight& f, int status, std::vector<float>&& controls) {
    Result r;
    r.status = status;
    r.controls = std::move(controls);
    r.latency_us = std::chrono::duration<double, std::micro>(Clock::now() - f.t_submit).count();
    s->results[f.ticket] = std::move(r);
    ++s->completed;
}

// A request admitted under the server's lock, launched after the lock is released (so that a
// submitting thread never waits for GPU launches).
struct Admitted {
    Inflight f;
    mppi_ctx* ctx;
    Request req;
};

void worker_loop(mppi_server* s) {
    cudaSetDevice(s->device);
    std::vector<float> scratch;
    std::vector<Admitted> todo;
    while (true) {
        bool progress = false, idle = false;
        todo.clear();
        {
            std::lock_guard<std::mutex> lock(s->mu);
            // completions
            for (size_t i = 0; i < s->inflight.size();) {
                const Inflight f = s->inflight[i];
                Drone& d = s->drones[f.drone];
                scratch.resize(static_cast<size_t>(d.cfg.H) * 4);
                const int rc = mppi::ctx_poll_host_step(d.ctx, scratch.data());
                if (rc == 1) {
                    ++i;
                    continue;
                }
                std::vector<float> ctrl(scratch.begin(), scratch.end());
                if (rc != MPPI_OK) sfail(s, rc, "drone %d: %s", f.drone, mppi_last_error(d.ctx));
                finish(s, f, rc, std::move(ctrl));
                d.busy = false;
                s->inflight.erase(s->inflight.begin() + static_cast<long>(i));
                progress = true;
            }
            // admissions, in arrival order; a drone with a request in flight keeps its later ones queued
            for (auto it = s->queue.begin(); it != s->queue.end();) {
                if (static_cast<int>(s->inflight.size()) >= s->cfg.max_inflight) break;
                Drone& d = s->drones[it->drone];
                if (d.busy) {
                    ++it;
                    continue;
                }
                const int rc = ensure_context(s, it->drone, d);
                if (rc == 1) break;                       // wait for memory to free up
                Inflight f{it->ticket, it->drone, it->t_submit};
                if (rc != MPPI_OK) {
                    finish(s, f, rc, {});
                    it = s->queue.erase(it);
                    continue;
                }
                // busy: no eviction and no second admission of this drone until it completes
                d.busy = true;
                d.last_use = ++s->lru_clock;
                ++s->admitted;
                s->inflight.push_back(f);
                todo.push_back(Admitted{f, d.ctx, std::move(*it)});
                it = s->queue.erase(it);
                progress = true;
            }
            idle = s->queue.empty() && s->inflight.empty();
            if (idle && s->stop) break;
        }
        // launches outside the lock (only this thread uses a busy drone's context); a request whose
        // launch fails is finished with its error under the lock
        for (Admitted& a : todo) {
            const Request& r = a.req;
            const int e = mppi::ctx_enqueue_host_step(a.ctx, r.state, r.n_gates, r.poses.empty() ? nullptr : r.poses.data(),
                                                      r.latents.empty() ? nullptr : r.latents.data());
            if (e != MPPI_OK) {
                std::lock_guard<std::mutex> lock(s->mu);
                sfail(s, e, "drone %d: %s", a.f.drone, mppi_last_error(a.ctx));
                finish(s, a.f, e, {});
                s->drones[a.f.drone].busy = false;
                for (size_t i = 0; i < s->inflight.size(); ++i)
                    if (s->inflight[i].ticket == a.f.ticket) {
                        s->inflight.erase(s->inflight.begin() + static_cast<long>(i));
                        break;
                    }
            }
        }
        if (idle)
            std::this_thread::sleep_for(std::chrono::microseconds(50));
        else if (!progress)
            std::this_thread::yield();
    }
}

// ---------------------------------------------------------------- batched mode
// Launch a prepared batch on the server's stream: one copy of its block (slots and inputs), the
// prep, rollout, SDF and update launches, and the completion event.  With positional encoding or
// the FP32 MLP the SDF runs per drone (the batched SDF launch is the tensor-core one without
// encoding), still on the batch's stream.
cudaError_t launch_batch(mppi_server* s, BatchBuf& b, int n, size_t in_floats, int roll_blocks, int tiles,
                         int upd_blocks, int max_h, int max_r, const std::vector<mppi_ctx*>& ctxs) {
    using namespace mppi;
    cudaStream_t st = b.stream;
    const BatchSlot* hs = reinterpret_cast<const BatchSlot*>(b.h);
    const BatchSlot* ds = reinterpret_cast<const BatchSlot*>(b.d);
    const float* din = reinterpret_cast<const float*>(b.d + s->slots_bytes);
    cudaError_t e = cudaMemcpyAsync(b.d, b.h, s->slots_bytes + in_floats * sizeof(float), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = launch_batch_prep(ds, n, din, st);
    if (e == cudaSuccess) e = launch_rollout_batch(ds, n, roll_blocks, max_h, st);
    const int mode = s->cfg.sdf_mode;
    if (e == cudaSuccess && mode != MPPI_SDF_ANALYTIC) {
        if (s->pe_levels == 0 && mode != MPPI_SDF_MLP_FP32) {
            e = launch_sdf_batch(mode, b.pair_tiles, ds, n, tiles, ctx_params(ctxs[0]), ctx_weights(ctxs[0]),
                                 b.d_err, ctx_num_sms(ctxs[0]), st);
        } else {
            for (int i = 0; i < n && e == cudaSuccess; ++i) {
                const MlpWeights W = ctx_weights(ctxs[i]);
                const int sms = ctx_num_sms(ctxs[i]);
                switch (mode) {
                    case MPPI_SDF_MLP_FP32: e = launch_sdf_mlp_fp32(hs[i].P, hs[i].B, W, sms, st); break;
                    case MPPI_SDF_MLP_BF16: e = launch_sdf_mlp_bf16(hs[i].P, hs[i].B, W, sms, st); break;
                    case MPPI_SDF_MLP_FP16: e = launch_sdf_mlp_fp16(hs[i].P, hs[i].B, W, sms, st); break;
                    default: e = launch_sdf_mlp_fp8(hs[i].P, hs[i].B, W, sms, st); break;
                }
            }
        }
    }
    if (e == cudaSuccess) e = launch_cost_update_batch(ds, n, upd_blocks, max_r, st);
    if (e == cudaSuccess) e = cudaEventRecord(b.done, st);
    return e;
}

void batched_worker_loop(mppi_server* s) {
    using namespace mppi;
    cudaSetDevice(s->device);
    std::vector<float> scratch;
    std::vector<mppi_ctx*> ctxs;
    while (true) {
        bool progress = false, idle = false;
        // a batch formed under the lock is launched after it is released (so that a submitting
        // thread never waits for GPU launches); its buffer is already in s->order, and the next
        // completion check (this thread, after the launch) sees its recorded event
        int launch_fb = -1, launch_n = 0, l_roll = 0, l_tiles = 0, l_upd = 0, l_max_h = 1, l_max_r = 32;
        size_t l_in = 0;
        {
            std::lock_guard<std::mutex> lock(s->mu);
            // completions (batches on different streams may finish in any order)
            for (size_t oi = 0; oi < s->order.size();) {
                BatchBuf& b = s->buf[s->order[oi]];
                const cudaError_t q = cudaEventQuery(b.done);
                if (q == cudaErrorNotReady) {
                    ++oi;
                    continue;
                }
                const int berr = *reinterpret_cast<volatile int*>(b.h_err);
                for (const Inflight& f : b.reqs) {
                    Drone& d = s->drones[f.drone];
                    scratch.assign(static_cast<size_t>(d.cfg.H) * 4, 0.f);
                    int rc;
                    if (q != cudaSuccess) {
                        rc = sfail(s, MPPI_E_CUDA, "batch failed: %s", cudaGetErrorString(q));
                    } else if (berr != 0) {
                        rc = sfail(s, MPPI_E_TIMEOUT, "a device-side wait of the batch timed out");
                    } else {
                        rc = ctx_batch_result(d.ctx, scratch.data());
                        if (rc != MPPI_OK) sfail(s, rc, "drone %d: %s", f.drone, mppi_last_error(d.ctx));
                    }
                    if (rc == MPPI_E_TIMEOUT) ctx_clear_error(d.ctx);
                    finish(s, f, rc, std::vector<float>(scratch.begin(), scratch.end()));
                    d.busy = false;
                }
                if (berr != 0) *reinterpret_cast<volatile int*>(b.h_err) = 0;
                b.reqs.clear();
                b.busy = false;
                s->order.erase(s->order.begin() + static_cast<long>(oi));
                progress = true;
            }
            // the next batch: every admissible queued request, in arrival order, into a free buffer
            int fb = -1;
            for (int i = 0; i < kBatchBufs && fb < 0; ++i)
                if (!s->buf[i].busy) fb = i;
            if (fb >= 0 && !s->queue.empty()) {
                BatchBuf& b = s->buf[fb];
                BatchSlot* slots = reinterpret_cast<BatchSlot*>(b.h);
                float* in = reinterpret_cast<float*>(b.h + s->slots_bytes);
                size_t inflight = 0;
                for (int i : s->order) inflight += s->buf[i].reqs.size();
                int n = 0, roll = 0, tiles = 0, upd = 0, max_h = 1, max_r = 32;
                size_t in_used = 0;
                // decided once per batch: the same flag lays out the tiles and picks the kernel form
                const bool pair_tiles = s->pe_levels == 0 && !s->cfg.sdf_single_cta &&
                                        sdf_batch_pairs_available(s->cfg.sdf_mode);
                b.pair_tiles = pair_tiles;
                ctxs.clear();
                for (auto it = s->queue.begin(); it != s->queue.end();) {
                    if (inflight + static_cast<size_t>(n) >= static_cast<size_t>(s->cfg.max_inflight)) break;
                    Drone& d = s->drones[it->drone];
                    if (d.busy) {
                        ++it;
                        continue;
                    }
                    const int rc = ensure_context(s, it->drone, d);
                    if (rc == 1) break;                   // wait for memory to free up
                    Inflight f{it->ticket, it->drone, it->t_submit};
                    if (rc != MPPI_OK) {
                        finish(s, f, rc, {});
                        it = s->queue.erase(it);
                        continue;
                    }
                    BatchSlot& sl = slots[n];
                    const int used = ctx_batch_slot(d.ctx, it->state, it->n_gates,
                                                    it->poses.empty() ? nullptr : it->poses.data(),
                                                    it->latents.empty() ? nullptr : it->latents.data(), &sl,
                                                    in + in_used);
                    if (used < 0) {
                        sfail(s, used, "drone %d: %s", it->drone, mppi_last_error(d.ctx));
                        finish(s, f, used, {});
                        it = s->queue.erase(it);
                        continue;
                    }
                    sl.in_off = static_cast<int>(in_used);
                    in_used += static_cast<size_t>(used);
                    sl.roll_form = rollout_form(sl.P);
                    sl.roll_block0 = roll;
                    roll += rollout_batch_blocks(sl.P);
                    sl.tile0 = tiles;
                    if (sl.mlp) {
                        const int t = (sl.P.K * sl.P.H + kTileRows - 1) / kTileRows;
                        tiles += pair_tiles ? (t + 1) & ~1 : t;     // a pair unit never spans two drones
                    }
                    sl.upd_R = update_rollouts_per_block(sl.P.K);
                    sl.upd_block0 = upd;
                    upd += (sl.P.K + sl.upd_R - 1) / sl.upd_R;
                    if (sl.P.H > max_h) max_h = sl.P.H;
                    if (sl.upd_R > max_r) max_r = sl.upd_R;
                    ctxs.push_back(d.ctx);
                    d.busy = true;
                    d.last_use = ++s->lru_clock;
                    ++s->admitted;
                    b.reqs.push_back(f);
                    ++n;
                    it = s->queue.erase(it);
                }
                if (n > 0) {
                    b.busy = true;
                    s->order.push_back(fb);
                    launch_fb = fb;
                    launch_n = n;
                    l_roll = roll;
                    l_tiles = tiles;
                    l_upd = upd;
                    l_max_h = max_h;
                    l_max_r = max_r;
                    l_in = in_used;
                    progress = true;
                }
            }
            idle = s->queue.empty() && s->order.empty();
            if (idle && s->stop) break;
        }
        if (launch_fb >= 0) {
            BatchBuf& b = s->buf[launch_fb];
            const cudaError_t le = launch_batch(s, b, launch_n, l_in, l_roll, l_tiles, l_upd, l_max_h, l_max_r, ctxs);
            std::lock_guard<std::mutex> lock(s->mu);
            if (le != cudaSuccess) {
                const int rc = sfail(s, MPPI_E_CUDA, "batch launch failed: %s", cudaGetErrorString(le));
                for (const Inflight& f : b.reqs) {
                    finish(s, f, rc, {});
                    s->drones[f.drone].busy = false;
                }
                b.reqs.clear();
                b.busy = false;
                for (size_t oi = 0; oi < s->order.size(); ++oi)
                    if (s->order[oi] == launch_fb) {
                        s->order.erase(s->order.begin() + static_cast<long>(oi));
                        break;
                    }
            } else {
                for (mppi_ctx* c : ctxs) ctx_batch_launched(c);
                ++s->batches;
            }
        }
        if (idle)
            std::this_thread::sleep_for(std::chrono::microseconds(50));
        else if (!progress)
            std::this_thread::yield();
    }
}

bool finite(const float* x, size_t n) {
    for (size_t i = 0; i < n; ++i)
        if (!(x[i] == x[i]) || x[i] > 3.0e38f || x[i] < -3.0e38f) return false;
    return true;
}

}  // namespace

extern "C" {

void mppi_server_config_default(mppi_server_config* c) {
    if (!c) return;
    std::memset(c, 0, sizeof(*c));
    c->hbm_budget_bytes = 0;
    c->max_inflight = 16;
    c->sdf_mode = MPPI_SDF_MLP_FP16;
    c->batching = 1;
    c->sdf_single_cta = 1;
}

int mppi_server_create(const mppi_server_config* cfg, mppi_server** out) {
    if (!out || !cfg) return sfail(nullptr, MPPI_E_INVALID, "NULL argument");
    *out = nullptr;
    if (cfg->max_inflight < 1 || cfg->max_inflight > 1024)
        return sfail(nullptr, MPPI_E_INVALID, "max_inflight=%d out of [1, 1024]", cfg->max_inflight);
    if (cfg->sdf_mode < MPPI_SDF_ANALYTIC || cfg->sdf_mode > MPPI_SDF_MLP_FP8)
        return sfail(nullptr, MPPI_E_INVALID, "sdf_mode=%d", cfg->sdf_mode);
    if (cfg->sdf_single_cta != 0 && cfg->sdf_single_cta != 1)
        return sfail(nullptr, MPPI_E_INVALID, "sdf_single_cta=%d", cfg->sdf_single_cta);
    mppi_server* s = new (std::nothrow) mppi_server();
    if (!s) return sfail(nullptr, MPPI_E_OOM, "host allocation failed");
    s->cfg = *cfg;
    if (cudaGetDevice(&s->device) != cudaSuccess) {
        delete s;
        return sfail(nullptr, MPPI_E_UNSUPPORTED, "no CUDA device");
    }
    if (cfg->batching) {
        // kBatchBufs batch buffers of max_inflight slots and inputs each, each with its stream and
        // its batch's error word
        s->slots_bytes = (static_cast<size_t>(cfg->max_inflight) * sizeof(mppi::BatchSlot) + 255) & ~size_t(255);
        const size_t bytes = s->slots_bytes + static_cast<size_t>(cfg->max_inflight) * kBatchInFloats * sizeof(float);
        bool ok = true;
        for (BatchBuf& b : s->buf) {
            ok = ok && cudaStreamCreateWithFlags(&b.stream, cudaStreamNonBlocking) == cudaSuccess &&
                 cudaMallocHost(&b.h, bytes) == cudaSuccess && cudaMalloc(&b.d, bytes) == cudaSuccess &&
                 cudaHostAlloc(&b.h_err, sizeof(int), cudaHostAllocMapped) == cudaSuccess &&
                 cudaHostGetDevicePointer(reinterpret_cast<void**>(&b.d_err), b.h_err, 0) == cudaSuccess &&
                 cudaEventCreateWithFlags(&b.done, cudaEventDisableTiming) == cudaSuccess;
            if (ok) *b.h_err = 0;
        }
        if (!ok) {
            cudaGetLastError();
            mppi_server_destroy(s);
            return sfail(nullptr, MPPI_E_OOM, "batch buffers could not be allocated");
        }
        s->worker = std::thread(batched_worker_loop, s);
    } else {
        s->worker = std::thread(worker_loop, s);
    }
    *out = s;
    return MPPI_OK;
}

void mppi_server_destroy(mppi_server* s) {
    if (!s) return;
    {
        std::lock_guard<std::mutex> lock(s->mu);
        s->stop = true;
    }
    if (s->worker.joinable()) s->worker.join();
    for (BatchBuf& b : s->buf)
        if (b.stream) cudaStreamSynchronize(b.stream);
    for (auto& kv : s->drones)
        if (kv.second.ctx) mppi_destroy(kv.second.ctx);
    for (BatchBuf& b : s->buf) {
        if (b.h) cudaFreeHost(b.h);
        if (b.d) cudaFree(b.d);
        if (b.h_err) cudaFreeHost(b.h_err);
        if (b.done) cudaEventDestroy(b.done);
        if (b.stream) cudaStreamDestroy(b.stream);
    }
    delete s;
}

const char* mppi_server_last_error(const mppi_server* s) { return s ? s->err : g_server_err; }

int mppi_server_set_sdf_weights(mppi_server* s, const float* const* layers, int n_layers, const float* fp8_scales) {
    if (!s) return sfail(nullptr, MPPI_E_INVALID, "server is NULL");
    if (!layers || n_layers != 2 * MPPI_MLP_LAYERS) return sfail(s, MPPI_E_INVALID, "expected 10 layer pointers");
    const size_t sizes[10] = {MPPI_HIDDEN * (3 + MPPI_LATENT_DIM), MPPI_HIDDEN, MPPI_HIDDEN * MPPI_HIDDEN, MPPI_HIDDEN,
                              MPPI_HIDDEN * MPPI_HIDDEN, MPPI_HIDDEN, MPPI_HIDDEN * MPPI_HIDDEN, MPPI_HIDDEN,
                              MPPI_HIDDEN, 1};
    std::lock_guard<std::mutex> lock(s->mu);
    if (!s->drones.empty()) return sfail(s, MPPI_E_INVALID, "set the weights before the first request");
    s->layers.clear();
    for (int i = 0; i < n_layers; ++i) {
        if (!layers[i] || !finite(layers[i], sizes[i])) return sfail(s, MPPI_E_INVALID, "layer array %d", i);
        s->layers.emplace_back(layers[i], layers[i] + sizes[i]);
    }
    s->fp8.clear();
    if (fp8_scales) s->fp8.assign(fp8_scales, fp8_scales + 3);
    s->have_weights = true;
    return MPPI_OK;
}

int mppi_server_submit(mppi_server* s, int drone_id, const mppi_config* cfg, const float* state, int n_gates,
                       const float* poses, const float* latents, uint64_t* ticket) {
    if (!s || !cfg || !state || !ticket) return sfail(s, MPPI_E_INVALID, "NULL argument");
    if (n_gates < 0 || n_gates > cfg->max_gates) return sfail(s, MPPI_E_INVALID, "n_gates=%d", n_gates);
    if (n_gates > 0 && !poses) return sfail(s, MPPI_E_INVALID, "poses is NULL");
    if (s->cfg.sdf_mode != MPPI_SDF_ANALYTIC && n_gates > 0 && !latents)
        return sfail(s, MPPI_E_INVALID, "latents are required by the MLP SDF");
    if (!finite(state, mppi_state_dim(cfg))) return sfail(s, MPPI_E_INVALID, "non-finite state");
    Request r;
    r.drone = drone_id;
    std::memcpy(r.state, state, sizeof(float) * mppi_state_dim(cfg));
    r.n_gates = n_gates;
    if (n_gates > 0) r.poses.assign(poses, poses + 7 * n_gates);
    if (n_gates > 0 && latents) r.latents.assign(latents, latents + MPPI_LATENT_DIM * n_gates);
    r.t_submit = Clock::now();
    std::lock_guard<std::mutex> lock(s->mu);
    if (s->cfg.sdf_mode != MPPI_SDF_ANALYTIC && !s->have_weights)
        return sfail(s, MPPI_E_NOT_READY, "no SDF weights set");
    if (s->cfg.batching) {
        // one batched SDF launch serves every drone: they share the softplus sharpness and encoding levels
        if (s->pe_levels < 0) {
            s->beta = cfg->softplus_beta;
            s->pe_levels = cfg->pe_levels;
        } else if (cfg->softplus_beta != s->beta || cfg->pe_levels != s->pe_levels) {
            return sfail(s, MPPI_E_INVALID, "drone %d: softplus_beta and pe_levels must match the server's drones",
                         drone_id);
        }
    }
    auto it = s->drones.find(drone_id);
    if (it == s->drones.end()) {
        Drone d;
        d.cfg = *cfg;
        d.cfg.sdf_mode = s->cfg.sdf_mode;
        s->drones.emplace(drone_id, d);
    } else {
        const mppi_config& c0 = it->second.cfg;
        if (c0.K != cfg->K || c0.H != cfg->H || c0.max_gates != cfg->max_gates)
            return sfail(s, MPPI_E_INVALID, "drone %d: K, H or max_gates differ from its first request", drone_id);
    }
    r.ticket = s->next_ticket++;
    *ticket = r.ticket;
    s->queue.push_back(std::move(r));
    return MPPI_OK;
}

int mppi_server_poll(mppi_server* s, uint64_t ticket, float* new_controls, double* latency_us) {
    if (!s) return sfail(nullptr, MPPI_E_INVALID, "server is NULL");
    std::lock_guard<std::mutex> lock(s->mu);
    auto it = s->results.find(ticket);
    if (it == s->results.end()) {
        if (ticket == 0 || ticket >= s->next_ticket) return sfail(s, MPPI_E_INVALID, "unknown ticket %llu",
                                                                  static_cast<unsigned long long>(ticket));
        return MPPI_PENDING;
    }
    const int status = it->second.status;
    if (status == MPPI_OK && new_controls)
        std::memcpy(new_controls, it->second.controls.data(), it->second.controls.size() * sizeof(float));
    if (latency_us) *latency_us = it->second.latency_us;
    s->results.erase(it);
    return status;
}

int mppi_server_next_result(mppi_server* s, uint64_t* ticket, float* new_controls, size_t cap_floats,
                            double* latency_us) {
    if (!s || !ticket) return sfail(s, MPPI_E_INVALID, "NULL argument");
    std::lock_guard<std::mutex> lock(s->mu);
    if (s->results.empty()) return MPPI_PENDING;
    auto it = s->results.begin();
    *ticket = it->first;
    const int status = it->second.status;
    if (status == MPPI_OK && new_controls) {
        if (it->second.controls.size() > cap_floats)
            return sfail(s, MPPI_E_INVALID, "new_controls holds %zu floats, the result has %zu", cap_floats,
                         it->second.controls.size());
        std::memcpy(new_controls, it->second.controls.data(), it->second.controls.size() * sizeof(float));
    }
    if (latency_us) *latency_us = it->second.latency_us;
    s->results.erase(it);
    return status;
}

int mppi_server_get_stats(mppi_server* s, mppi_server_stats* out) {
    if (!s || !out) return sfail(s, MPPI_E_INVALID, "NULL argument");
    std::lock_guard<std::mutex> lock(s->mu);
    out->submitted = s->next_ticket - 1;
    out->completed = s->completed;
    out->queued = s->queue.size();
    size_t batched = 0;
    for (int i : s->order) batched += s->buf[i].reqs.size();
    out->inflight = s->inflight.size() + batched;
    out->evictions = s->evictions;
    out->restores = s->restores;
    out->device_bytes = s->used_bytes;
    out->peak_device_bytes = s->peak_bytes;
    out->batches = s->batches;
    return MPPI_OK;
}

}  // extern "C"
