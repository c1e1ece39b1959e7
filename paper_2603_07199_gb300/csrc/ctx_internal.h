// Hooks of a controller context used by the serving engine (internal).
#pragma once

#include <cstddef>
#include <cstdint>

#include "mppi.h"

namespace mppi {

// Enqueue one step from host inputs on the context's stream without waiting:
// state (13), n_gates gates (poses n x 7, latents n x 64 or NULL in analytic
// mode).  The outputs land in the context's pinned staging; completion is
// recorded on an event.  One request per context may be in flight.
int ctx_enqueue_host_step(mppi_ctx* c, const float* state, int n_gates, const float* poses, const float* latents);
// 1 while the last enqueued step runs; MPPI_OK once done (new_controls H x 4 filled); or an error.
int ctx_poll_host_step(mppi_ctx* c, float* new_controls);
// Save / restore the device-resident warm start, true state and step counter (synchronous).
int ctx_save(mppi_ctx* c, float* nominal, float* state, uint64_t* step);
int ctx_restore(mppi_ctx* c, const float* nominal, const float* state, uint64_t step);
// Device bytes a context of this configuration allocates.
size_t ctx_device_bytes(const mppi_config& cfg);

// ---- batched serving steps (the server's own stream launches the step kernels of many contexts)
struct BatchSlot;
struct MlpWeights;
struct StepParams;
// Prepare the context's next step for a batch: checks the inputs like ctx_enqueue_host_step, fills
// the slot's parameters, buffers and pointers (outputs into the context's pinned staging) and packs
// state, gate poses and latents into `in` from in[0] on.  Returns the floats written (> 0) or an error.
int ctx_batch_slot(mppi_ctx* c, const float* state, int n_gates, const float* poses, const float* latents,
                   BatchSlot* slot, float* in);
// The step of the last batch slot of this context has been launched.
void ctx_batch_launched(mppi_ctx* c);
// After the batch completed: MPPI_OK with new_controls (H x 4) filled, or the step's error.
int ctx_batch_result(mppi_ctx* c, float* new_controls);
// Clear the context's device error word and barrier counter (after a timed-out batch).  Synchronous.
int ctx_clear_error(mppi_ctx* c);
// The context's SDF weights, parameters and device SM count (for the batched launches).
MlpWeights ctx_weights(const mppi_ctx* c);
StepParams ctx_params(const mppi_ctx* c);
int ctx_num_sms(const mppi_ctx* c);

}  // namespace mppi
