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

}  // namespace mppi
