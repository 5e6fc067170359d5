// lise_internal.h -- library-internal entry points shared by the sources of
// liblise.so (not part of the C ABI in include/lise.h).
#pragma once
#include "../../include/lise.h"

// lise_set_state without waiting for the device: enqueues the host-to-device
// copy, the finiteness check of the input and the series-expansion start on the
// context's stream and returns.  A non-finite input sets the context's error
// word, reported as LISE_ENONFINITE by the next synchronising call (lise_sync,
// lise_get_state, ...).  psi must stay valid until the stream has consumed it.
extern "C" int lise_set_state_enqueue(lise_ctx* c, const double* psi, double t0, double dt);

namespace lise {
// Validation of lise_params shared by lise_create and lise_rhs_noalloc: LISE_OK or LISE_EINVAL
// (lattice, spacing, state count, precision, finiteness of every physical parameter, the
// pairing options).
int check_params(const lise_params* p);
// The pairing coupling's kernel arguments (lise_kernels.cuh) for valid parameters.
struct Pairing;
Pairing make_pairing(const lise_params* p);
}  // namespace lise

// The stream a batch (lise_batch_*) enqueues its work on.
extern "C" void* lise_batch_stream(lise_batch* b);
