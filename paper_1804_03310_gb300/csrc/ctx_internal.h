// Hooks into a context for the library's own serving loop (not exported).
#pragma once

#include <cuda_runtime.h>

#include <string>

#include "../../include/afqmc.h"

namespace afqmc {

// Enqueue on the context's stream copies of the latest measurement (mixed
// energy, weight sum: two doubles) and of the status word into host memory
// (page-locked, so that the copies stay asynchronous).
cudaError_t ctx_enqueue_readback(afqmc_ctx* c, double* e2, int* status);

// Host step counter (steps issued so far).
long ctx_step(const afqmc_ctx* c);

// Error text for calls without a context (afqmc_last_error(NULL)).
void set_global_error(const std::string& msg);

}  // namespace afqmc
