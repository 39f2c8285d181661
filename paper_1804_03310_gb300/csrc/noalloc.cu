// Comb population control that allocates no device memory.
//
// Some callers cannot call cudaMalloc: applications whose device memory is
// all owned by another memory manager (a framework's caching allocator or a
// pool reserved at start-up), and real-time or certified hosts that forbid
// device allocation after initialisation. afqmc_comb_static gives them the
// comb with its prefix-sum scratch in a fixed-size file-scope device array
// instead of memory from a context; they pass only their own input and
// output buffers.
//
// In host code the array's name below is only a host-side stand-in; its
// device address is obtained once per device with cudaGetSymbolAddress (with
// that device current) and passed to the kernel.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "../../include/afqmc.h"
#include "kernels.h"

namespace afqmc {
void set_global_error(const std::string& msg);
}

namespace {

// Prefix sums of up to AFQMC_COMB_STATIC_MAX_WALKERS weights, plus one slot
// whose first four bytes hold the kernel's status word. Every GPU that loads
// the library keeps this array (512 KB + 8 bytes) until the process exits.
static __device__ __align__(256) double g_comb_scratch[AFQMC_COMB_STATIC_MAX_WALKERS + 1];

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
double* g_scratch_ptr[kMaxDevices] = {nullptr};

// Device address of g_comb_scratch on the current device, looked up on the
// first call for that device.
cudaError_t scratch_for_current_device(double** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_mutex);
  if (!g_scratch_ptr[dev]) {
    double* p = nullptr;
    e = cudaGetSymbolAddress((void**)&p, g_comb_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_ptr[dev] = p;
  }
  *out = g_scratch_ptr[dev];
  return cudaSuccess;
}

afqmc_status fail(afqmc_status s, const std::string& msg) {
  afqmc::set_global_error(msg);
  return s;
}

}  // namespace

extern "C" afqmc_status afqmc_comb_static(const double* d_weight, int32_t n_walkers,
                                          uint64_t seed, int32_t run_id, int64_t step,
                                          int32_t* d_parent, double* d_wnew,
                                          void* stream) {
  if (!d_weight || !d_parent || !d_wnew)
    return fail(AFQMC_E_INVALID, "afqmc_comb_static: null device pointer");
  if (n_walkers < 1 || n_walkers > AFQMC_COMB_STATIC_MAX_WALKERS)
    return fail(AFQMC_E_INVALID,
                "afqmc_comb_static: n_walkers must be in 1.." +
                    std::to_string(AFQMC_COMB_STATIC_MAX_WALKERS));
  if (run_id < 0 || run_id >= (1 << 29))
    return fail(AFQMC_E_INVALID, "afqmc_comb_static: run_id out of range");
  double* scratch = nullptr;
  cudaError_t e = scratch_for_current_device(&scratch);
  if (e != cudaSuccess)
    return fail(AFQMC_E_CUDA, std::string("afqmc_comb_static: scratch lookup: ") +
                                  cudaGetErrorString(e));
  cudaStream_t st = (cudaStream_t)stream;
  int* status = reinterpret_cast<int*>(scratch + AFQMC_COMB_STATIC_MAX_WALKERS);
  // The array keeps the previous call's contents: the status word must start
  // at zero (the prefix sums are fully rewritten by the kernel).
  e = cudaMemsetAsync(status, 0, sizeof(int), st);
  if (e == cudaSuccess)
    e = afqmc::launch_comb(st, n_walkers, d_weight, seed, run_id, nullptr, (long)step,
                           d_parent, scratch, d_wnew, status);
  if (e != cudaSuccess)
    return fail(AFQMC_E_CUDA, std::string("afqmc_comb_static: ") + cudaGetErrorString(e));
  return AFQMC_OK;
}
