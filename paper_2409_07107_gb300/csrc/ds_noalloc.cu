// sim_step_jac_noalloc: sim_step_jac with its workspace in a fixed array that the library module
// carries, for callers that cannot allocate device memory at call time.
#include <mutex>

#include "ds_common.cuh"

// Scratch shared by every call on a device; it lives as long as the library is loaded.
static __device__ __align__(256) unsigned char g_noalloc_scratch[DS_NOALLOC_SCRATCH_BYTES];

static std::mutex g_scratch_mu;
static void* g_scratch_ptr[64];  // device address of g_noalloc_scratch, per device

// The host-side name g_noalloc_scratch is not a device address: resolve it once per device, with
// that device current.
static ds_status scratch_for_current_device(void** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return DS_ECUDA;
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return DS_ECUDA;
    g_scratch_ptr[dev] = p;
  }
  *out = g_scratch_ptr[dev];
  return DS_OK;
}

extern "C" ds_status sim_step_jac_noalloc(const ds_model* const* models, int32_t nmodels, const ds_batch* batch,
                                          const ds_options* opt, const ds_step_out* out, double* dv_dq,
                                          double* dv_dv, double* dv_dtau, void* stream) {
  if (!models || nmodels <= 0 || !batch || !opt || !out) return DS_EINVAL;
  size_t need = 0;
  ds_status s = ds_workspace_size(models, nmodels, batch, opt, &need);
  if (s != DS_OK) return s;
  if (need > DS_NOALLOC_SCRATCH_BYTES) return DS_ETOOLARGE;
  void* ws = nullptr;
  s = scratch_for_current_device(&ws);
  if (s != DS_OK) return s;
  ds_allow_helper_streams(false);   // no stream or event creation on this path
  s = sim_step_jac(models, nmodels, batch, opt, out, dv_dq, dv_dv, dv_dtau, ws, DS_NOALLOC_SCRATCH_BYTES, stream);
  ds_allow_helper_streams(true);
  return s;
}
