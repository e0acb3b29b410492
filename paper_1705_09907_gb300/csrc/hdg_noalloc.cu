// Allocation-free variant of the condensed right-hand side.
//
// hdg_condense_rhs keeps its per-element partial results in a buffer the
// context allocated at set-up. Some callers cannot allocate device memory at
// the point where they need the right-hand side -- code that runs where a
// device allocation would synchronise the device or is simply forbidden, such
// as a solver step driven from inside another framework's memory-managed
// region or a real-time loop that owns all of its memory up front. For them,
// hdg_condense_rhs_noalloc does the same computation with its scratch in a
// fixed array that is part of the library image: every GPU that loads the
// library holds kNoAllocScratch doubles (4 MiB) until the process exits.
#include <mutex>

#include "hdg_internal.h"

namespace hdg {
cudaError_t launch_condense_into(Context* c, const double* f_q, double* b, int nrhs, double* scratch,
                                 cudaStream_t s);
}  // namespace hdg

using namespace hdg;

namespace {

constexpr size_t kNoAllocScratch = size_t(1) << 19;          // doubles (4 MiB)
constexpr int kMaxDevices = 64;

// File-scope scratch: per-element partial results [nel][4(k+1)].
static __device__ __align__(256) double g_condense_scratch[kNoAllocScratch];

std::mutex g_mu;
double* g_scratch_ptr[kMaxDevices] = {};                    // device address per device

// Device address of the scratch array on device `dev`, which must be the
// current device. The first lookup on a device asks the runtime for it (the
// array's name is only a host-side stand-in in host code; the lookup also loads
// the part of the library image that holds the array); later calls reuse the
// cached address.
cudaError_t scratch_for_device(int dev, double** out) {
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  cudaError_t e;
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_condense_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_ptr[dev] = static_cast<double*>(p);
  }
  *out = g_scratch_ptr[dev];
  return cudaSuccess;
}

}  // namespace

namespace hdg {
// Called by hdg_setup with the context's device current: looks the scratch
// address up while the caller is still setting up, so the entry point's own
// calls on that device find it cached.
cudaError_t noalloc_prepare_device(int dev) {
  double* p = nullptr;
  return scratch_for_device(dev, &p);
}
}  // namespace hdg

extern "C" int hdg_condense_rhs_noalloc(void* ctx, const double* f_q, double* b, int nrhs, void* stream) {
  Context* c = (Context*)ctx;
  if (!c || !f_q || !b || nrhs < 1) return HDG_ERR_INVALID_ARG;
  if ((size_t)c->nel * (size_t)c->ref.m > kNoAllocScratch) return HDG_ERR_INVALID_ARG;
  // the scratch is per device: use it only on the context's own device
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) return HDG_ERR_CUDA;
  if (dev != c->dev) return HDG_ERR_INVALID_ARG;
  double* scratch = nullptr;
  cudaError_t e = scratch_for_device(dev, &scratch);
  if (e != cudaSuccess) return HDG_ERR_CUDA;
  e = launch_condense_into(c, f_q, b, nrhs, scratch, (cudaStream_t)stream);
  return e == cudaSuccess ? HDG_OK : HDG_ERR_CUDA;
}
