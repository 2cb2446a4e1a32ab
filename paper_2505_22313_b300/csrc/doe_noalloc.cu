// doe_noalloc.cu -- doe_psf_noalloc: the PSF entry point for callers that cannot allocate.
//
// doe_psf needs a caller-provided device workspace.  Some callers cannot obtain one: a plugin
// running inside a host application that owns the whole device-memory budget and hands out
// only input and output buffers, a latency-critical loop that must never call cudaMalloc
// (an allocation can block on the device or fail under memory pressure), or an embedding
// that links only this library and has no allocator of its own.  For them this file keeps
// the scratch in a file-scope static device array instead.  Every GPU that loads the library
// holds the array (DOE_NOALLOC_SCRATCH_BYTES) until the process exits.
#include <cuda.h>  // CUcontext / CUresult types only: the driver entry point is looked up at run time
#include <cuda_runtime.h>

#include <mutex>

#include "doe.h"

static __device__ __align__(256) unsigned char g_noalloc_scratch[DOE_NOALLOC_SCRATCH_BYTES];

namespace {
constexpr int kMaxDevices = 64;
std::mutex g_mu;
struct Cached {
  CUcontext ctx;
  void* ptr;
};
Cached g_scratch[kMaxDevices] = {};

// The calling thread's current context, through the driver entry point the runtime hands out
// (the library does not link against the driver library itself).
CUcontext current_context() {
  using Fn = CUresult (*)(CUcontext*);
  static const Fn fn = [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      return (Fn) nullptr;
    return reinterpret_cast<Fn>(p);
  }();
  CUcontext c = nullptr;
  if (!fn || fn(&c) != CUDA_SUCCESS) return nullptr;
  return c;
}

// Device address of the scratch array on the current device.  In host code the array's
// name only stands in for the symbol; the address is looked up with that device current, once
// per device and context: a device reset or a new primary context reloads the module, and the
// array may then sit elsewhere, so a changed context triggers a new lookup.
int scratch_for_current_device(void** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return DOE_ECUDA;
  std::lock_guard<std::mutex> lk(g_mu);
  const CUcontext ctx = current_context();  // null before the runtime has made one current
  if (!g_scratch[dev].ptr || !ctx || g_scratch[dev].ctx != ctx) {
    void* p = nullptr;  // the lookup also makes the device's primary context current
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return DOE_ECUDA;
    g_scratch[dev] = {current_context(), p};
  }
  *out = g_scratch[dev].ptr;
  return DOE_OK;
}
}  // namespace

extern "C" int doe_psf_noalloc(const doe_geom* g, const float* h, const float* e_in, float* psf, void* stream) {
  const size_t need = doe_workspace_bytes(g, DOE_OP_PSF);
  if (need == 0) return doe_psf(g, h, e_in, psf, nullptr, 0, stream);  // reports the validation error
  if (need > DOE_NOALLOC_SCRATCH_BYTES) return DOE_ESCRATCH;
  void* ws = nullptr;
  const int rc = scratch_for_current_device(&ws);
  if (rc != DOE_OK) return rc;
  // Every location the passes read is written earlier in the same call (the padding columns
  // of the field buffer are never read into a result), so the previous call's contents need
  // no clearing.
  return doe_psf(g, h, e_in, psf, ws, DOE_NOALLOC_SCRATCH_BYTES, stream);
}
