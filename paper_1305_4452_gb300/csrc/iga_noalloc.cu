// iga_form_residual_noalloc: residual assembly that allocates no device memory.
//
// Some callers cannot call cudaMalloc at the moment they need a residual: code
// running under a memory budget fixed by another allocator that owns the device
// (a framework's caching pool, an embedded solver inside a larger application),
// real-time loops where an allocation's latency or possible failure is not
// acceptable, or callers that must not add any allocation of their own.
// iga_form_residual uses an element-vector buffer that iga_create allocated; this
// variant runs the same kernels with that buffer replaced by a fixed array in the
// library's own device memory, so the call itself never allocates.
//
// The array is a file-scope __device__ variable of IGA_NOALLOC_MAX_ELEMENT_VALUES
// doubles (16 MiB).  CUDA loads the code of this file, and reserves the array on a
// device, the first time its address is asked for on that device.  iga_create does
// that (noalloc_setup, with the handle's device current), so a device holds the
// array from its first handle's creation until the process exits, and the entry
// point itself neither loads code nor reserves memory.  Should that look-up have
// failed at creation, the first call on the handle repeats it (and may then be the
// one that reserves the array); make that call outside any stream capture.  All
// calls share the array, so calls that overlap on the GPU (different streams or
// different handles at the same time) race on it; the kernels overwrite every entry
// they later read, so no part of it has to start at zero and stale contents from an
// earlier call are never used.
#include <cuda_runtime.h>

#include <mutex>

#include "iga_internal.h"

static __device__ __align__(256) double g_residual_scratch[IGA_NOALLOC_MAX_ELEMENT_VALUES];

namespace {
constexpr int kMaxDevices = 64;
std::mutex g_mu;
double *g_addr[kMaxDevices] = {};

// Device address of the scratch array on the current device (looked up once per device).
// In host code g_residual_scratch names a host-side stand-in, not device memory: only
// the address returned by cudaGetSymbolAddress may be handed to a kernel.
cudaError_t scratch_address(double **out) {
  int dev = 0;
  cudaError_t ce = cudaGetDevice(&dev);
  if (ce != cudaSuccess) return ce;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_addr[dev]) {
    void *p = nullptr;
    ce = cudaGetSymbolAddress(&p, g_residual_scratch);
    if (ce != cudaSuccess) return ce;
    g_addr[dev] = (double *)p;
  }
  *out = g_addr[dev];
  return cudaSuccess;
}
}  // namespace

void noalloc_setup(iga_s *h) {
  double *p = nullptr;
  h->noalloc_scratch = (scratch_address(&p) == cudaSuccess) ? p : nullptr;
  cudaGetLastError();  // a failed look-up is retried by the first call; drop its error state here
}

extern "C" iga_status iga_form_residual_noalloc(iga_t h, const double *U, double *F) {
  if (!h) return IGA_EINVAL;
  if (!U || !F || U == F) {
    h->err = "U and F must be distinct non-NULL device pointers";
    return IGA_EINVAL;
  }
  if (h->inner) {
    h->err = "periodic handles have no allocation-free residual";
    return IGA_EINVAL;
  }
  int nen = (h->dim == 3) ? (h->p + 1) * (h->p + 1) * (h->p + 1) : (h->p + 1) * (h->p + 1);
  unsigned long long need = (unsigned long long)h->nelem * (unsigned long long)nen;
  if (need > (unsigned long long)IGA_NOALLOC_MAX_ELEMENT_VALUES) {
    h->err = iga_format("iga_form_residual_noalloc: %llu element values (elements x (p+1)^dim) exceed the fixed "
                        "scratch of %u; use iga_form_residual",
                        need, (unsigned)IGA_NOALLOC_MAX_ELEMENT_VALUES);
    return IGA_EINVAL;
  }
  int dev = -1;
  cudaError_t ce = cudaGetDevice(&dev);
  if (ce != cudaSuccess || dev != h->device) {
    h->err = iga_format("iga_form_residual_noalloc: current device %d is not the handle's device %d", dev, h->device);
    return IGA_EINVAL;
  }
  if (!h->noalloc_scratch) {
    double *p = nullptr;
    ce = scratch_address(&p);
    if (ce != cudaSuccess) {
      h->err = iga_format("iga_form_residual_noalloc: cudaGetSymbolAddress: %s", cudaGetErrorString(ce));
      return IGA_ECUDA;
    }
    h->noalloc_scratch = p;
  }
  ce = launch_residual_into(h, U, F, h->noalloc_scratch);
  if (ce != cudaSuccess) {
    h->err = iga_format("iga_form_residual_noalloc: %s", cudaGetErrorString(ce));
    return IGA_ECUDA;
  }
  return IGA_OK;
}
