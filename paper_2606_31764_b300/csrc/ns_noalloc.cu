// splat_forward_noalloc: the forward splat with its scratch memory in a
// fixed device array of this library instead of a caller-provided workspace.
//
// Some callers cannot call cudaMalloc (or any allocator) at the point where
// they render: a host application that owns and pre-plans all device memory
// (a game engine, an inference server with a fixed memory budget), a plugin
// that may only touch the buffers it was handed, or a render loop that must
// never trigger the device-wide synchronisation an allocation can cause.  For
// them this entry point takes only the inputs and the output image; the
// scratch it needs (tile pairs, sort buffers, tile ranges, per-pixel state,
// counters) lives in `g_noalloc_scratch` below.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "ns_internal.cuh"

namespace ns {

// 16 MiB of scratch, allocated with the module: every GPU that loads this
// library holds it until the process exits.
constexpr size_t kNoAllocBytes = size_t(16) << 20;
constexpr int64_t kNoAllocMaxGaussians = 1 << 16;
constexpr int64_t kNoAllocMaxPairs = 1 << 18;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

// Device address of the scratch array.  In host code the name
// g_noalloc_scratch is only a host-side stand-in, not a device address, so it
// is never passed to a kernel directly.  The address is looked up on every
// call that is not being captured into a CUDA graph (so a device reset or a
// new context on the same ordinal is picked up); a call made while its stream
// is capturing reuses the address the last uncaptured call on that device
// found, since the lookup may not be legal during capture.
static std::mutex g_noalloc_mutex;
static void* g_noalloc_ptr[64] = {nullptr};

static void* noalloc_scratch(int dev, bool capturing) {
  if (dev < 0 || dev >= 64) return nullptr;
  std::lock_guard<std::mutex> lock(g_noalloc_mutex);
  if (!capturing) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess) {
      cudaGetLastError();
      g_noalloc_ptr[dev] = nullptr;
      return nullptr;
    }
    g_noalloc_ptr[dev] = p;
  }
  return g_noalloc_ptr[dev];
}

}  // namespace ns

using namespace ns;

extern "C" ns_status splat_forward_noalloc(const ns_curves* curves, const ns_gaussians* g,
                                           const ns_raster_params* rp, float* image, ns_report* report,
                                           void* stream) {
  if (!curves || !g || !rp || !image) {
    set_error("splat_forward_noalloc: null argument");
    return NS_ERR_INVALID_ARG;
  }
  if (g->capacity < 0 || g->capacity > kNoAllocMaxGaussians) {
    set_error("splat_forward_noalloc: the Gaussian set's capacity exceeds the fixed scratch limit of 65536");
    return NS_ERR_INVALID_ARG;
  }
  // no sampling plans live in the scratch: bin one pair per Gaussian and tile
  ns_raster_params rpn = *rp;
  rpn.fill_layers = 0;
  rp = &rpn;
  ns_capacity cap;
  cap.gaussians = g->capacity;
  cap.pairs = kNoAllocMaxPairs;
  cap.boundary = 0;
  const size_t need = ns_workspace_size(curves, &cap, rp);
  if (need == 0) return NS_ERR_INVALID_ARG;   // message set by the layout check
  if (need > kNoAllocBytes) {
    set_error("splat_forward_noalloc: this batch needs " + std::to_string(need) +
              " bytes of scratch; the fixed scratch holds " + std::to_string(kNoAllocBytes) +
              " (fewer pixels, curves or Gaussians are needed)");
    return NS_ERR_INVALID_ARG;
  }
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    set_error("splat_forward_noalloc: no current device");
    return NS_ERR_CUDA;
  }
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(static_cast<cudaStream_t>(stream), &cs) != cudaSuccess) {
    cudaGetLastError();
    set_error("splat_forward_noalloc: invalid stream");
    return NS_ERR_CUDA;
  }
  void* ws = noalloc_scratch(dev, cs != cudaStreamCaptureStatusNone);
  if (!ws) {
    set_error(cs != cudaStreamCaptureStatusNone
                  ? "splat_forward_noalloc: the first call on a device must come before any stream capture"
                  : "splat_forward_noalloc: cudaGetSymbolAddress of the scratch array failed");
    return NS_ERR_CUDA;
  }
  // The scratch keeps the previous call's contents: start from a clear status.
  ns_status st = ns_clear_status(ws, stream);
  if (st != NS_OK) return st;
  st = splat_forward(curves, g, rp, &cap, image, ws, kNoAllocBytes, stream);
  if (st != NS_OK || !report) return st;
  st = ns_poll_status(ws, report, stream);
  if (st != NS_OK) return st;
  // the status word was cleared above, and with it the sampling counters:
  // report the Gaussians the set holds (its count) instead
  int count = 0;
  if (cudaMemcpy(&count, g->count, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) {
    set_error(std::string("splat_forward_noalloc: ") + cudaGetErrorString(cudaGetLastError()));
    return NS_ERR_CUDA;
  }
  report->gaussians = count;
  return NS_OK;
}
