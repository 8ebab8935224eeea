// epic_image_host_static: the host-buffer imaging call for callers that must
// not allocate device memory.
//
// epic_image_host stages the voltages and the image in device buffers that
// the plan grows with cudaMalloc on demand.  Some callers cannot allow that:
// a real-time correlator loop that may not add a device-wide synchronising
// cudaMalloc between intervals, a process that runs inside a fixed device
// memory budget reserved up front, or host code that runs where CUDA
// allocation calls are not permitted.  This variant stages through one
// file-scope device array of fixed size instead, so the call itself
// allocates nothing (the plan's own tables were allocated when the plan was
// created).  The imaging kernel and its arithmetic are the ones epic_image
// uses.
#include "../../include/epic.h"

#include <cuda_runtime.h>

#include <cstdio>
#include <mutex>
#include <string>

#include "epic_internal.h"

namespace {

// Staging area: the [C][N][N] float64 image first (256-byte aligned), then as
// many whole time samples of voltages as fit.  Every GPU that loads the
// library holds these 32 MiB until the process exits.
constexpr size_t kStaticScratchBytes = static_cast<size_t>(32) << 20;
static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

// Device address of g_static_scratch per device.  The symbol's name is a
// host-side stand-in in host code, so the address is looked up once per
// device with that device current.  The cached address belongs to the
// device's current context: it does not survive cudaDeviceReset (the module
// is loaded again into the new context and the array may move), so a caller
// that resets a device must not call this entry point on it afterwards.
constexpr int kMaxDevices = 64;
void* g_scratch_addr[kMaxDevices] = {};
std::mutex g_scratch_mu;

int scratch_address(int dev, void** out) {
  if (dev < 0 || dev >= kMaxDevices)
    return epic::set_error(EPIC_ERR_UNSUPPORTED, "device index beyond the static scratch table");
  std::lock_guard<std::mutex> lk(g_scratch_mu);
  if (!g_scratch_addr[dev]) {
    void* ptr = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&ptr, g_static_scratch);
    if (e != cudaSuccess || !ptr) {
      const std::string msg = std::string("cudaGetSymbolAddress(static scratch): ") + cudaGetErrorString(e);
      return epic::set_error(EPIC_ERR_CUDA, msg.c_str());
    }
    g_scratch_addr[dev] = ptr;
  }
  *out = g_scratch_addr[dev];
  return EPIC_OK;
}

}  // namespace

extern "C" epic_status epic_image_host_static(epic_plan_t p, const void* h_volt, long long n_time,
                                              double* h_image, int accumulate) {
  if (!p) return static_cast<epic_status>(epic::set_error(EPIC_ERR_INVALID_ARG, "plan is NULL"));
  if (!h_volt || !h_image)
    return static_cast<epic_status>(epic::set_error(EPIC_ERR_INVALID_ARG, "NULL host buffer"));
  if (n_time < 1)
    return static_cast<epic_status>(epic::set_error(EPIC_ERR_INVALID_ARG, "n_time must be >= 1"));
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess)
    return static_cast<epic_status>(epic::set_error(EPIC_ERR_CUDA, cudaGetErrorString(e)));
  if (dev != epic::plan_device(p))
    return static_cast<epic_status>(
        epic::set_error(EPIC_ERR_INVALID_ARG, "current device is not the plan's device"));
  // only the fused FP32 kernel images from the array alone; every other path
  // needs plan scratch.  Refused before anything touches the array.
  if (epic::plan_path(p) != EPIC_PATH_FUSED)
    return static_cast<epic_status>(epic::set_error(
        EPIC_ERR_UNSUPPORTED, "epic_image_host_static needs a plan on the fused FP32 path (EPIC_PATH_FUSED)"));

  const size_t img_bytes = epic::plan_image_elems(p) * sizeof(double);
  const size_t img_span = (img_bytes + 255) & ~static_cast<size_t>(255);
  const size_t frame = epic::plan_frame_bytes(p);
  if (img_span + frame > kStaticScratchBytes) {
    char msg[200];
    std::snprintf(msg, sizeof msg,
                  "image (%zu B) plus one time sample of voltages (%zu B) exceed the %zu B static "
                  "scratch of epic_image_host_static; use epic_image_host",
                  img_bytes, frame, kStaticScratchBytes);
    return static_cast<epic_status>(epic::set_error(EPIC_ERR_INVALID_ARG, msg));
  }
  void* base = nullptr;
  if (int s = scratch_address(dev, &base)) return static_cast<epic_status>(s);

  double* d_img = static_cast<double*>(base);
  unsigned char* d_volt = static_cast<unsigned char*>(base) + img_span;
  const long long chunk = static_cast<long long>((kStaticScratchBytes - img_span) / frame);
  cudaStream_t st = epic::plan_stream(p);

  // the array keeps the previous call's contents: set the image first
  e = accumulate ? cudaMemcpyAsync(d_img, h_image, img_bytes, cudaMemcpyHostToDevice, st)
                 : cudaMemsetAsync(d_img, 0, img_bytes, st);
  if (e != cudaSuccess)
    return static_cast<epic_status>(epic::set_error(EPIC_ERR_CUDA, cudaGetErrorString(e)));
  const double scale = 1.0 / static_cast<double>(n_time);
  const unsigned char* hv = static_cast<const unsigned char*>(h_volt);
  for (long long t0 = 0; t0 < n_time; t0 += chunk) {
    const long long n = (n_time - t0 < chunk) ? n_time - t0 : chunk;
    e = cudaMemcpyAsync(d_volt, hv + static_cast<size_t>(t0) * frame, static_cast<size_t>(n) * frame,
                        cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess)
      return static_cast<epic_status>(epic::set_error(EPIC_ERR_CUDA, cudaGetErrorString(e)));
    if (int s = epic::image_batch_scaled(p, d_volt, n, d_img, scale)) return static_cast<epic_status>(s);
  }
  e = cudaMemcpyAsync(h_image, d_img, img_bytes, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess)
    return static_cast<epic_status>(epic::set_error(EPIC_ERR_CUDA, cudaGetErrorString(e)));
  return EPIC_OK;
}
