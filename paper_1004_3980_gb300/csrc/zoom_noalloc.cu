// Back-projection for callers that cannot allocate device memory.
//
// Some callers of this library cannot call cudaMalloc or any allocator:
// code running inside another framework's memory budget that forbids
// allocations after start-up, real-time pipelines whose memory is fixed in
// advance, or callers recording work where an allocation would break the
// recording.  zoom_backproject_noalloc runs the same back-projection
// kernels as zoom_backproject, but its scratch memory (the second HR image
// of the ping-pong and the LR error image) is a fixed-size array that lives
// in this library's own device memory for as long as the library is loaded.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "zoom_internal.h"

namespace {

// The scratch array; every GPU that loads the library holds it until exit.
static __device__ __align__(256) float g_noalloc_scratch[ZOOM_NOALLOC_SCRATCH_FLOATS];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mu;
float* g_scratch_addr[kMaxDevices] = {};

// Device address of the scratch array on `device` (made current).  Looked
// up once per device; the host-side name of the array is not a device
// address and is never handed to a kernel.
cudaError_t scratch_address(int device, float** out) {
  std::lock_guard<std::mutex> lock(g_setup_mu);
  if (!g_scratch_addr[device]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_addr[device] = (float*)p;
  }
  *out = g_scratch_addr[device];
  return cudaSuccess;
}

}  // namespace

extern "C" zoom_status zoom_backproject_noalloc(int device, const zoom_degradation* degr,
                                                const float* lr, int32_t h, int32_t w,
                                                const zoom_upscale_params* prm, float* hr,
                                                void* stream) {
  if (!degr || !lr || !prm || !hr) {
    zoom_set_error("NULL argument");
    return ZOOM_ERR_INVALID_ARG;
  }
  int n_dev = 0;
  const cudaError_t ec = cudaGetDeviceCount(&n_dev);
  if (ec != cudaSuccess) {   // no driver, or a sticky error of the runtime: not an argument error
    cudaGetLastError();
    zoom_set_error(std::string("cudaGetDeviceCount: ") + cudaGetErrorString(ec));
    return ZOOM_ERR_CUDA;
  }
  if (device < 0 || device >= n_dev || device >= kMaxDevices) {
    zoom_set_error("no such device");
    return ZOOM_ERR_INVALID_ARG;
  }
  const int s = degr->scale;
  if (s < 1 || s > 4 || !(degr->blur_sigma > 0.0) || h < 1 || w < 1) {
    zoom_set_error("bad degradation or image size");
    return ZOOM_ERR_INVALID_ARG;
  }
  if (prm->bp_iters < 0 || prm->bp_iters > 64 || prm->bp_radius < 1 || prm->bp_radius > 7 ||
      !(prm->sigma_spatial > 0.f) || !(prm->sigma_range > 0.f)) {
    zoom_set_error("bad back-projection parameters");
    return ZOOM_ERR_INVALID_ARG;
  }
  // scratch: the HR ping-pong image, then (256-byte aligned) the LR error
  const size_t hr_floats = (size_t)s * h * s * w;
  const size_t err_off = (hr_floats + 63) / 64 * 64;
  const size_t need = err_off + (size_t)h * w;
  if (need > (size_t)ZOOM_NOALLOC_SCRATCH_FLOATS) {
    zoom_set_error("image too large for the static scratch: needs " + std::to_string(need) +
                   " floats, the maximum is " + std::to_string((size_t)ZOOM_NOALLOC_SCRATCH_FLOATS));
    return ZOOM_ERR_INVALID_ARG;
  }
  cudaError_t e = cudaSetDevice(device);
  float* scratch = nullptr;
  if (e == cudaSuccess) e = scratch_address(device, &scratch);
  if (e != cudaSuccess) {
    zoom_set_error(std::string("scratch set-up: ") + cudaGetErrorString(e));
    return ZOOM_ERR_CUDA;
  }
  cudaStream_t st = (cudaStream_t)stream;
  float* tmp = scratch;
  float* err = scratch + err_off;
  // Both scratch images are fully written before they are read in every
  // iteration, so nothing left by an earlier call needs clearing.
  float* a = hr;
  float* b = tmp;
  for (int it = 0; it < prm->bp_iters; ++it) {
    e = launch_bp_iteration(a, b, lr, err, h, w, s, degr->blur_sigma, prm->sigma_spatial,
                            prm->sigma_range, prm->bp_radius, st);
    if (e != cudaSuccess) {
      zoom_set_error(std::string("backproject: ") + cudaGetErrorString(e));
      return ZOOM_ERR_CUDA;
    }
    float* t = a;
    a = b;
    b = t;
  }
  if (a != hr) {
    e = cudaMemcpyAsync(hr, a, hr_floats * sizeof(float), cudaMemcpyDeviceToDevice, st);
    if (e != cudaSuccess) {
      zoom_set_error(std::string("copy back: ") + cudaGetErrorString(e));
      return ZOOM_ERR_CUDA;
    }
  }
  return ZOOM_OK;
}
