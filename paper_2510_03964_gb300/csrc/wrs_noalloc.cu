// wrs_push_frame_host without caller-allocated staging: the device copies of
// the host frame, fov map and resolved output live in one file-scope device
// array of fixed size, so a caller that cannot allocate device memory can
// still push host frames (its reservoir state buffer is still its own).
#include <cuda_runtime.h>

#include "wrs_internal.h"

namespace {

constexpr size_t kFrameBytes = static_cast<size_t>(WRS_NOALLOC_MAX_PIXELS) * 3 * sizeof(float);
constexpr size_t kFovBytes = (static_cast<size_t>(WRS_NOALLOC_MAX_PIXELS) + 255) / 256 * 256;
constexpr size_t kStageBytes = 2 * kFrameBytes + kFovBytes;  // frame, output, fov map

// frame copy at 0, output at kFrameBytes, fov map at 2 * kFrameBytes
static __device__ __align__(256) uint8_t g_stage[kStageBytes];

}  // namespace

extern "C" int wrs_push_frame_host_noalloc(wrs_ctx* x, const float* h_frame, float gx, float gy,
                                           const uint8_t* h_fov, float* h_out,
                                           wrs_stream_t stream) {
  wrs_clear_error();
  if (!x) return wrs_fail(WRS_ERR_ARG, "context is NULL");
  if (!h_frame || !h_out) return wrs_fail(WRS_ERR_ARG, "h_frame and h_out must be non-NULL");
  const size_t hw = static_cast<size_t>(x->cfg.width) * x->cfg.height;
  if (hw > static_cast<size_t>(WRS_NOALLOC_MAX_PIXELS))
    return wrs_fail(WRS_ERR_ARG, "%zu pixels exceed the static staging of %d pixels", hw,
                    WRS_NOALLOC_MAX_PIXELS);
  int cur = -1;
  cudaError_t e = cudaGetDevice(&cur);
  if (e != cudaSuccess) return wrs_cuda_fail(e, "wrs_push_frame_host_noalloc: device query");
  if (cur != x->device)
    return wrs_fail(WRS_ERR_ARG, "the stream's device (%d) must be current (is %d)", x->device, cur);
  // the array's address on the current device (each device has its own copy)
  void* base = nullptr;
  e = cudaGetSymbolAddress(&base, g_stage);
  if (e != cudaSuccess) return wrs_cuda_fail(e, "wrs_push_frame_host_noalloc: staging address");
  uint8_t* b = static_cast<uint8_t*>(base);
  float* d_frame = reinterpret_cast<float*>(b);
  float* d_out = reinterpret_cast<float*>(b + kFrameBytes);
  uint8_t* d_fov = b + 2 * kFrameBytes;
  // nothing here must start at zero: every staged byte the update reads is
  // first written by this call
  return wrs_push_frame_host(x, h_frame, gx, gy, h_fov, h_out, d_frame, h_fov ? d_fov : nullptr,
                             d_out, stream);
}
