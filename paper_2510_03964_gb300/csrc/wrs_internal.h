// Library-internal declarations shared by the translation units of libwrs.
#pragma once

#include <cuda_runtime.h>

#include "wrs.h"
#include "wrs_device.cuh"
#include "wrs_fov.cuh"

struct wrs_ctx {
  wrs_config cfg;
  wrs_layout lay;
  uint8_t* state;        // caller-owned device buffer: header (status, counters) + planes
  uint8_t* planes;       // buffer whose planes hold the current reservoirs: state or spare
  uint8_t* spare;        // caller-owned second buffer for reprojection (null until set)
  uint32_t t;            // frames pushed
  int block;             // threads per block of the plain kernel
  int px;                // requested pixels per thread of the plain kernel
  int device;            // CUDA device the state lives on
  int sms;               // its multiprocessor count
  int pipe;              // 1: use the pipelined kernel when the frame allows it
  int pipe_px;           // pipelined kernel: pixels per thread (tile = 256 * px)
  int pipe_stages;       // pipelined kernel: shared-memory stages
  int pipe_ctas;         // pipelined kernel: CTAs per SM (0: as many as fit)
  uint64_t timeout_ns;   // bound on every device-side wait
  uint32_t test_extra_tx;  // > 0 only to exercise the timeout path in tests
  int failed;             // 1 once wrs_check_status saw a wait give up: the reservoirs are
                          // undefined until wrs_import_state restores a saved state
  uint32_t base;          // the idx planes hold every sample index of frames < base; later
                          // ones are codes in the ring until a push or a fold applies them
};

constexpr int kDefaultBlock = 256;
constexpr int kDefaultPx = 4;
constexpr uint64_t kDefaultTimeoutNs = 2000000000ull;  // 2 s
constexpr size_t kSmemBudget = 227 * 1024 - 1024;       // dynamic shared memory per CTA we use

uint32_t* wrs_status_word(const wrs_ctx* x);
size_t wrs_pipe_smem_bytes(int K, bool f16, int px, int stages, bool resolve);
bool wrs_pipe_supported(const wrs_ctx* x, const float* frame, int64_t pitch, const float* out);
cudaError_t wrs_launch_pipe(const wrs::StreamDev& s, const wrs::FrameDev& f, bool f16, int px,
                            int stages, int sms, int ctas_per_sm, uint32_t* status,
                            uint64_t timeout_ns, uint32_t extra_tx, cudaStream_t st);
void wrs_default_pipe(int K, bool f16, int* px, int* stages);

void wrs_clear_error();
// WRS_OK, or WRS_ERR_STATE (with the message set) if the context's reservoirs are undefined.
int wrs_require_usable(const wrs_ctx* x);
int wrs_fail(int code, const char* fmt, ...);
int wrs_cuda_fail(cudaError_t e, const char* what);
int wrs_check_config(const wrs_config* c);
void wrs_make_layout(const wrs_config* c, wrs_layout* L);
float wrs_delta(const wrs_config* c);
wrs::StreamDev wrs_stream_dev(const wrs_ctx* x);
cudaError_t wrs_init_planes(const wrs_ctx* x, uint8_t* base, cudaStream_t st);
// First frame whose ring codes the band folded by the next push still applies.
uint32_t wrs_map_lo(const wrs_ctx* x);
// Folds every pending ring code into the current idx planes (a kernel on st);
// afterwards base = t.
cudaError_t wrs_fold_all(wrs_ctx* x, cudaStream_t st);
int wrs_effective_px(const wrs_ctx* x, const float* frame, int64_t pitch, const float* out);
// Validates a foveation source (image, mip buffer, radii, filter) and fills fv.
int wrs_fov_check_source(const float* d_img, int64_t pitch, const void* d_mip, size_t mip_bytes,
                   int32_t width, int32_t height, int32_t nradii, const float* radii,
                   int32_t filter, wrs::FovDev* fv);
// The pipelined kernel foveating the frame as it reads it (filter: WRS_FILTER_*).
cudaError_t wrs_launch_pipe_fov(const wrs::StreamDev& s, const wrs::FrameDev& f,
                                const wrs::FovDev& fv, int filter, bool f16, int stages, int sms,
                                int ctas_per_sm, uint32_t* status, uint64_t timeout_ns,
                                cudaStream_t st);
cudaError_t wrs_launch_push(const wrs::StreamDev& s, const wrs::FrameDev& f, int block, int px,
                            bool f16, cudaStream_t st);
