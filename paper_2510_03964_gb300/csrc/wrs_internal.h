// Library-internal declarations shared by the translation units of libwrs.
#pragma once

#include <cuda_runtime.h>

#include "wrs.h"
#include "wrs_device.cuh"

struct wrs_ctx {
  wrs_config cfg;
  wrs_layout lay;
  uint8_t* state;  // caller-owned device buffer
  uint32_t t;      // frames pushed
  int block;       // threads per block of the fused kernel
  int px;          // requested pixels per thread
};

constexpr int kDefaultBlock = 256;
constexpr int kDefaultPx = 4;

int wrs_fail(int code, const char* fmt, ...);
int wrs_cuda_fail(cudaError_t e, const char* what);
int wrs_check_config(const wrs_config* c);
void wrs_make_layout(const wrs_config* c, wrs_layout* L);
float wrs_delta(const wrs_config* c);
wrs::StreamDev wrs_stream_dev(const wrs_ctx* x);
int wrs_effective_px(const wrs_ctx* x, const float* frame, int64_t pitch, const float* out);
cudaError_t wrs_launch_push(const wrs::StreamDev& s, const wrs::FrameDev& f, int block, int px,
                            bool f16, cudaStream_t st);
