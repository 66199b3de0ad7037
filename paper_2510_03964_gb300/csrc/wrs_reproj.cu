// Temporal reprojection (Sec. 4.3, "Implementation"): each pixel gathers the
// previous frame's reservoir of the surface it now shows (through its motion
// vector, nearest pixel centre), drops it on a depth mismatch or when the
// source lies off screen, and then takes the frame's candidate exactly as the
// in-place push does. The gather reads another pixel's slots, so the update
// cannot run in place: it reads one state buffer and writes every slot to the
// other, and the buffers swap roles afterwards.
//
// One pixel per thread: under a pan the gathered rows are the current rows
// shifted, so neighbouring threads still read neighbouring addresses.
#include <cmath>

#include "wrs_internal.h"

namespace {

using wrs::FrameDev;
using wrs::StreamDev;

constexpr int kThreads = 256;

struct ReprojDev {
  const float2* motion;      // [H][W] or null
  const float* depth;        // [H][W] or null
  const float* prev_depth;   // [H][W] or null
  float tol;
};

template <bool F16, bool LIT, bool FOV>
__global__ void __launch_bounds__(kThreads) reproject_kernel(const __grid_constant__ StreamDev cur,
                                                             const __grid_constant__ StreamDev prev,
                                                             const __grid_constant__ FrameDev f,
                                                             const __grid_constant__ ReprojDev r) {
  __shared__ unsigned block_replaced;
  if (threadIdx.x == 0) block_replaced = 0;
  __syncthreads();
  const float d_f = wrs::fovea_density(cur);
  const float fw = static_cast<float>(cur.width), fh = static_cast<float>(cur.height);
  int replaced = 0;
  for (int64_t p = blockIdx.x * static_cast<int64_t>(kThreads) + threadIdx.x; p < cur.hw;
       p += static_cast<int64_t>(gridDim.x) * kThreads) {
    int y, x;
    wrs::row_col(cur, static_cast<int>(p), y, x);
    float mx = 0.0f, my = 0.0f;
    if (r.motion != nullptr) {
      const float2 m = r.motion[p];
      mx = m.x;
      my = m.y;
    }
    const float cx = __fsub_rn(__fadd_rn(static_cast<float>(x), 0.5f), mx);
    const float cy = __fsub_rn(__fadd_rn(static_cast<float>(y), 0.5f), my);
    bool ok = cx >= 0.0f && cx < fw && cy >= 0.0f && cy < fh;  // false for NaN
    int64_t q = p;
    if (ok) q = static_cast<int64_t>(floorf(cy)) * cur.width + static_cast<int64_t>(floorf(cx));
    if (ok && r.depth != nullptr) {
      const float dp = r.depth[p], dq = r.prev_depth[q];
      if (fabsf(__fsub_rn(dq, dp)) > __fmul_rn(r.tol, dp)) ok = false;
    }
    wrs::Src src;
    src.W = prev.W;
    src.P = prev.P;
    src.key = prev.key;
    src.idx = prev.idx;
    src.wt = prev.wt;
    src.col = prev.col;
    src.stride = prev.plane;
    src.at = q;
    src.frame = nullptr;
    src.u = nullptr;
    const int pi = static_cast<int>(p);
    if constexpr (LIT)
      replaced += wrs::push_group_literal<F16, 1, false, FOV, true>(cur, f, pi, src, d_f, !ok);
    else
      replaced += wrs::push_group<0, F16, 1, false, FOV, true>(cur, f, pi, src, d_f, !ok);
  }
  const unsigned c = __reduce_add_sync(0xffffffffu, static_cast<unsigned>(replaced));
  if ((threadIdx.x & 31) == 0 && c != 0) atomicAdd(&block_replaced, c);
  __syncthreads();
  if (threadIdx.x == 0 && block_replaced != 0)
    atomicAdd(cur.replacements, static_cast<unsigned long long>(block_replaced));
}

bool aligned(const void* p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

template <bool F16, bool LIT>
void launch(bool fov, unsigned grid, cudaStream_t st, const StreamDev& cur, const StreamDev& prev,
            const FrameDev& f, const ReprojDev& r) {
  if (fov)
    reproject_kernel<F16, LIT, true><<<grid, kThreads, 0, st>>>(cur, prev, f, r);
  else
    reproject_kernel<F16, LIT, false><<<grid, kThreads, 0, st>>>(cur, prev, f, r);
}

}  // namespace

extern "C" int wrs_set_reprojection_buffer(wrs_ctx* x, void* d_spare, size_t bytes,
                                           wrs_stream_t stream) {
  wrs_clear_error();
  if (!x) return wrs_fail(WRS_ERR_ARG, "context is NULL");
  const cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (d_spare == nullptr) {
    if (x->planes != x->state) {
      const int64_t hdr = x->lay.W_off;
      cudaError_t e = cudaMemcpyAsync(x->state + hdr, x->planes + hdr, x->lay.total_bytes - hdr,
                                      cudaMemcpyDeviceToDevice, st);
      if (e != cudaSuccess) return wrs_cuda_fail(e, "wrs_set_reprojection_buffer: copy back");
      x->planes = x->state;
    }
    x->spare = nullptr;
    return WRS_OK;
  }
  if (!aligned(d_spare, 256)) return wrs_fail(WRS_ERR_ARG, "d_spare must be 256-byte aligned");
  if (bytes < static_cast<size_t>(x->lay.total_bytes))
    return wrs_fail(WRS_ERR_BUDGET, "spare buffer holds %zu bytes, the stream needs %lld", bytes,
                    static_cast<long long>(x->lay.total_bytes));
  uint8_t* sp = static_cast<uint8_t*>(d_spare);
  if (sp == x->state || sp == x->planes)
    return wrs_fail(WRS_ERR_ARG, "d_spare must be a buffer other than the stream's state");
  if (x->planes != x->state) {
    // the current reservoirs live in the old spare: move them home first
    const int64_t hdr = x->lay.W_off;
    cudaError_t e = cudaMemcpyAsync(x->state + hdr, x->planes + hdr, x->lay.total_bytes - hdr,
                                    cudaMemcpyDeviceToDevice, st);
    if (e != cudaSuccess) return wrs_cuda_fail(e, "wrs_set_reprojection_buffer: copy back");
    x->planes = x->state;
  }
  // empty reservoirs in the spare: planes a reprojected push never writes
  // (the key and bias planes under the literal rule) keep defined values
  cudaError_t e = wrs_init_planes(x, sp, st);
  if (e != cudaSuccess) return wrs_cuda_fail(e, "wrs_set_reprojection_buffer: init");
  x->spare = sp;
  return WRS_OK;
}

extern "C" int wrs_push_frame_reproject(wrs_ctx* x, const float* d_frame, int64_t pitch, float gx,
                                        float gy, const float* d_motion, const float* d_depth,
                                        const float* d_prev_depth, float depth_tol,
                                        const uint8_t* d_fov, float* d_out, wrs_stream_t stream) {
  wrs_clear_error();
  if (!x) return wrs_fail(WRS_ERR_ARG, "context is NULL");
  if (!x->spare)
    return wrs_fail(WRS_ERR_STATE, "no spare state buffer: call wrs_set_reprojection_buffer");
  if (!d_frame) return wrs_fail(WRS_ERR_ARG, "d_frame is NULL");
  if (!aligned(d_frame, 4) || (d_out && !aligned(d_out, 4)))
    return wrs_fail(WRS_ERR_ARG, "frame and out must be 4-byte aligned");
  if (pitch < 3 * static_cast<int64_t>(x->cfg.width))
    return wrs_fail(WRS_ERR_ARG, "frame_pitch_elems %lld is below 3 * width",
                    static_cast<long long>(pitch));
  if (!std::isfinite(gx) || !std::isfinite(gy)) return wrs_fail(WRS_ERR_ARG, "gaze must be finite");
  if (d_motion && !aligned(d_motion, 8))
    return wrs_fail(WRS_ERR_ARG, "d_motion must be 8-byte aligned");
  if ((d_depth == nullptr) != (d_prev_depth == nullptr))
    return wrs_fail(WRS_ERR_ARG, "d_depth and d_prev_depth go together");
  if (d_depth && (!aligned(d_depth, 4) || !aligned(d_prev_depth, 4)))
    return wrs_fail(WRS_ERR_ARG, "depth buffers must be 4-byte aligned");
  if (d_depth && (!std::isfinite(depth_tol) || depth_tol < 0.0f))
    return wrs_fail(WRS_ERR_ARG, "depth_tol must be finite and >= 0");
  if (x->t == 0xFFFFFFFFu) return wrs_fail(WRS_ERR_STATE, "frame counter exhausted");

  uint8_t* src_planes = x->planes;
  uint8_t* dst_planes = x->planes == x->state ? x->spare : x->state;
  x->planes = src_planes;
  const StreamDev prev = wrs_stream_dev(x);
  x->planes = dst_planes;
  const StreamDev cur = wrs_stream_dev(x);
  x->planes = src_planes;  // until the launch has been enqueued

  FrameDev f;
  f.frame = d_frame;
  f.pitch = pitch;
  f.fov = d_fov;
  f.out = d_out;
  f.gx = gx;
  f.gy = gy;
  f.t = x->t;
  ReprojDev r;
  r.motion = reinterpret_cast<const float2*>(d_motion);
  r.depth = d_depth;
  r.prev_depth = d_prev_depth;
  r.tol = depth_tol;

  const int64_t hw = static_cast<int64_t>(x->cfg.width) * x->cfg.height;
  const int64_t want = (hw + kThreads - 1) / kThreads;
  const int64_t cap = static_cast<int64_t>(x->sms) * 8 * 16;
  const unsigned grid = static_cast<unsigned>(want < cap ? want : cap);
  const cudaStream_t st = static_cast<cudaStream_t>(stream);
  const bool f16 = x->cfg.color_fp16 != 0;
  const bool lit = x->cfg.update_rule == WRS_RULE_LITERAL;
  const bool fov = d_fov != nullptr;
  if (f16) {
    if (lit) launch<true, true>(fov, grid, st, cur, prev, f, r);
    else launch<true, false>(fov, grid, st, cur, prev, f, r);
  } else {
    if (lit) launch<false, true>(fov, grid, st, cur, prev, f, r);
    else launch<false, false>(fov, grid, st, cur, prev, f, r);
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return wrs_cuda_fail(e, "wrs_push_frame_reproject: launch");
  x->planes = dst_planes;
  x->t += 1;
  return WRS_OK;
}
