// Pipelined host-buffer frames. On GB300 the host link moves about 200 GB/s
// each way, so a 4K frame in (99.5 MB) and its resolved frame out each take
// longer than the update itself. Three CUDA streams overlap them:
// the copy of frame n in, the update of frame n-1 and the copy of frame n-2's
// output run at once, through kDepth device staging slots for frames and for
// outputs. Events order each slot's reuse; the host waits only for frame
// n - kDepth to be fully done before it enqueues frame n, which bounds the
// frames in flight to kDepth and keeps the caller's host buffers of older
// frames free. With two slots the upload of frame n could not start before
// frame n-2's download ended, so a frame cost (up + update + down) / 2, more
// than the link alone; three slots leave the link as the bound.
#include <new>

#include "wrs_internal.h"

namespace {
constexpr int kDepth = 3;  // staging slots = frames in flight
}  // namespace

struct wrs_host_pipe {
  wrs_ctx* x;
  int with_fov;
  float* d_frame[kDepth];
  float* d_out[kDepth];
  uint8_t* d_fov[kDepth];
  cudaStream_t s_in, s_comp, s_out;
  cudaEvent_t in_done[kDepth], comp_done[kDepth], out_done[kDepth];
  uint64_t n;  // frames enqueued
};

namespace {

size_t round256(size_t b) { return (b + 255) / 256 * 256; }

// The pipeline's streams belong to the context's device: it must be current.
int check_device(const wrs_ctx* x, const char* what) {
  int cur = -1;
  const cudaError_t e = cudaGetDevice(&cur);
  if (e != cudaSuccess) return wrs_cuda_fail(e, what);
  if (cur != x->device)
    return wrs_fail(WRS_ERR_ARG, "%s: the stream's device (%d) must be current (is %d)", what,
                    x->device, cur);
  return WRS_OK;
}

void destroy_handles(wrs_host_pipe* p) {
  for (int i = 0; i < kDepth; ++i) {
    if (p->in_done[i]) cudaEventDestroy(p->in_done[i]);
    if (p->comp_done[i]) cudaEventDestroy(p->comp_done[i]);
    if (p->out_done[i]) cudaEventDestroy(p->out_done[i]);
  }
  if (p->s_in) cudaStreamDestroy(p->s_in);
  if (p->s_comp) cudaStreamDestroy(p->s_comp);
  if (p->s_out) cudaStreamDestroy(p->s_out);
}

}  // namespace

extern "C" size_t wrs_host_pipe_stage_bytes(const wrs_ctx* x, int with_fov) {
  if (!x) return 0;
  const size_t hw = static_cast<size_t>(x->cfg.width) * x->cfg.height;
  return kDepth * (2 * round256(hw * 3 * sizeof(float)) + (with_fov ? round256(hw) : 0));
}

extern "C" int wrs_host_pipe_create(wrs_ctx* x, void* d_stage, size_t bytes, int with_fov,
                                    wrs_host_pipe** out) {
  wrs_clear_error();
  if (!out) return wrs_fail(WRS_ERR_ARG, "output pointer is NULL");
  *out = nullptr;
  if (!x) return wrs_fail(WRS_ERR_ARG, "context is NULL");
  if (with_fov != 0 && with_fov != 1) return wrs_fail(WRS_ERR_ARG, "with_fov must be 0 or 1");
  if (!d_stage || reinterpret_cast<uintptr_t>(d_stage) % 256 != 0)
    return wrs_fail(WRS_ERR_ARG, "d_stage is NULL or not 256-byte aligned");
  if (int rc = check_device(x, "wrs_host_pipe_create")) return rc;
  const size_t need = wrs_host_pipe_stage_bytes(x, with_fov);
  if (bytes < need)
    return wrs_fail(WRS_ERR_BUDGET, "stage holds %zu bytes, the pipeline needs %zu", bytes, need);
  wrs_host_pipe* p = new (std::nothrow) wrs_host_pipe{};
  if (!p) return wrs_fail(WRS_ERR_ARG, "out of host memory for the pipeline");
  p->x = x;
  p->with_fov = with_fov;
  const size_t hw = static_cast<size_t>(x->cfg.width) * x->cfg.height;
  uint8_t* b = static_cast<uint8_t*>(d_stage);
  for (int i = 0; i < kDepth; ++i) {
    p->d_frame[i] = reinterpret_cast<float*>(b);
    b += round256(hw * 3 * sizeof(float));
    p->d_out[i] = reinterpret_cast<float*>(b);
    b += round256(hw * 3 * sizeof(float));
    p->d_fov[i] = with_fov ? b : nullptr;
    if (with_fov) b += round256(hw);
  }
  cudaError_t e = cudaStreamCreateWithFlags(&p->s_in, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&p->s_comp, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&p->s_out, cudaStreamNonBlocking);
  for (int i = 0; i < kDepth && e == cudaSuccess; ++i) {
    e = cudaEventCreateWithFlags(&p->in_done[i], cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&p->comp_done[i], cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&p->out_done[i], cudaEventDisableTiming);
  }
  if (e != cudaSuccess) {
    destroy_handles(p);
    delete p;
    return wrs_cuda_fail(e, "wrs_host_pipe_create");
  }
  *out = p;
  return WRS_OK;
}

extern "C" int wrs_host_pipe_push(wrs_host_pipe* p, const float* h_frame, float gx, float gy,
                                  const uint8_t* h_fov, float* h_out) {
  wrs_clear_error();
  if (!p) return wrs_fail(WRS_ERR_ARG, "pipeline is NULL");
  if (!h_frame || !h_out) return wrs_fail(WRS_ERR_ARG, "h_frame and h_out must be non-NULL");
  if (h_fov && !p->with_fov)
    return wrs_fail(WRS_ERR_ARG, "this pipeline was created without fov-map slots");
  const int s = static_cast<int>(p->n % kDepth);
  wrs_ctx* x = p->x;
  if (int rc = check_device(x, "wrs_host_pipe_push")) return rc;
  const size_t hw = static_cast<size_t>(x->cfg.width) * x->cfg.height;
  cudaError_t e = cudaSuccess;
  // frame n - kDepth used this slot: its output must have reached the host
  if (p->n >= kDepth) e = cudaEventSynchronize(p->out_done[s]);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(p->d_frame[s], h_frame, hw * 3 * sizeof(float), cudaMemcpyHostToDevice,
                        p->s_in);
  if (e == cudaSuccess && h_fov)
    e = cudaMemcpyAsync(p->d_fov[s], h_fov, hw, cudaMemcpyHostToDevice, p->s_in);
  if (e == cudaSuccess) e = cudaEventRecord(p->in_done[s], p->s_in);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(p->s_comp, p->in_done[s], 0);
  if (e != cudaSuccess) return wrs_cuda_fail(e, "wrs_host_pipe_push: upload");
  const int rc = wrs_push_frame(x, p->d_frame[s], 3 * static_cast<int64_t>(x->cfg.width), gx, gy,
                                h_fov ? p->d_fov[s] : nullptr, p->d_out[s], p->s_comp);
  if (rc != WRS_OK) return rc;
  e = cudaEventRecord(p->comp_done[s], p->s_comp);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(p->s_out, p->comp_done[s], 0);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(h_out, p->d_out[s], hw * 3 * sizeof(float), cudaMemcpyDeviceToHost,
                        p->s_out);
  if (e == cudaSuccess) e = cudaEventRecord(p->out_done[s], p->s_out);
  if (e != cudaSuccess) return wrs_cuda_fail(e, "wrs_host_pipe_push: download");
  p->n += 1;
  return WRS_OK;
}

extern "C" int wrs_host_pipe_finish(wrs_host_pipe* p) {
  wrs_clear_error();
  if (!p) return wrs_fail(WRS_ERR_ARG, "pipeline is NULL");
  cudaError_t e = cudaSuccess;
  for (uint64_t k = p->n >= kDepth ? p->n - kDepth : 0; k < p->n && e == cudaSuccess; ++k)
    e = cudaEventSynchronize(p->out_done[k % kDepth]);
  return e == cudaSuccess ? WRS_OK : wrs_cuda_fail(e, "wrs_host_pipe_finish");
}

extern "C" int wrs_host_pipe_destroy(wrs_host_pipe* p) {
  wrs_clear_error();
  if (!p) return WRS_OK;
  const int rc = wrs_host_pipe_finish(p);
  destroy_handles(p);
  delete p;
  return rc;
}
