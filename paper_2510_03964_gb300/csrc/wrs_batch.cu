// Batched form: many streams of uneven resolution, K and colour precision in
// one persistent launch, captured once in a CUDA graph.
//
// The launch's descriptor (every stream's planes, frame, gaze, frame index and
// first tile) travels by value as the kernel parameter, so a batch needs no
// device memory of its own. Tiles of T = 256 * PX pixels of all streams are
// numbered stream after stream and dealt to the persistent CTAs round-robin,
// which spreads every stream (and so every K) evenly over the CTAs. Each tile
// goes through the same bulk-copy / uniform / compute pipeline as the
// single-stream kernel (wrs_async.cuh), with the arithmetic chosen per tile by
// the stream's K and colour precision; results are bit-identical to pushing
// each stream on its own.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <new>

#include "wrs.h"
#include "wrs_batch_kernel.cuh"
#include "wrs_internal.h"

namespace {

template <int PX>
const void* batch_fn(int fam) {
  switch (fam) {
    case kFamF16K48: return reinterpret_cast<const void*>(&batch_kernel<PX, kFamF16K48>);
    case kFamF32K48: return reinterpret_cast<const void*>(&batch_kernel<PX, kFamF32K48>);
    default: return reinterpret_cast<const void*>(&batch_kernel<PX, kFamAll>);
  }
}

const void* batch_kernel_for(int px, int fam) {
  switch (px) {
    case 4: return batch_fn<4>(fam);
    case 2: return batch_fn<2>(fam);
    default: return batch_fn<1>(fam);
  }
}

// 3 pixels-per-thread choices x 3 families, then 3 families x 2 filters of
// the foveating form (one pixel per thread)
constexpr int kSlots = 15;

}  // namespace

// The foveating variants (wrs_batch_fov.cu): family x filter.
const void* wrs_batch_fov_kernel(int fam, int filter);

struct wrs_batch {
  int max_streams;
  int px, stages, ctas_per_sm, use_graph;
  BatchArgs* args;            // host copy of the launch descriptor
  // one captured graph per pixels-per-thread choice and family
  cudaGraph_t graph[kSlots];
  cudaGraphExec_t exec[kSlots];
  cudaGraphNode_t node[kSlots];
  size_t configured_smem[kSlots];
  int device;
  int rebuilds;  // graph nodes rebuilt because an in-place update was refused
};

static int px_slot(int px) { return px == 4 ? 2 : (px == 2 ? 1 : 0); }

static int family_of(const BatchArgs& a) {
  bool f16 = true, f32 = true;
  for (int i = 0; i < a.n; ++i) {
    f16 = f16 && (a.e[i].code == 0 || a.e[i].code == 1);
    f32 = f32 && (a.e[i].code == 2 || a.e[i].code == 3);
  }
  return f16 ? kFamF16K48 : (f32 ? kFamF32K48 : kFamAll);
}

extern "C" int wrs_batch_create(int max_streams, wrs_batch** out) {
  if (!out) return wrs_fail(WRS_ERR_ARG, "output pointer is NULL");
  *out = nullptr;
  if (max_streams < 1 || max_streams > kMaxBatch)
    return wrs_fail(WRS_ERR_ARG, "max_streams must be in 1..%d", kMaxBatch);
  wrs_batch* b = new (std::nothrow) wrs_batch;
  if (!b) return wrs_fail(WRS_ERR_ARG, "out of host memory");
  std::memset(b, 0, sizeof *b);
  b->args = new (std::nothrow) BatchArgs;
  if (!b->args) {
    delete b;
    return wrs_fail(WRS_ERR_ARG, "out of host memory");
  }
  std::memset(b->args, 0, sizeof(BatchArgs));
  b->max_streams = max_streams;
  b->px = 1;
  b->stages = 0;
  b->ctas_per_sm = 0;
  b->use_graph = 1;
  b->device = -1;
  *out = b;
  return WRS_OK;
}

extern "C" int wrs_batch_destroy(wrs_batch* b) {
  if (!b) return WRS_OK;
  for (int i = 0; i < kSlots; ++i) {
    if (b->exec[i]) cudaGraphExecDestroy(b->exec[i]);
    if (b->graph[i]) cudaGraphDestroy(b->graph[i]);
  }
  delete b->args;
  delete b;
  return WRS_OK;
}

extern "C" int wrs_batch_set_launch(wrs_batch* b, int px_per_thread, int stages, int ctas_per_sm,
                                    int use_graph) {
  if (!b) return wrs_fail(WRS_ERR_ARG, "batch is NULL");
  if (px_per_thread == 0) px_per_thread = 1;
  if (px_per_thread != 1 && px_per_thread != 2 && px_per_thread != 4)
    return wrs_fail(WRS_ERR_ARG, "px_per_thread must be 1, 2 or 4");
  if (stages < 0 || stages > 8) return wrs_fail(WRS_ERR_ARG, "stages must be in 0..8");
  if (ctas_per_sm < 0 || ctas_per_sm > 8) return wrs_fail(WRS_ERR_ARG, "ctas_per_sm must be in 0..8");
  b->px = px_per_thread;
  b->stages = stages;
  b->ctas_per_sm = ctas_per_sm;
  b->use_graph = use_graph ? 1 : 0;
  return WRS_OK;
}

extern "C" int wrs_batch_get_launch(const wrs_batch* b, int* px_per_thread, int* stages,
                                    int* ctas_per_sm, int* use_graph) {
  if (!b || !px_per_thread || !stages || !ctas_per_sm || !use_graph)
    return wrs_fail(WRS_ERR_ARG, "NULL argument");
  *px_per_thread = b->px;
  *stages = b->stages;
  *ctas_per_sm = b->ctas_per_sm;
  *use_graph = b->use_graph;
  return WRS_OK;
}

static int code_of(const wrs_config& c) {
  const bool f16 = c.color_fp16 != 0;
  if (c.update_rule == WRS_RULE_LITERAL) return f16 ? 6 : 7;
  if (c.K == 4) return f16 ? 0 : 2;
  if (c.K == 8) return f16 ? 1 : 3;
  return f16 ? 4 : 5;
}

// Validates and launches one batch; sources == NULL: the frames are in
// d_frames; else stream i's frame is foveated on read from sources[i] with
// `filter` (d_frames unused).
static int push_batch(wrs_batch* b, int n, wrs_ctx* const* ctxs, const float* const* d_frames,
                      const wrs_fov_source* sources, int32_t filter, const float* gaze_xy,
                      const uint8_t* const* d_fov_maps, float* const* d_outs, wrs_stream_t stream) {
  const bool fov = sources != nullptr;
  if (!b || !ctxs || (!d_frames && !fov) || !gaze_xy) return wrs_fail(WRS_ERR_ARG, "NULL argument");
  if (n < 1 || n > b->max_streams)
    return wrs_fail(WRS_ERR_ARG, "n must be in 1..%d (got %d)", b->max_streams, n);
  if (fov && filter != WRS_FILTER_BOX && filter != WRS_FILTER_BILINEAR)
    return wrs_fail(WRS_ERR_ARG, "filter must be WRS_FILTER_BOX or WRS_FILTER_BILINEAR");
  BatchArgs& a = *b->args;
  // the foveating form takes one pixel per thread (256-pixel tiles)
  const int px = fov ? 1 : b->px;
  const int T = 256 * px;
  int64_t tiles = 0;
  uint32_t stage_bytes = 0;
  int device = -1;
  for (int i = 0; i < n; ++i) {
    wrs_ctx* x = ctxs[i];
    if (!x) return wrs_fail(WRS_ERR_ARG, "ctxs[%d] is NULL", i);
    for (int j = 0; j < i; ++j)
      if (ctxs[j] == x) return wrs_fail(WRS_ERR_ARG, "stream %d appears twice in the batch", i);
    if (device < 0) device = x->device;
    if (x->device != device) return wrs_fail(WRS_ERR_ARG, "all streams of a batch must share a device");
    float* out = d_outs ? d_outs[i] : nullptr;
    const float* fr = nullptr;
    BatchEntry& e = a.e[i];
    if (fov) {
      // foveated on read: the stream's own source, checked as wrs_foveate checks it
      if (x->cfg.width % 4 != 0 || (out && (reinterpret_cast<uintptr_t>(out) & 15u)))
        return wrs_fail(WRS_ERR_ARG, "stream %d: foveating batches need width %% 4 == 0 and a "
                        "16-byte aligned out", i);
      const wrs_fov_source& src = sources[i];
      if (int rc = wrs_fov_check_source(src.d_img, src.img_pitch_elems, src.d_mip, src.mip_bytes,
                                  x->cfg.width, x->cfg.height, src.nradii, src.radii, filter, &e.fv))
        return rc;
    } else {
      fr = d_frames[i];
      if (!fr || !wrs_pipe_supported(x, fr, 3 * static_cast<int64_t>(x->cfg.width), out))
        return wrs_fail(WRS_ERR_ARG,
                        "stream %d: batched frames need width %% 4 == 0 and 16-byte aligned, "
                        "unpadded frame and out",
                        i);
      e.fv = wrs::FovDev{};
    }
    const float gx = gaze_xy[2 * i], gy = gaze_xy[2 * i + 1];
    if (!std::isfinite(gx) || !std::isfinite(gy))
      return wrs_fail(WRS_ERR_ARG, "stream %d: gaze must be finite", i);
    if (x->t == 0xFFFFFFFFu) return wrs_fail(WRS_ERR_STATE, "stream %d: frame counter exhausted", i);
    if (wrs_require_usable(x) != WRS_OK)
      return wrs_fail(WRS_ERR_STATE, "stream %d: a device-side wait gave up on it; restore a saved "
                      "state with wrs_import_state first", i);
    e.s = wrs_stream_dev(x);
    e.f.frame = fr;
    e.f.pitch = 3 * static_cast<int64_t>(x->cfg.width);
    e.f.fov = d_fov_maps ? d_fov_maps[i] : nullptr;
    e.f.out = out;
    e.f.gx = gx;
    e.f.gy = gy;
    e.f.t = x->t;
    e.f.map_lo = wrs_map_lo(x);
    e.status = wrs_status_word(x);
    e.tile0 = static_cast<int>(tiles);
    e.code = code_of(x->cfg);
    tiles += (static_cast<int64_t>(e.s.hw) + T - 1) / T;
    const bool records = out != nullptr || x->cfg.temporal_bias == 2;
    const uint32_t sb = wrs::stage_layout(T, x->cfg.K, x->cfg.color_fp16 ? 2 : 4, records).bytes;
    if (sb > stage_bytes) stage_bytes = sb;
  }
  if (tiles > 0x7FFFFFFF) return wrs_fail(WRS_ERR_ARG, "batch too large");
  int stages = b->stages;
  if (stages == 0) {
    // as many stages (up to 4) as keep two CTAs on an SM, else what one CTA holds
    constexpr size_t kSmPerSm = 228 * 1024, kReservedPerCta = 1024;
    stages = 4;
    while (stages > 2 && 2 * (wrs::ring_bytes(stage_bytes, T, stages) + kReservedPerCta) > kSmPerSm)
      --stages;
    while (stages > 1 && wrs::ring_bytes(stage_bytes, T, stages) > kSmemBudget) --stages;
  }
  const size_t smem = wrs::ring_bytes(stage_bytes, T, stages);
  if (smem > kSmemBudget)
    return wrs_fail(WRS_ERR_ARG, "%d stages of %u B exceed shared memory", stages, stage_bytes);
  a.n = n;
  a.ntiles = static_cast<int>(tiles);
  a.stages = stages;
  a.stage_bytes = stage_bytes;
  a.timeout_ns = ctxs[0]->timeout_ns;

  const int fam = family_of(a);
  const int slot = fov ? 9 + fam * 2 + filter : px_slot(px) * 3 + fam;
  const void* fn = fov ? wrs_batch_fov_kernel(fam, filter) : batch_kernel_for(px, fam);
  cudaError_t e = cudaSuccess;
  if (b->device != device) {
    // a new device: drop graphs and attribute settings made for another one
    for (int i = 0; i < kSlots; ++i) {
      if (b->exec[i]) cudaGraphExecDestroy(b->exec[i]);
      if (b->graph[i]) cudaGraphDestroy(b->graph[i]);
      b->exec[i] = nullptr;
      b->graph[i] = nullptr;
      b->configured_smem[i] = 0;
    }
    b->device = device;
  }
  if (b->configured_smem[slot] == 0) {
    // allow the whole budget once, before any graph is built: a graph keeps the
    // limit it was instantiated under, and later batches may need larger stages
    e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             static_cast<int>(kSmemBudget));
    if (e != cudaSuccess) return wrs_cuda_fail(e, "push_batch: shared memory attribute");
    b->configured_smem[slot] = kSmemBudget;
  }
  int fit = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&fit, fn, kBatchThreads, smem);
  if (e != cudaSuccess) return wrs_cuda_fail(e, "push_batch: occupancy");
  if (fit < 1) return wrs_fail(WRS_ERR_ARG, "batch kernel does not fit on an SM");
  const int per_sm = b->ctas_per_sm > 0 && b->ctas_per_sm < fit ? b->ctas_per_sm : fit;
  const int64_t want = static_cast<int64_t>(ctxs[0]->sms) * per_sm;
  const int grid = static_cast<int>(tiles < want ? tiles : want);

  cudaKernelNodeParams kp;
  std::memset(&kp, 0, sizeof kp);
  void* params[1] = {&a};
  kp.func = const_cast<void*>(fn);
  kp.gridDim = dim3(grid);
  kp.blockDim = dim3(kBatchThreads);
  kp.sharedMemBytes = static_cast<unsigned>(smem);
  kp.kernelParams = params;
  const cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (b->use_graph) {
    if (b->exec[slot]) {
      e = cudaGraphExecKernelNodeSetParams(b->exec[slot], b->node[slot], &kp);
      if (e != cudaSuccess) {
        // the in-place update was refused: rebuild the node below
        (void)cudaGetLastError();
        cudaGraphExecDestroy(b->exec[slot]);
        cudaGraphDestroy(b->graph[slot]);
        b->exec[slot] = nullptr;
        b->graph[slot] = nullptr;
        b->rebuilds += 1;
      }
    }
    if (!b->exec[slot]) {
      e = cudaGraphCreate(&b->graph[slot], 0);
      if (e == cudaSuccess) e = cudaGraphAddKernelNode(&b->node[slot], b->graph[slot], nullptr, 0, &kp);
      if (e == cudaSuccess) e = cudaGraphInstantiate(&b->exec[slot], b->graph[slot], 0);
      if (e != cudaSuccess) return wrs_cuda_fail(e, "push_batch: graph build");
    }
    e = cudaGraphLaunch(b->exec[slot], st);
    if (e != cudaSuccess) return wrs_cuda_fail(e, "push_batch: graph launch");
  } else {
    e = cudaLaunchKernel(fn, kp.gridDim, kp.blockDim, params, smem, st);
    if (e != cudaSuccess) return wrs_cuda_fail(e, "push_batch: launch");
  }
  for (int i = 0; i < n; ++i) ctxs[i]->t += 1;
  return WRS_OK;
}

extern "C" int wrs_push_batch(wrs_batch* b, int n, wrs_ctx* const* ctxs,
                              const float* const* d_frames, const float* gaze_xy,
                              const uint8_t* const* d_fov_maps, float* const* d_outs,
                              wrs_stream_t stream) {
  wrs_clear_error();
  return push_batch(b, n, ctxs, d_frames, nullptr, WRS_FILTER_BOX, gaze_xy, d_fov_maps, d_outs,
                    stream);
}

extern "C" int wrs_push_batch_foveated(wrs_batch* b, int n, wrs_ctx* const* ctxs,
                                       const wrs_fov_source* sources, int32_t filter,
                                       const float* gaze_xy, const uint8_t* const* d_fov_maps,
                                       float* const* d_outs, wrs_stream_t stream) {
  wrs_clear_error();
  if (!sources) return wrs_fail(WRS_ERR_ARG, "sources is NULL");
  return push_batch(b, n, ctxs, nullptr, sources, filter, gaze_xy, d_fov_maps, d_outs, stream);
}
