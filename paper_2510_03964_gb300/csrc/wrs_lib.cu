// libwrs: C-ABI entry points (include/wrs.h) and the single-stream kernels.
//
// One kernel per frame does the whole per-pixel path of the paper (weight,
// key, temporal bias, combine, resolve); see wrs_device.cuh for the
// arithmetic. The host side only validates arguments, places the state planes
// and picks a kernel instantiation.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>

#include "wrs.h"
#include "wrs_device.cuh"
#include "wrs_internal.h"

using wrs::FrameDev;
using wrs::StreamDev;

// ---------------------------------------------------------------- errors

static thread_local char g_err[512] = "";

int wrs_fail(int code, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof g_err, fmt, ap);
  va_end(ap);
  return code;
}

void wrs_clear_error() { g_err[0] = '\0'; }

extern "C" const char* wrs_last_error(void) { return g_err; }

int wrs_cuda_fail(cudaError_t e, const char* what) {
  return wrs_fail(WRS_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

int wrs_require_usable(const wrs_ctx* x) {
  if (!x->failed) return WRS_OK;
  return wrs_fail(WRS_ERR_STATE,
                  "a device-side wait gave up on this stream, so its reservoirs are undefined: "
                  "restore a saved state with wrs_import_state first");
}

// ---------------------------------------------------------------- config, layout

static constexpr int64_t kPlaneAlign = 64;                 // entries; 256 B for 4-byte planes
static constexpr int64_t kMaxPixels = (1ll << 31) - 64;
static constexpr int64_t kStatusBytes = 256;                // status header before the planes
static constexpr int64_t kMapFrames = wrs::kRingFrames;     // ring of replacement-code planes

int wrs_check_config(const wrs_config* c) {
  if (!c) return wrs_fail(WRS_ERR_ARG, "config is NULL");
  if (c->width < 1 || c->height < 1)
    return wrs_fail(WRS_ERR_ARG, "width and height must be >= 1 (got %d x %d)", c->width,
                    c->height);
  if (static_cast<int64_t>(c->width) * c->height > kMaxPixels)
    return wrs_fail(WRS_ERR_ARG, "width * height must be below 2^31 - 64");
  if (c->K < 1 || c->K > WRS_MAX_K)
    return wrs_fail(WRS_ERR_ARG, "K must be in 1..%d (got %d)", WRS_MAX_K, c->K);
  if (!(c->fovea_radius_px > 0.0f) || !std::isfinite(c->fovea_radius_px))
    return wrs_fail(WRS_ERR_ARG, "fovea_radius_px must be finite and > 0");
  if (!std::isfinite(c->deg_per_px))
    return wrs_fail(WRS_ERR_ARG, "deg_per_px must be finite");
  if (c->color_fp16 != 0 && c->color_fp16 != 1)
    return wrs_fail(WRS_ERR_ARG, "color_fp16 must be 0 or 1");
  if (c->temporal_bias < 0 || c->temporal_bias > 2)
    return wrs_fail(WRS_ERR_ARG, "temporal_bias must be 0, 1 or 2");
  if (c->update_rule != WRS_RULE_KEYS && c->update_rule != WRS_RULE_LITERAL)
    return wrs_fail(WRS_ERR_ARG, "update_rule must be WRS_RULE_KEYS or WRS_RULE_LITERAL");
  if (c->update_rule == WRS_RULE_LITERAL && c->K != 1)
    return wrs_fail(WRS_ERR_ARG, "the literal update rule holds one sample: K must be 1");
  return WRS_OK;
}

void wrs_make_layout(const wrs_config* c, wrs_layout* L) {
  const int64_t hw = static_cast<int64_t>(c->width) * c->height;
  const int64_t pl = (hw + kPlaneAlign - 1) / kPlaneAlign * kPlaneAlign;
  L->plane_px = pl;
  L->plane_bytes4 = pl * 4;
  L->plane_bytes_col = pl * (c->color_fp16 ? 8 : 16);
  L->plane_bytes_wt = c->color_fp16 ? pl * 2 : 0;
  L->status_off = 0;
  L->W_off = kStatusBytes;
  L->P_off = L->W_off + L->plane_bytes4;
  L->key_off = L->P_off + L->plane_bytes4;
  L->idx_off = L->key_off + c->K * L->plane_bytes4;
  if (c->color_fp16) {
    // low halves of the slot weights (uint16), then 8-byte records {r, g, b, w_hi}
    L->wt_off = L->idx_off + c->K * L->plane_bytes4;
    L->col_off = (L->wt_off + c->K * L->plane_bytes_wt + 255) / 256 * 256;
  } else {
    // FP32 colour: weight and colour of a slot in one float4 record
    L->wt_off = -1;
    L->col_off = L->idx_off + c->K * L->plane_bytes4;
  }
  // one code byte per pixel and frame for the last kMapFrames frames; none
  // for one or two slots, whose kernels write the sample indices directly
  L->map_off = L->col_off + c->K * L->plane_bytes_col;
  L->map_frames = c->K <= 2 ? 0 : kMapFrames;
  L->total_bytes = L->map_off + L->map_frames * pl;
}

float wrs_delta(const wrs_config* c) {
  // default: the fovea radius spans 2.5 degrees (IEEE single division)
  return c->deg_per_px > 0.0f ? c->deg_per_px : 2.5f / c->fovea_radius_px;
}

StreamDev wrs_stream_dev(const wrs_ctx* x) {
  StreamDev s;
  uint8_t* b = x->planes;
  s.W = reinterpret_cast<float*>(b + x->lay.W_off);
  s.P = reinterpret_cast<float*>(b + x->lay.P_off);
  s.key = reinterpret_cast<float*>(b + x->lay.key_off);
  s.idx = reinterpret_cast<uint32_t*>(b + x->lay.idx_off);
  s.wt = x->lay.wt_off >= 0 ? reinterpret_cast<uint16_t*>(b + x->lay.wt_off) : nullptr;
  s.col = b + x->lay.col_off;
  s.plane = x->lay.plane_px;
  s.width = x->cfg.width;
  s.height = x->cfg.height;
  s.K = x->cfg.K;
  s.hw = x->cfg.width * x->cfg.height;
  s.width_rcp = x->cfg.width == 1
                    ? 0xFFFFFFFFu
                    : static_cast<uint32_t>(((1ull << 32) + x->cfg.width - 1) / x->cfg.width);
  s.r_f = x->cfg.fovea_radius_px;
  s.delta = wrs_delta(&x->cfg);
  s.seed_lo = static_cast<uint32_t>(x->cfg.seed);
  s.seed_hi = static_cast<uint32_t>(x->cfg.seed >> 32);
  s.stream_id = x->cfg.stream_id;
  s.bias = x->cfg.temporal_bias;
  s.literal = x->cfg.update_rule == WRS_RULE_LITERAL ? 1 : 0;
  s.replacements = reinterpret_cast<unsigned long long*>(x->state + x->lay.status_off + 8);
  // the ring stays in the primary buffer (none for one or two slots)
  s.maps = x->lay.map_frames > 0 ? x->state + x->lay.map_off : nullptr;
  s.check = reinterpret_cast<uint32_t*>(x->state + x->lay.status_off + 16);
  return s;
}

uint32_t wrs_map_lo(const wrs_ctx* x) {
  if (x->lay.map_frames == 0) return x->t;  // no ring: nothing to fold
  const uint32_t back = static_cast<uint32_t>(x->lay.map_frames - 1);
  const uint32_t oldest = x->t >= back ? x->t - back : 0u;  // oldest frame the ring still holds
  return x->base > oldest ? x->base : oldest;
}

uint32_t* wrs_status_word(const wrs_ctx* x) {
  return reinterpret_cast<uint32_t*>(x->state + x->lay.status_off);
}

// Stages of `px` pixels per thread: as many (up to four) as keep two CTAs on
// an SM, else what one CTA holds. More stages keep more bytes in flight; the
// kernels wait on copies, not on arithmetic.
static int wrs_default_stages(int K, bool f16, int px) {
  constexpr size_t kSmPerSm = 228 * 1024, kReservedPerCta = 1024;
  int st = 4;
  while (st > 2 && 2 * (wrs_pipe_smem_bytes(K, f16, px, st, true) + kReservedPerCta) > kSmPerSm) --st;
  while (st > 1 && wrs_pipe_smem_bytes(K, f16, px, st, true) > kSmemBudget) --st;
  return st;
}

void wrs_default_pipe(int K, bool f16, int* px, int* stages) {
  // 256-pixel tiles with the stages above (K = 8 FP32 gets two stages at two
  // CTAs per SM, K = 8 FP16 three, K = 4 four); one or two slots take two
  // pixels per thread (512-pixel tiles, four stages): their kernels are bound
  // by instruction issue, and a thread's second pixel shares its per-tile work
  *px = K <= 2 ? 2 : 1;
  *stages = wrs_default_stages(K, f16, *px);
}

extern "C" size_t wrs_state_bytes(const wrs_config* cfg) {
  if (wrs_check_config(cfg) != WRS_OK) return 0;
  wrs_layout L;
  wrs_make_layout(cfg, &L);
  return static_cast<size_t>(L.total_bytes);
}

extern "C" int wrs_state_layout(const wrs_config* cfg, wrs_layout* out) {
  if (!out) return wrs_fail(WRS_ERR_ARG, "layout output is NULL");
  const int rc = wrs_check_config(cfg);
  if (rc != WRS_OK) return rc;
  wrs_make_layout(cfg, out);
  return WRS_OK;
}

// ---------------------------------------------------------------- kernels

namespace {

// Every slot empty, W = 0, P = 1 (padding entries included).
__global__ void init_kernel(StreamDev s) {
  const int64_t n = s.plane;
  const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
       i += stride) {
    s.W[i] = 0.0f;
    s.P[i] = 1.0f;
    for (int j = 0; j < s.K; ++j) {
      s.key[j * n + i] = wrs::kInf;
      s.idx[j * n + i] = wrs::kEmpty;
      if (s.wt) s.wt[j * n + i] = 0;  // records are zeroed with the colour region
    }
  }
}

// Folds every pending ring code into the idx planes: pixel p's block was
// last folded by the push of the latest frame below t with that frame % ring
// == the block's band (if it is not below base); codes of later frames apply.
__global__ void fold_all_kernel(StreamDev s, uint32_t base, uint32_t t) {
  const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
  for (int64_t p = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; p < s.hw;
       p += stride) {
    uint32_t lo = base;
    if (t > 0) {
      const uint32_t d = ((t - 1u) - wrs::fold_band(p)) & wrs::kRingMask;
      if (t - 1u >= d) {
        const uint32_t last = (t - 1u) - d;  // the last push that folded this block
        if (last >= base) lo = last + 1u;
      }
    }
    if (lo < t) {
      wrs::FoldIn<WRS_MAX_K> in;
      wrs::fold_load(s, s.idx, s.K, t, p, in);
      wrs::fold_store(s, s.idx, s.K, t, lo, p, in, wrs::kCodeKeep);
    }
  }
}

__global__ void zero_kernel(uint8_t* p, int64_t bytes) {
  const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < bytes / 16;
       i += stride)
    reinterpret_cast<uint4*>(p)[i] = make_uint4(0, 0, 0, 0);
}

template <int KT, bool F16, int PX, bool VEC, bool LIT>
__global__ void __launch_bounds__(256, PX == 4 ? 2 : 3) push_kernel(const __grid_constant__ StreamDev s,
                                                      const __grid_constant__ FrameDev f) {
  __shared__ unsigned block_replaced;
  if (threadIdx.x == 0) block_replaced = 0;
  __syncthreads();
  const int64_t g = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  const int64_t p0 = g * PX;
  int replaced = 0;
  if (p0 < s.hw) {
    const float d_f = wrs::fovea_density(s);
    const wrs::Src src = wrs::global_src(s, f, static_cast<int>(p0), VEC);
    if constexpr (LIT) {
      if (f.fov != nullptr)
        replaced = wrs::push_group_literal<F16, PX, VEC, true>(s, f, static_cast<int>(p0), src, d_f);
      else
        replaced = wrs::push_group_literal<F16, PX, VEC, false>(s, f, static_cast<int>(p0), src, d_f);
    } else {
      if (f.fov != nullptr)
        replaced = wrs::push_group<KT, F16, PX, VEC, true>(s, f, static_cast<int>(p0), src, d_f);
      else
        replaced = wrs::push_group<KT, F16, PX, VEC, false>(s, f, static_cast<int>(p0), src, d_f);
    }
  }
  // one atomic per block for the stream's replacement count
  const unsigned c = __reduce_add_sync(0xffffffffu, static_cast<unsigned>(replaced));
  if ((threadIdx.x & 31) == 0 && c != 0) atomicAdd(&block_replaced, c);
  __syncthreads();
  if (threadIdx.x == 0 && block_replaced != 0)
    atomicAdd(s.replacements, static_cast<unsigned long long>(block_replaced));
}

template <int KT, bool F16, int PX>
__global__ void __launch_bounds__(256, PX == 4 ? 2 : 3) resolve_kernel(const __grid_constant__ StreamDev s,
                                                         float* __restrict__ out) {
  const int64_t g = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  const int64_t p0 = g * PX;
  if (p0 >= s.hw) return;
  wrs::resolve_group<KT, F16, PX>(s, out, static_cast<int>(p0));
}

template <int KT, bool F16, int PX, bool VEC, bool LIT = false>
cudaError_t launch_push_t(const StreamDev& s, const FrameDev& f, int block, cudaStream_t st) {
  const int64_t groups = (static_cast<int64_t>(s.hw) + PX - 1) / PX;
  const int64_t grid = (groups + block - 1) / block;
  push_kernel<KT, F16, PX, VEC, LIT><<<static_cast<unsigned>(grid), block, 0, st>>>(s, f);
  return cudaGetLastError();
}

template <int KT, bool F16, bool LIT = false>
cudaError_t launch_push_px(const StreamDev& s, const FrameDev& f, int block, int px,
                           cudaStream_t st) {
  switch (px) {
    case 4: return launch_push_t<KT, F16, 4, true, LIT>(s, f, block, st);
    case 2: return launch_push_t<KT, F16, 2, true, LIT>(s, f, block, st);
    default: return launch_push_t<KT, F16, 1, false, LIT>(s, f, block, st);
  }
}

template <bool F16>
cudaError_t launch_push_k(const StreamDev& s, const FrameDev& f, int block, int px,
                          cudaStream_t st) {
  if (s.literal) return launch_push_px<1, F16, true>(s, f, block, px, st);
  switch (s.K) {
    case 1: return launch_push_px<1, F16>(s, f, block, px, st);
    case 2: return launch_push_px<2, F16>(s, f, block, px, st);
    case 4: return launch_push_px<4, F16>(s, f, block, px, st);
    case 8: return launch_push_px<8, F16>(s, f, block, px, st);
    default: return launch_push_px<0, F16>(s, f, block, px, st);
  }
}

template <int KT, bool F16, int PX>
cudaError_t launch_resolve_t(const StreamDev& s, float* out, int block, cudaStream_t st) {
  const int64_t groups = (static_cast<int64_t>(s.hw) + PX - 1) / PX;
  const int64_t grid = (groups + block - 1) / block;
  resolve_kernel<KT, F16, PX><<<static_cast<unsigned>(grid), block, 0, st>>>(s, out);
  return cudaGetLastError();
}

template <bool F16>
cudaError_t launch_resolve_k(const StreamDev& s, float* out, int block, int px,
                             cudaStream_t st) {
  const bool p4 = px == 4;
  switch (s.K) {
    case 1: return p4 ? launch_resolve_t<1, F16, 4>(s, out, block, st) : launch_resolve_t<1, F16, 1>(s, out, block, st);
    case 2: return p4 ? launch_resolve_t<2, F16, 4>(s, out, block, st) : launch_resolve_t<2, F16, 1>(s, out, block, st);
    case 4: return p4 ? launch_resolve_t<4, F16, 4>(s, out, block, st) : launch_resolve_t<4, F16, 1>(s, out, block, st);
    case 8: return p4 ? launch_resolve_t<8, F16, 4>(s, out, block, st) : launch_resolve_t<8, F16, 1>(s, out, block, st);
    default: return p4 ? launch_resolve_t<0, F16, 4>(s, out, block, st) : launch_resolve_t<0, F16, 1>(s, out, block, st);
  }
}

bool aligned(const void* p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

}  // namespace

// Pixels per thread that the frame/out pointers and the width allow, given the request.
int wrs_effective_px(const wrs_ctx* x, const float* frame, int64_t pitch, const float* out) {
  int px = x->px;
  while (px > 1) {
    const size_t a = px == 4 ? 16 : 8;
    const bool ok = (x->cfg.width % px == 0) && (pitch % px == 0) && aligned(frame, a) &&
                    (out == nullptr || aligned(out, a));
    if (ok) break;
    px /= 2;
  }
  return px;
}

cudaError_t wrs_launch_push(const StreamDev& s, const FrameDev& f, int block, int px,
                            bool f16, cudaStream_t st) {
  return f16 ? launch_push_k<true>(s, f, block, px, st)
             : launch_push_k<false>(s, f, block, px, st);
}

cudaError_t wrs_fold_all(wrs_ctx* x, cudaStream_t st) {
  if (x->lay.map_frames == 0) x->base = x->t;  // indices written directly
  if (x->base == x->t) return cudaSuccess;
  const StreamDev s = wrs_stream_dev(x);
  fold_all_kernel<<<static_cast<unsigned>(x->sms) * 8, 256, 0, st>>>(s, x->base, x->t);
  const cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) x->base = x->t;
  return e;
}

// ---------------------------------------------------------------- C-ABI

cudaError_t wrs_init_planes(const wrs_ctx* x, uint8_t* base, cudaStream_t st) {
  // colour planes zeroed, then empty slots, W = 0, P = 1 in the planes at `base`
  wrs_ctx tmp = *x;
  tmp.planes = base;
  const StreamDev s = wrs_stream_dev(&tmp);
  zero_kernel<<<1216, 256, 0, st>>>(base + x->lay.col_off, x->lay.total_bytes - x->lay.col_off);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) {
    init_kernel<<<1216, 256, 0, st>>>(s);
    e = cudaGetLastError();
  }
  return e;
}

extern "C" int wrs_create(const wrs_config* cfg, void* d_state, size_t state_bytes,
                          wrs_stream_t stream, wrs_ctx** out) {
  wrs_clear_error();
  if (!out) return wrs_fail(WRS_ERR_ARG, "output context pointer is NULL");
  *out = nullptr;
  int rc = wrs_check_config(cfg);
  if (rc != WRS_OK) return rc;
  if (!d_state) return wrs_fail(WRS_ERR_ARG, "d_state is NULL");
  if (!aligned(d_state, 256)) return wrs_fail(WRS_ERR_ARG, "d_state must be 256-byte aligned");
  wrs_layout L;
  wrs_make_layout(cfg, &L);
  if (state_bytes < static_cast<size_t>(L.total_bytes))
    return wrs_fail(WRS_ERR_BUDGET, "state buffer holds %zu bytes, the stream needs %lld",
                    state_bytes, static_cast<long long>(L.total_bytes));
  wrs_ctx* x = new (std::nothrow) wrs_ctx;
  if (!x) return wrs_fail(WRS_ERR_ARG, "out of host memory for the context");
  x->cfg = *cfg;
  x->lay = L;
  x->state = static_cast<uint8_t*>(d_state);
  x->planes = x->state;
  x->spare = nullptr;
  x->t = 0;
  x->block = kDefaultBlock;
  x->px = kDefaultPx;
  x->pipe = 1;
  x->pipe_ctas = 0;
  wrs_default_pipe(cfg->K, cfg->color_fp16 != 0, &x->pipe_px, &x->pipe_stages);
  x->timeout_ns = kDefaultTimeoutNs;
  x->test_extra_tx = 0;
  x->failed = 0;
  x->base = 0;
  cudaError_t e = cudaGetDevice(&x->device);
  if (e == cudaSuccess)
    e = cudaDeviceGetAttribute(&x->sms, cudaDevAttrMultiProcessorCount, x->device);
  if (e != cudaSuccess) {
    delete x;
    return wrs_cuda_fail(e, "wrs_create: device query");
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  // status word and colour planes start zeroed; then the per-slot fields
  zero_kernel<<<1, 32, 0, st>>>(x->state + L.status_off, kStatusBytes);
  e = cudaGetLastError();
  if (e == cudaSuccess) e = wrs_init_planes(x, x->state, st);
  if (e != cudaSuccess) {
    delete x;
    return wrs_cuda_fail(e, "wrs_create: init launch");
  }
  *out = x;
  return WRS_OK;
}

extern "C" int wrs_push_frame(wrs_ctx* x, const float* d_frame, int64_t pitch, float gx,
                              float gy, const uint8_t* d_fov, float* d_out,
                              wrs_stream_t stream) {
  wrs_clear_error();
  if (!x) return wrs_fail(WRS_ERR_ARG, "context is NULL");
  if (!d_frame) return wrs_fail(WRS_ERR_ARG, "d_frame is NULL");
  if (!aligned(d_frame, 4) || (d_out && !aligned(d_out, 4)))
    return wrs_fail(WRS_ERR_ARG, "frame and out must be 4-byte aligned");
  if (pitch < 3 * static_cast<int64_t>(x->cfg.width))
    return wrs_fail(WRS_ERR_ARG, "frame_pitch_elems %lld is below 3 * width",
                    static_cast<long long>(pitch));
  if (!std::isfinite(gx) || !std::isfinite(gy))
    return wrs_fail(WRS_ERR_ARG, "gaze must be finite");
  if (int rc = wrs_require_usable(x)) return rc;
  if (x->t == 0xFFFFFFFFu) return wrs_fail(WRS_ERR_STATE, "frame counter exhausted");
  const StreamDev s = wrs_stream_dev(x);
  FrameDev f;
  f.frame = d_frame;
  f.pitch = pitch;
  f.fov = d_fov;
  f.out = d_out;
  f.gx = gx;
  f.gy = gy;
  f.t = x->t;
  f.map_lo = wrs_map_lo(x);
  cudaError_t e;
  if (x->pipe && wrs_pipe_supported(x, d_frame, pitch, d_out)) {
    e = wrs_launch_pipe(s, f, x->cfg.color_fp16 != 0, x->pipe_px, x->pipe_stages, x->sms,
                        x->pipe_ctas, wrs_status_word(x), x->timeout_ns, x->test_extra_tx,
                        static_cast<cudaStream_t>(stream));
  } else {
    const int px = wrs_effective_px(x, d_frame, pitch, d_out);
    e = wrs_launch_push(s, f, x->block, px, x->cfg.color_fp16 != 0,
                        static_cast<cudaStream_t>(stream));
  }
  if (e != cudaSuccess) return wrs_cuda_fail(e, "wrs_push_frame: launch");
  x->t += 1;
  return WRS_OK;
}

extern "C" int wrs_push_foveated(wrs_ctx* x, const float* d_img, int64_t img_pitch,
                                 const void* d_mip, size_t mip_bytes, int32_t nradii,
                                 const float* radii, int32_t filter, float gx, float gy,
                                 const uint8_t* d_fov, float* d_out, wrs_stream_t stream) {
  wrs_clear_error();
  if (!x) return wrs_fail(WRS_ERR_ARG, "context is NULL");
  if (x->cfg.width % 4 != 0)
    return wrs_fail(WRS_ERR_ARG, "foveating on read needs width %% 4 == 0 (got %d)",
                    x->cfg.width);
  if (d_out && !aligned(d_out, 16)) return wrs_fail(WRS_ERR_ARG, "d_out must be 16-byte aligned");
  if (!std::isfinite(gx) || !std::isfinite(gy))
    return wrs_fail(WRS_ERR_ARG, "gaze must be finite");
  wrs::FovDev fv;
  if (int rc = wrs_fov_check_source(d_img, img_pitch, d_mip, mip_bytes, x->cfg.width, x->cfg.height,
                              nradii, radii, filter, &fv))
    return rc;
  if (int rc = wrs_require_usable(x)) return rc;
  if (x->t == 0xFFFFFFFFu) return wrs_fail(WRS_ERR_STATE, "frame counter exhausted");
  const StreamDev s = wrs_stream_dev(x);
  FrameDev f;
  f.frame = nullptr;  // the consumers foveate the frame into shared memory
  f.pitch = 3 * static_cast<int64_t>(x->cfg.width);
  f.fov = d_fov;
  f.out = d_out;
  f.gx = gx;
  f.gy = gy;
  f.t = x->t;
  f.map_lo = wrs_map_lo(x);
  int px = x->pipe_px, stages = x->pipe_stages;
  // the foveating form takes one pixel per thread: its own stage count then
  if (px != 1) stages = wrs_default_stages(x->cfg.K, x->cfg.color_fp16 != 0, 1);
  cudaError_t e = wrs_launch_pipe_fov(s, f, fv, filter, x->cfg.color_fp16 != 0, stages, x->sms,
                                      x->pipe_ctas, wrs_status_word(x), x->timeout_ns,
                                      static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return wrs_cuda_fail(e, "wrs_push_foveated: launch");
  x->t += 1;
  return WRS_OK;
}

extern "C" int wrs_resolve(wrs_ctx* x, float* d_out, wrs_stream_t stream) {
  wrs_clear_error();
  if (!x) return wrs_fail(WRS_ERR_ARG, "context is NULL");
  if (!d_out || !aligned(d_out, 4)) return wrs_fail(WRS_ERR_ARG, "d_out is NULL or unaligned");
  if (int rc = wrs_require_usable(x)) return rc;
  const StreamDev s = wrs_stream_dev(x);
  const int px = (x->px == 4) ? 4 : 1;
  const cudaStream_t st = static_cast<cudaStream_t>(stream);
  const cudaError_t e = x->cfg.color_fp16 ? launch_resolve_k<true>(s, d_out, x->block, px, st)
                                          : launch_resolve_k<false>(s, d_out, x->block, px, st);
  if (e != cudaSuccess) return wrs_cuda_fail(e, "wrs_resolve: launch");
  return WRS_OK;
}

extern "C" int wrs_destroy(wrs_ctx* x) {
  wrs_clear_error();
  delete x;
  return WRS_OK;
}

extern "C" int wrs_push_frame_host(wrs_ctx* x, const float* h_frame, float gx, float gy,
                                   const uint8_t* h_fov, float* h_out, float* d_frame_stage,
                                   uint8_t* d_fov_stage, float* d_out_stage,
                                   wrs_stream_t stream) {
  wrs_clear_error();
  if (!x) return wrs_fail(WRS_ERR_ARG, "context is NULL");
  if (!h_frame || !h_out || !d_frame_stage || !d_out_stage)
    return wrs_fail(WRS_ERR_ARG, "frame, out and their staging buffers must be non-NULL");
  if (h_fov && !d_fov_stage) return wrs_fail(WRS_ERR_ARG, "h_fov_map needs d_fov_stage");
  const cudaStream_t st = static_cast<cudaStream_t>(stream);
  const size_t hw = static_cast<size_t>(x->cfg.width) * x->cfg.height;
  cudaError_t e = cudaMemcpyAsync(d_frame_stage, h_frame, hw * 3 * sizeof(float),
                                  cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess && h_fov)
    e = cudaMemcpyAsync(d_fov_stage, h_fov, hw, cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return wrs_cuda_fail(e, "wrs_push_frame_host: upload");
  const int rc = wrs_push_frame(x, d_frame_stage, 3 * static_cast<int64_t>(x->cfg.width), gx,
                                gy, h_fov ? d_fov_stage : nullptr, d_out_stage, stream);
  if (rc != WRS_OK) return rc;
  e = cudaMemcpyAsync(h_out, d_out_stage, hw * 3 * sizeof(float), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return wrs_cuda_fail(e, "wrs_push_frame_host: download");
  return WRS_OK;
}

extern "C" int wrs_export_state(wrs_ctx* x, void* h_dst, size_t bytes, wrs_stream_t stream) {
  wrs_clear_error();
  if (!x || !h_dst) return wrs_fail(WRS_ERR_ARG, "context or destination is NULL");
  if (bytes < static_cast<size_t>(x->lay.total_bytes))
    return wrs_fail(WRS_ERR_BUDGET, "destination holds %zu bytes, the state is %lld", bytes,
                    static_cast<long long>(x->lay.total_bytes));
  const cudaStream_t st = static_cast<cudaStream_t>(stream);
  // complete sample indices first, then the header from the primary buffer and
  // the planes from whichever buffer holds them
  cudaError_t e = wrs_fold_all(x, st);
  if (e != cudaSuccess) return wrs_cuda_fail(e, "wrs_export_state: fold");
  const int64_t hdr = x->lay.W_off;
  uint8_t* dst = static_cast<uint8_t*>(h_dst);
  e = cudaMemcpyAsync(dst, x->state, hdr, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(dst + hdr, x->planes + hdr, x->lay.map_off - hdr, cudaMemcpyDeviceToHost,
                        st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return wrs_cuda_fail(e, "wrs_export_state");
  std::memset(dst + x->lay.map_off, 0, static_cast<size_t>(x->lay.total_bytes - x->lay.map_off));
  return WRS_OK;
}

extern "C" int wrs_import_state(wrs_ctx* x, const void* h_src, size_t bytes,
                                uint32_t frame_index, wrs_stream_t stream) {
  wrs_clear_error();
  if (!x || !h_src) return wrs_fail(WRS_ERR_ARG, "context or source is NULL");
  if (bytes < static_cast<size_t>(x->lay.total_bytes))
    return wrs_fail(WRS_ERR_BUDGET, "source holds %zu bytes, the state is %lld", bytes,
                    static_cast<long long>(x->lay.total_bytes));
  const cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int64_t hdr = x->lay.W_off;
  const uint8_t* src = static_cast<const uint8_t*>(h_src);
  cudaError_t e = cudaMemcpyAsync(x->state, src, hdr, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(x->planes + hdr, src + hdr, x->lay.map_off - hdr, cudaMemcpyHostToDevice,
                        st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return wrs_cuda_fail(e, "wrs_import_state");
  x->t = frame_index;
  x->base = frame_index;  // imported indices are complete; the ring's codes are stale
  x->failed = 0;          // the reservoirs are defined again
  return WRS_OK;
}

extern "C" uint32_t wrs_frame_index(const wrs_ctx* x) { return x ? x->t : 0u; }

extern "C" int wrs_set_launch(wrs_ctx* x, int block_threads, int px_per_thread) {
  wrs_clear_error();
  if (!x) return wrs_fail(WRS_ERR_ARG, "context is NULL");
  if (block_threads == 0) block_threads = kDefaultBlock;
  if (px_per_thread == 0) px_per_thread = kDefaultPx;
  if (block_threads < 64 || block_threads > 256 || block_threads % 32 != 0)
    return wrs_fail(WRS_ERR_ARG, "block_threads must be a multiple of 32 in 64..256");
  if (px_per_thread != 1 && px_per_thread != 2 && px_per_thread != 4)
    return wrs_fail(WRS_ERR_ARG, "px_per_thread must be 1, 2 or 4");
  x->block = block_threads;
  x->px = px_per_thread;
  return WRS_OK;
}

extern "C" int wrs_get_launch(const wrs_ctx* x, int* block_threads, int* px_per_thread) {
  if (!x || !block_threads || !px_per_thread)
    return wrs_fail(WRS_ERR_ARG, "NULL argument");
  *block_threads = x->block;
  *px_per_thread = x->px;
  return WRS_OK;
}

extern "C" int wrs_set_pipeline(wrs_ctx* x, int enable, int px_per_thread, int stages,
                                int ctas_per_sm) {
  wrs_clear_error();
  if (!x) return wrs_fail(WRS_ERR_ARG, "context is NULL");
  int dpx, dst;
  wrs_default_pipe(x->cfg.K, x->cfg.color_fp16 != 0, &dpx, &dst);
  const bool f16 = x->cfg.color_fp16 != 0;
  if (px_per_thread == 0) px_per_thread = dpx;
  if (px_per_thread != 1 && px_per_thread != 2 && px_per_thread != 4)
    return wrs_fail(WRS_ERR_ARG, "px_per_thread must be 1, 2 or 4");
  if (stages == 0) stages = wrs_default_stages(x->cfg.K, f16, px_per_thread);
  if (stages < 1 || stages > 8) return wrs_fail(WRS_ERR_ARG, "stages must be in 1..8");
  if (ctas_per_sm < 0 || ctas_per_sm > 8) return wrs_fail(WRS_ERR_ARG, "ctas_per_sm must be in 0..8");
  const size_t need = wrs_pipe_smem_bytes(x->cfg.K, f16, px_per_thread, stages, true);
  if (enable && need > kSmemBudget)
    return wrs_fail(WRS_ERR_ARG, "%d stages of %d px/thread need %zu B of shared memory (> %zu)",
                    stages, px_per_thread, need, kSmemBudget);
  x->pipe = enable ? 1 : 0;
  x->pipe_px = px_per_thread;
  x->pipe_stages = stages;
  x->pipe_ctas = ctas_per_sm;
  return WRS_OK;
}

extern "C" int wrs_get_pipeline(const wrs_ctx* x, int* enable, int* px_per_thread, int* stages,
                                int* ctas_per_sm) {
  if (!x || !enable || !px_per_thread || !stages || !ctas_per_sm)
    return wrs_fail(WRS_ERR_ARG, "NULL argument");
  *enable = x->pipe;
  *px_per_thread = x->pipe_px;
  *stages = x->pipe_stages;
  *ctas_per_sm = x->pipe_ctas;
  return WRS_OK;
}

extern "C" int wrs_set_wait_limit(wrs_ctx* x, uint64_t timeout_ns, uint32_t test_extra_tx) {
  wrs_clear_error();
  if (!x) return wrs_fail(WRS_ERR_ARG, "context is NULL");
  if (timeout_ns == 0) timeout_ns = kDefaultTimeoutNs;
  if (timeout_ns > 60ull * 1000000000ull) return wrs_fail(WRS_ERR_ARG, "timeout above 60 s");
  if (test_extra_tx > 4096) return wrs_fail(WRS_ERR_ARG, "test_extra_tx above 4096");
  x->timeout_ns = timeout_ns;
  x->test_extra_tx = test_extra_tx;
  return WRS_OK;
}

extern "C" int wrs_checked_build(void) {
#ifdef WRS_CHECKED
  return 1;
#else
  return 0;
#endif
}

extern "C" int wrs_check_status(wrs_ctx* x, wrs_stream_t stream) {
  wrs_clear_error();
  if (!x) return wrs_fail(WRS_ERR_ARG, "context is NULL");
  const cudaStream_t st = static_cast<cudaStream_t>(stream);
  uint32_t head[5] = {0, 0, 0, 0, 0};  // status word at +0, check word at +16
  cudaError_t e = cudaMemcpyAsync(head, wrs_status_word(x), sizeof head, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return wrs_cuda_fail(e, "wrs_check_status");
  const uint32_t word = head[0], bounds = head[4];
  if (bounds != 0) {
    e = cudaMemsetAsync(reinterpret_cast<uint8_t*>(wrs_status_word(x)) + 16, 0, sizeof bounds, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return wrs_cuda_fail(e, "wrs_check_status: clear");
    x->failed = 1;
    return wrs_fail(WRS_ERR_CHECK,
                    "checked build: indices outside their buffers were skipped (bits 0x%x: 1 state "
                    "plane, 2 source/stage entry, 4 frame pixel, 8 output, 16 bulk-copy range, 32 "
                    "reprojection source, 64 stage size); the reservoirs are undefined",
                    bounds);
  }
  if (word == WRS_OK) return WRS_OK;
  e = cudaMemsetAsync(wrs_status_word(x), 0, sizeof word, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return wrs_cuda_fail(e, "wrs_check_status: clear");
  x->failed = 1;
  return wrs_fail(static_cast<int>(word),
                  "a device-side wait gave up after %llu ns: the reservoirs are undefined and "
                  "further pushes are refused until wrs_import_state restores a saved state",
                  static_cast<unsigned long long>(x->timeout_ns));
}

extern "C" int wrs_get_stats(wrs_ctx* x, uint64_t* replacements, wrs_stream_t stream) {
  wrs_clear_error();
  if (!x || !replacements) return wrs_fail(WRS_ERR_ARG, "NULL argument");
  const cudaStream_t st = static_cast<cudaStream_t>(stream);
  unsigned long long v = 0;
  cudaError_t e = cudaMemcpyAsync(&v, x->state + x->lay.status_off + 8, sizeof v,
                                  cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return wrs_cuda_fail(e, "wrs_get_stats");
  *replacements = v;
  return WRS_OK;
}
