// Temporal reprojection (Sec. 4.3, "Implementation"): each pixel gathers the
// previous frame's reservoir of the surface it now shows (through its motion
// vector, nearest pixel centre), drops it on a depth mismatch or when the
// source lies off screen, and then takes the frame's candidate exactly as the
// in-place push does. The gather reads another pixel's slots, so the update
// cannot run in place: it reads one state buffer and writes every slot to the
// other, and the buffers swap roles afterwards.
//
// One pixel per thread, its whole history gathered into the thread's column of
// shared memory by asynchronous copies (the key race) or into registers (the
// literal rule, one slot): under a pan the gathered rows are the current rows
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

// Where pixel p's history comes from: the previous frame's pixel containing
// the centre moved back by the motion vector; `ok` is false when that point
// is off screen or the depth test rejects it (q is then p, a valid address).
__device__ __forceinline__ int64_t source_pixel(const StreamDev& s, const ReprojDev& r, int64_t p,
                                                int x, int y, float dp, bool& ok) {
  float mx = 0.0f, my = 0.0f;
  if (r.motion != nullptr) {
    const float2 m = r.motion[p];
    mx = m.x;
    my = m.y;
  }
  const float cx = __fsub_rn(__fadd_rn(static_cast<float>(x), 0.5f), mx);
  const float cy = __fsub_rn(__fadd_rn(static_cast<float>(y), 0.5f), my);
  ok = cx >= 0.0f && cx < static_cast<float>(s.width) && cy >= 0.0f &&
       cy < static_cast<float>(s.height);  // false for NaN
  int64_t q = p;
  if (ok) q = static_cast<int64_t>(floorf(cy)) * s.width + static_cast<int64_t>(floorf(cx));
  if (ok && r.depth != nullptr) {
    const float dq = r.prev_depth[q];
    if (fabsf(__fsub_rn(dq, dp)) > __fmul_rn(r.tol, dp)) ok = false;
  }
  return q;
}

// Asynchronous 4/8/16-byte global -> shared copies (no register holds the
// data in flight), completed by cp.async.wait_all.
__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void cp_async4(void* dst, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(smem_addr(dst)), "l"(src)
               : "memory");
}
__device__ __forceinline__ void cp_async8(void* dst, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(smem_addr(dst)), "l"(src)
               : "memory");
}
__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_addr(dst)), "l"(src)
               : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.wait_all;" ::: "memory");
}

// Shared staging of one block's gathered histories, one column per thread:
// W, P, key[KT], idx[KT], then (FP32 colour) KT float4 records {w, r, g, b}
// or (FP16 colour) KT words of the weight-low plane (the aligned pair of
// entries holding the source pixel's) and KT 8-byte records {r, g, b, w_hi}.
template <int KT, bool F16>
struct Hist {
  static constexpr int kW = 0;
  static constexpr int kP = kW + 4 * kThreads;
  static constexpr int kKey = kP + 4 * kThreads;
  static constexpr int kIdx = kKey + 4 * KT * kThreads;
  static constexpr int kWt = kIdx + 4 * KT * kThreads;               // FP16 only
  static constexpr int kRec = F16 ? kWt + 4 * KT * kThreads : kWt;   // 16-byte aligned
  static constexpr int kBytes = kRec + (F16 ? 8 : 16) * KT * kThreads;
};

// The key race for one pixel whose history the thread gathers into its
// column of shared memory with asynchronous copies: the copies of the whole
// source reservoir are issued at once, the uniform, weight and key are
// computed while they fly, and the update then reads the history from shared
// memory. The arithmetic is the in-place update's, step for step
// (push_group): Eq. (full-temporal-bias) factor from the history's resolved
// colour, Eq. (temporal-bias), the key race, the fused resolve, then every
// slot written to the other buffer. KT >= K bounds the staging.
template <int KT, bool F16, bool FOV>
__device__ __forceinline__ int reproject_keys(const StreamDev& cur, const StreamDev& prev,
                                              const FrameDev& f, const ReprojDev& r, int64_t p,
                                              float d_f, uint8_t* smem) {
  using namespace wrs;
  using H = Hist<KT, F16>;
  const int K = cur.K;
  const int64_t pl = cur.plane;
  const int tid = threadIdx.x;
  float* sW = reinterpret_cast<float*>(smem + H::kW) + tid;
  float* sP = reinterpret_cast<float*>(smem + H::kP) + tid;
  float* sKey = reinterpret_cast<float*>(smem + H::kKey) + tid;
  uint32_t* sIdx = reinterpret_cast<uint32_t*>(smem + H::kIdx) + tid;
  uint32_t* sWt = reinterpret_cast<uint32_t*>(smem + H::kWt) + tid;
  uint8_t* sRec = smem + H::kRec + (F16 ? 8 : 16) * tid;
  constexpr int kRecStride = (F16 ? 8 : 16) * kThreads;

  int y, x;
  row_col(cur, static_cast<int>(p), y, x);
  const float dp = r.depth != nullptr ? r.depth[p] : 0.0f;
  bool ok;
  const int64_t q = source_pixel(cur, r, p, x, y, dp, ok);
  if (!WRS_IN(cur, q >= 0 && q < cur.hw && p < cur.hw && y < cur.height && x < cur.width &&
                       static_cast<int64_t>(y) * cur.width + x == p,
              kChkGather))
    return 0;
  cp_async4(sW, prev.W + q);
  cp_async4(sP, prev.P + q);
  for (int j = 0; j < K; ++j) {
    cp_async4(sKey + j * kThreads, prev.key + j * pl + q);
    cp_async4(sIdx + j * kThreads, prev.idx + j * pl + q);
    if constexpr (F16) {
      // 2-byte entries: copy the 4-byte pair holding q's (in the plane: its length is even)
      cp_async4(sWt + j * kThreads, prev.wt + j * pl + (q & ~static_cast<int64_t>(1)));
      cp_async8(sRec + j * kRecStride, static_cast<const uint2*>(prev.col) + j * pl + q);
    } else {
      cp_async16(sRec + j * kRecStride, static_cast<const float4*>(prev.col) + j * pl + q);
    }
  }

  const float* fp = f.frame + static_cast<int64_t>(y) * f.pitch + 3 * x;
  float rgb[3] = {fp[0], fp[1], fp[2]};
  bool flush = (FOV && f.fov[p] == 0xFFu) || !ok;
  const uint4 blk = philox4x32_10(make_uint4(static_cast<uint32_t>(p) >> 2, f.t, cur.stream_id, 0u),
                                  cur.seed_lo, cur.seed_hi);
  const float u = unit_uniform(word(blk, static_cast<int>(p) & 3));
  const float w = pixel_weight(cur, d_f, x, y, f.gx, f.gy);
  const float k = fdiv(-log_pos(u), w);
  cp_async_wait_all();

  // slot j of the gathered history, from this thread's column
  const int lo_shift = 16 * static_cast<int>(q & 1);  // q's half of each weight-low pair
  auto slot = [&](int j, float& a, float& cr, float& cg, float& cb) {
    if constexpr (F16) {
      const uint2 v = *reinterpret_cast<const uint2*>(sRec + j * kRecStride);
      a = slot_weight_f16(v.y, sWt[j * kThreads] >> lo_shift);
      cr = __half2float(__ushort_as_half(static_cast<unsigned short>(v.x & 0xffffu)));
      cg = __half2float(__ushort_as_half(static_cast<unsigned short>(v.x >> 16)));
      cb = __half2float(__ushort_as_half(static_cast<unsigned short>(v.y & 0xffffu)));
    } else {
      const float4 v = *reinterpret_cast<const float4*>(sRec + j * kRecStride);
      a = v.x; cr = v.y; cg = v.z; cb = v.w;
    }
  };

  float W = *sW, P = *sP;
  float gl = 1.0f;
  if (cur.bias == 2) {
    float n0 = 0.0f, n1 = 0.0f, n2 = 0.0f, dn = 0.0f;
    for (int j = 0; j < K; ++j) {
      float a, cr, cg, cb;
      slot(j, a, cr, cg, cb);
      n0 = __fmaf_rn(a, cr, n0);
      n1 = __fmaf_rn(a, cg, n1);
      n2 = __fmaf_rn(a, cb, n2);
      dn = fadd(dn, a);
    }
    if (!flush && W > 0.0f) {
      gl = lightness_factor(n0, n1, n2, dn, rgb);
      if (gl <= 0.0f) flush = true;
    }
  }
  if (flush) { W = 0.0f; P = 1.0f; }
  bool rescale;
  const float ks = bias_and_sum(cur.bias, w, k, W, P, rescale, gl);

  float kmax = -1.0f;
  int jm = 0;
  for (int j = 0; j < K; ++j) {
    const float kj = race_key(sKey[j * kThreads], flush, rescale);
    if (kj > kmax) { kmax = kj; jm = j; }
  }
  const bool repl = ks < kmax;
  const float c0 = stored_colour<F16>(rgb[0]), c1 = stored_colour<F16>(rgb[1]),
              c2 = stored_colour<F16>(rgb[2]);

  if (f.out != nullptr) {
    float n0 = 0.0f, n1 = 0.0f, n2 = 0.0f, dn = 0.0f;
    for (int j = 0; j < K; ++j) {
      float aa, rr, gg, bb;
      slot(j, aa, rr, gg, bb);
      if (flush) { aa = 0.0f; rr = gg = bb = 0.0f; }
      if (repl && jm == j) { aa = w; rr = c0; gg = c1; bb = c2; }
      n0 = __fmaf_rn(aa, rr, n0);
      n1 = __fmaf_rn(aa, gg, n1);
      n2 = __fmaf_rn(aa, bb, n2);
      dn = fadd(dn, aa);
    }
    const float inv = dn > 0.0f ? __frcp_rn(dn) : 0.0f;
    float* o = f.out + p * 3;
    o[0] = fmul(n0, inv);
    o[1] = fmul(n1, inv);
    o[2] = fmul(n2, inv);
  }

  cur.W[p] = W;
  cur.P[p] = P;
  for (int j = 0; j < K; ++j) {
    if (repl && j == jm) {
      cur.key[j * pl + p] = ks;
      cur.idx[j * pl + p] = f.t;
      store_slot<F16>(cur.wt, cur.col, K, j, pl, p, w, rgb[0], rgb[1], rgb[2]);
    } else if (flush) {
      cur.key[j * pl + p] = kInf;
      cur.idx[j * pl + p] = kEmpty;
      store_slot<F16>(cur.wt, cur.col, K, j, pl, p, 0.0f, 0.0f, 0.0f, 0.0f);
    } else {
      float kj = sKey[j * kThreads];
      if (rescale && kj != kInf) kj = fminf(fmul(kj, kPScale), kFltMax);
      cur.key[j * pl + p] = kj;
      cur.idx[j * pl + p] = sIdx[j * kThreads];
      if constexpr (F16) {
        // the record moves unchanged; the low half of its weight beside it
        cur.wt[j * pl + p] = static_cast<uint16_t>(sWt[j * kThreads] >> lo_shift);
        static_cast<uint2*>(cur.col)[j * pl + p] =
            *reinterpret_cast<const uint2*>(sRec + j * kRecStride);
      } else {
        static_cast<float4*>(cur.col)[j * pl + p] =
            *reinterpret_cast<const float4*>(sRec + j * kRecStride);
      }
    }
  }
  return repl ? 1 : 0;
}

// The literal n = 1 rule (Alg. 2 with Eq. (temporal-bias)) for one pixel with
// its gathered history, step for step as push_group_literal; the key and bias
// planes are neither read nor written.
template <bool F16, bool FOV>
__device__ __forceinline__ int reproject_literal(const StreamDev& cur, const StreamDev& prev,
                                                 const FrameDev& f, const ReprojDev& r, int64_t p,
                                                 float d_f) {
  using namespace wrs;
  const int64_t pl = cur.plane;
  int y, x;
  row_col(cur, static_cast<int>(p), y, x);
  const float* fp = f.frame + static_cast<int64_t>(y) * f.pitch + 3 * x;
  float rgb[3] = {fp[0], fp[1], fp[2]};
  const float dp = r.depth != nullptr ? r.depth[p] : 0.0f;
  bool flush = FOV && f.fov[p] == 0xFFu;
  const uint4 blk = philox4x32_10(make_uint4(static_cast<uint32_t>(p) >> 2, f.t, cur.stream_id, 0u),
                                  cur.seed_lo, cur.seed_hi);
  const float u = unit_uniform(word(blk, static_cast<int>(p) & 3));
  const float w = pixel_weight(cur, d_f, x, y, f.gx, f.gy);

  bool ok;
  const int64_t q = source_pixel(cur, r, p, x, y, dp, ok);
  if (!WRS_IN(cur, q >= 0 && q < cur.hw && p < cur.hw && y < cur.height && x < cur.width &&
                       static_cast<int64_t>(y) * cur.width + x == p,
              kChkGather))
    return 0;
  float W = prev.W[q];
  const uint32_t id0 = prev.idx[q];
  float a1[1], r1[1], g1[1], b1[1];
  load_slot<F16, 1>(prev.wt, prev.col, 1, 0, pl, q, a1, r1, g1, b1);
  flush = flush || !ok;

  float gl = 1.0f;
  if (cur.bias == 2 && !flush && W > 0.0f) {
    gl = lightness_factor(__fmaf_rn(a1[0], r1[0], 0.0f), __fmaf_rn(a1[0], g1[0], 0.0f),
                          __fmaf_rn(a1[0], b1[0], 0.0f), fadd(0.0f, a1[0]), rgb);
    if (gl <= 0.0f) flush = true;
  }
  if (flush) W = 0.0f;
  if (cur.bias && W > 0.0f) {
    float fb = fdiv(W, fadd(W, w));
    if (cur.bias == 2) fb = fmul(fb, gl);
    W = fmul(W, fb);
  }
  const float tot = fadd(W, w);
  const bool take = !(fmul(u, tot) <= W);  // Alg. 2: R1 kept on <=
  W = tot;

  if (f.out != nullptr) {
    float aa = a1[0], rr = r1[0], gg = g1[0], bb = b1[0];
    if (take) {
      aa = w;
      rr = stored_colour<F16>(rgb[0]);
      gg = stored_colour<F16>(rgb[1]);
      bb = stored_colour<F16>(rgb[2]);
    }
    const float n0 = __fmaf_rn(aa, rr, 0.0f), n1 = __fmaf_rn(aa, gg, 0.0f),
                n2 = __fmaf_rn(aa, bb, 0.0f);
    const float den = fadd(0.0f, aa);
    const float inv = den > 0.0f ? __frcp_rn(den) : 0.0f;
    float* o = f.out + p * 3;
    o[0] = fmul(n0, inv);
    o[1] = fmul(n1, inv);
    o[2] = fmul(n2, inv);
  }
  cur.W[p] = W;
  if (take) {
    cur.idx[p] = f.t;
    store_slot<F16>(cur.wt, cur.col, 1, 0, pl, p, w, rgb[0], rgb[1], rgb[2]);
  } else {
    cur.idx[p] = id0;
    store_slot<F16>(cur.wt, cur.col, 1, 0, pl, p, a1[0], r1[0], g1[0], b1[0]);
  }
  return take ? 1 : 0;
}

// KT > 0: the key race with K <= KT slots, histories staged in dynamic
// shared memory (Hist<KT, F16>::kBytes); KT == 0: the literal rule.
template <int KT, bool F16, bool FOV>
__global__ void __launch_bounds__(kThreads) reproject_kernel(const __grid_constant__ StreamDev cur,
                                                             const __grid_constant__ StreamDev prev,
                                                             const __grid_constant__ FrameDev f,
                                                             const __grid_constant__ ReprojDev r) {
  extern __shared__ __align__(16) uint8_t hist_smem[];
  __shared__ unsigned block_replaced;
  if (threadIdx.x == 0) block_replaced = 0;
  __syncthreads();
  const float d_f = wrs::fovea_density(cur);
  int replaced = 0;
  for (int64_t p = blockIdx.x * static_cast<int64_t>(kThreads) + threadIdx.x; p < cur.hw;
       p += static_cast<int64_t>(gridDim.x) * kThreads) {
    if constexpr (KT == 0)
      replaced += reproject_literal<F16, FOV>(cur, prev, f, r, p, d_f);
    else
      replaced += reproject_keys<KT, F16, FOV>(cur, prev, f, r, p, d_f, hist_smem);
  }
  const unsigned c = __reduce_add_sync(0xffffffffu, static_cast<unsigned>(replaced));
  if ((threadIdx.x & 31) == 0 && c != 0) atomicAdd(&block_replaced, c);
  __syncthreads();
  if (threadIdx.x == 0 && block_replaced != 0)
    atomicAdd(cur.replacements, static_cast<unsigned long long>(block_replaced));
}

bool aligned(const void* p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

template <int KT, bool F16, bool FOV>
cudaError_t launch_fov(unsigned grid, cudaStream_t st, const StreamDev& cur, const StreamDev& prev,
                       const FrameDev& f, const ReprojDev& r) {
  const size_t smem = KT > 0 ? Hist<(KT > 0 ? KT : 1), F16>::kBytes : 0;
  if (smem > 48 * 1024) {
    // per instantiation and device: allow the staging once
    static bool configured[64] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    if (!configured[dev]) {
      e = cudaFuncSetAttribute(reproject_kernel<KT, F16, FOV>,
                               cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
      if (e != cudaSuccess) return e;
      configured[dev] = true;
    }
  }
  reproject_kernel<KT, F16, FOV><<<grid, kThreads, smem, st>>>(cur, prev, f, r);
  return cudaGetLastError();
}

template <int KT, bool F16>
cudaError_t launch(bool fov, unsigned grid, cudaStream_t st, const StreamDev& cur,
                   const StreamDev& prev, const FrameDev& f, const ReprojDev& r) {
  return fov ? launch_fov<KT, F16, true>(grid, st, cur, prev, f, r)
             : launch_fov<KT, F16, false>(grid, st, cur, prev, f, r);
}

template <bool F16>
cudaError_t launch_k(int K, bool lit, bool fov, unsigned grid, cudaStream_t st,
                     const StreamDev& cur, const StreamDev& prev, const FrameDev& f,
                     const ReprojDev& r) {
  if (lit) return launch<0, F16>(fov, grid, st, cur, prev, f, r);
  if (K <= 4) return launch<4, F16>(fov, grid, st, cur, prev, f, r);
  if (K <= 8) return launch<8, F16>(fov, grid, st, cur, prev, f, r);
  return launch<16, F16>(fov, grid, st, cur, prev, f, r);
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
      cudaError_t e = cudaMemcpyAsync(x->state + hdr, x->planes + hdr, x->lay.map_off - hdr,
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
    cudaError_t e = cudaMemcpyAsync(x->state + hdr, x->planes + hdr, x->lay.map_off - hdr,
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
  if (int rc = wrs_require_usable(x)) return rc;
  if (x->t == 0xFFFFFFFFu) return wrs_fail(WRS_ERR_STATE, "frame counter exhausted");

  const cudaStream_t st = static_cast<cudaStream_t>(stream);
  // the gather copies whole reservoirs, sample indices included: complete them
  cudaError_t e = wrs_fold_all(x, st);
  if (e != cudaSuccess) return wrs_cuda_fail(e, "wrs_push_frame_reproject: fold");
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
  f.map_lo = x->t;  // unused: a reprojected push writes every sample index itself
  ReprojDev r;
  r.motion = reinterpret_cast<const float2*>(d_motion);
  r.depth = d_depth;
  r.prev_depth = d_prev_depth;
  r.tol = depth_tol;

  const int64_t hw = static_cast<int64_t>(x->cfg.width) * x->cfg.height;
  const int64_t want = (hw + kThreads - 1) / kThreads;
  const int64_t cap = static_cast<int64_t>(x->sms) * 8 * 16;
  const unsigned grid = static_cast<unsigned>(want < cap ? want : cap);
  const bool f16 = x->cfg.color_fp16 != 0;
  const bool lit = x->cfg.update_rule == WRS_RULE_LITERAL;
  const bool fov = d_fov != nullptr;
  e = f16 ? launch_k<true>(x->cfg.K, lit, fov, grid, st, cur, prev, f, r)
          : launch_k<false>(x->cfg.K, lit, fov, grid, st, cur, prev, f, r);
  if (e != cudaSuccess) return wrs_cuda_fail(e, "wrs_push_frame_reproject: launch");
  x->planes = dst_planes;
  x->t += 1;
  x->base = x->t;  // every index of the new planes is written
  return WRS_OK;
}
