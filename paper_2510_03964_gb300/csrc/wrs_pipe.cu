// Pipelined persistent form of the fused update + resolve (sm_103a).
//
// One CTA per SM walks the image in tiles of T = 256 * PX pixels. Warp 0
// streams the planes a tile needs (frame RGB, W, P, the K key planes and, for
// the fused resolve, the K weight and 3K colour planes) into a ring of S
// shared-memory stages with 1-D bulk asynchronous copies (cp.async.bulk)
// that complete on one transaction-count mbarrier per stage, while all 256
// threads compute the previous tile from shared memory. Writes go straight to
// global memory. The per-pixel arithmetic is push_group, the same code as the
// plain kernel, so results are bit-identical.
//
// Every wait is bounded by %globaltimer. A wait that runs out records
// WRS_ERR_TIMEOUT in the stream's status word, waits (again bounded) for the
// copies this CTA still has in flight, and returns; the host reads the word
// with wrs_check_status.
#include <cuda_runtime.h>

#include "wrs.h"
#include "wrs_device.cuh"
#include "wrs_internal.h"

using wrs::FrameDev;
using wrs::StreamDev;

namespace {

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
               : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}

// global -> shared bulk copy of `bytes` (multiple of 16, both addresses 16-byte
// aligned), completing `bytes` transactions on `bar`
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes,
                                         uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
          "r"(smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Waits for phase `parity` of `bar` to complete; false once limit_ns has passed.
__device__ __noinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, uint64_t limit_ns) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = global_ns();
  for (;;) {
    if (mbar_try_wait(bar, parity)) return true;
    if (global_ns() - t0 > limit_ns) return false;
  }
}

// Byte offsets of one stage's planes in shared memory.
struct StageLayout {
  uint32_t frame, W, P, key, wt, col, bytes;
};

__host__ __device__ __forceinline__ StageLayout stage_layout(int T, int K, int cs, bool resolve) {
  StageLayout L;
  L.frame = 0;
  L.W = 12u * T;
  L.P = L.W + 4u * T;
  L.key = L.P + 4u * T;
  L.wt = L.key + 4u * K * T;
  L.col = L.wt + (resolve ? 4u * K * T : 0u);
  L.bytes = L.col + (resolve ? static_cast<uint32_t>(cs) * 3u * K * T : 0u);
  return L;
}

struct PipeArgs {
  int stages;
  int ntiles;
  int resolve;             // copy weight/colour planes (f.out != null)
  uint32_t* status;        // stream status word (WRS_OK or WRS_ERR_TIMEOUT)
  uint64_t timeout_ns;
  uint32_t extra_tx;       // added to the expected bytes: > 0 only to test the timeout path
};

template <int KT, bool F16, int PX>
__device__ __forceinline__ void issue_tile(const StreamDev& s, const FrameDev& f,
                                           const PipeArgs& a, const StageLayout& L,
                                           uint8_t* stage, uint64_t* bar, int tile, int lane) {
  constexpr int T = 256 * PX;
  constexpr int cs = F16 ? 2 : 4;
  const int K = KT > 0 ? KT : s.K;
  const int64_t p0 = static_cast<int64_t>(tile) * T;
  const int64_t rem_plane = s.plane - p0, rem_px = s.hw - p0;
  const uint32_t n = static_cast<uint32_t>(rem_plane < T ? rem_plane : T);  // plane entries (x64)
  const uint32_t np = static_cast<uint32_t>(rem_px < T ? rem_px : T);       // pixels (x4)
  const int ncopy = 3 + K + (a.resolve ? 4 * K : 0);
  if (lane == 0) {
    uint32_t bytes = 12u * np + 8u * n + 4u * K * n;
    if (a.resolve) bytes += 4u * K * n + static_cast<uint32_t>(cs) * 3u * K * n;
    mbar_arrive_expect_tx(bar, bytes + a.extra_tx);
  }
  __syncwarp();
  const int64_t pl = s.plane;
  for (int c = lane; c < ncopy; c += 32) {
    if (c == 0) {
      bulk_g2s(stage + L.frame, f.frame + 3 * p0, 12u * np, bar);
    } else if (c == 1) {
      bulk_g2s(stage + L.W, s.W + p0, 4u * n, bar);
    } else if (c == 2) {
      bulk_g2s(stage + L.P, s.P + p0, 4u * n, bar);
    } else if (c < 3 + K) {
      const int j = c - 3;
      bulk_g2s(stage + L.key + 4u * T * j, s.key + j * pl + p0, 4u * n, bar);
    } else if (c < 3 + 2 * K) {
      const int j = c - 3 - K;
      bulk_g2s(stage + L.wt + 4u * T * j, s.wt + j * pl + p0, 4u * n, bar);
    } else {
      const int m = c - 3 - 2 * K;  // channel * K + slot
      const uint8_t* src = static_cast<const uint8_t*>(s.col) + static_cast<int64_t>(cs) * (m * pl + p0);
      bulk_g2s(stage + L.col + static_cast<uint32_t>(cs) * T * m, src, cs * n, bar);
    }
  }
}

template <int KT, bool F16, int PX>
__global__ void __launch_bounds__(256, 1)
    pipe_kernel(const __grid_constant__ StreamDev s, const __grid_constant__ FrameDev f,
                const PipeArgs a) {
  extern __shared__ __align__(128) uint8_t smem[];
  constexpr int T = 256 * PX;
  constexpr int cs = F16 ? 2 : 4;
  const int K = KT > 0 ? KT : s.K;
  const int S = a.stages;
  const StageLayout L = stage_layout(T, K, cs, a.resolve != 0);
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + S * L.bytes);
  const int tid = threadIdx.x;
  const int lane = tid & 31;

  if (tid == 0) {
    for (int i = 0; i < S; ++i) mbar_init(&bars[i], 1);
    fence_mbar_init();
  }
  __syncthreads();

  const int first = blockIdx.x;
  const int step = gridDim.x;
  const int my_tiles = first < a.ntiles ? (a.ntiles - 1 - first) / step + 1 : 0;
  const int prologue = min(S - 1, my_tiles);
  if (tid < 32)
    for (int it = 0; it < prologue; ++it)
      issue_tile<KT, F16, PX>(s, f, a, L, smem + (it % S) * L.bytes, &bars[it % S],
                              first + it * step, lane);

  const float d_f = wrs::fovea_density(s);
  int it = 0;
  bool ok = true;
  for (; it < my_tiles; ++it) {
    const int nxt = it + S - 1;
    if (tid < 32 && nxt < my_tiles)
      issue_tile<KT, F16, PX>(s, f, a, L, smem + (nxt % S) * L.bytes, &bars[nxt % S],
                              first + nxt * step, lane);
    const int stg = it % S;
    // every thread waits; the block then agrees on the outcome, so that no
    // thread leaves the loop while others wait at the barrier below
    const bool landed = mbar_wait_bounded(&bars[stg], (it / S) & 1u, a.timeout_ns);
    if (!__syncthreads_and(landed)) {
      ok = false;
      break;
    }
    uint8_t* st = smem + stg * L.bytes;
    const int tl = tid * PX;
    const int p = (first + it * step) * T + tl;
    if (p < s.hw) {
      wrs::Src src;
      src.W = reinterpret_cast<const float*>(st + L.W);
      src.P = reinterpret_cast<const float*>(st + L.P);
      src.key = reinterpret_cast<const float*>(st + L.key);
      src.wt = reinterpret_cast<const float*>(st + L.wt);
      src.col = st + L.col;
      src.stride = T;
      src.at = tl;
      src.frame = reinterpret_cast<const float*>(st + L.frame) + 3 * tl;
      wrs::push_group<KT, F16, PX, true>(s, f, p, src, d_f);
    }
    __syncthreads();
  }
  if (!ok) {
    // record the timeout, then let every copy this CTA issued land before the
    // shared memory is released: tiles it .. min(it + S - 1, my_tiles - 1)
    if (tid == 0) atomicExch(a.status, static_cast<uint32_t>(WRS_ERR_TIMEOUT));
    const int last = min(it + S, my_tiles);
    for (int j = it; j < last; ++j) mbar_wait_bounded(&bars[j % S], (j / S) & 1u, a.timeout_ns);
  }
}

template <int KT, bool F16, int PX>
cudaError_t launch_pipe_t(const StreamDev& s, const FrameDev& f, PipeArgs a, int sms,
                          cudaStream_t st) {
  constexpr int T = 256 * PX;
  const StageLayout L = stage_layout(T, s.K, F16 ? 2 : 4, a.resolve != 0);
  const size_t smem = static_cast<size_t>(a.stages) * L.bytes + 8 * a.stages;
  // per instantiation and device: the largest dynamic shared memory already allowed
  static size_t configured[64] = {};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  if (smem > configured[dev]) {
    e = cudaFuncSetAttribute(pipe_kernel<KT, F16, PX>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             static_cast<int>(smem));
    if (e != cudaSuccess) return e;
    configured[dev] = smem;
  }
  a.ntiles = static_cast<int>((static_cast<int64_t>(s.hw) + T - 1) / T);
  const int grid = a.ntiles < sms ? a.ntiles : sms;
  pipe_kernel<KT, F16, PX><<<grid, 256, smem, st>>>(s, f, a);
  return cudaGetLastError();
}

template <int KT, bool F16>
cudaError_t launch_pipe_px(const StreamDev& s, const FrameDev& f, const PipeArgs& a, int px,
                           int sms, cudaStream_t st) {
  switch (px) {
    case 4: return launch_pipe_t<KT, F16, 4>(s, f, a, sms, st);
    case 2: return launch_pipe_t<KT, F16, 2>(s, f, a, sms, st);
    default: return launch_pipe_t<KT, F16, 1>(s, f, a, sms, st);
  }
}

template <bool F16>
cudaError_t launch_pipe_k(const StreamDev& s, const FrameDev& f, const PipeArgs& a, int px,
                          int sms, cudaStream_t st) {
  switch (s.K) {
    case 1: return launch_pipe_px<1, F16>(s, f, a, px, sms, st);
    case 2: return launch_pipe_px<2, F16>(s, f, a, px, sms, st);
    case 4: return launch_pipe_px<4, F16>(s, f, a, px, sms, st);
    case 8: return launch_pipe_px<8, F16>(s, f, a, px, sms, st);
    default: return launch_pipe_px<0, F16>(s, f, a, px, sms, st);
  }
}

}  // namespace

// Shared memory one stage of the pipelined kernel needs.
size_t wrs_pipe_stage_bytes(int K, bool f16, int px, bool resolve) {
  return stage_layout(256 * px, K, f16 ? 2 : 4, resolve).bytes;
}

bool wrs_pipe_supported(const wrs_ctx* x, const float* frame, int64_t pitch, const float* out) {
  const auto al = [](const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; };
  return x->cfg.width % 4 == 0 && pitch == 3 * static_cast<int64_t>(x->cfg.width) && al(frame) &&
         (out == nullptr || al(out));
}

cudaError_t wrs_launch_pipe(const StreamDev& s, const FrameDev& f, bool f16, int px, int stages,
                            int sms, uint32_t* status, uint64_t timeout_ns, uint32_t extra_tx,
                            cudaStream_t st) {
  PipeArgs a;
  a.stages = stages;
  a.ntiles = 0;
  a.resolve = f.out != nullptr ? 1 : 0;
  a.status = status;
  a.timeout_ns = timeout_ns;
  a.extra_tx = extra_tx;
  return f16 ? launch_pipe_k<true>(s, f, a, px, sms, st) : launch_pipe_k<false>(s, f, a, px, sms, st);
}
