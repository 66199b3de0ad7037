// Bulk asynchronous copies and transaction-count barriers (sm_90+ PTX, used on
// sm_103a), and the tile pipeline shared by the single-stream and batched
// persistent kernels.
#pragma once

#include <stdint.h>

#include "wrs_device.cuh"

namespace wrs {

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
static __device__ __noinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, uint64_t limit_ns) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = global_ns();
  for (;;) {
    if (mbar_try_wait(bar, parity)) return true;
    if (global_ns() - t0 > limit_ns) return false;
  }
}

// Byte offsets of one stage's planes in shared memory (tile of T pixels).
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

// Warp-wide: lane 0 arms `bar` for the tile's bytes (plus extra_tx, which is
// non-zero only to test the timeout path), then the lanes issue one bulk copy
// per plane segment. The tile starts at pixel p0 (a multiple of T >= 256);
// requires frame rows without padding, width % 4 == 0 and 16-byte aligned
// frame and state planes.
template <int T>
__device__ __forceinline__ void issue_tile_copies(const StreamDev& s, const FrameDev& f, int K,
                                                  int cs, bool resolve, const StageLayout& L,
                                                  uint8_t* stage, uint64_t* bar, int64_t p0,
                                                  uint32_t extra_tx, int lane) {
  const int64_t rem_plane = s.plane - p0, rem_px = s.hw - p0;
  const uint32_t n = static_cast<uint32_t>(rem_plane < T ? rem_plane : T);  // plane entries (x64)
  const uint32_t np = static_cast<uint32_t>(rem_px < T ? rem_px : T);       // pixels (x4)
  const int ncopy = 3 + K + (resolve ? 4 * K : 0);
  if (lane == 0) {
    uint32_t bytes = 12u * np + 8u * n + 4u * K * n;
    if (resolve) bytes += 4u * K * n + static_cast<uint32_t>(cs) * 3u * K * n;
    mbar_arrive_expect_tx(bar, bytes + extra_tx);
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
      const uint8_t* src =
          static_cast<const uint8_t*>(s.col) + static_cast<int64_t>(cs) * (m * pl + p0);
      bulk_g2s(stage + L.col + static_cast<uint32_t>(cs) * T * m, src, cs * n, bar);
    }
  }
}

// The tile's uniforms: one Philox block per 4 pixels, written to u[0 .. T-1].
// Threads tid < T/4 each draw one block.
template <int T>
__device__ __forceinline__ void draw_tile_uniforms(const StreamDev& s, const FrameDev& f,
                                                   int64_t p0, float* u, int tid) {
  if (tid < T / 4) {
    const uint32_t q = static_cast<uint32_t>((p0 >> 2) + tid);
    const uint4 b = philox4x32_10(make_uint4(q, f.t, s.stream_id, 0u), s.seed_lo, s.seed_hi);
    float4 v;
    v.x = unit_uniform(b.x);
    v.y = unit_uniform(b.y);
    v.z = unit_uniform(b.z);
    v.w = unit_uniform(b.w);
    reinterpret_cast<float4*>(u)[tid] = v;
  }
}

// Computes the thread's PX pixels of a landed tile from shared memory.
template <int KT, bool F16, int PX, int T>
__device__ __forceinline__ void compute_tile(const StreamDev& s, const FrameDev& f,
                                             const StageLayout& L, const uint8_t* st,
                                             const float* u, int64_t p0, float d_f, int tid) {
  const int tl = tid * PX;
  const int64_t p = p0 + tl;
  if (p >= s.hw) return;
  Src src;
  src.W = reinterpret_cast<const float*>(st + L.W);
  src.P = reinterpret_cast<const float*>(st + L.P);
  src.key = reinterpret_cast<const float*>(st + L.key);
  src.wt = reinterpret_cast<const float*>(st + L.wt);
  src.col = st + L.col;
  src.stride = T;
  src.at = tl;
  src.frame = reinterpret_cast<const float*>(st + L.frame) + 3 * tl;
  src.u = u + tl;
  if (f.fov != nullptr)
    push_group<KT, F16, PX, true, true>(s, f, static_cast<int>(p), src, d_f);
  else
    push_group<KT, F16, PX, true, false>(s, f, static_cast<int>(p), src, d_f);
}

}  // namespace wrs
