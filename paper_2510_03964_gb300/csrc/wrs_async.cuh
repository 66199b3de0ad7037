// Bulk asynchronous copies and transaction-count barriers (sm_90+ PTX, used on
// sm_103a), and the tile pipeline shared by the single-stream and batched
// persistent kernels.
#pragma once

#include <stdint.h>

#include "wrs_device.cuh"
#include "wrs_fov.cuh"

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

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
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
// cs = 2 (FP16 colour: K planes of the weights' low 16 bits, then K planes of
// 8-byte records {r, g, b, w_hi}) or 4 (FP32 colour: K float4 {w, r, g, b}
// record planes, starting at `col`; `wt` == `col`).
struct StageLayout {
  uint32_t frame, W, P, key, wt, col, bytes;
};

__host__ __device__ __forceinline__ StageLayout stage_layout(int T, int K, int cs, bool resolve) {
  StageLayout L;
  L.frame = 0;
  L.W = 12u * T;
  L.P = L.W + 4u * T;
  L.key = L.P + 4u * T;
  if (cs == 2) {
    L.wt = L.key + 4u * K * T;
    L.col = L.wt + (resolve ? 2u * K * T : 0u);
    L.bytes = L.col + (resolve ? 8u * K * T : 0u);
  } else {
    L.wt = L.col = L.key + 4u * K * T;
    L.bytes = L.col + (resolve ? 16u * K * T : 0u);
  }
  return L;
}

// Warp-wide: lane 0 arms `bar` for the tile's bytes (plus extra_tx, which is
// non-zero only to test the timeout path), then the lanes issue one bulk copy
// per plane segment. The tile starts at pixel p0 (a multiple of T >= 256);
// requires frame rows without padding, width % 4 == 0 and 16-byte aligned
// frame and state planes. copy_frame = false leaves the frame segment to the
// consumers (they foveate the frame into it themselves).
template <int T>
__device__ __forceinline__ void issue_tile_copies(const StreamDev& s, const FrameDev& f, int K,
                                                  int cs, bool resolve, const StageLayout& L,
                                                  uint8_t* stage, uint64_t* bar, int64_t p0,
                                                  uint32_t extra_tx, int lane,
                                                  bool copy_frame = true,
                                                  uint32_t stage_cap = 0xFFFFFFFFu) {
  const int64_t rem_plane = s.plane - p0, rem_px = s.hw - p0;
  const uint32_t n = static_cast<uint32_t>(rem_plane < T ? rem_plane : T);  // plane entries (x64)
  const uint32_t np = static_cast<uint32_t>(rem_px < T ? rem_px : T);       // pixels (x4)
#ifdef WRS_CHECKED
  // every copy's global range inside its plane or the frame, and the stage's
  // layout inside the ring's stage; otherwise no copy is issued and the
  // barrier completes empty (the consumers then compute stale data, flagged)
  {
    bool ok = WRS_IN(s, p0 >= 0 && p0 < s.hw && p0 + n <= s.plane && p0 + np <= s.hw &&
                            n % 64 == 0 && np % 4 == 0 && K >= 1 && K <= WRS_MAX_K,
                     kChkCopy);
    ok = WRS_IN(s, L.bytes <= stage_cap, kChkStageSize) && ok;
    if (!ok) {
      if (lane == 0) mbar_arrive_expect_tx(bar, 0u);
      __syncwarp();
      return;
    }
  }
#else
  (void)stage_cap;
#endif
  // the literal rule (K = 1) reads no P and no key plane: copies 2 and 3 are skipped
  const int skip = s.literal ? 2 : 0;
  const int ncopy = 3 + K + (resolve ? (cs == 2 ? 2 * K : K) : 0);
  if (lane == 0) {
    uint32_t bytes = (copy_frame ? 12u * np : 0u) + 8u * n + 4u * K * n;
    if (skip) bytes -= 4u * n + 4u * K * n;
    if (resolve) bytes += cs == 2 ? (2u * K * n + 8u * K * n) : 16u * K * n;
    mbar_arrive_expect_tx(bar, bytes + extra_tx);
  }
  __syncwarp();
  const int64_t pl = s.plane;
  for (int c = lane; c < ncopy; c += 32) {
    if (skip && (c == 2 || c == 3)) continue;
    if (c == 0 && !copy_frame) continue;
    if (c == 0) {
      bulk_g2s(stage + L.frame, f.frame + 3 * p0, 12u * np, bar);
    } else if (c == 1) {
      bulk_g2s(stage + L.W, s.W + p0, 4u * n, bar);
    } else if (c == 2) {
      bulk_g2s(stage + L.P, s.P + p0, 4u * n, bar);
    } else if (c < 3 + K) {
      const int j = c - 3;
      bulk_g2s(stage + L.key + 4u * T * j, s.key + j * pl + p0, 4u * n, bar);
    } else if (cs == 4) {
      const int j = c - 3 - K;  // FP32 colour: record plane j
      bulk_g2s(stage + L.col + 16u * T * j,
               static_cast<const float4*>(s.col) + j * pl + p0, 16u * n, bar);
    } else if (c < 3 + 2 * K) {
      const int j = c - 3 - K;
      bulk_g2s(stage + L.wt + 2u * T * j, s.wt + j * pl + p0, 2u * n, bar);
    } else {
      const int j = c - 3 - 2 * K;  // FP16 colour: record plane j
      bulk_g2s(stage + L.col + 8u * T * j, static_cast<const uint2*>(s.col) + j * pl + p0,
               8u * n, bar);
    }
  }
}

// The tile's uniforms, drawn by one warp: one Philox block per 4 pixels,
// written to u[0 .. T-1].
template <int T>
__device__ __forceinline__ void draw_tile_uniforms_warp(const StreamDev& s, const FrameDev& f,
                                                        int64_t p0, float* u, int lane) {
  for (int q = lane; q < T / 4; q += 32) {
    const uint32_t blk = static_cast<uint32_t>((p0 >> 2) + q);
    const uint4 b = philox4x32_10(make_uint4(blk, f.t, s.stream_id, 0u), s.seed_lo, s.seed_hi);
    float4 v;
    v.x = unit_uniform(b.x);
    v.y = unit_uniform(b.y);
    v.z = unit_uniform(b.z);
    v.w = unit_uniform(b.w);
    reinterpret_cast<float4*>(u)[q] = v;
  }
}

// Computes consumer thread `tid`'s PX pixels of a landed tile from shared
// memory; returns how many of them replaced a slot. LIT: the literal n = 1
// rule (KT = 1).
template <int KT, bool F16, int PX, int T, bool LIT = false, int KM = FoldCap<KT>::value>
__device__ __forceinline__ int compute_tile(const StreamDev& s, const FrameDev& f,
                                            const StageLayout& L, const uint8_t* st,
                                            const float* u, int64_t p0, float d_f, int tid,
                                            const FoldIn<KM>* pre = nullptr) {
  const int tl = tid * PX;
  const int64_t p = p0 + tl;
  if (p >= s.hw) return 0;
  Src src;
  src.W = reinterpret_cast<const float*>(st + L.W);
  src.P = reinterpret_cast<const float*>(st + L.P);
  src.key = reinterpret_cast<const float*>(st + L.key);
  src.wt = reinterpret_cast<const uint16_t*>(st + L.wt);
  src.col = st + L.col;
  src.stride = T;
  src.at = tl;
  src.frame = reinterpret_cast<const float*>(st + L.frame) + 3 * tl;
  src.u = u + tl;
  if constexpr (LIT) {
    if (f.fov != nullptr) return push_group_literal<F16, PX, true, true>(s, f, static_cast<int>(p), src, d_f);
    return push_group_literal<F16, PX, true, false>(s, f, static_cast<int>(p), src, d_f);
  } else {
    if (f.fov != nullptr) return push_group<KT, F16, PX, true, true, KM>(s, f, static_cast<int>(p), src, d_f, pre);
    return push_group<KT, F16, PX, true, false, KM>(s, f, static_cast<int>(p), src, d_f, pre);
  }
}

// Before a consumer waits for its tile: if the tile's pixel of thread `tid`
// (one pixel per thread) is in the band this frame folds, load the fold's
// inputs now, so that their latency passes while the tile is still in flight.
// Returns whether `in` was filled.
template <int KM, int PX>
__device__ __forceinline__ bool prefetch_fold(const StreamDev& s, const FrameDev& f, int64_t p0,
                                              int tid, FoldIn<KM>& in) {
  if constexpr (PX == 1) {
    const int64_t p = p0 + tid;
    if (s.K > 2 && s.K <= KM && p < s.hw && folds_now(f, p)) {
      fold_load(s, s.idx, s.K, f.t, p, in);
      return true;
    }
  }
  return false;
}

// Adds a warp's counts to a running total: one atomic per warp.
// As compute_tile, with the thread's PX pixels of the frame foveated from
// `fv` into the stage's frame segment first (the producer copied no frame);
// each thread writes and then reads only its own pixels there.
template <int KT, bool F16, int PX, int T, bool LIT, int FILTER, int KM = FoldCap<KT>::value>
__device__ __forceinline__ int compute_tile_fov(const StreamDev& s, const FrameDev& f,
                                                const FovDev& fv, const StageLayout& L,
                                                uint8_t* st, const float* u, int64_t p0,
                                                float d_f, int tid,
                                                const FoldIn<KM>* pre = nullptr) {
  const int tl = tid * PX;
  const int64_t p = p0 + tl;
  if (p >= s.hw) return 0;
  int y, x;
  row_col(s, static_cast<int>(p), y, x);
  float* fr = reinterpret_cast<float*>(st + L.frame) + 3 * tl;
#pragma unroll
  for (int i = 0; i < PX; ++i) fov_pixel<FILTER>(fv, f.gx, f.gy, x + i, y, fr + 3 * i);
  return compute_tile<KT, F16, PX, T, LIT, KM>(s, f, L, st, u, p0, d_f, tid, pre);
}

__device__ __forceinline__ void add_warp_count(unsigned long long* total, int count, int lane) {
  const unsigned c = __reduce_add_sync(0xffffffffu, static_cast<unsigned>(count));
  if (lane == 0 && c != 0) atomicAdd(total, static_cast<unsigned long long>(c));
}

// ---------------------------------------------------------------- warp-specialised loop

// Shared-memory ring of S stages, each holding one tile's planes followed by
// its uniforms, then the S "full" and S "empty" barriers and a flag word.
struct Ring {
  uint8_t* base;
  uint32_t stage_bytes;  // planes of the largest tile layout used
  uint32_t stride;       // stage_bytes + 4 * T
  int S;
  uint64_t* full;
  uint64_t* empty;
  int* flag;             // non-zero once some wait gave up

  __device__ uint8_t* stage(int i) const { return base + i * stride; }
  __device__ float* u(int i) const { return reinterpret_cast<float*>(base + i * stride + stage_bytes); }
};

__host__ __device__ __forceinline__ size_t ring_bytes(uint32_t stage_bytes, int T, int S) {
  return static_cast<size_t>(S) * (stage_bytes + 4u * T) + 16u * S + 16u;
}

__device__ __forceinline__ Ring make_ring(uint8_t* smem, uint32_t stage_bytes, int T, int S) {
  Ring r;
  r.base = smem;
  r.stage_bytes = stage_bytes;
  r.stride = stage_bytes + 4u * T;
  r.S = S;
  r.full = reinterpret_cast<uint64_t*>(smem + static_cast<size_t>(S) * r.stride);
  r.empty = r.full + S;
  r.flag = reinterpret_cast<int*>(r.empty + S);
  return r;
}

// Thread 0 initialises the barriers (full: one arrival, the producer's;
// empty: one arrival per consumer warp) and the flag; the caller then
// synchronises the block.
__device__ __forceinline__ void init_ring(const Ring& r, int consumer_warps) {
  for (int i = 0; i < r.S; ++i) {
    mbar_init(&r.full[i], 1);
    mbar_init(&r.empty[i], consumer_warps);
  }
  *r.flag = 0;
  fence_mbar_init();
}

__device__ __forceinline__ void raise_flag(const Ring& r) {
  atomicExch(r.flag, 1);
}

__device__ __forceinline__ bool flag_raised(const Ring& r) {
  return *reinterpret_cast<volatile int*>(r.flag) != 0;
}

// Producer warp: for each of its tiles, waits until the stage is free, draws
// the tile's uniforms into the stage, arms the stage's full barrier and
// issues the tile's copies. `tile_fn(it, stage, u, full_bar, lane)` does the
// drawing and the copies for iteration it. Returns the number of tiles issued.
template <typename TileFn>
__device__ __forceinline__ int produce(const Ring& r, int my_tiles, uint64_t timeout_ns, int lane,
                                       TileFn tile_fn) {
  int it = 0;
  for (; it < my_tiles; ++it) {
    const int stg = it % r.S;
    if (it >= r.S && !mbar_wait_bounded(&r.empty[stg], ((it / r.S) - 1) & 1u, timeout_ns)) {
      raise_flag(r);
      break;
    }
    if (flag_raised(r)) break;
    tile_fn(it, r.stage(stg), r.u(stg), &r.full[stg], lane);
  }
  return it;
}

// Consumer warp: for each tile, runs `before_fn(it)` (loads that need not
// wait for the stage), waits for its stage to land, computes it
// (`compute_fn(it, stage, u)`), and releases the stage.
template <typename BeforeFn, typename ComputeFn>
__device__ __forceinline__ void consume(const Ring& r, int my_tiles, uint64_t timeout_ns, int lane,
                                        BeforeFn before_fn, ComputeFn compute_fn) {
  for (int it = 0; it < my_tiles; ++it) {
    const int stg = it % r.S;
    before_fn(it);
    if (!mbar_wait_bounded(&r.full[stg], (it / r.S) & 1u, timeout_ns)) {
      raise_flag(r);
      break;
    }
    compute_fn(it, r.stage(stg), r.u(stg));
    __syncwarp();
    if (lane == 0) mbar_arrive(&r.empty[stg]);
  }
}

// After the loops (and a block barrier): if a wait gave up, the producer warp
// waits (bounded) on the full barriers of the last S tiles it issued, giving
// their copies time to land before the CTA exits. A barrier whose expected
// bytes can never all arrive (the test_extra_tx fault injection) does not
// complete even after its copies have landed, so there this wait only spends
// the limit once per stage: the guarantee then rests on the copies finishing
// within that time (they take microseconds; the limit is milliseconds), not on
// observing the barrier.
__device__ __forceinline__ void drain(const Ring& r, int issued, uint64_t timeout_ns) {
  const int from = issued > r.S ? issued - r.S : 0;
  for (int j = from; j < issued; ++j)
    mbar_wait_bounded(&r.full[j % r.S], (j / r.S) & 1u, timeout_ns);
}

}  // namespace wrs
