// The batched persistent kernel (template), shared by the translation unit of
// the plain batches (wrs_batch.cu, frames in memory) and that of the
// foveating batches (wrs_batch_fov.cu, frames foveated on read), which each
// instantiate their own variants.
#pragma once

#include <cuda_runtime.h>

#include "wrs.h"
#include "wrs_async.cuh"
#include "wrs_device.cuh"
#include "wrs_fov.cuh"

using wrs::FrameDev;
using wrs::StageLayout;
using wrs::StreamDev;

namespace {

constexpr int kMaxBatch = WRS_MAX_BATCH;

struct BatchEntry {
  StreamDev s;
  FrameDev f;
  wrs::FovDev fv;  // the stream's rendered image and mip levels (foveating batches only)
  uint32_t* status;
  int tile0;   // first global tile of this stream
  int code;    // arithmetic variant: 0 K=4 f16, 1 K=8 f16, 2 K=4 f32, 3 K=8 f32, 4 any K f16,
               // 5 any K f32, 6 literal f16, 7 literal f32
};

// The slot records are staged when the fused resolve needs them or the full
// temporal bias forms the history's resolved colour from them.
__device__ __forceinline__ bool stage_records(const BatchEntry& e) {
  return e.f.out != nullptr || e.s.bias == 2;
}

struct BatchArgs {
  int n;
  int ntiles;
  int stages;
  uint32_t stage_bytes;  // largest stage of any stream in the batch
  uint64_t timeout_ns;
  BatchEntry e[kMaxBatch];
};
// kernel parameters may take up to 32764 bytes on sm_70 and later (CUDA 12.1+)
static_assert(sizeof(BatchArgs) <= 32000, "batch descriptor too large for a kernel parameter");

// The entry (stream) of global tile g: the last entry with tile0 <= g. A CTA
// visits its tiles in ascending order, so each of its warps keeps the entry of
// its previous tile in `e` and moves it forward (a few steps per stream
// boundary instead of a search per tile).
__device__ __forceinline__ int entry_after(const BatchArgs& a, int g, int e) {
  while (e + 1 < a.n && a.e[e + 1].tile0 <= g) ++e;
  return e;
}

__device__ __forceinline__ bool entry_f16(const BatchEntry& e) {
  return e.code == 0 || e.code == 1 || e.code == 4 || e.code == 6;
}

constexpr int kConsumerWarps = 8;
constexpr int kBatchThreads = (kConsumerWarps + 1) * 32;

// Adds a warp's running count of replacements in entry ei to the CTA's
// per-stream total and clears it: once per stream a warp leaves, not per tile.
__device__ __forceinline__ void flush_count(unsigned long long* replaced_s, int ei, int& count,
                                            int lane) {
  const unsigned c = __reduce_add_sync(0xffffffffu, static_cast<unsigned>(count));
  if (lane == 0 && c != 0) atomicAdd(&replaced_s[ei], static_cast<unsigned long long>(c));
  count = 0;
}

// Arithmetic families: a batch whose streams all use FP16 colour with K = 4
// or 8 (the serving mix) or all FP32 colour with K = 4 or 8 gets a kernel
// holding only those two variants; any other mix gets the kernel with all.
constexpr int kFamF16K48 = 0, kFamF32K48 = 1, kFamAll = 2;

// One tile of entry e: the update from the staged frame, or (FOVF >= 0) from
// the frame foveated on read.
// pre: the fold inputs loaded before the wait (for up to 8 slots, used as
// they are: no narrowed copy, which would have to live in local memory), or
// null. The generic-K and literal forms take none.
template <int KT, bool F16, int PX, int T, bool LIT, int FOVF>
__device__ __forceinline__ int tile(const BatchEntry& e, const StageLayout& L, uint8_t* st,
                                    const float* u, int64_t p0, float d_f, int tid,
                                    const wrs::FoldIn<8>* pre = nullptr) {
  if constexpr (KT == 4 || KT == 8) {
    if constexpr (FOVF >= 0)
      return wrs::compute_tile_fov<KT, F16, PX, T, LIT, FOVF, 8>(e.s, e.f, e.fv, L, st, u, p0, d_f, tid, pre);
    else
      return wrs::compute_tile<KT, F16, PX, T, LIT, 8>(e.s, e.f, L, st, u, p0, d_f, tid, pre);
  } else {
    if constexpr (FOVF >= 0)
      return wrs::compute_tile_fov<KT, F16, PX, T, LIT, FOVF>(e.s, e.f, e.fv, L, st, u, p0, d_f, tid);
    else
      return wrs::compute_tile<KT, F16, PX, T, LIT>(e.s, e.f, L, st, u, p0, d_f, tid);
  }
}

// The producer's work for one tile of entry e: its uniforms, then its bulk
// copies. KT, CS > 0 fix the slot count and colour bytes at compile time (the
// K = 4 / 8 families), so the copy sizes and stage offsets fold to constants.
template <int T, int KT, int CS, bool COPY_FRAME>
__device__ __forceinline__ void produce_tile(const BatchEntry& e, int64_t p0, uint8_t* st, float* u,
                                             uint64_t* full, int ln, uint32_t stage_cap) {
  const int K = KT > 0 ? KT : e.s.K;
  const int cs = CS > 0 ? CS : (entry_f16(e) ? 2 : 4);
  const bool resolve = stage_records(e);
  const StageLayout L = wrs::stage_layout(T, K, cs, resolve);
  wrs::draw_tile_uniforms_warp<T>(e.s, e.f, p0, u, ln);
  __syncwarp();
  wrs::issue_tile_copies<T>(e.s, e.f, K, cs, resolve, L, st, full, p0, 0u, ln, COPY_FRAME, stage_cap);
}

// Warp-specialised like the single-stream pipelined kernel: warp 8 draws each
// tile's uniforms and issues its copies, warps 0..7 compute it. FOVF >= 0:
// no frame is copied; the consumers foveate each pixel from the stream's
// image and mip levels (filter FOVF, WRS_FILTER_*) into the stage first.
template <int PX, int FAM, int FOVF = -1>
__global__ void __launch_bounds__(kBatchThreads, PX == 1 ? 2 : 1)
    batch_kernel(const __grid_constant__ BatchArgs a) {
  static_assert(FOVF < 0 || PX == 1, "foveating batches take one pixel per thread");
  extern __shared__ __align__(128) uint8_t smem[];
  __shared__ unsigned long long replaced_s[kMaxBatch];  // per stream, this CTA
  __shared__ float d_f_s[kMaxBatch];                    // per stream: density at the fovea edge
  __shared__ uint32_t failed_s[kMaxBatch];              // per stream: an earlier wait gave up
  constexpr int T = kConsumerWarps * 32 * PX;
  const wrs::Ring r = wrs::make_ring(smem, a.stage_bytes, T, a.stages);
  const int tid = threadIdx.x;
  const int warp = tid >> 5;
  const int lane = tid & 31;
  if (tid == 0) wrs::init_ring(r, kConsumerWarps);
  if (tid < kMaxBatch) replaced_s[tid] = 0;
  // each stream's Eq. (phat) normaliser, once per CTA instead of once per tile
  if (tid < a.n) {
    d_f_s[tid] = wrs::fovea_density(a.e[tid].s);
    // a stream whose earlier push timed out (not yet seen by the host) has
    // undefined reservoirs: its tiles are copied but not computed or written
    failed_s[tid] = *reinterpret_cast<volatile const uint32_t*>(a.e[tid].status);
  }
  __syncthreads();

  const int first = blockIdx.x, step = gridDim.x;
  const int my_tiles = first < a.ntiles ? (a.ntiles - 1 - first) / step + 1 : 0;
  int issued = 0;
  if (warp == kConsumerWarps) {
    int pe = 0;  // entry of the producer's current tile
    issued = wrs::produce(r, my_tiles, a.timeout_ns, lane,
                          [&](int it, uint8_t* st, float* u, uint64_t* full, int ln) {
                            const int g = first + it * step;
                            pe = entry_after(a, g, pe);
                            const BatchEntry& e = a.e[pe];
                            const int64_t p0 = static_cast<int64_t>(g - e.tile0) * T;
                            constexpr bool cf = FOVF < 0;
                            if constexpr (FAM == kFamF16K48) {
                              if (e.code == 0) produce_tile<T, 4, 2, cf>(e, p0, st, u, full, ln, r.stage_bytes);
                              else produce_tile<T, 8, 2, cf>(e, p0, st, u, full, ln, r.stage_bytes);
                            } else if constexpr (FAM == kFamF32K48) {
                              if (e.code == 2) produce_tile<T, 4, 4, cf>(e, p0, st, u, full, ln, r.stage_bytes);
                              else produce_tile<T, 8, 4, cf>(e, p0, st, u, full, ln, r.stage_bytes);
                            } else {
                              produce_tile<T, 0, 0, cf>(e, p0, st, u, full, ln, r.stage_bytes);
                            }
                          });
  } else {
    // fold inputs of entries that compute with K = 4 or 8, loaded before the
    // wait; the generic-K arithmetic loads its own (the literal rule has none)
    wrs::FoldIn<8> fin;
    bool folding = false;
    int ei = 0;        // entry of the consumer's current tile
    int replaced = 0;  // this thread's replacements in entry ei so far
    wrs::consume(r, my_tiles, a.timeout_ns, lane, [&](int it) {
      const int g = first + it * step;
      const int next = entry_after(a, g, ei);
      if (next != ei) {
        flush_count(replaced_s, ei, replaced, lane);
        ei = next;
      }
      const BatchEntry& e = a.e[ei];
      const int64_t p0 = static_cast<int64_t>(g - e.tile0) * T;
      folding = e.code < 4 && wrs::prefetch_fold<8, PX>(e.s, e.f, p0, tid, fin);
    }, [&](int it, uint8_t* st, const float* u) {
      const int g = first + it * step;
      const BatchEntry& e = a.e[ei];
      const int64_t p0 = static_cast<int64_t>(g - e.tile0) * T;
      const bool resolve = stage_records(e);
      const float d_f = d_f_s[ei];
      if (failed_s[ei] != 0) return;
      const wrs::FoldIn<8>* pre = folding ? &fin : nullptr;
      int rc;
      if constexpr (FAM == kFamF16K48) {
        rc = e.code == 0
                 ? tile<4, true, PX, T, false, FOVF>(e, wrs::stage_layout(T, 4, 2, resolve), st, u, p0, d_f, tid, pre)
                 : tile<8, true, PX, T, false, FOVF>(e, wrs::stage_layout(T, 8, 2, resolve), st, u, p0, d_f, tid, pre);
      } else if constexpr (FAM == kFamF32K48) {
        rc = e.code == 2
                 ? tile<4, false, PX, T, false, FOVF>(e, wrs::stage_layout(T, 4, 4, resolve), st, u, p0, d_f, tid, pre)
                 : tile<8, false, PX, T, false, FOVF>(e, wrs::stage_layout(T, 8, 4, resolve), st, u, p0, d_f, tid, pre);
      } else {
        switch (e.code) {
        case 0: rc = tile<4, true, PX, T, false, FOVF>(e, wrs::stage_layout(T, 4, 2, resolve), st, u, p0, d_f, tid, pre); break;
        case 1: rc = tile<8, true, PX, T, false, FOVF>(e, wrs::stage_layout(T, 8, 2, resolve), st, u, p0, d_f, tid, pre); break;
        case 2: rc = tile<4, false, PX, T, false, FOVF>(e, wrs::stage_layout(T, 4, 4, resolve), st, u, p0, d_f, tid, pre); break;
        case 3: rc = tile<8, false, PX, T, false, FOVF>(e, wrs::stage_layout(T, 8, 4, resolve), st, u, p0, d_f, tid, pre); break;
        case 4: rc = tile<0, true, PX, T, false, FOVF>(e, wrs::stage_layout(T, e.s.K, 2, resolve), st, u, p0, d_f, tid); break;
        case 6: rc = tile<1, true, PX, T, true, FOVF>(e, wrs::stage_layout(T, 1, 2, resolve), st, u, p0, d_f, tid, pre); break;
        case 7: rc = tile<1, false, PX, T, true, FOVF>(e, wrs::stage_layout(T, 1, 4, resolve), st, u, p0, d_f, tid, pre); break;
        default: rc = tile<0, false, PX, T, false, FOVF>(e, wrs::stage_layout(T, e.s.K, 4, resolve), st, u, p0, d_f, tid); break;
        }
      }
      replaced += rc;
    });
    flush_count(replaced_s, ei, replaced, lane);
  }
  __syncthreads();
  if (tid < a.n && replaced_s[tid] != 0) atomicAdd(a.e[tid].s.replacements, replaced_s[tid]);
  if (wrs::flag_raised(r)) {
    if (warp == kConsumerWarps) wrs::drain(r, issued, a.timeout_ns);
    // the batch ran out of time as a whole: report it on every stream
    if (tid < a.n) atomicExch(a.e[tid].status, static_cast<uint32_t>(WRS_ERR_TIMEOUT));
  }
}

}  // namespace
