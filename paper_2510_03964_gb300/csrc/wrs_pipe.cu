// Pipelined persistent form of the fused update + resolve (sm_103a).
//
// Persistent CTAs (one or more per SM) walk the image in tiles of
// T = 256 * PX pixels. A producer warp streams the planes a tile needs (frame
// RGB, W, P, the K key planes and, for the fused resolve, the K weight and 3K
// colour planes) into a ring of S shared-memory stages with 1-D bulk
// asynchronous copies (cp.async.bulk) that complete on one transaction-count
// "full" mbarrier per stage, after drawing the tile's uniforms (one Philox
// block per 4 pixels) into the stage. Eight consumer warps compute each
// landed tile from shared memory with the same per-pixel code as the plain
// kernel (bit-identical results), write straight to global memory and free
// the stage through its "empty" mbarrier. No block-wide barrier sits inside
// the loop.
//
// Every wait is bounded by %globaltimer. A wait that runs out records
// WRS_ERR_TIMEOUT in the stream's status word, waits (again bounded) for the
// copies this CTA still has in flight, and returns; the host reads the word
// with wrs_check_status.
#include <cuda_runtime.h>

#include <mutex>

#include "wrs.h"
#include "wrs_async.cuh"
#include "wrs_device.cuh"
#include "wrs_internal.h"

using wrs::FovDev;
using wrs::FrameDev;
using wrs::StageLayout;
using wrs::StreamDev;

namespace {

struct PipeArgs {
  int stages;
  int ntiles;
  int resolve;             // copy weight/colour planes (fused resolve or full temporal bias)
  uint32_t* status;        // stream status word (WRS_OK or WRS_ERR_TIMEOUT)
  uint64_t timeout_ns;
  uint32_t extra_tx;       // added to the expected bytes: > 0 only to test the timeout path
};

constexpr int kConsumerWarps = 8;
constexpr int kPipeThreads = (kConsumerWarps + 1) * 32;

// Warp-specialised: warps 0..7 compute (consumers, PX pixels per thread), warp 8
// draws uniforms and issues copies (producer). Consumers and producer meet
// only at the per-stage full/empty barriers, never at a block-wide barrier.
// FOVF >= 0: the frame is not copied but foveated by the consumers from `fv`
// with filter FOVF (WRS_FILTER_*) as they compute; FOVF < 0: `fv` is unused.
// Resident CTAs per SM the compiler is asked to fit: three for one or two
// slots (their stages are small, and the extra warps hide the per-pixel
// arithmetic's latency), two for one pixel per thread, else one.
template <int KT, int PX>
constexpr int pipe_min_blocks() {
  return PX != 1 ? 1 : ((KT == 1 || KT == 2) ? 3 : 2);
}

template <int KT, bool F16, int PX, bool LIT, int FOVF = -1>
__global__ void __launch_bounds__(kPipeThreads, pipe_min_blocks<KT, PX>())
    pipe_kernel(const __grid_constant__ StreamDev s, const __grid_constant__ FrameDev f,
                const PipeArgs a, const __grid_constant__ FovDev fv) {
  extern __shared__ __align__(128) uint8_t smem[];
  constexpr int T = kConsumerWarps * 32 * PX;
  constexpr int cs = F16 ? 2 : 4;
  const int K = KT > 0 ? KT : s.K;
  const bool resolve = a.resolve != 0;
  const StageLayout L = wrs::stage_layout(T, K, cs, resolve);
  const wrs::Ring r = wrs::make_ring(smem, L.bytes, T, a.stages);
  const int tid = threadIdx.x;
  const int warp = tid >> 5;
  const int lane = tid & 31;
  __shared__ uint32_t failed;
  if (tid == 0) {
    wrs::init_ring(r, kConsumerWarps);
    // a wait of an earlier push gave up and the host has not yet seen it: the
    // reservoirs are undefined, so leave them (and the waits) alone
    failed = *reinterpret_cast<volatile const uint32_t*>(a.status);
  }
  __syncthreads();
  if (failed != 0) return;

  const int first = blockIdx.x;
  const int step = gridDim.x;
  const int my_tiles = first < a.ntiles ? (a.ntiles - 1 - first) / step + 1 : 0;
  int issued = 0;
  int replaced = 0;
  if (warp == kConsumerWarps) {
    issued = wrs::produce(r, my_tiles, a.timeout_ns, lane,
                          [&](int it, uint8_t* st, float* u, uint64_t* full, int ln) {
                            const int64_t p0 = static_cast<int64_t>(first + it * step) * T;
                            wrs::draw_tile_uniforms_warp<T>(s, f, p0, u, ln);
                            __syncwarp();
                            wrs::issue_tile_copies<T>(s, f, K, cs, resolve, L, st, full, p0,
                                                      a.extra_tx, ln, FOVF < 0, r.stage_bytes);
                          });
  } else {
    const float d_f = wrs::fovea_density(s);
    wrs::FoldFor<KT> fin;
    bool folding = false;
    wrs::consume(
        r, my_tiles, a.timeout_ns, lane,
        [&](int it) {
          const int64_t p0 = static_cast<int64_t>(first + it * step) * T;
          if constexpr (KT > 2) folding = wrs::prefetch_fold<wrs::FoldCap<KT>::value, PX>(s, f, p0, tid, fin);
        },
        [&](int it, uint8_t* st, const float* u) {
          const int64_t p0 = static_cast<int64_t>(first + it * step) * T;
          const wrs::FoldFor<KT>* pre = folding ? &fin : nullptr;
          if constexpr (FOVF >= 0)
            replaced += wrs::compute_tile_fov<KT, F16, PX, T, LIT, FOVF>(s, f, fv, L, st, u, p0,
                                                                         d_f, tid, pre);
          else
            replaced += wrs::compute_tile<KT, F16, PX, T, LIT>(s, f, L, st, u, p0, d_f, tid, pre);
        });
  }
  __syncthreads();
  if (warp < kConsumerWarps) wrs::add_warp_count(s.replacements, replaced, lane);
  if (wrs::flag_raised(r)) {
    if (warp == kConsumerWarps) wrs::drain(r, issued, a.timeout_ns);
    if (tid == 0) atomicExch(a.status, static_cast<uint32_t>(WRS_ERR_TIMEOUT));
  }
}

template <int KT, bool F16, int PX, bool LIT = false, int FOVF = -1>
cudaError_t launch_pipe_t(const StreamDev& s, const FrameDev& f, PipeArgs a, int sms,
                          int ctas_per_sm, cudaStream_t st, const FovDev& fv = FovDev{}) {
  constexpr int T = kConsumerWarps * 32 * PX;
  const StageLayout L = wrs::stage_layout(T, s.K, F16 ? 2 : 4, a.resolve != 0);
  const size_t smem = wrs::ring_bytes(L.bytes, T, a.stages);
  // per instantiation and device: the largest dynamic shared memory already
  // allowed; the lock keeps two host threads from lowering each other's limit
  static size_t configured[64] = {};
  static std::mutex lock;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  {
    std::lock_guard<std::mutex> hold(lock);
    if (smem > configured[dev]) {
      e = cudaFuncSetAttribute(pipe_kernel<KT, F16, PX, LIT, FOVF>,
                               cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
      if (e != cudaSuccess) return e;
      configured[dev] = smem;
    }
  }
  int fit = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&fit, pipe_kernel<KT, F16, PX, LIT, FOVF>,
                                                    kPipeThreads, smem);
  if (e != cudaSuccess) return e;
  if (fit < 1) return cudaErrorInvalidConfiguration;
  const int per_sm = ctas_per_sm > 0 && ctas_per_sm < fit ? ctas_per_sm : fit;
  a.ntiles = static_cast<int>((static_cast<int64_t>(s.hw) + T - 1) / T);
  const int64_t want = static_cast<int64_t>(sms) * per_sm;
  const int grid = static_cast<int>(a.ntiles < want ? a.ntiles : want);
  pipe_kernel<KT, F16, PX, LIT, FOVF><<<grid, kPipeThreads, smem, st>>>(s, f, a, fv);
  return cudaGetLastError();
}

// The foveating form: one pixel per thread (the default tile), K = 4, 8 or
// any other through the generic instantiation, and the literal rule.
template <bool F16, int FILTER>
cudaError_t launch_pipe_fov_k(const StreamDev& s, const FrameDev& f, const FovDev& fv,
                              const PipeArgs& a, int sms, int ctas, cudaStream_t st) {
  if (s.literal) return launch_pipe_t<1, F16, 1, true, FILTER>(s, f, a, sms, ctas, st, fv);
  switch (s.K) {
    case 4: return launch_pipe_t<4, F16, 1, false, FILTER>(s, f, a, sms, ctas, st, fv);
    case 8: return launch_pipe_t<8, F16, 1, false, FILTER>(s, f, a, sms, ctas, st, fv);
    default: return launch_pipe_t<0, F16, 1, false, FILTER>(s, f, a, sms, ctas, st, fv);
  }
}

template <int KT, bool F16, bool LIT = false>
cudaError_t launch_pipe_px(const StreamDev& s, const FrameDev& f, const PipeArgs& a, int px,
                           int sms, int ctas, cudaStream_t st) {
  switch (px) {
    case 4: return launch_pipe_t<KT, F16, 4, LIT>(s, f, a, sms, ctas, st);
    case 2: return launch_pipe_t<KT, F16, 2, LIT>(s, f, a, sms, ctas, st);
    default: return launch_pipe_t<KT, F16, 1, LIT>(s, f, a, sms, ctas, st);
  }
}

template <bool F16>
cudaError_t launch_pipe_k(const StreamDev& s, const FrameDev& f, const PipeArgs& a, int px,
                          int sms, int ctas, cudaStream_t st) {
  if (s.literal) return launch_pipe_px<1, F16, true>(s, f, a, px, sms, ctas, st);
  switch (s.K) {
    case 1: return launch_pipe_px<1, F16>(s, f, a, px, sms, ctas, st);
    case 2: return launch_pipe_px<2, F16>(s, f, a, px, sms, ctas, st);
    case 4: return launch_pipe_px<4, F16>(s, f, a, px, sms, ctas, st);
    case 8: return launch_pipe_px<8, F16>(s, f, a, px, sms, ctas, st);
    default: return launch_pipe_px<0, F16>(s, f, a, px, sms, ctas, st);
  }
}

}  // namespace

// Shared memory one CTA of the pipelined kernel needs.
size_t wrs_pipe_smem_bytes(int K, bool f16, int px, int stages, bool resolve) {
  const int T = kConsumerWarps * 32 * px;
  return wrs::ring_bytes(wrs::stage_layout(T, K, f16 ? 2 : 4, resolve).bytes, T, stages);
}

bool wrs_pipe_supported(const wrs_ctx* x, const float* frame, int64_t pitch, const float* out) {
  const auto al = [](const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; };
  return x->cfg.width % 4 == 0 && pitch == 3 * static_cast<int64_t>(x->cfg.width) && al(frame) &&
         (out == nullptr || al(out));
}

cudaError_t wrs_launch_pipe_fov(const StreamDev& s, const FrameDev& f, const FovDev& fv, int filter,
                                bool f16, int stages, int sms, int ctas_per_sm, uint32_t* status,
                                uint64_t timeout_ns, cudaStream_t st) {
  PipeArgs a;
  a.stages = stages;
  a.ntiles = 0;
  a.resolve = (f.out != nullptr || s.bias == 2) ? 1 : 0;  // records: resolve or Delta L
  a.status = status;
  a.timeout_ns = timeout_ns;
  a.extra_tx = 0;
  if (filter == WRS_FILTER_BOX)
    return f16 ? launch_pipe_fov_k<true, WRS_FILTER_BOX>(s, f, fv, a, sms, ctas_per_sm, st)
               : launch_pipe_fov_k<false, WRS_FILTER_BOX>(s, f, fv, a, sms, ctas_per_sm, st);
  return f16 ? launch_pipe_fov_k<true, WRS_FILTER_BILINEAR>(s, f, fv, a, sms, ctas_per_sm, st)
             : launch_pipe_fov_k<false, WRS_FILTER_BILINEAR>(s, f, fv, a, sms, ctas_per_sm, st);
}

cudaError_t wrs_launch_pipe(const StreamDev& s, const FrameDev& f, bool f16, int px, int stages,
                            int sms, int ctas_per_sm, uint32_t* status, uint64_t timeout_ns,
                            uint32_t extra_tx, cudaStream_t st) {
  PipeArgs a;
  a.stages = stages;
  a.ntiles = 0;
  a.resolve = (f.out != nullptr || s.bias == 2) ? 1 : 0;  // records: resolve or Delta L
  a.status = status;
  a.timeout_ns = timeout_ns;
  a.extra_tx = extra_tx;
  return f16 ? launch_pipe_k<true>(s, f, a, px, sms, ctas_per_sm, st)
             : launch_pipe_k<false>(s, f, a, px, sms, ctas_per_sm, st);
}
