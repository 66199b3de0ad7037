// Foveation post-process (Sec. 4.3, "Implementation"): the rendered frame is
// mip-mapped and each ring around the gaze is reconstructed from a coarser
// level, by nearest lookup or bilinear filtering. Two kernels:
//
//  mip_kernel     one pass over the image builds every stored level. A CTA
//                 stages a 2^M-row strip of 2048 pixels in shared memory
//                 (M = top level), then forms the level sums bottom-up in
//                 shared memory with the quad-tree order (s00 + s01) +
//                 (s10 + s11) and writes each level's means as 16-byte
//                 texels. The image is read once; levels >= 1 are written
//                 once.
//  foveate4_kernel four adjacent pixels per thread (foveate_kernel: one, for
//                 widths not divisible by 4 or unaligned frames): FP32 ring
//                 test, then a copy of the image pixel (level 0) or one (box)
//                 or four (bilinear) texel reads, which the 129 MB L2 serves
//                 for the coarse levels; writes the colours as 16-byte stores
//                 and the ring levels as one word.
//
// Every arithmetic step that decides a bit of the output is a single
// round-to-nearest intrinsic, so the results are reproducible on any IEEE
// FP32 implementation of the same sequence.
#include <cmath>
#include <cstring>

#include "wrs_fov.cuh"
#include "wrs_internal.h"

using wrs::FovDev;
using wrs::MipLevelDev;

namespace {

constexpr int kMipThreads = 256;
constexpr int kTilePx = 2048;          // pixels per CTA strip: 2^M rows x (2048 >> M) columns
constexpr int kFovThreads = 256;

// Writable view of a stored level, for the build.
struct MipLevelOut {
  float4* texels;
  int32_t wb, hb;
};

struct MipArgs {
  const float* img;
  int64_t pitch;
  int32_t width, height;
  int32_t top;                          // highest level built, 1..WRS_MAX_MIP_LEVELS-1
  MipLevelOut lev[WRS_MAX_MIP_LEVELS];  // [0] unused
};

struct FovArgs {
  FovDev fv;
  float* frame;
  int64_t frame_pitch;
  uint8_t* ring;
  int32_t width, height;
  float gx, gy;
};

__device__ __forceinline__ int32_t block_extent(int32_t n, int32_t i, int L) {
  const int64_t lo = (int64_t)i << L;
  const int64_t hi = lo + ((int64_t)1 << L);
  return (int32_t)((hi < n ? hi : n) - lo);
}

// Shared memory of one strip: the pixels, then the sums of levels 1..M.
// Level L of the strip holds (2^M >> L) rows x ((2048 >> M) >> L) texels x 3.
template <int M, bool VEC>
__global__ void __launch_bounds__(kMipThreads) mip_kernel(MipArgs a) {
  constexpr int TH = 1 << M;
  constexpr int TW = kTilePx >> M;
  constexpr int kRowF = TW * 3;
  __shared__ __align__(16) float s_px[kTilePx * 3];
  // levels 1..M of a strip hold sum_L 2048 / 4^L < 2048 / 3 texels
  __shared__ float s_sum[(kTilePx / 3 + 1) * 3];

  const int tid = threadIdx.x;
  const int64_t ty0 = (int64_t)blockIdx.y * TH;
  const int64_t tx0 = (int64_t)blockIdx.x * TW;
  const int64_t row_f = 3 * (int64_t)a.width;

  // stage the strip (zero outside the image), coalesced along each row
  if (VEC) {
    // 16-byte loads: rows start 16-byte aligned (pitch % 4 == 0, tx0 % 4 == 0);
    // all of a thread's loads are issued before any is stored to shared memory
    constexpr int kRowQ = kRowF / 4;
    constexpr int kPer = kTilePx * 3 / 4 / kMipThreads;
    float4 v[kPer];
#pragma unroll
    for (int j = 0; j < kPer; ++j) {
      const int q = tid + j * kMipThreads;
      const int r = q / kRowQ, c4 = q - r * kRowQ;
      const int64_t y = ty0 + r;
      const int64_t lim = y < a.height ? row_f - 3 * tx0 : 0;
      const float* src = a.img + (y < a.height ? y : 0) * a.pitch + 3 * tx0 + 4 * c4;
      const int64_t f0 = 4 * (int64_t)c4;
      if (f0 + 4 <= lim) {
        v[j] = __ldg(reinterpret_cast<const float4*>(src));
      } else {
        v[j].x = f0 < lim ? __ldg(src) : 0.0f;
        v[j].y = f0 + 1 < lim ? __ldg(src + 1) : 0.0f;
        v[j].z = f0 + 2 < lim ? __ldg(src + 2) : 0.0f;
        v[j].w = 0.0f;
      }
    }
#pragma unroll
    for (int j = 0; j < kPer; ++j)
      reinterpret_cast<float4*>(s_px)[tid + j * kMipThreads] = v[j];
  } else {
    for (int r = 0; r < TH; ++r) {
      const int64_t y = ty0 + r;
      // floats of this row inside the image (none below the last row)
      const int64_t lim = y < a.height ? row_f - 3 * tx0 : 0;
      const float* src = a.img + (y < a.height ? y : 0) * a.pitch + 3 * tx0;
      for (int i = tid; i < kRowF; i += kMipThreads)
        s_px[r * kRowF + i] = i < lim ? __ldg(src + i) : 0.0f;
    }
  }
  __syncthreads();

  // level L sums from level L-1 (level 0 = the staged pixels)
  const float* prev = s_px;
  int prev_w = TW;
  float* cur = s_sum;
#pragma unroll
  for (int L = 1; L <= M; ++L) {
    const int lw = TW >> L;
    const int lh = TH >> L;
    const int n = lw * lh;
    const MipLevelOut lv = a.lev[L];
    for (int i = tid; i < n; i += kMipThreads) {
      const int r = i / lw, c = i - r * lw;
      const float* p0 = prev + ((2 * r) * prev_w + 2 * c) * 3;
      const float* p1 = p0 + prev_w * 3;
      float s[3];
#pragma unroll
      for (int ch = 0; ch < 3; ++ch) {
        const float top = __fadd_rn(p0[ch], p0[3 + ch]);
        const float bot = __fadd_rn(p1[ch], p1[3 + ch]);
        s[ch] = __fadd_rn(top, bot);
        cur[i * 3 + ch] = s[ch];
      }
      const int32_t gy = (int32_t)(ty0 >> L) + r;
      const int32_t gx = (int32_t)(tx0 >> L) + c;
      if (gy < lv.hb && gx < lv.wb) {
        const float cnt = (float)(block_extent(a.height, gy, L) * block_extent(a.width, gx, L));
        lv.texels[(int64_t)gy * lv.wb + gx] =
            make_float4(__fdiv_rn(s[0], cnt), __fdiv_rn(s[1], cnt), __fdiv_rn(s[2], cnt), 0.0f);
      }
    }
    __syncthreads();
    prev = cur;
    prev_w = lw;
    cur += n * 3;
  }
}

// One pixel per thread (any width, pitch and alignment).
template <int FILTER>
__global__ void __launch_bounds__(kFovThreads) foveate_kernel(FovArgs a) {
  const int64_t n = (int64_t)a.width * a.height;
  for (int64_t p = (int64_t)blockIdx.x * kFovThreads + threadIdx.x; p < n;
       p += (int64_t)gridDim.x * kFovThreads) {
    const int32_t y = (int32_t)(p / a.width);
    const int32_t x = (int32_t)(p - (int64_t)y * a.width);
    float rgb[3];
    const int L = wrs::fov_pixel<FILTER>(a.fv, a.gx, a.gy, x, y, rgb);
    float* o = a.frame + (int64_t)y * a.frame_pitch + 3 * (int64_t)x;
    o[0] = rgb[0];
    o[1] = rgb[1];
    o[2] = rgb[2];
    if (a.ring) a.ring[p] = (uint8_t)L;
  }
}

// Four horizontally adjacent pixels per thread: width % 4 == 0, the frame's
// rows 16-byte aligned and the ring map 4-byte aligned, so a thread writes
// its 48 bytes of colour as three 16-byte stores and its levels as one word.
template <int FILTER>
__global__ void __launch_bounds__(kFovThreads) foveate4_kernel(FovArgs a) {
  const int32_t wq = a.width >> 2;
  const int64_t nq = (int64_t)wq * a.height;
  for (int64_t q = (int64_t)blockIdx.x * kFovThreads + threadIdx.x; q < nq;
       q += (int64_t)gridDim.x * kFovThreads) {
    const int32_t y = (int32_t)(q / wq);
    const int32_t x0 = 4 * (int32_t)(q - (int64_t)y * wq);
    float rgb[12];
    const uint32_t lv = wrs::fov_quad<FILTER>(a.fv, a.gx, a.gy, x0, y, rgb);
    float4* o = reinterpret_cast<float4*>(a.frame + (int64_t)y * a.frame_pitch + 3 * (int64_t)x0);
    o[0] = make_float4(rgb[0], rgb[1], rgb[2], rgb[3]);
    o[1] = make_float4(rgb[4], rgb[5], rgb[6], rgb[7]);
    o[2] = make_float4(rgb[8], rgb[9], rgb[10], rgb[11]);
    if (a.ring) *reinterpret_cast<uint32_t*>(a.ring + (int64_t)y * a.width + x0) = lv;
  }
}

bool aligned(const void* p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

int check_image(int32_t width, int32_t height) {
  if (width < 1 || height < 1)
    return wrs_fail(WRS_ERR_ARG, "image size must be >= 1 x 1 (got %d x %d)", width, height);
  if ((int64_t)width * height >= ((int64_t)1 << 31))
    return wrs_fail(WRS_ERR_ARG, "width * height must be below 2^31");
  return WRS_OK;
}

template <typename Level>
void fill_levels(const wrs_mip_layout& L, const void* base, Level* lev) {
  for (int l = 1; l < L.levels; ++l) {
    lev[l].texels = reinterpret_cast<float4*>(const_cast<uint8_t*>(
        static_cast<const uint8_t*>(base) + L.offset[l]));
    lev[l].wb = L.width[l];
    lev[l].hb = L.height[l];
  }
}

int device_sms(int* sms) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(sms, cudaDevAttrMultiProcessorCount, dev);
  return e == cudaSuccess ? WRS_OK : wrs_cuda_fail(e, "device query");
}

}  // namespace

extern "C" int wrs_mip_layout_get(int32_t width, int32_t height, int32_t levels,
                                  wrs_mip_layout* out) {
  wrs_clear_error();
  if (!out) return wrs_fail(WRS_ERR_ARG, "layout output is NULL");
  if (int rc = check_image(width, height)) return rc;
  if (levels < 1 || levels > WRS_MAX_MIP_LEVELS)
    return wrs_fail(WRS_ERR_ARG, "levels must be in 1..%d (got %d)", WRS_MAX_MIP_LEVELS, levels);
  std::memset(out, 0, sizeof(*out));
  out->levels = levels;
  out->width[0] = width;
  out->height[0] = height;
  out->offset[0] = -1;
  int64_t off = 0;
  for (int l = 1; l < levels; ++l) {
    out->width[l] = (int32_t)(((int64_t)width + (1 << l) - 1) >> l);
    out->height[l] = (int32_t)(((int64_t)height + (1 << l) - 1) >> l);
    out->offset[l] = off;
    off += ((int64_t)out->width[l] * out->height[l] * 16 + 255) / 256 * 256;
  }
  out->total_bytes = off;
  return WRS_OK;
}

extern "C" int wrs_mip_build(const float* d_img, int64_t pitch, int32_t width, int32_t height,
                             int32_t levels, void* d_mip, size_t mip_bytes, wrs_stream_t stream) {
  wrs_clear_error();
  wrs_mip_layout L;
  if (int rc = wrs_mip_layout_get(width, height, levels, &L)) return rc;
  if (levels == 1) return WRS_OK;
  if (!d_img || !aligned(d_img, 4)) return wrs_fail(WRS_ERR_ARG, "d_img is NULL or unaligned");
  if (pitch < 3 * (int64_t)width)
    return wrs_fail(WRS_ERR_ARG, "img_pitch_elems %lld is below 3 * width", (long long)pitch);
  if (!d_mip || !aligned(d_mip, 256))
    return wrs_fail(WRS_ERR_ARG, "d_mip is NULL or not 256-byte aligned");
  if ((int64_t)mip_bytes < L.total_bytes)
    return wrs_fail(WRS_ERR_BUDGET, "mip buffer holds %zu bytes, the layout needs %lld", mip_bytes,
                    (long long)L.total_bytes);
  MipArgs a{};
  a.img = d_img;
  a.pitch = pitch;
  a.width = width;
  a.height = height;
  a.top = levels - 1;
  fill_levels(L, d_mip, a.lev);
  const int M = levels - 1;
  const int TH = 1 << M, TW = kTilePx >> M;
  const dim3 grid((unsigned)((width + TW - 1) / TW), (unsigned)((height + TH - 1) / TH));
  if (grid.y > 65535u) return wrs_fail(WRS_ERR_ARG, "image too tall for the mip build");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const bool vec = pitch % 4 == 0 && aligned(d_img, 16);
#define WRS_MIP_LAUNCH(m)                                                   \
  (vec ? mip_kernel<m, true><<<grid, kMipThreads, 0, st>>>(a)               \
       : mip_kernel<m, false><<<grid, kMipThreads, 0, st>>>(a))
  switch (M) {
    case 1: WRS_MIP_LAUNCH(1); break;
    case 2: WRS_MIP_LAUNCH(2); break;
    case 3: WRS_MIP_LAUNCH(3); break;
    case 4: WRS_MIP_LAUNCH(4); break;
    default: WRS_MIP_LAUNCH(5); break;
  }
#undef WRS_MIP_LAUNCH
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? WRS_OK : wrs_cuda_fail(e, "wrs_mip_build: launch");
}

int wrs_fov_check_source(const float* d_img, int64_t pitch, const void* d_mip, size_t mip_bytes,
                   int32_t width, int32_t height, int32_t nradii, const float* radii,
                   int32_t filter, FovDev* out) {
  if (int rc = check_image(width, height)) return rc;
  if (nradii < 1 || nradii > WRS_MAX_MIP_LEVELS - 1 || !radii)
    return wrs_fail(WRS_ERR_ARG, "nradii must be in 1..%d with a radii array",
                    WRS_MAX_MIP_LEVELS - 1);
  if (filter != WRS_FILTER_BOX && filter != WRS_FILTER_BILINEAR)
    return wrs_fail(WRS_ERR_ARG, "filter must be WRS_FILTER_BOX or WRS_FILTER_BILINEAR");
  if (!d_img || !aligned(d_img, 4)) return wrs_fail(WRS_ERR_ARG, "d_img is NULL or unaligned");
  if (pitch < 3 * (int64_t)width)
    return wrs_fail(WRS_ERR_ARG, "img_pitch_elems %lld is below 3 * width", (long long)pitch);
  if (!d_mip || !aligned(d_mip, 256))
    return wrs_fail(WRS_ERR_ARG, "d_mip is NULL or not 256-byte aligned");
  FovDev fv{};
  for (int i = 0; i < nradii; ++i) {
    if (!std::isfinite(radii[i]) || !(radii[i] > 0.0f) || (i > 0 && radii[i] < radii[i - 1]))
      return wrs_fail(WRS_ERR_ARG, "radii must be finite, positive and ascending");
    fv.r2[i] = radii[i] * radii[i];
  }
  wrs_mip_layout L;
  if (int rc = wrs_mip_layout_get(width, height, nradii + 1, &L)) return rc;
  if ((int64_t)mip_bytes < L.total_bytes)
    return wrs_fail(WRS_ERR_BUDGET, "mip buffer holds %zu bytes, %d levels need %lld", mip_bytes,
                    nradii + 1, (long long)L.total_bytes);
  fv.img = d_img;
  fv.pitch = pitch;
  fv.nradii = nradii;
  fill_levels(L, d_mip, fv.lev);
  *out = fv;
  return WRS_OK;
}

extern "C" int wrs_foveate(const float* d_img, int64_t pitch, const void* d_mip, size_t mip_bytes,
                           int32_t width, int32_t height, int32_t nradii, const float* radii,
                           float gx, float gy, int32_t filter, float* d_frame,
                           int64_t frame_pitch, uint8_t* d_ring, wrs_stream_t stream) {
  wrs_clear_error();
  if (!std::isfinite(gx) || !std::isfinite(gy)) return wrs_fail(WRS_ERR_ARG, "gaze must be finite");
  if (!d_frame || !aligned(d_frame, 4))
    return wrs_fail(WRS_ERR_ARG, "d_frame must be non-NULL and 4-byte aligned");
  if (frame_pitch < 3 * (int64_t)width)
    return wrs_fail(WRS_ERR_ARG, "pitches must be >= 3 * width");
  FovArgs a{};
  if (int rc = wrs_fov_check_source(d_img, pitch, d_mip, mip_bytes, width, height, nradii, radii, filter,
                              &a.fv))
    return rc;
  a.frame = d_frame;
  a.frame_pitch = frame_pitch;
  a.ring = d_ring;
  a.width = width;
  a.height = height;
  a.gx = gx;
  a.gy = gy;
  int sms = 0;
  if (int rc = device_sms(&sms)) return rc;
  const bool quad = width % 4 == 0 && frame_pitch % 4 == 0 && aligned(d_frame, 16) &&
                    (!d_ring || aligned(d_ring, 4));
  const int64_t n = (int64_t)width * height / (quad ? 4 : 1);
  const int64_t want = (n + kFovThreads - 1) / kFovThreads;
  const int64_t cap = (int64_t)sms * 8 * 16;  // 8 resident CTAs per SM x 16 waves
  const unsigned grid = (unsigned)(want < cap ? want : cap);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (quad) {
    if (filter == WRS_FILTER_BOX)
      foveate4_kernel<WRS_FILTER_BOX><<<grid, kFovThreads, 0, st>>>(a);
    else
      foveate4_kernel<WRS_FILTER_BILINEAR><<<grid, kFovThreads, 0, st>>>(a);
  } else if (filter == WRS_FILTER_BOX) {
    foveate_kernel<WRS_FILTER_BOX><<<grid, kFovThreads, 0, st>>>(a);
  } else {
    foveate_kernel<WRS_FILTER_BILINEAR><<<grid, kFovThreads, 0, st>>>(a);
  }
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? WRS_OK : wrs_cuda_fail(e, "wrs_foveate: launch");
}
