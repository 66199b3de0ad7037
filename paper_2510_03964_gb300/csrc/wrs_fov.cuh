// The per-pixel foveation post-process (Sec. 4.3, "Implementation"), shared
// by the standalone foveation kernels and the push kernel that foveates the
// frame as it reads it. Every arithmetic step that decides a bit of the
// result is one round-to-nearest intrinsic.
#pragma once

#include <stdint.h>

#include "wrs.h"

namespace wrs {

// One stored mip level: [hb][wb] texels {r, g, b, 0}.
struct MipLevelDev {
  const float4* texels;
  int32_t wb, hb;
};

// A rendered image, its mip levels and the ring radii (squared, FP32).
struct FovDev {
  const float* img;                     // [H][pitch] RGB triples
  int64_t pitch;
  int32_t nradii;                       // 1..WRS_MAX_MIP_LEVELS-1
  float r2[WRS_MAX_MIP_LEVELS - 1];     // r_i * r_i, rounded once
  MipLevelDev lev[WRS_MAX_MIP_LEVELS];  // [1..nradii]; [0] unused (the image)
};

// Level coordinate of pixel index i at level L: u = (i + 0.5) * 2^-L - 0.5
// clamped to [0, nb - 1]; integer part, right neighbour (clamped) and fraction.
__device__ __forceinline__ void texel_coord(int32_t i, int L, int32_t nb, int32_t* i0,
                                            int32_t* i1, float* f) {
  const float inv_b = __int_as_float((127 - L) << 23);  // 2^-L, exact
  float u = __fsub_rn(__fmul_rn(__fadd_rn((float)i, 0.5f), inv_b), 0.5f);
  u = fminf(fmaxf(u, 0.0f), (float)(nb - 1));
  const float fl = floorf(u);
  *i0 = (int32_t)fl;
  *i1 = *i0 + 1 < nb ? *i0 + 1 : nb - 1;
  *f = __fsub_rn(u, fl);
}

__device__ __forceinline__ float lerp2(float a, float b, float one_minus_f, float f) {
  return __fadd_rn(__fmul_rn(a, one_minus_f), __fmul_rn(b, f));
}

// Ring level of pixel x of a row whose squared vertical offset is dy2: the
// number of radii with (x + 0.5 - gx)^2 + dy2 > r^2 (FP32).
__device__ __forceinline__ int ring_level(const FovDev& a, float gx, float dy2, int32_t x) {
  const float dx = __fsub_rn(__fadd_rn((float)x, 0.5f), gx);
  const float d2 = __fadd_rn(__fmul_rn(dx, dx), dy2);
  int L = 0;
#pragma unroll
  for (int i = 0; i < WRS_MAX_MIP_LEVELS - 1; ++i)
    if (i < a.nradii) L += d2 > a.r2[i];
  return L;
}

__device__ __forceinline__ float row_dy2(float gy, int32_t y) {
  const float dy = __fsub_rn(__fadd_rn((float)y, 0.5f), gy);
  return __fmul_rn(dy, dy);
}

// Colour of pixel (x, y) of the foveated frame at ring level L: level 0
// copies the image pixel; level L takes the level's texel (box) or the
// bilinear blend of its four nearest texel centres.
template <int FILTER>
__device__ __forceinline__ void level_colour(const FovDev& a, int L, int32_t x, int32_t y,
                                             float* rgb) {
  if (L == 0) {
    const float* s = a.img + (int64_t)y * a.pitch + 3 * (int64_t)x;
    rgb[0] = __ldg(s);
    rgb[1] = __ldg(s + 1);
    rgb[2] = __ldg(s + 2);
  } else {
    const MipLevelDev lv = a.lev[L];
    if (FILTER == WRS_FILTER_BOX) {
      const float4 t = __ldg(lv.texels + (int64_t)(y >> L) * lv.wb + (x >> L));
      rgb[0] = t.x;
      rgb[1] = t.y;
      rgb[2] = t.z;
    } else {
      int32_t x0, x1, y0, y1;
      float fx, fy;
      texel_coord(x, L, lv.wb, &x0, &x1, &fx);
      texel_coord(y, L, lv.hb, &y0, &y1, &fy);
      const float4 t00 = __ldg(lv.texels + (int64_t)y0 * lv.wb + x0);
      const float4 t01 = __ldg(lv.texels + (int64_t)y0 * lv.wb + x1);
      const float4 t10 = __ldg(lv.texels + (int64_t)y1 * lv.wb + x0);
      const float4 t11 = __ldg(lv.texels + (int64_t)y1 * lv.wb + x1);
      const float gx_ = __fsub_rn(1.0f, fx), gy_ = __fsub_rn(1.0f, fy);
      rgb[0] = lerp2(lerp2(t00.x, t01.x, gx_, fx), lerp2(t10.x, t11.x, gx_, fx), gy_, fy);
      rgb[1] = lerp2(lerp2(t00.y, t01.y, gx_, fx), lerp2(t10.y, t11.y, gx_, fx), gy_, fy);
      rgb[2] = lerp2(lerp2(t00.z, t01.z, gx_, fx), lerp2(t10.z, t11.z, gx_, fx), gy_, fy);
    }
  }
}

// Colour of pixel (x, y) of the foveated frame for gaze (gx, gy), and its ring
// level (see ring_level and level_colour).
template <int FILTER>
__device__ __forceinline__ int fov_pixel(const FovDev& a, float gx, float gy, int32_t x,
                                         int32_t y, float* rgb) {
  const int L = ring_level(a, gx, row_dy2(gy, y), x);
  level_colour<FILTER>(a, L, x, y, rgb);
  return L;
}

// Four adjacent pixels x0 .. x0+3 of row y: the same colours and levels as
// fov_pixel, with the row's vertical offset computed once and, for bilinear
// filtering when all four share a level, the level's vertical texel
// coordinate and weights too (the common case away from ring boundaries).
// Returns the four levels, one per byte.
template <int FILTER>
__device__ __forceinline__ uint32_t fov_quad(const FovDev& a, float gx, float gy, int32_t x0,
                                             int32_t y, float* rgb) {
  const float dy2 = row_dy2(gy, y);
  int L[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) L[i] = ring_level(a, gx, dy2, x0 + i);
  if (FILTER == WRS_FILTER_BILINEAR && L[0] > 0 && L[0] == L[1] && L[0] == L[2] && L[0] == L[3]) {
    const int l = L[0];
    const MipLevelDev lv = a.lev[l];
    int32_t y0, y1;
    float fy;
    texel_coord(y, l, lv.hb, &y0, &y1, &fy);
    const float gy_ = __fsub_rn(1.0f, fy);
    const float4* row0 = lv.texels + (int64_t)y0 * lv.wb;
    const float4* row1 = lv.texels + (int64_t)y1 * lv.wb;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      int32_t xa, xb;
      float fx;
      texel_coord(x0 + i, l, lv.wb, &xa, &xb, &fx);
      const float4 t00 = __ldg(row0 + xa), t01 = __ldg(row0 + xb);
      const float4 t10 = __ldg(row1 + xa), t11 = __ldg(row1 + xb);
      const float gx_ = __fsub_rn(1.0f, fx);
      float* c = rgb + 3 * i;
      c[0] = lerp2(lerp2(t00.x, t01.x, gx_, fx), lerp2(t10.x, t11.x, gx_, fx), gy_, fy);
      c[1] = lerp2(lerp2(t00.y, t01.y, gx_, fx), lerp2(t10.y, t11.y, gx_, fx), gy_, fy);
      c[2] = lerp2(lerp2(t00.z, t01.z, gx_, fx), lerp2(t10.z, t11.z, gx_, fx), gy_, fy);
    }
  } else {
#pragma unroll
    for (int i = 0; i < 4; ++i) level_colour<FILTER>(a, L[i], x0 + i, y, rgb + 3 * i);
  }
  return (uint32_t)L[0] | ((uint32_t)L[1] << 8) | ((uint32_t)L[2] << 16) | ((uint32_t)L[3] << 24);
}

}  // namespace wrs
