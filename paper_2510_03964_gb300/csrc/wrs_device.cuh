// Device-side arithmetic of the per-pixel weighted reservoir update (sm_103a).
//
// "Enhancing Foveated Rendering with Weighted Reservoir Sampling"
// (arXiv 2510.03964): weight Eq. (cone_retinal_density) + Eq. (phat) (Sec. 4.1),
// A-ES keys (Sec. 3.1), Eq. (temporal-bias) (Sec. 4.2), Alg. 2 (Sec. 3.2).
//
// Every floating-point step that decides which sample a slot holds is an
// explicit round-to-nearest intrinsic (__fadd_rn, __fmul_rn, __fdiv_rn,
// __fsqrt_rn, __fmaf_rn), so the compiler cannot contract or reorder it: the
// stored keys, indices, weights, W and P are a fixed function of the inputs,
// bit for bit.
// The resolve accumulates with explicit fused multiply-adds in slot order, so
// the fused and standalone resolves agree bit for bit too.
#pragma once

#include <cuda_fp16.h>
#include "wrs.h"
#include <stdint.h>

namespace wrs {

constexpr uint32_t kEmpty = 0xFFFFFFFFu;
// planes in the ring of per-frame replacement codes (a power of two)
constexpr int kRingFrames = 16;
constexpr uint32_t kRingMask = kRingFrames - 1;
constexpr float kInf = __builtin_huge_valf();
constexpr float kFltMax = 3.40282346638528859812e+38f;

// ---------------------------------------------------------------- constants
// ln 2 = LN2_HI + LN2_LO with LN2_HI the 12-significant-bit rounding of ln 2
// (n * LN2_HI exact for |n| < 4096) and LN2_LO the float nearest the rest.
constexpr float kLn2Hi = 0x1.62ep-1f;
constexpr float kLn2Lo = 0x1.0bfbe8p-15f;
constexpr float kLog2e = 0x1.715476p+0f;   // float nearest 1/ln 2
constexpr float kSqrt2 = 0x1.6a09e6p+0f;   // float nearest sqrt 2
// floats nearest 1/k! (k = 3..7) and 1/(2k+1) (k = 1..4)
constexpr float kF3 = 0x1.555556p-3f, kF4 = 0x1.555556p-5f, kF5 = 0x1.111112p-7f,
                kF6 = 0x1.6c16c2p-10f, kF7 = 0x1.a01a02p-13f;
constexpr float kQ3 = 0x1.555556p-2f, kQ5 = 0x1.99999ap-3f, kQ7 = 0x1.24924ap-3f,
                kQ9 = 0x1.c71c72p-4f;
// Watson's density parameters as printed with Eq. (cone_retinal_density); r_m,
// absent from the paper, is the cited formula's 41.03 deg.
constexpr float kA = 0.9851f;
// floats nearest 1 / r_2, 1 / r_e, 1 / r_m (each radius first rounded to float)
constexpr float kInvR2 = 0x1.e3ee96p-1f, kInvRe = 0x1.720250p-5f, kInvRm = 0x1.8f514ep-6f;
constexpr float kEccMax = 180.0f;           // eccentricity clamp, degrees
constexpr float kPFloor = 0x1p-64f;         // rescale the bias product below this
constexpr float kPScale = 0x1p64f;

__device__ __forceinline__ float fadd(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float fsub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float fmul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float fdiv(float a, float b) { return __fdiv_rn(a, b); }
__device__ __forceinline__ float ffma(float a, float b, float c) { return __fmaf_rn(a, b, c); }

// exp(x) for x <= 0: x = n ln2 + r, |r| <= ln2/2; Taylor series of exp(r) to
// degree 7 in Horner form; times 2^n through the exponent field.
__device__ __forceinline__ float exp_nonpos(float x) {
  x = fminf(fmaxf(x, -87.0f), 0.0f);
  const float n = rintf(fmul(x, kLog2e));
  float r = ffma(-n, kLn2Hi, x);
  r = ffma(-n, kLn2Lo, r);
  float p = ffma(r, kF7, kF6);
  p = ffma(r, p, kF5);
  p = ffma(r, p, kF4);
  p = ffma(r, p, kF3);
  p = ffma(r, p, 0.5f);
  p = ffma(r, p, 1.0f);
  p = ffma(r, p, 1.0f);
  const int ni = __float2int_rn(n);
  return fmul(p, __uint_as_float(static_cast<uint32_t>(ni + 127) << 23));
}

// ln(u) for normal u > 0: u = m 2^e, m in [sqrt(1/2), sqrt 2); ln m = 2 atanh(s),
// s = (m-1)/(m+1), series in s^2 to s^8/9.
__device__ __forceinline__ float log_pos(float u) {
  const uint32_t b = __float_as_uint(u);
  int e = static_cast<int>((b >> 23) & 0xffu) - 127;
  float m = __uint_as_float((b & 0x007fffffu) | 0x3f800000u);
  if (m > kSqrt2) {
    m = fmul(m, 0.5f);
    e += 1;
  }
  const float s = fdiv(fsub(m, 1.0f), fadd(m, 1.0f));
  const float z = fmul(s, s);
  float q = ffma(z, kQ9, kQ7);
  q = ffma(z, q, kQ5);
  q = ffma(z, q, kQ3);
  q = ffma(z, q, 1.0f);
  const float lnm = fmul(fmul(2.0f, s), q);
  const float fe = __int2float_rn(e);
  return ffma(fe, kLn2Hi, ffma(fe, kLn2Lo, lnm));
}

// Philox4x32-10 (Salmon et al., SC'11): ten rounds, key bumped by the Weyl
// constants between rounds.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r > 0) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
    const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
    c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
  }
  return c;
}

__device__ __forceinline__ uint32_t word(const uint4& v, int i) {
  return i == 0 ? v.x : (i == 1 ? v.y : (i == 2 ? v.z : v.w));
}

// top 24 bits, forced odd, scaled by 2^-24: exact and strictly inside (0, 1)
__device__ __forceinline__ float unit_uniform(uint32_t x) {
  return fmul(__uint2float_rn((x >> 8) | 1u), 0x1p-24f);
}

// d(e) / (2 d_c(0)) of Eq. (cone_retinal_density) as num / den over one
// denominator: num = a + (1-a) exp(-e/r_e) (1+e/r_2)^2,
// den = (1+e/r_2)^2 (1+e/r_m).
__device__ __forceinline__ void density_parts(float e, float& num, float& den) {
  const float t2 = ffma(e, kInvR2, 1.0f);
  const float q = fmul(t2, t2);
  const float tm = ffma(e, kInvRm, 1.0f);
  const float b_term = fmul(fsub(1.0f, kA), exp_nonpos(-fmul(e, kInvRe)));
  num = ffma(b_term, q, kA);
  den = fmul(q, tm);
}

__device__ __forceinline__ float density(float e) {
  float num, den;
  density_parts(e, num, den);
  return fdiv(num, den);
}

// ---------------------------------------------------------------- parameters

struct StreamDev {
  float* W;          // [plane]
  float* P;          // [plane]
  float* key;        // [K][plane]
  uint32_t* idx;     // [K][plane]
  uint16_t* wt;      // FP16 colour: [K][plane] low 16 bits of the slot weights; FP32: unused
  void* col;         // FP32 colour: [K][plane] float4 records {w, r, g, b} (weight and colour
                     // of a slot in one 16-byte entry); FP16 colour: [K][plane] 8-byte
                     // records {r, g, b, w_hi}: the colour as IEEE halves and the high 16
                     // bits of the slot weight (with `wt`, the FP32 weight bit for bit)
  int64_t plane;     // entries per plane (multiple of 64)
  int32_t width, height, K, hw;
  uint32_t width_rcp; // ceil(2^32 / width) (0xFFFFFFFF for width 1): see row_of
  float r_f;         // fovea radius, px
  float delta;       // degrees per px
  uint32_t seed_lo, seed_hi, stream_id;
  int32_t bias;
  int32_t literal;   // 1: the literal n = 1 rule (push_group_literal)
  unsigned long long* replacements;  // running count of slot replacements (stream header)
  uint8_t* maps;     // ring of replacement-code planes [kRingFrames][plane] (primary buffer)
  uint32_t* check;   // checked build: bits of the bounds checks that failed (stream header)
};

// ---------------------------------------------------------------- checked build
// Compiled with WRS_CHECKED, every group of pixels tests the indices it is
// about to use (state planes, shared-memory stage, frame, output, flush map,
// gathered source pixel, bulk-copy ranges) against their buffers first. A
// failed test sets its bit in the stream's check word (state header + 16) and
// the access is skipped; nothing traps. wrs_check_status reports the word.
// Without WRS_CHECKED the tests compile to nothing.
constexpr uint32_t kChkPlane = 1u, kChkStage = 2u, kChkFrame = 4u, kChkOut = 8u, kChkCopy = 16u,
                   kChkGather = 32u, kChkStageSize = 64u;
#ifdef WRS_CHECKED
__device__ __forceinline__ bool in_bounds(uint32_t* word, bool ok, uint32_t bit) {
  if (!ok) atomicOr(word, bit);
  return ok;
}
#define WRS_IN(s, cond, bit) ::wrs::in_bounds((s).check, (cond), (bit))
#else
#define WRS_IN(s, cond, bit) true
#endif

struct FrameDev {
  const float* frame;  // [H][pitch]
  int64_t pitch;
  const uint8_t* fov;  // [H][W] or null
  float* out;          // [H][W][3] or null
  float gx, gy;
  uint32_t t;
  uint32_t map_lo;     // first frame whose codes a folding block still has to apply
};

// (y, x) of pixel p: y = p / width by a multiply-high with ceil(2^32 / width),
// which is off by at most one, then corrected with the remainder.
__device__ __forceinline__ void row_col(const StreamDev& s, int p, int& y, int& x) {
  int q = static_cast<int>(__umulhi(static_cast<uint32_t>(p), s.width_rcp));
  int r = p - q * s.width;
  if (r < 0) {
    q -= 1;
    r += s.width;
  } else if (r >= s.width) {
    q += 1;
    r -= s.width;
  }
  y = q;
  x = r;
}

// CIE 1976 lightness L* of linear-light sRGB (D65): Y = 0.2126 r + 0.7152 g +
// 0.0722 b clamped to [0, 1]; 116 Y^(1/3) - 16 above (6/29)^3 (cube root as
// exp(ln Y / 3) with the routines above), (29/3)^3 Y below.
constexpr float kLumaR = 0.2126f, kLumaG = 0.7152f, kLumaB = 0.0722f;
constexpr float kLabEps = 0x1.22354ep-7f;     // float nearest (6/29)^3 = 216/24389
constexpr float kLabKappa = 0x1.c3a5eep+9f;   // float nearest (29/3)^3 = 24389/27
constexpr float kThird = 0x1.555556p-2f;      // float nearest 1/3

__device__ __forceinline__ float lightness(float r, float g, float b) {
  float Y = ffma(kLumaB, b, ffma(kLumaG, g, fmul(kLumaR, r)));
  Y = fminf(fmaxf(Y, 0.0f), 1.0f);
  if (Y > kLabEps) return ffma(116.0f, exp_nonpos(fmul(log_pos(Y), kThird)), -16.0f);
  return fmul(kLabKappa, Y);
}

// The factor 1 - |Delta L| of Eq. (full-temporal-bias): Delta L is the L*
// difference / 100 (clamped to 1) between the resolved colour of the slots
// before the push and the new sample.
__device__ __forceinline__ float lightness_factor(float n0, float n1, float n2, float den,
                                                  const float (&rgb)[3]) {
  if (!(den > 0.0f)) return 1.0f;
  const float inv = __frcp_rn(den);
  const float l_old = lightness(fmul(n0, inv), fmul(n1, inv), fmul(n2, inv));
  const float l_new = lightness(rgb[0], rgb[1], rgb[2]);
  const float dl = fminf(fmul(fabsf(fsub(l_old, l_new)), 0.01f), 1.0f);
  return fsub(1.0f, dl);
}

// density at the fovea edge, the normaliser of Eq. (phat)
__device__ __forceinline__ float fovea_density(const StreamDev& s) {
  return density(fminf(fmul(s.r_f, s.delta), kEccMax));
}

// Eq. (phat) for one pixel centre; d_f = fovea_density(s).
__device__ __forceinline__ float pixel_weight(const StreamDev& s, float d_f, int x, int y,
                                              float gx, float gy) {
  const float dx = fsub(fadd(__int2float_rn(x), 0.5f), gx);
  const float dy = fsub(fadd(__int2float_rn(y), 0.5f), gy);
  const float d = __fsqrt_rn(fadd(fmul(dx, dx), fmul(dy, dy)));
  if (d <= s.r_f) return 1.0f;
  const float e = fminf(fmul(d, s.delta), kEccMax);
  float num, den;
  density_parts(e, num, den);
  return fminf(fdiv(num, fmul(den, d_f)), 1.0f);
}

// ---------------------------------------------------------------- vector I/O

template <int N> struct VecF;
template <> struct VecF<1> { using T = float; };
template <> struct VecF<2> { using T = float2; };
template <> struct VecF<4> { using T = float4; };

template <int N>
__device__ __forceinline__ void load_f(const float* p, float (&v)[N]) {
  typename VecF<N>::T t = *reinterpret_cast<const typename VecF<N>::T*>(p);
  const float* tf = reinterpret_cast<const float*>(&t);
#pragma unroll
  for (int i = 0; i < N; ++i) v[i] = tf[i];
}

template <int N>
__device__ __forceinline__ void store_f(float* p, const float (&v)[N]) {
  typename VecF<N>::T t;
  float* tf = reinterpret_cast<float*>(&t);
#pragma unroll
  for (int i = 0; i < N; ++i) tf[i] = v[i];
  *reinterpret_cast<typename VecF<N>::T*>(p) = t;
}

// FP16 colour: a slot's FP32 weight from the high half stored in its record's
// fourth half word (rec_hi = the record's second 32-bit word) and the low half
// from the weight plane.
__device__ __forceinline__ float slot_weight_f16(uint32_t rec_hi, uint32_t lo) {
  return __uint_as_float((rec_hi & 0xffff0000u) | (lo & 0xffffu));
}

// Weight and colour of slot j for a group of N pixels whose first entry is at
// `at` in planes of `stride` entries. FP32 colour: one float4 record
// {w, r, g, b} per entry in `col`; FP16 colour: an 8-byte record
// {r, g, b, w_hi} per entry in `col` (colour as halves) and the low 16 bits of
// the weight in the uint16 plane `wt`.
template <bool F16, int N>
__device__ __forceinline__ void load_slot(const uint16_t* wt, const void* col, int K, int j,
                                          int64_t stride, int64_t at, float (&a)[N],
                                          float (&r)[N], float (&g)[N], float (&b)[N]) {
  if constexpr (F16) {
    const uint16_t* lo = wt + j * stride + at;
    const uint2* rec = static_cast<const uint2*>(col) + j * stride + at;
#pragma unroll
    for (int i = 0; i < N; ++i) {
      const uint2 v = rec[i];
      a[i] = slot_weight_f16(v.y, lo[i]);
      r[i] = __half2float(__ushort_as_half(static_cast<unsigned short>(v.x & 0xffffu)));
      g[i] = __half2float(__ushort_as_half(static_cast<unsigned short>(v.x >> 16)));
      b[i] = __half2float(__ushort_as_half(static_cast<unsigned short>(v.y & 0xffffu)));
    }
  } else {
    const float4* rec = static_cast<const float4*>(col) + j * stride + at;
#pragma unroll
    for (int i = 0; i < N; ++i) {
      const float4 v = rec[i];
      a[i] = v.x;
      r[i] = v.y;
      g[i] = v.z;
      b[i] = v.w;
    }
  }
}

// Writes slot j of pixel p (global planes of `plane` entries).
template <bool F16>
__device__ __forceinline__ void store_slot(uint16_t* wt, void* col, int K, int j, int64_t plane,
                                           int64_t p, float w, float r, float g, float b) {
  if constexpr (F16) {
    const uint32_t wb = __float_as_uint(w);
    wt[j * plane + p] = static_cast<uint16_t>(wb & 0xffffu);
    const uint32_t rb = __half_as_ushort(__float2half_rn(r));
    const uint32_t gb = __half_as_ushort(__float2half_rn(g));
    const uint32_t bb = __half_as_ushort(__float2half_rn(b));
    static_cast<uint2*>(col)[j * plane + p] = make_uint2(rb | (gb << 16), bb | (wb & 0xffff0000u));
  } else {
    static_cast<float4*>(col)[j * plane + p] = make_float4(w, r, g, b);
  }
}

// colour as it will be stored in a slot (FP16 storage rounds to nearest even)
template <bool F16>
__device__ __forceinline__ float stored_colour(float c) {
  if constexpr (F16) return __half2float(__float2half_rn(c));
  else return c;
}

// ---------------------------------------------------------------- per-pixel steps

// Eq. (temporal-bias) on the history, then Alg. 2's sum. Returns the race key
// k * P of the new candidate; `rescale` reports a 2^64 rescale of P (the
// stored keys must then be rescaled by the same factor).
__device__ __forceinline__ float bias_and_sum(int bias, float w, float k, float& W, float& P,
                                              bool& rescale, float g = 1.0f) {
  rescale = false;
  if (bias && W > 0.0f) {
    float fb = fdiv(W, fadd(W, w));  // 1 - w / (W + w)
    if (bias == 2) fb = fmul(fb, g);  // Eq. (full-temporal-bias): times 1 - |Delta L|
    W = fmul(W, fb);
    P = fmul(P, fb);
    if (P < kPFloor) {
      P = fmul(P, kPScale);
      rescale = true;
    }
  }
  W = fadd(W, w);
  return fmul(k, P);
}

// stored key as the race sees it this frame (after a flush or a rescale)
__device__ __forceinline__ float race_key(float kv, bool flush, bool rescale) {
  float kj = flush ? kInf : kv;
  if (rescale && kj != kInf) kj = fminf(fmul(kj, kPScale), kFltMax);
  return kj;
}

// Where one group's reservoir planes are read from: global memory (plane
// stride = plane entries, index = pixel) or a shared-memory tile (stride = tile
// entries, index = position in the tile). `frame` points at the group's first
// RGB triple when the group's colours are contiguous, else is null.
struct Src {
  const float* W;
  const float* P;
  const float* key;
  const uint16_t* wt;
  const void* col;
  int64_t stride;
  int64_t at;
  const float* frame;
  const float* u;  // the group's uniforms (u[0..PX-1]) if already drawn, else null
};

__device__ __forceinline__ Src global_src(const StreamDev& s, const FrameDev& f, int p0, bool vec) {
  Src r;
  r.W = s.W; r.P = s.P; r.key = s.key; r.wt = s.wt; r.col = s.col;
  r.stride = s.plane;
  r.at = p0;
  r.frame = nullptr;
  r.u = nullptr;
  if (vec) {
    int y, x;
    row_col(s, p0, y, x);
    r.frame = f.frame + static_cast<int64_t>(y) * f.pitch + 3 * x;
  }
  return r;
}

template <int N>
__device__ __forceinline__ void load_rgb(const float* src, float (&rgb)[N][3]) {
  float v[3 * N];
  if constexpr (N == 4) {
    float a[4], b[4], c[4];
    load_f<4>(src, a);
    load_f<4>(src + 4, b);
    load_f<4>(src + 8, c);
#pragma unroll
    for (int i = 0; i < 4; ++i) { v[i] = a[i]; v[4 + i] = b[i]; v[8 + i] = c[i]; }
  } else if constexpr (N == 2) {
    float a[2], b[2], c[2];
    load_f<2>(src, a);
    load_f<2>(src + 2, b);
    load_f<2>(src + 4, c);
    v[0] = a[0]; v[1] = a[1]; v[2] = b[0]; v[3] = b[1]; v[4] = c[0]; v[5] = c[1];
  } else {
    v[0] = src[0]; v[1] = src[1]; v[2] = src[2];
  }
#pragma unroll
  for (int i = 0; i < N; ++i) {
    rgb[i][0] = v[3 * i]; rgb[i][1] = v[3 * i + 1]; rgb[i][2] = v[3 * i + 2];
  }
}

template <int N>
__device__ __forceinline__ void store_rgb(float* dst, const float (&o)[N][3]) {
  if constexpr (N == 4) {
    float a[4] = {o[0][0], o[0][1], o[0][2], o[1][0]};
    float b[4] = {o[1][1], o[1][2], o[2][0], o[2][1]};
    float c[4] = {o[2][2], o[3][0], o[3][1], o[3][2]};
    store_f<4>(dst, a);
    store_f<4>(dst + 4, b);
    store_f<4>(dst + 8, c);
  } else if constexpr (N == 2) {
    float a[2] = {o[0][0], o[0][1]};
    float b[2] = {o[0][2], o[1][0]};
    float c[2] = {o[1][1], o[1][2]};
    store_f<2>(dst, a);
    store_f<2>(dst + 2, b);
    store_f<2>(dst + 4, c);
  } else {
    dst[0] = o[0][0]; dst[1] = o[0][1]; dst[2] = o[0][2];
  }
}

// ---------------------------------------------------------------- sample indices

// With one or two slots the update writes each sample index straight into
// idx[j] and the state has no code ring: such kernels are bound by
// instruction issue, not by DRAM, and at their low replacement rates the
// ring's per-pixel work costs more than the scattered index writes it saves.
template <int KT>
__device__ __forceinline__ bool direct_index(const StreamDev& s) {
  if constexpr (KT == 1 || KT == 2) return true;
  else if constexpr (KT == 0) return s.K <= 2;
  else return false;
}

// Replacement codes: the slot that took the frame's sample (0..K-1), that
// slot plus kCodeFlush when the history was dropped first (every other slot
// is then empty), or kCodeKeep when the reservoir kept its samples.
constexpr uint8_t kCodeKeep = 0xFFu, kCodeFlush = 0x80u;

// Sample index of slot j after frame `fr` with code c (v before it).
__device__ __forceinline__ uint32_t after_code(uint32_t v, int j, uint8_t c, uint32_t fr) {
  if (c == kCodeKeep) return v;
  if (c & kCodeFlush) return (c & 0x1Fu) == static_cast<uint32_t>(j) ? fr : kEmpty;
  return c == static_cast<uint8_t>(j) ? fr : v;
}

// The band of 256-pixel block b: (b + b/16 + b/256) mod 16. The persistent
// kernels deal tiles to CTAs in arithmetic progressions whose step (the grid,
// 152 SMs x CTAs per SM) is a multiple of 8 or 16, so a band of b % 16 would
// give each CTA all of its folds in one frame out of 16 (the slowest CTA then
// sets the frame's time). Adding the higher base-16 digits makes each CTA's
// blocks run through every band: with 152 or 304 CTAs no CTA folds more than
// 1.05 times its share in any frame.
__device__ __forceinline__ uint32_t fold_band(int64_t p) {
  const uint32_t b = static_cast<uint32_t>(p >> 8);
  return (b + (b >> 4) + (b >> 8)) & kRingMask;
}

// Whether this frame's push folds pixel p's pending codes into its idx
// planes: one band of blocks per frame, band(block) == t % ring.
__device__ __forceinline__ bool folds_now(const FrameDev& f, int64_t p) {
  return ((fold_band(p) ^ f.t) & kRingMask) == 0u;
}

// What a fold reads: pixel p's K sample indices (K <= KM) and its ring codes
// of the frames t-15 .. t-1 (byte k of the 16: frame t-15+k). All loads are
// issued at once, so a fold costs one memory round trip, and the pipelined
// kernels issue them before waiting for the tile, hiding even that.
template <int KM>
struct FoldIn {
  uint32_t v[KM];
  uint32_t code[kRingFrames / 4];
};

// Capacity of the fold inputs of a kernel instantiated for KT slots (0: any
// K): exactly KT, so that a kernel for few slots holds no unused registers.
template <int KT>
struct FoldCap {
  static constexpr int value = (KT > 0 && KT <= 8) ? KT : WRS_MAX_K;
};

template <int KT>
using FoldFor = FoldIn<FoldCap<KT>::value>;

template <int KM>
__device__ __forceinline__ void fold_load(const StreamDev& s, const uint32_t* idx, int K,
                                          uint32_t t, int64_t p, FoldIn<KM>& in) {
  const int64_t pl = s.plane;
#pragma unroll
  for (int j = 0; j < KM; ++j) in.v[j] = j < K ? idx[j * pl + p] : kEmpty;
  uint8_t b[kRingFrames];
#pragma unroll
  for (int k = 0; k < kRingFrames - 1; ++k) {
    const uint32_t fr = t - static_cast<uint32_t>(kRingFrames - 1) + k;
    b[k] = s.maps[static_cast<int64_t>(fr & kRingMask) * pl + p];
  }
  b[kRingFrames - 1] = kCodeKeep;
#pragma unroll
  for (int w = 0; w < kRingFrames / 4; ++w)
    in.code[w] = static_cast<uint32_t>(b[4 * w]) | (static_cast<uint32_t>(b[4 * w + 1]) << 8) |
                 (static_cast<uint32_t>(b[4 * w + 2]) << 16) |
                 (static_cast<uint32_t>(b[4 * w + 3]) << 24);
}

// Applies the loaded codes of frames lo .. t-1 (older ring entries, and
// entries of frames before lo, are skipped) and then, if c_now is not
// kCodeKeep, code c_now of frame t; writes pixel p's K indices to `idx`.
template <int KM>
__device__ __forceinline__ void fold_store(const StreamDev& s, uint32_t* idx, int K, uint32_t t,
                                           uint32_t lo, int64_t p, const FoldIn<KM>& in,
                                           uint8_t c_now) {
  const int64_t pl = s.plane;
  uint32_t v[KM];
#pragma unroll
  for (int j = 0; j < KM; ++j) v[j] = in.v[j];
#pragma unroll
  for (int k = 0; k < kRingFrames - 1; ++k) {
    const uint32_t fr = t - static_cast<uint32_t>(kRingFrames - 1) + k;
    const uint8_t c = static_cast<uint8_t>(in.code[k >> 2] >> (8 * (k & 3)));
    if (fr >= lo && fr < t && c != kCodeKeep) {
#pragma unroll
      for (int j = 0; j < KM; ++j) v[j] = after_code(v[j], j, c, fr);
    }
  }
  if (c_now != kCodeKeep) {
#pragma unroll
    for (int j = 0; j < KM; ++j) v[j] = after_code(v[j], j, c_now, t);
  }
#pragma unroll
  for (int j = 0; j < KM; ++j)
    if (j < K) idx[j * pl + p] = v[j];
}

// This frame's code of pixel p into the ring and, for the band this frame
// folds, every pending code into the idx planes (from `pre` when the fold's
// inputs were loaded ahead, else loaded here). KM >= K: the capacity of the
// preloaded inputs (a batched kernel loads for up to 8 slots whatever the
// stream's K; entries past K are dead code once K is a constant).
template <int KT, int KM = FoldCap<KT>::value>
__device__ __forceinline__ void record_code(const StreamDev& s, const FrameDev& f, int64_t p,
                                            uint8_t c, const FoldIn<KM>* pre) {
  const int K = KT > 0 ? KT : s.K;
  s.maps[static_cast<int64_t>(f.t & kRingMask) * s.plane + p] = c;
  if (!folds_now(f, p)) return;
  if (pre != nullptr) {
    fold_store(s, s.idx, K, f.t, f.map_lo, p, *pre, c);
  } else {
    FoldFor<KT> in;
    fold_load(s, s.idx, K, f.t, p, in);
    fold_store(s, s.idx, K, f.t, f.map_lo, p, in, c);
  }
}

// ---------------------------------------------------------------- the pixel group

// Checked build: the indices a group of PX pixels at p0 uses, against their
// buffers: state-plane entries p0 .. p0+PX-1 (writes, and reads through
// global planes), source entries at src.at in planes of src.stride entries
// (the shared-memory stage or the global planes), the pixels' frame rows and
// columns and the output. True in the default build.
template <int PX, bool VEC>
__device__ __forceinline__ bool group_in_bounds(const StreamDev& s, const FrameDev& f, int p0,
                                                const Src& src, const bool (&valid)[PX],
                                                const int (&xs)[PX], const int (&ys)[PX]) {
#ifdef WRS_CHECKED
  bool ok = WRS_IN(s, p0 >= 0 && static_cast<int64_t>(p0) + PX <= s.plane, kChkPlane);
  ok = WRS_IN(s, src.at >= 0 && src.at + PX <= src.stride, kChkStage) && ok;
#pragma unroll
  for (int i = 0; i < PX; ++i) {
    if (!valid[i]) continue;
    ok = WRS_IN(s, ys[i] >= 0 && ys[i] < s.height && xs[i] >= 0 && xs[i] < s.width &&
                       static_cast<int64_t>(ys[i]) * s.width + xs[i] == static_cast<int64_t>(p0) + i,
                kChkFrame) && ok;
    if (f.frame != nullptr && (src.frame == nullptr || src.stride == s.plane))
      ok = WRS_IN(s, static_cast<int64_t>(ys[i]) * f.pitch + 3 * xs[i] + 3 <=
                         static_cast<int64_t>(s.height) * f.pitch,
                  kChkFrame) && ok;
  }
  if (VEC && f.out != nullptr)
    ok = WRS_IN(s, (static_cast<int64_t>(ys[0]) * s.width + xs[0] + PX) * 3 <= 3ll * s.hw, kChkOut) && ok;
  return ok;
#else
  (void)s; (void)f; (void)p0; (void)src; (void)valid; (void)xs; (void)ys;
  return true;
#endif
}

// One thread's group of PX consecutive pixels p0 .. p0+PX-1 (p0 % PX == 0):
// weight, key, bias, key race over the K slots, fused resolve, stores. Reads
// the reservoir through `src` (global planes or a shared-memory tile); writes
// always go to the global planes. KT > 0 fixes K at compile time. VEC: the
// group lies in one row and src.frame / f.out take vector accesses; otherwise
// every pixel is addressed on its own (and may lie past the end of the image).
// FOV: a flush map is present (f.fov != null); without one the flush logic is
// compiled out.
template <int KT, bool F16, int PX, bool VEC, bool FOV, int KM = FoldCap<KT>::value>
__device__ __forceinline__ int push_group(const StreamDev& s, const FrameDev& f, int p0,
                                          const Src& src, float d_f,
                                          const FoldIn<KM>* pre = nullptr) {
  const int K = KT > 0 ? KT : s.K;
  const int64_t pl = s.plane;
  const int64_t ss = src.stride;
  const int64_t sa = src.at;

  bool valid[PX];
  int xs[PX], ys[PX];
  if constexpr (VEC) {
    int y, x;
    row_col(s, p0, y, x);
#pragma unroll
    for (int i = 0; i < PX; ++i) {
      valid[i] = true;
      xs[i] = x + i;
      ys[i] = y;
    }
  } else {
#pragma unroll
    for (int i = 0; i < PX; ++i) {
      const int p = p0 + i;
      valid[i] = p < s.hw;
      ys[i] = 0;
      xs[i] = 0;
      if (valid[i]) row_col(s, p, ys[i], xs[i]);
    }
  }

  if (!group_in_bounds<PX, VEC>(s, f, p0, src, valid, xs, ys)) return 0;

  // incoming colours
  float rgb[PX][3];
  if constexpr (VEC) {
    load_rgb<PX>(src.frame, rgb);
  } else {
#pragma unroll
    for (int i = 0; i < PX; ++i) {
      if (valid[i]) {
        const float* fp = src.frame ? src.frame + 3 * i
                                    : f.frame + static_cast<int64_t>(ys[i]) * f.pitch + 3 * xs[i];
        rgb[i][0] = fp[0]; rgb[i][1] = fp[1]; rgb[i][2] = fp[2];
      } else {
        rgb[i][0] = rgb[i][1] = rgb[i][2] = 0.0f;
      }
    }
  }

  bool flush[PX];
#pragma unroll
  for (int i = 0; i < PX; ++i) flush[i] = FOV && valid[i] && f.fov[p0 + i] == 0xFFu;

  // uniforms: one Philox block per 4 consecutive pixels, word p mod 4 (PX divides
  // 4 and p0 % PX == 0, so the group never straddles two blocks)
  static_assert(4 % PX == 0, "pixels per thread must divide 4");
  float u[PX];
  if (src.u != nullptr) {
#pragma unroll
    for (int i = 0; i < PX; ++i) u[i] = src.u[i];
  } else {
    const uint4 blk = philox4x32_10(
        make_uint4(static_cast<uint32_t>(p0) >> 2, f.t, s.stream_id, 0u), s.seed_lo, s.seed_hi);
#pragma unroll
    for (int i = 0; i < PX; ++i) u[i] = unit_uniform(word(blk, (p0 + i) & 3));
  }

  // weight (Eq. phat) and A-ES key -ln(u)/w
  float w[PX], k[PX];
#pragma unroll
  for (int i = 0; i < PX; ++i) {
    w[i] = valid[i] ? pixel_weight(s, d_f, xs[i], ys[i], f.gx, f.gy) : 1.0f;
    k[i] = fdiv(-log_pos(u[i]), w[i]);
  }

  // Eq. (temporal-bias) on the history, then Alg. 2's sum
  float Wv[PX], Pv[PX];
  load_f<PX>(src.W + sa, Wv);
  load_f<PX>(src.P + sa, Pv);
  float gl[PX];
#pragma unroll
  for (int i = 0; i < PX; ++i) gl[i] = 1.0f;
  if (s.bias == 2) {
    // Eq. (full-temporal-bias): resolved colour of the slots before the push
    float n0[PX], n1[PX], n2[PX], dn[PX];
#pragma unroll
    for (int i = 0; i < PX; ++i) { n0[i] = n1[i] = n2[i] = dn[i] = 0.0f; }
    for (int j = 0; j < K; ++j) {
      float a[PX], r[PX], g[PX], b[PX];
      load_slot<F16, PX>(src.wt, src.col, K, j, ss, sa, a, r, g, b);
#pragma unroll
      for (int i = 0; i < PX; ++i) {
        n0[i] = __fmaf_rn(a[i], r[i], n0[i]);
        n1[i] = __fmaf_rn(a[i], g[i], n1[i]);
        n2[i] = __fmaf_rn(a[i], b[i], n2[i]);
        dn[i] = fadd(dn[i], a[i]);
      }
    }
#pragma unroll
    for (int i = 0; i < PX; ++i) {
      if (!valid[i] || flush[i] || !(Wv[i] > 0.0f)) continue;
      gl[i] = lightness_factor(n0[i], n1[i], n2[i], dn[i], rgb[i]);
      if (gl[i] <= 0.0f) flush[i] = true;  // no weight left in the history
    }
  }
  bool rescale[PX];
  float ks[PX];
#pragma unroll
  for (int i = 0; i < PX; ++i) {
    rescale[i] = false;
    if (!valid[i]) { ks[i] = kInf; continue; }
    if (flush[i]) { Wv[i] = 0.0f; Pv[i] = 1.0f; }
    ks[i] = bias_and_sum(s.bias, w[i], k[i], Wv[i], Pv[i], rescale[i], gl[i]);
  }

  // key race: the slot holding the largest key (lowest index on ties; an empty
  // slot holds +inf) is replaced iff the new key is strictly smaller
  float kmax[PX];
  int jm[PX];
#pragma unroll
  for (int i = 0; i < PX; ++i) { kmax[i] = -1.0f; jm[i] = 0; }
#pragma unroll 8
  for (int j = 0; j < K; ++j) {
    float kv[PX];
    load_f<PX>(src.key + j * ss + sa, kv);
#pragma unroll
    for (int i = 0; i < PX; ++i) {
      const float kj = race_key(kv[i], flush[i], rescale[i]);
      if (kj > kmax[i]) { kmax[i] = kj; jm[i] = j; }
    }
  }
  bool repl[PX];
  float cst[PX][3];
#pragma unroll
  for (int i = 0; i < PX; ++i) {
    repl[i] = valid[i] && ks[i] < kmax[i];
    cst[i][0] = stored_colour<F16>(rgb[i][0]);
    cst[i][1] = stored_colour<F16>(rgb[i][1]);
    cst[i][2] = stored_colour<F16>(rgb[i][2]);
  }

  // fused resolve over the slots as they will be after this push
  if (f.out != nullptr) {
    float num[PX][3], den[PX];
#pragma unroll
    for (int i = 0; i < PX; ++i) { num[i][0] = num[i][1] = num[i][2] = 0.0f; den[i] = 0.0f; }
#pragma unroll 4
    for (int j = 0; j < K; ++j) {
      float wv[PX], c0[PX], c1[PX], c2[PX];
      load_slot<F16, PX>(src.wt, src.col, K, j, ss, sa, wv, c0, c1, c2);
#pragma unroll
      for (int i = 0; i < PX; ++i) {
        float a = wv[i], r = c0[i], g = c1[i], b = c2[i];
        if (flush[i]) { a = 0.0f; r = g = b = 0.0f; }
        if (repl[i] && jm[i] == j) { a = w[i]; r = cst[i][0]; g = cst[i][1]; b = cst[i][2]; }
        num[i][0] = __fmaf_rn(a, r, num[i][0]);
        num[i][1] = __fmaf_rn(a, g, num[i][1]);
        num[i][2] = __fmaf_rn(a, b, num[i][2]);
        den[i] = fadd(den[i], a);
      }
    }
    float o[PX][3];
#pragma unroll
    for (int i = 0; i < PX; ++i) {
      const float inv = den[i] > 0.0f ? __frcp_rn(den[i]) : 0.0f;
      o[i][0] = fmul(num[i][0], inv);
      o[i][1] = fmul(num[i][1], inv);
      o[i][2] = fmul(num[i][2], inv);
    }
    if constexpr (VEC) {
      store_rgb<PX>(f.out + (static_cast<int64_t>(ys[0]) * s.width + xs[0]) * 3, o);
    } else {
#pragma unroll
      for (int i = 0; i < PX; ++i) {
        if (!valid[i]) continue;
        float* dst = f.out + static_cast<int64_t>(p0 + i) * 3;
        dst[0] = o[i][0]; dst[1] = o[i][1]; dst[2] = o[i][2];
      }
    }
  }

  // stores: running sums, the replaced slot, rescaled keys, flushed slots
  store_f<PX>(s.W + p0, Wv);
  store_f<PX>(s.P + p0, Pv);
#pragma unroll
  for (int i = 0; i < PX; ++i) {
    if (!valid[i]) continue;
    const int64_t p = p0 + i;
    if (rescale[i] && !flush[i]) {
      for (int j = 0; j < K; ++j) {
        const float kj = src.key[j * ss + sa + i];
        if (kj != kInf) s.key[j * pl + p] = fminf(fmul(kj, kPScale), kFltMax);
      }
    }
    const bool direct = direct_index<KT>(s);
    if (flush[i]) {
      for (int j = 0; j < K; ++j) {
        if (j == jm[i]) continue;
        s.key[j * pl + p] = kInf;
        if (direct) s.idx[j * pl + p] = kEmpty;
        store_slot<F16>(s.wt, s.col, K, j, pl, p, 0.0f, 0.0f, 0.0f, 0.0f);
      }
    }
    if (repl[i]) {
      const int j = jm[i];
      s.key[j * pl + p] = ks[i];
      if (direct) s.idx[j * pl + p] = f.t;
      store_slot<F16>(s.wt, s.col, K, j, pl, p, w[i], rgb[i][0], rgb[i][1], rgb[i][2]);
    }
    if (!direct) {
      // the sample index goes to the ring as a code
      const uint8_t code = repl[i] ? static_cast<uint8_t>(jm[i] | (flush[i] ? kCodeFlush : 0u))
                                   : (flush[i] ? kCodeFlush : kCodeKeep);
      record_code<KT, KM>(s, f, p, code, PX == 1 ? pre : nullptr);
    }
  }
  int replaced = 0;
#pragma unroll
  for (int i = 0; i < PX; ++i) replaced += repl[i] ? 1 : 0;
  return replaced;
}

// The paper's n = 1 update taken literally (Sec. 4.2): Eq. (temporal-bias) on
// W = R1.wsum, then Alg. 2 keeps R1 iff u * (W' + w) <= W', else takes the new
// sample; W <- W' + w. One slot (K = 1), no key and no bias product: the P
// and key planes are neither read nor written. Same frame, weight, uniform,
// resolve and store code as the key race.
template <bool F16, int PX, bool VEC, bool FOV>
__device__ __forceinline__ int push_group_literal(const StreamDev& s, const FrameDev& f, int p0,
                                                  const Src& src, float d_f) {
  const int64_t pl = s.plane;
  const int64_t ss = src.stride;
  const int64_t sa = src.at;
  bool valid[PX];
  int xs[PX], ys[PX];
  if constexpr (VEC) {
    int y, x;
    row_col(s, p0, y, x);
#pragma unroll
    for (int i = 0; i < PX; ++i) {
      valid[i] = true;
      xs[i] = x + i;
      ys[i] = y;
    }
  } else {
#pragma unroll
    for (int i = 0; i < PX; ++i) {
      const int p = p0 + i;
      valid[i] = p < s.hw;
      ys[i] = 0;
      xs[i] = 0;
      if (valid[i]) row_col(s, p, ys[i], xs[i]);
    }
  }
  if (!group_in_bounds<PX, VEC>(s, f, p0, src, valid, xs, ys)) return 0;
  float rgb[PX][3];
  if constexpr (VEC) {
    load_rgb<PX>(src.frame, rgb);
  } else {
#pragma unroll
    for (int i = 0; i < PX; ++i) {
      if (valid[i]) {
        const float* fp = src.frame ? src.frame + 3 * i
                                    : f.frame + static_cast<int64_t>(ys[i]) * f.pitch + 3 * xs[i];
        rgb[i][0] = fp[0]; rgb[i][1] = fp[1]; rgb[i][2] = fp[2];
      } else {
        rgb[i][0] = rgb[i][1] = rgb[i][2] = 0.0f;
      }
    }
  }
  bool flush[PX];
#pragma unroll
  for (int i = 0; i < PX; ++i) flush[i] = FOV && valid[i] && f.fov[p0 + i] == 0xFFu;
  static_assert(4 % PX == 0, "pixels per thread must divide 4");
  float u[PX];
  if (src.u != nullptr) {
#pragma unroll
    for (int i = 0; i < PX; ++i) u[i] = src.u[i];
  } else {
    const uint4 blk = philox4x32_10(
        make_uint4(static_cast<uint32_t>(p0) >> 2, f.t, s.stream_id, 0u), s.seed_lo, s.seed_hi);
#pragma unroll
    for (int i = 0; i < PX; ++i) u[i] = unit_uniform(word(blk, (p0 + i) & 3));
  }
  float w[PX];
#pragma unroll
  for (int i = 0; i < PX; ++i) w[i] = valid[i] ? pixel_weight(s, d_f, xs[i], ys[i], f.gx, f.gy) : 1.0f;

  float Wv[PX];
  load_f<PX>(src.W + sa, Wv);
  float gl[PX];
#pragma unroll
  for (int i = 0; i < PX; ++i) gl[i] = 1.0f;
  if (s.bias == 2) {
    // Eq. (full-temporal-bias): Delta L against the resident sample
    float a[PX], r[PX], g[PX], b[PX];
    load_slot<F16, PX>(src.wt, src.col, 1, 0, ss, sa, a, r, g, b);
#pragma unroll
    for (int i = 0; i < PX; ++i) {
      if (!valid[i] || flush[i] || !(Wv[i] > 0.0f)) continue;
      gl[i] = lightness_factor(__fmaf_rn(a[i], r[i], 0.0f), __fmaf_rn(a[i], g[i], 0.0f),
                               __fmaf_rn(a[i], b[i], 0.0f), fadd(0.0f, a[i]), rgb[i]);
      if (gl[i] <= 0.0f) flush[i] = true;
    }
  }
  bool take[PX];
#pragma unroll
  for (int i = 0; i < PX; ++i) {
    take[i] = false;
    if (!valid[i]) continue;
    if (flush[i]) Wv[i] = 0.0f;
    if (s.bias && Wv[i] > 0.0f) {
      float fb = fdiv(Wv[i], fadd(Wv[i], w[i]));
      if (s.bias == 2) fb = fmul(fb, gl[i]);
      Wv[i] = fmul(Wv[i], fb);
    }
    const float tot = fadd(Wv[i], w[i]);
    take[i] = !(fmul(u[i], tot) <= Wv[i]);  // Alg. 2: R1 kept on <=
    Wv[i] = tot;
  }

  if (f.out != nullptr) {
    float wv[PX], c0[PX], c1[PX], c2[PX];
    load_slot<F16, PX>(src.wt, src.col, 1, 0, ss, sa, wv, c0, c1, c2);
    float o[PX][3];
#pragma unroll
    for (int i = 0; i < PX; ++i) {
      float a = wv[i], r = c0[i], g = c1[i], b = c2[i];
      if (take[i]) {
        a = w[i];
        r = stored_colour<F16>(rgb[i][0]);
        g = stored_colour<F16>(rgb[i][1]);
        b = stored_colour<F16>(rgb[i][2]);
      }
      const float num0 = __fmaf_rn(a, r, 0.0f), num1 = __fmaf_rn(a, g, 0.0f),
                  num2 = __fmaf_rn(a, b, 0.0f);
      const float den = fadd(0.0f, a);
      const float inv = den > 0.0f ? __frcp_rn(den) : 0.0f;
      o[i][0] = fmul(num0, inv);
      o[i][1] = fmul(num1, inv);
      o[i][2] = fmul(num2, inv);
    }
    if constexpr (VEC) {
      store_rgb<PX>(f.out + (static_cast<int64_t>(ys[0]) * s.width + xs[0]) * 3, o);
    } else {
#pragma unroll
      for (int i = 0; i < PX; ++i) {
        if (!valid[i]) continue;
        float* dst = f.out + static_cast<int64_t>(p0 + i) * 3;
        dst[0] = o[i][0]; dst[1] = o[i][1]; dst[2] = o[i][2];
      }
    }
  }
  store_f<PX>(s.W + p0, Wv);
  int taken = 0;
#pragma unroll
  for (int i = 0; i < PX; ++i) {
    if (!valid[i]) continue;
    const int64_t p = p0 + i;
    if (take[i]) {
      s.idx[p] = f.t;  // one slot: the index is written directly (direct_index)
      store_slot<F16>(s.wt, s.col, 1, 0, pl, p, w[i], rgb[i][0], rgb[i][1], rgb[i][2]);
      taken += 1;
    }
  }
  return taken;
}

// Standalone resolve of one group: the same accumulation as the fused resolve.
template <int KT, bool F16, int PX>
__device__ __forceinline__ void resolve_group(const StreamDev& s, float* out, int p0) {
  const int K = KT > 0 ? KT : s.K;
  const int64_t pl = s.plane;
  if (!WRS_IN(s, p0 >= 0 && static_cast<int64_t>(p0) + PX <= pl, kChkPlane)) return;
  float num[PX][3], den[PX];
#pragma unroll
  for (int i = 0; i < PX; ++i) { num[i][0] = num[i][1] = num[i][2] = 0.0f; den[i] = 0.0f; }
#pragma unroll 4
  for (int j = 0; j < K; ++j) {
    float wv[PX], c0[PX], c1[PX], c2[PX];
    load_slot<F16, PX>(s.wt, s.col, K, j, pl, p0, wv, c0, c1, c2);
#pragma unroll
    for (int i = 0; i < PX; ++i) {
      num[i][0] = __fmaf_rn(wv[i], c0[i], num[i][0]);
      num[i][1] = __fmaf_rn(wv[i], c1[i], num[i][1]);
      num[i][2] = __fmaf_rn(wv[i], c2[i], num[i][2]);
      den[i] = fadd(den[i], wv[i]);
    }
  }
#pragma unroll
  for (int i = 0; i < PX; ++i) {
    if (p0 + i >= s.hw) continue;
    const float inv = den[i] > 0.0f ? __frcp_rn(den[i]) : 0.0f;
    float* dst = out + static_cast<int64_t>(p0 + i) * 3;
    dst[0] = fmul(num[i][0], inv);
    dst[1] = fmul(num[i][1], inv);
    dst[2] = fmul(num[i][2], inv);
  }
}

}  // namespace wrs
