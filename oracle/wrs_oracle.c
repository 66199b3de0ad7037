/*
 * CPU oracle for per-pixel weighted reservoir sampling (WRS) on foveated frame
 * streams. TEST INFRASTRUCTURE ONLY: see wrs_oracle.h.
 *
 * Build: gcc -std=c11 -O2 -ffp-contract=off (no fast-math). Every float
 * expression below is evaluated as written, one IEEE round-to-nearest-even
 * operation at a time; the only fused multiply-adds are the explicit fmaf
 * calls (one rounding each), never contracted ones.
 *
 * Paper references are to "Enhancing Foveated Rendering with Weighted
 * Reservoir Sampling" (arXiv 2510.03964):
 *   Eq. (cone_retinal_density)  retinal density d(e), Sec. 4.1
 *   Eq. (phat)                  perceptual weight w(e), Sec. 4.1
 *   Eq. (chao-selection-probability), Alg. 1 (A-Chao), Sec. 3.1
 *   A-ES random keys (largest u^(1/w) kept), Sec. 3.1
 *   Alg. 2 (Combine Reservoirs), Sec. 3.2
 *   Eq. (p_survive_reservoir), Eq. (temporal-bias), Sec. 4.2
 */
#include "wrs_oracle.h"

#include <float.h>
#include <math.h>
#include <pthread.h>
#include <stdlib.h>
#include <string.h>

/* ---------------------------------------------------------------- exp, log */

/* ln 2 split for range reduction: LN2_HI is ln 2 rounded to 12 significant
 * bits, so n * LN2_HI is exact for |n| < 2^12; LN2_LO is the float nearest
 * to ln 2 - LN2_HI. */
static const float LN2_HI = 0x1.62ep-1f;
static const float LN2_LO = 0x1.0bfbe8p-15f;
static const float LOG2E = 0x1.715476p+0f;   /* float nearest to 1 / ln 2 */
static const float SQRT2 = 0x1.6a09e6p+0f;   /* float nearest to sqrt(2) */

static float scale_pow2(float p, int n) {
  /* p * 2^n for -126 <= n <= 127 via the exponent field (exact product). */
  union { uint32_t u; float f; } s;
  s.u = (uint32_t)(n + 127) << 23;
  return p * s.f;
}

float orc_exp(float x) {
  /* exp(x) = 2^n exp(r), n = rint(x / ln 2), r = x - n ln 2 in [-ln2/2, ln2/2].
   * exp(r) by its Taylor series to r^7/7! (truncation < 2^-27 relative), in
   * Horner form with fused multiply-adds (fmaf: one IEEE rounding each).
   * Coefficients are the floats nearest to 1/k!. */
  if (x < -87.0f) x = -87.0f;
  if (x > 0.0f) x = 0.0f;
  float n = rintf(x * LOG2E);
  float r = fmaf(-n, LN2_HI, x);
  r = fmaf(-n, LN2_LO, r);
  const float c2 = 1.0f / 2.0f, c3 = 1.0f / 6.0f, c4 = 1.0f / 24.0f, c5 = 1.0f / 120.0f,
              c6 = 1.0f / 720.0f, c7 = 1.0f / 5040.0f;
  float p = fmaf(r, c7, c6);
  p = fmaf(r, p, c5);
  p = fmaf(r, p, c4);
  p = fmaf(r, p, c3);
  p = fmaf(r, p, c2);
  p = fmaf(r, p, 1.0f);
  p = fmaf(r, p, 1.0f);
  return scale_pow2(p, (int)n);
}

float orc_log(float u) {
  /* u = m 2^e with m in [sqrt(1/2), sqrt(2)); ln m = 2 atanh(s), s = (m-1)/(m+1),
   * atanh(s) = s (1 + s^2/3 + s^4/5 + s^6/7 + s^8/9 + ...), |s| <= 0.1716, so the
   * dropped terms are below 2^-27 relative. ln u = e ln 2 + ln m. */
  union { float f; uint32_t u; } b;
  b.f = u;
  int e = (int)((b.u >> 23) & 0xffu) - 127;
  union { uint32_t u; float f; } mb;
  mb.u = (b.u & 0x007fffffu) | 0x3f800000u;   /* m in [1, 2) */
  float m = mb.f;
  if (m > SQRT2) {
    m = m * 0.5f;
    e = e + 1;
  }
  float s = (m - 1.0f) / (m + 1.0f);
  float z = s * s;
  const float q3 = 1.0f / 3.0f, q5 = 1.0f / 5.0f, q7 = 1.0f / 7.0f, q9 = 1.0f / 9.0f;
  float q = fmaf(z, q9, q7);
  q = fmaf(z, q, q5);
  q = fmaf(z, q, q3);
  q = fmaf(z, q, 1.0f);
  float lnm = (2.0f * s) * q;
  float fe = (float)e;
  return fmaf(fe, LN2_HI, fmaf(fe, LN2_LO, lnm));
}

/* ---------------------------------------------------------------- Philox */

/* Philox4x32-10 as published by Salmon, Moraes, Dror and Shaw ("Parallel
 * random numbers: as easy as 1, 2, 3", SC'11): ten rounds of two 32x32->64
 * multiplications on the counter, with the key bumped by the Weyl constants
 * between rounds. */
static const uint32_t PHILOX_M0 = 0xD2511F53u, PHILOX_M1 = 0xCD9E8D57u;
static const uint32_t PHILOX_W0 = 0x9E3779B9u, PHILOX_W1 = 0xBB67AE85u;

void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
  uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
  uint32_t k0 = key[0], k1 = key[1];
  for (int round = 0; round < 10; ++round) {
    if (round > 0) {
      k0 += PHILOX_W0;
      k1 += PHILOX_W1;
    }
    uint64_t p0 = (uint64_t)PHILOX_M0 * (uint64_t)c0;
    uint64_t p1 = (uint64_t)PHILOX_M1 * (uint64_t)c2;
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t n0 = hi1 ^ c1 ^ k0;
    uint32_t n1 = lo1;
    uint32_t n2 = hi0 ^ c3 ^ k1;
    uint32_t n3 = lo0;
    c0 = n0; c1 = n1; c2 = n2; c3 = n3;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

float orc_uniform(uint64_t seed, uint32_t stream_id, uint32_t t, int64_t p) {
  /* One Philox block serves four consecutive pixels: counter (p/4, t, stream, 0),
   * word p mod 4. The top 24 bits, forced odd, times 2^-24: exact, in (0, 1). */
  uint32_t ctr[4] = {(uint32_t)(p >> 2), t, stream_id, 0u};
  uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  uint32_t out[4];
  orc_philox4x32_10(ctr, key, out);
  uint32_t x = out[p & 3];
  return (float)((x >> 8) | 1u) * 0x1p-24f;
}

/* ---------------------------------------------------------------- weight */

/* Watson's parameters as the paper lists them (Sec. 4.1): a_k, r_2k, r_ek,
 * d_c(0). The paper omits r_m; 41.03 deg is the value in the cited Watson
 * (2014) formula. */
static const double AK_D = 0.9851, R2_D = 1.058, RE_D = 22.14, RM_D = 41.03, DC0_D = 14804.6;
static const float AK_F = 0.9851f;
/* reciprocals of the radii, each the float nearest 1 / (float radius) */
static const float INV_R2_F = 1.0f / 1.058f, INV_RE_F = 1.0f / 22.14f, INV_RM_F = 1.0f / 41.03f;
/* Eccentricities are clamped to this many degrees (beyond the visual field). */
static const float E_MAX = 180.0f;

double orc_density64(double e) {
  /* Eq. (cone_retinal_density), term by term. */
  double radial = 1.0 / (1.0 + e / RM_D);
  double near = AK_D * pow(1.0 + e / R2_D, -2.0);
  double far = (1.0 - AK_D) * exp(-e / RE_D);
  return 2.0 * DC0_D * radial * (near + far);
}

/* d(e) / (2 d_c(0)) of Eq. (cone_retinal_density) over one common denominator:
 *   [a (1+e/r_2)^-2 + (1-a) exp(-e/r_e)] / (1+e/r_m)
 *     = [a + (1-a) exp(-e/r_e) (1+e/r_2)^2] / [(1+e/r_2)^2 (1+e/r_m)]
 * in the fixed order
 *   t2 = fma(e, 1/r_2, 1);  q = t2*t2;  tm = fma(e, 1/r_m, 1);
 *   B = (1-a) exp(-(e * (1/r_e)));  num = fma(B, q, a);  den = q*tm. */
static void orc_density_parts(float e, float* num, float* den) {
  float t2 = fmaf(e, INV_R2_F, 1.0f);
  float q = t2 * t2;
  float tm = fmaf(e, INV_RM_F, 1.0f);
  float one_minus_a = 1.0f - AK_F;
  float B = one_minus_a * orc_exp(-(e * INV_RE_F));
  *num = fmaf(B, q, AK_F);
  *den = q * tm;
}

float orc_density32(float e) {
  float num, den;
  orc_density_parts(e, &num, &den);
  return num / den;
}

float orc_delta(const orc_config* cfg) {
  /* Default pixel scale: the foveal radius spans the 2.5 deg at which the
   * paper normalises the weight (Fig. phat caption). */
  return cfg->deg_per_px > 0.0f ? cfg->deg_per_px : 2.5f / cfg->r_f;
}

float orc_weight32(const orc_config* cfg, int32_t x, int32_t y, float gx, float gy) {
  /* Eq. (phat): 1 inside the fovea (e <= r_f, tested in pixels), else
   * d(e) / d(r_f), clamped to 1 against FP32 rounding. */
  float dx = ((float)x + 0.5f) - gx;
  float dy = ((float)y + 0.5f) - gy;
  float d = sqrtf(dx * dx + dy * dy);
  if (d <= cfg->r_f) return 1.0f;
  float delta = orc_delta(cfg);
  float e = d * delta;
  if (e > E_MAX) e = E_MAX;
  float ef = cfg->r_f * delta;
  if (ef > E_MAX) ef = E_MAX;
  /* d(e)/d(e_f) = num / (den * d(e_f)) with d(e_f) = num_f / den_f */
  float num, den;
  orc_density_parts(e, &num, &den);
  float w = num / (den * orc_density32(ef));
  if (w > 1.0f) w = 1.0f;
  return w;
}

/* ---------------------------------------------------------------- lightness */

/* CIE 1976 L*: 116 f(Y) - 16 with f(Y) = Y^(1/3) above (6/29)^3 and the
 * linear segment (29/3)^3 Y below; Y from linear sRGB primaries (D65). */
static const float LUMA_R = 0.2126f, LUMA_G = 0.7152f, LUMA_B = 0.0722f;
static const float LAB_EPS = 216.0f / 24389.0f;   /* (6/29)^3 */
static const float LAB_KAPPA = 24389.0f / 27.0f;  /* (29/3)^3 */
static const float THIRD = 1.0f / 3.0f;

float orc_lightness(float r, float g, float b) {
  float Y = fmaf(LUMA_B, b, fmaf(LUMA_G, g, LUMA_R * r));
  if (Y < 0.0f) Y = 0.0f;
  if (Y > 1.0f) Y = 1.0f;
  if (Y > LAB_EPS) {
    float c = orc_exp(orc_log(Y) * THIRD);   /* Y^(1/3), Y in (eps, 1] */
    return fmaf(116.0f, c, -16.0f);
  }
  return LAB_KAPPA * Y;
}

static float stored(float c, int fp16) { return fp16 ? (float)(_Float16)c : c; }

float orc_lightness_factor(int K, const float* wt, const float* rgb, int fp16,
                           const float rgb_in[3]) {
  /* resolved colour of the slots before the push, in the GPU's FP32 order */
  float n0 = 0.0f, n1 = 0.0f, n2 = 0.0f, den = 0.0f;
  for (int j = 0; j < K; ++j) {
    n0 = fmaf(wt[j], stored(rgb[3 * j + 0], fp16), n0);
    n1 = fmaf(wt[j], stored(rgb[3 * j + 1], fp16), n1);
    n2 = fmaf(wt[j], stored(rgb[3 * j + 2], fp16), n2);
    den = den + wt[j];
  }
  if (!(den > 0.0f)) return 1.0f;
  float inv = 1.0f / den;
  float L_old = orc_lightness(n0 * inv, n1 * inv, n2 * inv);
  float L_new = orc_lightness(rgb_in[0], rgb_in[1], rgb_in[2]);
  float dl = fabsf(L_old - L_new) * 0.01f;
  if (dl > 1.0f) dl = 1.0f;
  return 1.0f - dl;
}

void orc_lightness_n(const float* rgb, float* L, int64_t n) {
  for (int64_t i = 0; i < n; ++i) L[i] = orc_lightness(rgb[3 * i], rgb[3 * i + 1], rgb[3 * i + 2]);
}

/* ---------------------------------------------------------------- reservoir */

static const float P_FLOOR = 0x1p-64f;   /* renormalise the bias product below this */
static const float P_RESCALE = 0x1p64f;

void orc_pixel_step(int K, int bias, float w, float u, uint32_t t, const float rgb_in[3],
                    int flush, float* W, float* P, float* key, uint32_t* idx, float* wt,
                    float* rgb) {
  orc_pixel_step_full(K, bias, 0, w, u, t, rgb_in, flush, W, P, key, idx, wt, rgb);
}

void orc_pixel_step_full(int K, int bias, int fp16, float w, float u, uint32_t t,
                         const float rgb_in[3], int flush, float* W, float* P, float* key,
                         uint32_t* idx, float* wt, float* rgb) {
  /* Eq. (full-temporal-bias): the history's weight also shrinks by 1 - |Delta L|;
   * a factor of 0 leaves it no weight at all, which is a flush */
  float g = 1.0f;
  if (bias == 2 && !flush && *W > 0.0f) {
    g = orc_lightness_factor(K, wt, rgb, fp16, rgb_in);
    if (g <= 0.0f) flush = 1;
  }
  if (flush) {
    /* occlusion / disocclusion: drop the history (Sec. 4.3, Sec. 6) */
    for (int j = 0; j < K; ++j) {
      key[j] = INFINITY;
      idx[j] = ORC_EMPTY;
      wt[j] = 0.0f;
      rgb[3 * j + 0] = rgb[3 * j + 1] = rgb[3 * j + 2] = 0.0f;
    }
    *W = 0.0f;
    *P = 1.0f;
  }

  /* A-ES key in exponential form: u^(1/w) largest <=> -ln(u)/w smallest. */
  float E = -orc_log(u);
  float k = E / w;

  /* Eq. (temporal-bias): R1.wsum <- R1.wsum * (1 - R2.wsum / (R1.wsum + R2.wsum)),
   * with R2.wsum = w; the factor 1 - w/(W+w) is evaluated as W/(W+w). The same
   * factor scales every stored sample's weight, which the keys carry through
   * the running product P. Skipped while the reservoir is empty (the factor
   * would be 0 * (1 - w/w)). */
  if (bias && *W > 0.0f) {
    float f = *W / (*W + w);
    if (bias == 2) f = f * g;
    *W = *W * f;
    *P = *P * f;
    if (*P < P_FLOOR) {
      /* exact power-of-two rescale of P and of every stored key */
      *P = *P * P_RESCALE;
      for (int j = 0; j < K; ++j) {
        if (idx[j] != ORC_EMPTY) {
          float s = key[j] * P_RESCALE;
          key[j] = s > FLT_MAX ? FLT_MAX : s;
        }
      }
    }
  }

  /* Alg. 2: R_out.wsum = R1.wsum + R2.wsum. */
  *W = *W + w;

  /* Alg. 2 selection as a key race: the new sample enters iff its key is
   * below the largest stored key (the first empty slot counts as +inf).
   * Ties keep the stored sample, as Alg. 2 keeps R1 on equality. */
  float ks = k * *P;
  int jmax = 0;
  for (int j = 1; j < K; ++j)
    if (key[j] > key[jmax]) jmax = j;
  if (ks < key[jmax]) {
    key[jmax] = ks;
    idx[jmax] = t;
    wt[jmax] = w;
    rgb[3 * jmax + 0] = rgb_in[0];
    rgb[3 * jmax + 1] = rgb_in[1];
    rgb[3 * jmax + 2] = rgb_in[2];
  }
}

void orc_pixel_step_literal(int bias, float w, float u, uint32_t t, const float rgb_in[3],
                            int flush, float* W, uint32_t* idx, float* wt, float* rgb) {
  orc_pixel_step_literal_full(bias, 0, w, u, t, rgb_in, flush, W, idx, wt, rgb);
}

void orc_pixel_step_literal_full(int bias, int fp16, float w, float u, uint32_t t,
                                 const float rgb_in[3], int flush, float* W, uint32_t* idx,
                                 float* wt, float* rgb) {
  float g = 1.0f;
  if (bias == 2 && !flush && *W > 0.0f) {
    g = orc_lightness_factor(1, wt, rgb, fp16, rgb_in);
    if (g <= 0.0f) flush = 1;
  }
  if (flush) {
    *idx = ORC_EMPTY;
    *wt = 0.0f;
    rgb[0] = rgb[1] = rgb[2] = 0.0f;
    *W = 0.0f;
  }
  /* Eq. (temporal-bias) on R1.wsum, the factor 1 - w/(W+w) evaluated as W/(W+w) */
  if (bias && *W > 0.0f) {
    float f = *W / (*W + w);
    if (bias == 2) f = f * g;
    *W = *W * f;
  }
  /* Alg. 2 with R2 = the new sample alone: keep R1 iff rand * (R1 + R2) <= R1 */
  float tot = *W + w;
  if (!(u * tot <= *W)) {
    *idx = t;
    *wt = w;
    rgb[0] = rgb_in[0];
    rgb[1] = rgb_in[1];
    rgb[2] = rgb_in[2];
  }
  /* R_out.wsum = R1.wsum + R2.wsum */
  *W = tot;
}

void orc_resolve_pixel(int K, const uint32_t* idx, const float* wt, const float* rgb,
                       double out[3]) {
  /* out = sum_j wt_j c_j / sum_j wt_j over occupied slots. With K = 1 this is
   * the resident sample itself, the paper's n = 1 output (Sec. 4.2). */
  double num[3] = {0.0, 0.0, 0.0}, den = 0.0;
  for (int j = 0; j < K; ++j) {
    if (idx[j] == ORC_EMPTY) continue;
    double w = (double)wt[j];
    num[0] += w * (double)rgb[3 * j + 0];
    num[1] += w * (double)rgb[3 * j + 1];
    num[2] += w * (double)rgb[3 * j + 2];
    den += w;
  }
  for (int c = 0; c < 3; ++c) out[c] = den > 0.0 ? num[c] / den : 0.0;
}

void orc_init_state(int K, int64_t n, float* W, float* P, float* key, uint32_t* idx,
                    float* wt, float* rgb) {
  for (int64_t i = 0; i < n; ++i) {
    W[i] = 0.0f;
    P[i] = 1.0f;
    for (int j = 0; j < K; ++j) {
      key[i * K + j] = INFINITY;
      idx[i * K + j] = ORC_EMPTY;
      wt[i * K + j] = 0.0f;
      rgb[(i * K + j) * 3 + 0] = rgb[(i * K + j) * 3 + 1] = rgb[(i * K + j) * 3 + 2] = 0.0f;
    }
  }
}

/* ---------------------------------------------------------------- frames */

typedef struct {
  const orc_config* cfg;
  uint32_t t;
  const float* frame;
  int64_t pitch;
  float gx, gy;
  const uint8_t* fov_map;
  const int64_t* pix;
  float *W, *P, *key, *wt, *rgb;
  uint32_t* idx;
  int64_t i0, i1;
} orc_job;

static void push_range(orc_job* j) {
  const orc_config* c = j->cfg;
  const int K = c->K;
  for (int64_t i = j->i0; i < j->i1; ++i) {
    int64_t p = j->pix ? j->pix[i] : i;
    int32_t x = (int32_t)(p % c->width), y = (int32_t)(p / c->width);
    float w = orc_weight32(c, x, y, j->gx, j->gy);
    float u = orc_uniform(c->seed, c->stream_id, j->t, p);
    const float* src = j->frame + (int64_t)y * j->pitch + 3 * (int64_t)x;
    int flush = j->fov_map ? (j->fov_map[p] == 0xFF) : 0;
    if (c->rule == 1)
      orc_pixel_step_literal_full(c->temporal_bias, c->color_fp16, w, u, j->t, src, flush,
                                  &j->W[i], &j->idx[i], &j->wt[i], &j->rgb[i * 3]);
    else
      orc_pixel_step_full(K, c->temporal_bias, c->color_fp16, w, u, j->t, src, flush, &j->W[i],
                          &j->P[i], &j->key[i * K], &j->idx[i * K], &j->wt[i * K],
                          &j->rgb[i * K * 3]);
  }
}

static void* push_thread(void* arg) {
  push_range((orc_job*)arg);
  return NULL;
}

static void run_jobs(orc_job* base, int64_t n, int nthreads, void* (*fn)(void*)) {
  if (nthreads < 1) nthreads = 1;
  if (nthreads > 256) nthreads = 256;
  if ((int64_t)nthreads > n) nthreads = n > 0 ? (int)n : 1;
  orc_job jobs[256];
  pthread_t th[256];
  for (int k = 0; k < nthreads; ++k) {
    jobs[k] = *base;
    jobs[k].i0 = n * k / nthreads;
    jobs[k].i1 = n * (k + 1) / nthreads;
  }
  if (nthreads == 1) {
    fn(&jobs[0]);
    return;
  }
  for (int k = 0; k < nthreads; ++k) pthread_create(&th[k], NULL, fn, &jobs[k]);
  for (int k = 0; k < nthreads; ++k) pthread_join(th[k], NULL);
}

int orc_push_frame(const orc_config* cfg, uint32_t t, const float* frame, int64_t pitch,
                   float gx, float gy, const uint8_t* fov_map, int64_t npix,
                   const int64_t* pix, float* W, float* P, float* key, uint32_t* idx,
                   float* wt, float* rgb, int nthreads) {
  if (!cfg || !frame || cfg->width <= 0 || cfg->height <= 0 || cfg->K < 1 || cfg->K > 16 ||
      (cfg->rule != 0 && cfg->rule != 1) || (cfg->rule == 1 && cfg->K != 1) ||
      cfg->temporal_bias < 0 || cfg->temporal_bias > 2 ||
      pitch < 3 * (int64_t)cfg->width || !(cfg->r_f > 0.0f) || !isfinite(gx) || !isfinite(gy))
    return -1;
  int64_t hw = (int64_t)cfg->width * cfg->height;
  if (!pix && npix != hw) return -1;
  if (pix)
    for (int64_t i = 0; i < npix; ++i)
      if (pix[i] < 0 || pix[i] >= hw) return -1;
  orc_job job;
  memset(&job, 0, sizeof job);
  job.cfg = cfg; job.t = t; job.frame = frame; job.pitch = pitch; job.gx = gx; job.gy = gy;
  job.fov_map = fov_map; job.pix = pix; job.W = W; job.P = P; job.key = key; job.idx = idx;
  job.wt = wt; job.rgb = rgb;
  run_jobs(&job, npix, nthreads, push_thread);
  return 0;
}

typedef struct {
  int K;
  const uint32_t* idx;
  const float *wt, *rgb;
  double* out;
  int64_t i0, i1;
} orc_rjob;

static void* resolve_thread(void* arg) {
  orc_rjob* j = (orc_rjob*)arg;
  for (int64_t i = j->i0; i < j->i1; ++i)
    orc_resolve_pixel(j->K, &j->idx[i * j->K], &j->wt[i * j->K], &j->rgb[i * j->K * 3],
                      &j->out[3 * i]);
  return NULL;
}

void orc_resolve(int K, int64_t npix, const uint32_t* idx, const float* wt, const float* rgb,
                 double* out, int nthreads) {
  if (nthreads < 1) nthreads = 1;
  if (nthreads > 256) nthreads = 256;
  if ((int64_t)nthreads > npix) nthreads = npix > 0 ? (int)npix : 1;
  orc_rjob jobs[256];
  pthread_t th[256];
  for (int k = 0; k < nthreads; ++k) {
    jobs[k].K = K; jobs[k].idx = idx; jobs[k].wt = wt; jobs[k].rgb = rgb; jobs[k].out = out;
    jobs[k].i0 = npix * k / nthreads;
    jobs[k].i1 = npix * (k + 1) / nthreads;
  }
  if (nthreads == 1) {
    resolve_thread(&jobs[0]);
    return;
  }
  for (int k = 0; k < nthreads; ++k) pthread_create(&th[k], NULL, resolve_thread, &jobs[k]);
  for (int k = 0; k < nthreads; ++k) pthread_join(th[k], NULL);
}

/* ---------------------------------------------------------------- reprojection */

typedef struct {
  orc_job base;
  const float *motion, *depth, *prev_depth;
  float tol;
  const float *W0, *P0, *key0, *wt0, *rgb0;
  const uint32_t* idx0;
} orc_rpjob;

static void* reproject_thread(void* arg) {
  orc_rpjob* r = (orc_rpjob*)arg;
  orc_job* j = &r->base;
  const orc_config* c = j->cfg;
  const int K = c->K;
  for (int64_t p = j->i0; p < j->i1; ++p) {
    int32_t x = (int32_t)(p % c->width), y = (int32_t)(p / c->width);
    float mx = r->motion ? r->motion[2 * p] : 0.0f;
    float my = r->motion ? r->motion[2 * p + 1] : 0.0f;
    float cx = ((float)x + 0.5f) - mx;
    float cy = ((float)y + 0.5f) - my;
    int valid = cx >= 0.0f && cx < (float)c->width && cy >= 0.0f && cy < (float)c->height;
    int64_t q = p;
    if (valid) q = (int64_t)floorf(cy) * c->width + (int64_t)floorf(cx);
    if (valid && r->depth) {
      float dp = r->depth[p], dq = r->prev_depth[q];
      if (fabsf(dq - dp) > r->tol * dp) valid = 0;
    }
    /* the history of p is the previous reservoir at q */
    j->W[p] = r->W0[q];
    j->P[p] = r->P0[q];
    for (int s = 0; s < K; ++s) {
      j->key[p * K + s] = r->key0[q * K + s];
      j->idx[p * K + s] = r->idx0[q * K + s];
      j->wt[p * K + s] = r->wt0[q * K + s];
      for (int ch = 0; ch < 3; ++ch) j->rgb[(p * K + s) * 3 + ch] = r->rgb0[(q * K + s) * 3 + ch];
    }
    float w = orc_weight32(c, x, y, j->gx, j->gy);
    float u = orc_uniform(c->seed, c->stream_id, j->t, p);
    const float* src = j->frame + (int64_t)y * j->pitch + 3 * (int64_t)x;
    int flush = !valid || (j->fov_map ? (j->fov_map[p] == 0xFF) : 0);
    if (c->rule == 1)
      orc_pixel_step_literal_full(c->temporal_bias, c->color_fp16, w, u, j->t, src, flush,
                                  &j->W[p], &j->idx[p], &j->wt[p], &j->rgb[p * 3]);
    else
      orc_pixel_step_full(K, c->temporal_bias, c->color_fp16, w, u, j->t, src, flush, &j->W[p],
                          &j->P[p], &j->key[p * K], &j->idx[p * K], &j->wt[p * K],
                          &j->rgb[p * K * 3]);
  }
  return NULL;
}

int orc_push_frame_reproject(const orc_config* cfg, uint32_t t, const float* frame, int64_t pitch,
                             float gx, float gy, const float* motion, const float* depth,
                             const float* prev_depth, float depth_tol, const uint8_t* fov_map,
                             const float* W0, const float* P0, const float* key0,
                             const uint32_t* idx0, const float* wt0, const float* rgb0, float* W,
                             float* P, float* key, uint32_t* idx, float* wt, float* rgb,
                             int nthreads) {
  if (!cfg || !frame || cfg->width <= 0 || cfg->height <= 0 || cfg->K < 1 || cfg->K > 16 ||
      (cfg->rule != 0 && cfg->rule != 1) || (cfg->rule == 1 && cfg->K != 1) ||
      cfg->temporal_bias < 0 || cfg->temporal_bias > 2 ||
      pitch < 3 * (int64_t)cfg->width || !(cfg->r_f > 0.0f) || !isfinite(gx) || !isfinite(gy))
    return -1;
  if ((depth == NULL) != (prev_depth == NULL)) return -1;
  if (depth && (!isfinite(depth_tol) || depth_tol < 0.0f)) return -1;
  const int64_t hw = (int64_t)cfg->width * cfg->height;
  if (nthreads < 1) nthreads = 1;
  if (nthreads > 256) nthreads = 256;
  if ((int64_t)nthreads > hw) nthreads = (int)hw;
  orc_rpjob jobs[256];
  pthread_t th[256];
  for (int k = 0; k < nthreads; ++k) {
    memset(&jobs[k], 0, sizeof jobs[k]);
    orc_job* j = &jobs[k].base;
    j->cfg = cfg; j->t = t; j->frame = frame; j->pitch = pitch; j->gx = gx; j->gy = gy;
    j->fov_map = fov_map; j->W = W; j->P = P; j->key = key; j->idx = idx; j->wt = wt;
    j->rgb = rgb;
    j->i0 = hw * k / nthreads;
    j->i1 = hw * (k + 1) / nthreads;
    jobs[k].motion = motion; jobs[k].depth = depth; jobs[k].prev_depth = prev_depth;
    jobs[k].tol = depth_tol;
    jobs[k].W0 = W0; jobs[k].P0 = P0; jobs[k].key0 = key0; jobs[k].idx0 = idx0;
    jobs[k].wt0 = wt0; jobs[k].rgb0 = rgb0;
  }
  if (nthreads == 1) {
    reproject_thread(&jobs[0]);
    return 0;
  }
  for (int k = 0; k < nthreads; ++k) pthread_create(&th[k], NULL, reproject_thread, &jobs[k]);
  for (int k = 0; k < nthreads; ++k) pthread_join(th[k], NULL);
  return 0;
}

/* ---------------------------------------------------------------- statistics */

void orc_run_streams(int K, int bias, int64_t n_trials, int n_items, const float* w,
                     const float* u, uint32_t* final_idx, float* final_W) {
  float key[16], wt[16], rgb[48];
  uint32_t idx[16];
  const float zero[3] = {0.0f, 0.0f, 0.0f};
  for (int64_t i = 0; i < n_trials; ++i) {
    float W, P;
    orc_init_state(K, 1, &W, &P, key, idx, wt, rgb);
    for (int s = 0; s < n_items; ++s)
      orc_pixel_step(K, bias, w[s], u[i * n_items + s], (uint32_t)s, zero, 0, &W, &P, key, idx,
                     wt, rgb);
    for (int j = 0; j < K; ++j) final_idx[i * K + j] = idx[j];
    if (final_W) final_W[i] = W;
  }
}

void orc_chao_literal(int bias, int64_t n_trials, int n_items, const float* w,
                      const float* u, uint32_t* final_idx) {
  const float zero[3] = {0.0f, 0.0f, 0.0f};
  for (int64_t i = 0; i < n_trials; ++i) {
    uint32_t x = ORC_EMPTY;
    float W = 0.0f, wt = 0.0f, rgb[3];
    for (int s = 0; s < n_items; ++s)
      orc_pixel_step_literal(bias, w[s], u[i * n_items + s], (uint32_t)s, zero, 0, &W, &x, &wt,
                             rgb);
    final_idx[i] = x;
  }
}

/* ---------------------------------------------------------------- foveation */

/* Sum of channel c over the aligned 2^L block (by, bx): the quad tree of its
 * four quadrants, top pair then bottom pair, each pair left then right. */
static float block_sum(const float* img, int64_t pitch, int32_t w, int32_t h, int32_t L,
                       int64_t by, int64_t bx, int c) {
  if (L == 0) return (by < h && bx < w) ? img[by * pitch + 3 * bx + c] : 0.0f;
  float s00 = block_sum(img, pitch, w, h, L - 1, 2 * by, 2 * bx, c);
  float s01 = block_sum(img, pitch, w, h, L - 1, 2 * by, 2 * bx + 1, c);
  float s10 = block_sum(img, pitch, w, h, L - 1, 2 * by + 1, 2 * bx, c);
  float s11 = block_sum(img, pitch, w, h, L - 1, 2 * by + 1, 2 * bx + 1, c);
  float top = s00 + s01;
  float bot = s10 + s11;
  return top + bot;
}

static int64_t ceil_shift(int64_t n, int L) { return (n + ((int64_t)1 << L) - 1) >> L; }

void orc_mip_means(const float* img, int64_t pitch, int32_t w, int32_t h, int32_t L, float* out) {
  const int64_t b = (int64_t)1 << L;
  const int64_t hb = ceil_shift(h, L), wb = ceil_shift(w, L);
  for (int64_t by = 0; by < hb; ++by)
    for (int64_t bx = 0; bx < wb; ++bx) {
      int64_t rows = (by * b + b < h ? by * b + b : h) - by * b;
      int64_t cols = (bx * b + b < w ? bx * b + b : w) - bx * b;
      float n = (float)(rows * cols);
      for (int c = 0; c < 3; ++c)
        out[(by * wb + bx) * 3 + c] = block_sum(img, pitch, w, h, L, by, bx, c) / n;
    }
}

/* Level coordinate of pixel index i at level L, clamped to [0, nb - 1]:
 * integer part i0, neighbour i1 and fraction f. */
static void texel_coord(int32_t i, int32_t L, int64_t nb, int64_t* i0, int64_t* i1, float* f) {
  float inv_b = 1.0f / (float)(1 << L);
  float u = ((float)i + 0.5f) * inv_b - 0.5f;
  if (u < 0.0f) u = 0.0f;
  if (u > (float)(nb - 1)) u = (float)(nb - 1);
  float fl = floorf(u);
  *i0 = (int64_t)fl;
  *i1 = *i0 + 1 < nb ? *i0 + 1 : nb - 1;
  *f = u - fl;
}

int orc_foveate(const float* img, int64_t pitch, int32_t w, int32_t h, int32_t nradii,
                const float* radii, float gx, float gy, int32_t filter, float* frame,
                uint8_t* ring_map) {
  if (!img || !frame || w < 1 || h < 1 || pitch < 3 * (int64_t)w) return -1;
  if (nradii < 1 || nradii > ORC_MAX_MIP_LEVELS - 1 || !radii) return -1;
  if (filter != ORC_FILTER_BOX && filter != ORC_FILTER_BILINEAR) return -1;
  if (!isfinite(gx) || !isfinite(gy)) return -1;
  float r2[ORC_MAX_MIP_LEVELS];
  for (int i = 0; i < nradii; ++i) {
    if (!(radii[i] > 0.0f) || !isfinite(radii[i]) || (i > 0 && radii[i] < radii[i - 1])) return -1;
    r2[i] = radii[i] * radii[i];
  }
  float* means[ORC_MAX_MIP_LEVELS] = {0};
  int64_t wbs[ORC_MAX_MIP_LEVELS], hbs[ORC_MAX_MIP_LEVELS];
  for (int L = 1; L <= nradii; ++L) {
    hbs[L] = ceil_shift(h, L);
    wbs[L] = ceil_shift(w, L);
    means[L] = (float*)malloc((size_t)(hbs[L] * wbs[L] * 3) * sizeof(float));
    orc_mip_means(img, pitch, w, h, L, means[L]);
  }
  for (int32_t y = 0; y < h; ++y)
    for (int32_t x = 0; x < w; ++x) {
      float dx = ((float)x + 0.5f) - gx;
      float dy = ((float)y + 0.5f) - gy;
      float d2 = dx * dx + dy * dy;
      int L = 0;
      for (int i = 0; i < nradii; ++i) L += d2 > r2[i];
      float* o = frame + ((int64_t)y * w + x) * 3;
      if (ring_map) ring_map[(int64_t)y * w + x] = (uint8_t)L;
      if (L == 0) {
        for (int c = 0; c < 3; ++c) o[c] = img[(int64_t)y * pitch + 3 * (int64_t)x + c];
      } else if (filter == ORC_FILTER_BOX) {
        const float* t = means[L] + (((int64_t)y >> L) * wbs[L] + ((int64_t)x >> L)) * 3;
        for (int c = 0; c < 3; ++c) o[c] = t[c];
      } else {
        int64_t x0, x1, y0, y1;
        float fx, fy;
        texel_coord(x, L, wbs[L], &x0, &x1, &fx);
        texel_coord(y, L, hbs[L], &y0, &y1, &fy);
        const float* m = means[L];
        for (int c = 0; c < 3; ++c) {
          float t00 = m[(y0 * wbs[L] + x0) * 3 + c], t01 = m[(y0 * wbs[L] + x1) * 3 + c];
          float t10 = m[(y1 * wbs[L] + x0) * 3 + c], t11 = m[(y1 * wbs[L] + x1) * 3 + c];
          float top = t00 * (1.0f - fx) + t01 * fx;
          float bot = t10 * (1.0f - fx) + t11 * fx;
          o[c] = top * (1.0f - fy) + bot * fy;
        }
      }
    }
  for (int L = 1; L <= nradii; ++L) free(means[L]);
  return 0;
}

/* ---------------------------------------------------------------- helpers */

void orc_exp_n(const float* x, float* y, int64_t n) {
  for (int64_t i = 0; i < n; ++i) y[i] = orc_exp(x[i]);
}
void orc_log_n(const float* x, float* y, int64_t n) {
  for (int64_t i = 0; i < n; ++i) y[i] = orc_log(x[i]);
}
void orc_density32_n(const float* e, float* y, int64_t n) {
  for (int64_t i = 0; i < n; ++i) y[i] = orc_density32(e[i]);
}
void orc_density64_n(const double* e, double* y, int64_t n) {
  for (int64_t i = 0; i < n; ++i) y[i] = orc_density64(e[i]);
}
void orc_uniform_n(uint64_t seed, uint32_t stream_id, uint32_t t, int64_t p0, int64_t n,
                   float* u) {
  for (int64_t i = 0; i < n; ++i) u[i] = orc_uniform(seed, stream_id, t, p0 + i);
}
void orc_weight32_grid(const orc_config* cfg, float gx, float gy, float* w) {
  for (int32_t y = 0; y < cfg->height; ++y)
    for (int32_t x = 0; x < cfg->width; ++x)
      w[(int64_t)y * cfg->width + x] = orc_weight32(cfg, x, y, gx, gy);
}
