/*
 * CPU oracle for per-pixel weighted reservoir sampling on foveated frame
 * streams ("Enhancing Foveated Rendering with Weighted Reservoir Sampling").
 *
 * TEST INFRASTRUCTURE ONLY. Plain, slow, obviously correct C. Only the test
 * suite, the smoke check and the CPU-baseline leg of the benchmark may load
 * it; the product path never does. It shares no source, header, table or
 * constant with the CUDA library: both follow the same written operation
 * sequence independently.
 *
 * Parity status of each function is given beside it; "pinned" names what
 * outside fact checks it in tests/test_oracle_pins.py.
 */
#ifndef WRS_ORACLE_H
#define WRS_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define ORC_EMPTY 0xFFFFFFFFu

typedef struct {
  int32_t width, height;   /* frame size in pixels */
  int32_t K;               /* reservoir slots per pixel, 1..16 */
  float r_f;               /* foveal radius in pixels */
  float deg_per_px;        /* eccentricity per pixel in degrees; <= 0 selects 2.5 / r_f */
  uint64_t seed;           /* Philox key */
  uint32_t stream_id;      /* third Philox counter word */
  int32_t temporal_bias;   /* 0: none; 1: Eq. (temporal-bias); 2: Eq. (full-temporal-bias) */
  int32_t rule;            /* 0: key race over K slots; 1: literal Alg. 2 (K == 1) */
  int32_t color_fp16;      /* slot colours as the GPU stores them: 1 = rounded to IEEE half */
} orc_config;

/* FP32 exp for x in [-87, 0]: range reduction by ln 2 and a degree-7 Taylor
 * polynomial. Pinned: libm exp within 4 ulp (closed form). */
float orc_exp(float x);
/* FP32 natural log for u in (0, 1): mantissa/exponent split and the atanh
 * series. Pinned: libm log within 4 ulp. */
float orc_log(float u);
/* Philox4x32-10 (Salmon et al., SC'11). Pinned: curand's Philox4_32_10
 * (GPU test) and uniformity statistics. */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
/* The uniform draw of pixel p at frame t, in (0, 1). */
float orc_uniform(uint64_t seed, uint32_t stream_id, uint32_t t, int64_t p);
/* Eq. (cone_retinal_density), plain FP64 with libm exp. Pinned: d(0), the
 * derivative at 0 and the large-e asymptote (closed forms). */
double orc_density64(double e);
/* The same density without the cancelling factor 2 d_c(0), in the fixed FP32
 * sequence the bit-exact path uses. Pinned: orc_density64 within 1e-6. */
float orc_density32(float e);
/* Eq. (phat) for the pixel (x, y) and gaze (gx, gy), fixed FP32 sequence.
 * Pinned: w = 1 inside the fovea, continuity at r_f, monotone decrease,
 * 0 < w <= 1, FP64 value within 1e-6. */
float orc_weight32(const orc_config* cfg, int32_t x, int32_t y, float gx, float gy);
float orc_delta(const orc_config* cfg);

/* CIELAB lightness L* of linear-light sRGB (D65) colour, fixed FP32 sequence:
 * Y = 0.2126 r + 0.7152 g + 0.0722 b clamped to [0, 1]; L* = 116 Y^(1/3) - 16
 * above (6/29)^3, else (29/3)^3 Y; the cube root as exp(ln(Y)/3) with orc_exp
 * and orc_log. Pinned: L*(0) = 0, L*(1) = 100, 18% grey = 49.50, continuity at
 * the junction. */
float orc_lightness(float r, float g, float b);
/* The factor 1 - |Delta L| of Eq. (full-temporal-bias), Delta L the L*
 * difference / 100 between the reservoir's resolved colour before the push
 * (FP32, slot order, as the GPU resolves) and the new sample. */
float orc_lightness_factor(int K, const float* wt, const float* rgb, int fp16,
                           const float rgb_in[3]);

/* One candidate entering one pixel's reservoir: Eq. (temporal-bias) on the
 * history, then Alg. 2 in its exponential-key form (keep the K smallest keys
 * E/w scaled by the running bias product P). Pinned statistically:
 * Eq. (chao-selection-probability) for K = 1, successive sampling without
 * replacement for K > 1 (brute force), uniform subsets for equal weights,
 * literal Alg. 2 equivalence, size <= K. */
void orc_pixel_step(int K, int bias, float w, float u, uint32_t t, const float rgb_in[3],
                    int flush, float* W, float* P, float* key, uint32_t* idx, float* wt,
                    float* rgb);
/* As orc_pixel_step; bias = 2 applies Eq. (full-temporal-bias): the history's
 * weight is scaled by (1 - |Delta L|) as well (a factor of 0 drops the
 * history, as a flush does). fp16: colours as stored in FP16 slots. */
void orc_pixel_step_full(int K, int bias, int fp16, float w, float u, uint32_t t,
                         const float rgb_in[3], int flush, float* W, float* P, float* key,
                         uint32_t* idx, float* wt, float* rgb);
/* The paper's n = 1 update taken literally: Eq. (temporal-bias) on R1.wsum,
 * then Alg. 2 keeps R1 iff rand * (R1.wsum + R2.wsum) <= R1.wsum, else takes
 * the new sample (R2 holds only it: R2.wsum = w). One slot, no key. Pinned:
 * the selection law of Eq. (chao-selection-probability) with effective
 * weights (statistics), and its distributional equality with the key race. */
void orc_pixel_step_literal(int bias, float w, float u, uint32_t t, const float rgb_in[3],
                            int flush, float* W, uint32_t* idx, float* wt, float* rgb);
void orc_pixel_step_literal_full(int bias, int fp16, float w, float u, uint32_t t,
                                 const float rgb_in[3], int flush, float* W, uint32_t* idx,
                                 float* wt, float* rgb);
void orc_lightness_n(const float* rgb, float* L, int64_t n);

/* Weighted combination of the occupied slots, FP64. Pinned: K = 1 returns the
 * resident sample, equal colours return that colour, no slot returns 0. */
void orc_resolve_pixel(int K, const uint32_t* idx, const float* wt, const float* rgb,
                       double out[3]);

/* Pixel-major state of n pixels: W[n], P[n], key[n][K], idx[n][K], wt[n][K],
 * rgb[n][K][3]. */
void orc_init_state(int K, int64_t n, float* W, float* P, float* key, uint32_t* idx,
                    float* wt, float* rgb);
/* One frame. frame is [height][pitch] floats holding RGB triples; fov_map is
 * [height][width] bytes or NULL (0xFF flushes the pixel). pix lists the
 * pixels to simulate (state index i belongs to pixel pix[i]); NULL means all
 * pixels in row-major order. Returns 0, or -1 on bad arguments. */
int orc_push_frame(const orc_config* cfg, uint32_t t, const float* frame, int64_t pitch,
                   float gx, float gy, const uint8_t* fov_map, int64_t npix,
                   const int64_t* pix, float* W, float* P, float* key, uint32_t* idx,
                   float* wt, float* rgb, int nthreads);
void orc_resolve(int K, int64_t npix, const uint32_t* idx, const float* wt, const float* rgb,
                 double* out, int nthreads);
/* One frame with temporal reprojection (Sec. 4.3): pixel p = (x, y) takes as
 * its history the previous frame's reservoir at q = (floor(x + 0.5 - mx),
 * floor(y + 0.5 - my)), (mx, my) = motion[p] the screen motion in pixels since
 * the previous frame (FP32 sub/add); the history is flushed when that centre
 * lies outside the frame or, with depth buffers, when
 * |prev_depth[q] - depth[p]| > depth_tol * depth[p] (FP32), as well as where
 * fov_map is 0xFF. The new candidate is then combined as in orc_push_frame.
 * Reads the previous state (all pixels, pixel-major) and writes the next one;
 * the two must not overlap. motion [h][w][2] or NULL (no motion); depth and
 * prev_depth [h][w] both or neither. Pinned: zero motion equals
 * orc_push_frame, slot provenance under integer pans (closed form), flushes
 * at depth edges and screen edges, nearest-centre rounding. Returns 0 or -1. */
int orc_push_frame_reproject(const orc_config* cfg, uint32_t t, const float* frame, int64_t pitch,
                             float gx, float gy, const float* motion, const float* depth,
                             const float* prev_depth, float depth_tol, const uint8_t* fov_map,
                             const float* W0, const float* P0, const float* key0,
                             const uint32_t* idx0, const float* wt0, const float* rgb0, float* W,
                             float* P, float* key, uint32_t* idx, float* wt, float* rgb,
                             int nthreads);

/* Statistics harness: n_trials independent single-pixel streams of n_items
 * candidates with weights w[n_items] and uniforms u[n_trials][n_items].
 * Writes the final slot frame indices [n_trials][K] and final W. */
void orc_run_streams(int K, int bias, int64_t n_trials, int n_items, const float* w,
                     const float* u, uint32_t* final_idx, float* final_W);
/* Literal n = 1 form: Eq. (temporal-bias) then Alg. 2 with rand * (R1 + R2) <= R1. */
void orc_chao_literal(int bias, int64_t n_trials, int n_items, const float* w,
                      const float* u, uint32_t* final_idx);

/* Foveation post-process (Sec. 4.3: foveated rendering simulated by a
 * mip-map of the rendered frame, reconstructed with filtering). */
#define ORC_MAX_MIP_LEVELS 6
#define ORC_FILTER_BOX 0
#define ORC_FILTER_BILINEAR 1
/* Means of the aligned 2^L x 2^L blocks of an RGB image, [ceil(h/2^L)][ceil(w/2^L)][3].
 * A block's sum is the quad tree (s00 + s01) + (s10 + s11) of its level-(L-1)
 * quadrants in FP32, pixels outside the image counting 0; the mean is that
 * sum / the pixel count, one FP32 division. Pinned: constant images, dyadic
 * ramps (exact closed forms), FP64 means within the rounding bound. */
void orc_mip_means(const float* img, int64_t pitch, int32_t w, int32_t h, int32_t L, float* out);
/* One foveated frame and its ring map. Ring level of pixel (x, y) =
 * #{i : d2 > r_i * r_i} with dx = ((float)x + 0.5f) - gx, dy likewise,
 * d2 = dx*dx + dy*dy (FP32, each rounded). Level 0 copies the image; level L
 * takes the level-L block means, by nearest lookup (box) or bilinear
 * filtering at u = ((float)x + 0.5f) * 2^-L - 0.5f clamped to the texel
 * centres, top = t00 (1 - fx) + t01 fx, bot = t10 (1 - fx) + t11 fx,
 * colour = top (1 - fy) + bot fy. Radii ascending, 1..5 of them. Pinned:
 * constant image, dyadic ramps, exact ring boundaries, mirror symmetry.
 * Returns 0, or -1 on bad arguments. */
int orc_foveate(const float* img, int64_t pitch, int32_t w, int32_t h, int32_t nradii,
                const float* radii, float gx, float gy, int32_t filter, float* frame,
                uint8_t* ring_map);

/* Element-wise helpers for tests. */
void orc_exp_n(const float* x, float* y, int64_t n);
void orc_log_n(const float* x, float* y, int64_t n);
void orc_density32_n(const float* e, float* y, int64_t n);
void orc_density64_n(const double* e, double* y, int64_t n);
void orc_uniform_n(uint64_t seed, uint32_t stream_id, uint32_t t, int64_t p0, int64_t n,
                   float* u);
void orc_weight32_grid(const orc_config* cfg, float gx, float gy, float* w);

#ifdef __cplusplus
}
#endif
#endif
