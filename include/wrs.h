/*
 * libwrs: per-pixel weighted reservoir sampling of foveated frame streams on
 * NVIDIA GB300 (sm_103a).
 *
 * Method: "Enhancing Foveated Rendering with Weighted Reservoir Sampling"
 * (arXiv 2510.03964). Every pixel location is an independent stream that
 * receives one candidate sample per frame (Sec. 4.1). The candidate's weight
 * is the normalised retinal density at its eccentricity from that frame's
 * gaze point (Eq. (cone_retinal_density), Eq. (phat)). The history held in
 * the reservoir is biased by the new candidate's survival odds
 * (Eq. (p_survive_reservoir), Eq. (temporal-bias)) and then combined with it
 * (Alg. 2). With K slots the combine keeps the K smallest exponential keys
 * -ln(u)/w (the A-ES key u^(1/w), Sec. 3.1, in log form), u drawn from
 * Philox4x32-10; with K = 1 this is Alg. 2 in distribution. The output pixel
 * is the weight-averaged colour of the occupied slots.
 *
 * Conventions shared by every call:
 *  - Status: every int-returning call returns WRS_OK (0) or a WRS_ERR_* code;
 *    wrs_last_error() then holds a one-line message for the calling thread.
 *    A call that fails leaves the reservoir state and the frame counter as
 *    they were. Failures found on the device after a call has returned (a
 *    wait that gave up) are reported by wrs_check_status instead: see there.
 *  - Streams: calls enqueue work on the given CUDA stream (a cudaStream_t
 *    passed as void*; NULL is the legacy default stream) and return without
 *    synchronising, except wrs_export_state / wrs_import_state and
 *    wrs_push_frame_host, which wait for their copies.
 *  - Memory: all d_* pointers are device memory owned by the caller and only
 *    borrowed for the call; h_* pointers are host memory (pinned memory gives
 *    asynchronous copies). The library owns only the context object.
 *  - Frame counter: t starts at 0 at wrs_create and advances by one on every
 *    successful push.
 *  - Images are row-major; colours are RGB float triples.
 */
#ifndef WRS_H
#define WRS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define WRS_OK 0
#define WRS_ERR_ARG 1      /* invalid argument (null, size, alignment, range) */
#define WRS_ERR_CUDA 2     /* a CUDA call failed (message holds its error string) */
#define WRS_ERR_BUDGET 3   /* state buffer smaller than wrs_state_bytes() */
#define WRS_ERR_TIMEOUT 4  /* a bounded device-side wait gave up */
#define WRS_ERR_STATE 5    /* context in the wrong state (e.g. counter exhausted) */
#define WRS_ERR_CHECK 6    /* checked build only: an index or copy range fell outside its
                              buffer and was skipped (reported by wrs_check_status) */

#define WRS_MAX_K 16
#define WRS_MAX_BATCH 64  /* streams in one wrs_push_batch launch */
#define WRS_RULE_KEYS 0
#define WRS_RULE_LITERAL 1
#define WRS_EMPTY_SLOT 0xFFFFFFFFu /* sample index of an unoccupied slot */
/* foveation post-process (Sec. 4.3): mip levels and reconstruction filters */
#define WRS_MAX_MIP_LEVELS 6   /* level 0 (the image) .. level 5 (32 x 32 blocks) */
#define WRS_FILTER_BOX 0       /* nearest lookup of the level's block mean */
#define WRS_FILTER_BILINEAR 1  /* bilinear filtering of the level's block means */

typedef struct wrs_ctx wrs_ctx;
typedef void* wrs_stream_t; /* cudaStream_t */

/* One frame stream. */
typedef struct {
  int32_t width, height;   /* pixels, >= 1; width * height < 2^31 - 64 */
  int32_t K;               /* reservoir slots per pixel, 1..16 (the paper uses n = 1) */
  float fovea_radius_px;   /* r_f in pixels (> 0): weight 1 at or inside it (Eq. (phat)) */
  float deg_per_px;        /* eccentricity scale in degrees per pixel; <= 0 selects
                              2.5 / fovea_radius_px, so r_f sits at the 2.5 deg where the
                              paper normalises the weight (Fig. (phat_figure) caption) */
  uint64_t seed;           /* Philox key */
  uint32_t stream_id;      /* third Philox counter word; distinct per stream in a batch */
  int32_t color_fp16;      /* 0: FP32 slot colours; 1: FP16 slot colours (keys, weights and
                              accumulation stay FP32) */
  int32_t temporal_bias;   /* 1: apply Eq. (temporal-bias) before each combine (paper);
                              2: Eq. (full-temporal-bias): also scale the history by
                                 1 - |Delta L|, Delta L the CIELAB L* difference / 100
                                 between the reservoir's resolved colour (linear sRGB, D65)
                                 and the new sample; a factor of 0 acts as a flush;
                              0: plain weighted sampling */
  int32_t update_rule;     /* WRS_RULE_KEYS (0): exponential-key race over K slots;
                              WRS_RULE_LITERAL (1): the paper's n = 1 update taken
                              literally, Alg. 2 keeping R1 iff rand*(R1+R2) <= R1 after
                              Eq. (temporal-bias); needs K == 1, uses no key or P plane */
} wrs_config;

/* Placement of the state planes inside the caller's state buffer. Every plane
 * holds `plane_px` entries (width*height rounded up to 64), pixel p at entry p.
 * Offsets are in bytes from the start of the buffer:
 *   W        float   running weight sum R.wsum (Alg. 2), biased (Eq. (temporal-bias))
 *   P        float   product of bias factors since the last rescale
 *   key[j]   float   stored key of slot j (+inf when empty), at key_off + j*plane_bytes4
 *   idx[j]   uint32  frame index of the slot's sample (WRS_EMPTY_SLOT when empty),
 *                    at idx_off + j*plane_bytes4
 * and the slot weights w (perceptual weight of the slot's sample) and colours,
 * 0 when empty:
 *   FP32 colour: rec[j] float4 {w, r, g, b} at col_off + j*plane_bytes_col
 *                (plane_bytes_col = 16*plane_px; wt_off = -1). One record per
 *                slot keeps a replacement's writes in one 16-byte entry.
 *   FP16 colour: rec[j], 8-byte records {r, g, b, w_hi} at col_off +
 *                j*plane_bytes_col (plane_bytes_col = 8*plane_px): the colour as
 *                IEEE halves and the high 16 bits of the FP32 weight w; wlo[j]
 *                uint16 at wt_off + j*plane_bytes_wt (plane_bytes_wt =
 *                2*plane_px) holds its low 16 bits, so w's bits are
 *                (w_hi << 16) | wlo. col_off is wt_off + K*plane_bytes_wt rounded
 *                up to 256 bytes.
 * After the planes, a ring of map_frames replacement-code planes of plane_px
 * bytes (map_off + r*plane_px, r = frame % map_frames): per frame and pixel,
 * which slot took that frame's sample (0..K-1), 0x80 + j (the history was
 * flushed, then slot j took the sample) or 0xFF (no change). The update writes this
 * code, one coalesced byte per pixel, instead of scattering the sample index
 * into idx[j]; every push also folds the pending codes of one band of
 * 256-pixel blocks into the idx planes: block b (pixels 256b .. 256b+255) is
 * folded by the pushes of the frames whose index % map_frames equals its band,
 * (b + b/16 + b/256) % 16 (integer divisions), which spreads the folding
 * blocks evenly over the CTAs of the persistent kernels. The idx planes of the other blocks therefore lag by up to
 * map_frames - 1 frames between pushes; wrs_export_state folds every pending
 * code first, so exported states always hold complete sample indices, and
 * the ring is not part of an exported or imported state. With K <= 2 there
 * is no ring (map_frames = 0): those kernels are bound by instruction issue
 * rather than DRAM, so they write each sample index into idx[j] directly. */
typedef struct {
  int64_t plane_px;
  int64_t plane_bytes4;     /* plane_px * 4 */
  int64_t plane_bytes_col;  /* plane_px * 16 (FP32 colour) or * 8 (FP16 colour) */
  int64_t plane_bytes_wt;   /* plane_px * 2 (FP16 colour) or 0 (FP32 colour) */
  int64_t status_off;       /* 256-byte header: uint32 status word (WRS_OK or WRS_ERR_TIMEOUT)
                               at +0, uint64 count of slot replacements at +8, uint32 check
                               word of the checked build at +16 */
  int64_t W_off, P_off, key_off, idx_off, wt_off, col_off;
  int64_t map_off;          /* ring of replacement-code planes (bytes), 256-byte aligned */
  int64_t map_frames;       /* planes in the ring (16), or 0 for K <= 2 */
  int64_t total_bytes;
} wrs_layout;

/* Bytes of device memory one stream's reservoir state needs (its planes are
 * described by wrs_state_layout), or 0 if cfg is invalid. Host only; no CUDA
 * call. */
size_t wrs_state_bytes(const wrs_config* cfg);
int wrs_state_layout(const wrs_config* cfg, wrs_layout* out);

/* Creates a stream context over d_state (device, >= wrs_state_bytes(cfg),
 * 256-byte aligned; caller-owned and never freed by the library) and enqueues
 * its initialisation on `stream`: every slot empty, W = 0, P = 1, t = 0.
 * Errors: WRS_ERR_ARG (cfg, pointers, alignment), WRS_ERR_BUDGET (too small),
 * WRS_ERR_CUDA (launch). */
int wrs_create(const wrs_config* cfg, void* d_state, size_t state_bytes, wrs_stream_t stream,
               wrs_ctx** out);

/* Pushes frame t into every pixel's reservoir and, if d_out is not NULL,
 * resolves it in the same pass (one kernel). Per pixel (Sec. 4, in order):
 * weight w from the eccentricity of the pixel centre to (gaze_x, gaze_y)
 * (Eq. (cone_retinal_density), Eq. (phat)); key -ln(u)/w from Philox
 * (A-ES, Sec. 3.1); Eq. (temporal-bias) on the history; Alg. 2 as the key
 * race over the K slots; then out = sum_j wt_j col_j / sum_j wt_j.
 *   d_frame     device float [height][frame_pitch_elems], RGB triples in the first
 *               3*width floats of each row; 4-byte aligned.
 *   frame_pitch_elems  floats per frame row, >= 3*width.
 *   gaze_x/y    gaze in pixel coordinates (pixel (x, y) has centre (x+0.5, y+0.5));
 *               must be finite, may lie outside the image.
 *   d_fov_map   NULL, or device uint8 [height][width]: 0xFF drops that pixel's
 *               history before the push (occlusion flush, Sec. 4.3); other
 *               values are ignored.
 *   d_out       NULL, or device float [height][width][3]: the resolved frame.
 * Errors: WRS_ERR_ARG, WRS_ERR_STATE (t would overflow), WRS_ERR_CUDA. */
int wrs_push_frame(wrs_ctx* ctx, const float* d_frame, int64_t frame_pitch_elems, float gaze_x,
                   float gaze_y, const uint8_t* d_fov_map, float* d_out, wrs_stream_t stream);

/* Resolves the current reservoirs into d_out (device float [height][width][3])
 * without pushing: bit-identical to the fused resolve of the last push. Pixels
 * with no occupied slot resolve to 0. */
int wrs_resolve(wrs_ctx* ctx, float* d_out, wrs_stream_t stream);

/* Frees the context object (not d_state). NULL is accepted. */
int wrs_destroy(wrs_ctx* ctx);

/* ------------------------------------------------------------------ extras */

/* Same as wrs_push_frame with host buffers: copies h_frame (float
 * [height][width][3], contiguous) and h_fov_map (optional) into the caller's
 * device staging buffers d_frame_stage / d_fov_stage, pushes with fused
 * resolve into d_out_stage, copies the result to h_out, and waits for the
 * copies on `stream`. */
int wrs_push_frame_host(wrs_ctx* ctx, const float* h_frame, float gaze_x, float gaze_y,
                        const uint8_t* h_fov_map, float* h_out, float* d_frame_stage,
                        uint8_t* d_fov_stage, float* d_out_stage, wrs_stream_t stream);

/* Largest frame (pixels) wrs_push_frame_host_noalloc stages: 3840 x 2160. */
#define WRS_NOALLOC_MAX_PIXELS 8294400

/* wrs_push_frame_host for callers that cannot allocate device memory: the
 * device copies of the frame, the fov map and the resolved output live in a
 * file-scope device array of the library (2 * 12 + 1 bytes per pixel of
 * WRS_NOALLOC_MAX_PIXELS, one copy per device), found with
 * cudaGetSymbolAddress for the stream's device, which must be current. The
 * caller still owns the reservoir state buffer. The paper has no counterpart:
 * this only moves frames between host memory and the device. Arguments,
 * results and errors as wrs_push_frame_host, plus WRS_ERR_ARG for frames
 * above WRS_NOALLOC_MAX_PIXELS or another device being current. The call
 * itself allocates nothing (no cudaMalloc, no allocating library routine).
 * The array (207 MB) is device memory all the same: the CUDA runtime backs it
 * when the library's device code is loaded on a device, which under lazy
 * module loading (CUDA's default) happens at this entry point's first call on
 * that device. If the device is then short of memory (a server close to its
 * budget), that first call fails with WRS_ERR_CUDA: make a warm-up call at
 * start-up, before memory fills up and before any stream capture. Later calls
 * reuse the array. Calls that overlap (from several host threads, or on
 * several CUDA streams of one device, for any stream) share the one staging
 * array and race; serialise them. The call waits for its copies, as
 * wrs_push_frame_host does. */
int wrs_push_frame_host_noalloc(wrs_ctx* ctx, const float* h_frame, float gaze_x, float gaze_y,
                                const uint8_t* h_fov_map, float* h_out, wrs_stream_t stream);

/* Pipelined host-buffer frames: the upload of frame n, the update of frame
 * n-1 and the download of frame n-2's resolved output overlap on three CUDA
 * streams the pipeline owns, through three device staging slots for frames
 * and outputs (and fov maps) in a caller-owned buffer. Each frame gets the same
 * update and output as wrs_push_frame_host. Not a step of the paper's method:
 * it moves frames between host memory and the device. */
typedef struct wrs_host_pipe wrs_host_pipe;

/* Device staging bytes the pipeline needs: three frames and three outputs of
 * width * height RGB floats (and three width * height fov maps if with_fov),
 * each 256-byte aligned. 0 for a NULL context. */
size_t wrs_host_pipe_stage_bytes(const wrs_ctx* ctx, int with_fov);

/* Creates a pipeline for `ctx` on d_stage (caller-owned, 256-byte aligned,
 * at least wrs_host_pipe_stage_bytes bytes, on the context's device, which
 * must be current). The pipeline owns its streams and events. Errors:
 * WRS_ERR_ARG, WRS_ERR_BUDGET, WRS_ERR_CUDA. */
int wrs_host_pipe_create(wrs_ctx* ctx, void* d_stage, size_t bytes, int with_fov,
                         wrs_host_pipe** out);

/* Enqueues one frame: h_frame [height][width][3] floats is uploaded
 * asynchronously, the context's update and fused resolve run, and the
 * resolved frame is downloaded to h_out asynchronously. Before enqueuing
 * frame n the call waits until frame n-3 is complete, so at most three frames
 * are in flight and the host buffers of frame n-3 and older are free again.
 * h_frame, h_fov_map (nullable) and h_out of the last three frames must stay
 * valid and unmodified until wrs_host_pipe_finish (pinned host memory makes
 * the copies asynchronous). The context's device must be current. Errors: as
 * wrs_push_frame, WRS_ERR_ARG for another current device, WRS_ERR_CUDA. */
int wrs_host_pipe_push(wrs_host_pipe* p, const float* h_frame, float gaze_x, float gaze_y,
                       const uint8_t* h_fov_map, float* h_out);

/* Waits until every enqueued frame's output is in its host buffer. */
int wrs_host_pipe_finish(wrs_host_pipe* p);

/* Finishes, then releases the streams and events (not the stage buffer). */
int wrs_host_pipe_destroy(wrs_host_pipe* p);

/* Copies the state (the header and the planes of wrs_state_layout, bytes
 * 0 .. map_off) to / from host memory and waits for the copy; h_dst / h_src
 * hold total_bytes, and export writes zeros over the ring's part of h_dst.
 * Export first folds every pending replacement code into the idx planes (a
 * kernel on `stream`), so the exported planes are complete. Used for
 * checkpoints, migration of a stream between devices, and tests. Import also
 * sets the frame counter and makes a context whose wait gave up usable again
 * (wrs_check_status). */
int wrs_export_state(wrs_ctx* ctx, void* h_dst, size_t bytes, wrs_stream_t stream);
int wrs_import_state(wrs_ctx* ctx, const void* h_src, size_t bytes, uint32_t frame_index,
                     wrs_stream_t stream);

/* Frame counter: frames pushed since create (or the imported index). */
uint32_t wrs_frame_index(const wrs_ctx* ctx);

/* Launch shape of the fused kernel: threads per block (64..1024, multiple of
 * 32) and pixels per thread (1, 2 or 4). 0 restores the default. Pixels per
 * thread above 1 need width divisible by it for vector frame I/O; otherwise
 * the kernel falls back to per-pixel frame access. */
int wrs_set_launch(wrs_ctx* ctx, int block_threads, int px_per_thread);
int wrs_get_launch(const wrs_ctx* ctx, int* block_threads, int* px_per_thread);

/* Kernel choice for wrs_push_frame. enable = 1 (default) uses the pipelined
 * persistent kernel whenever width % 4 == 0, frame_pitch_elems == 3 * width and
 * frame/out are 16-byte aligned (else the plain kernel runs): persistent CTAs
 * (ctas_per_sm per SM; 0 = as many as registers and shared memory allow)
 * stream tiles of 256 * px_per_thread pixels (1, 2 or 4) through `stages`
 * shared-memory stages with bulk asynchronous copies. 0 for px_per_thread
 * selects 256-pixel tiles; 0 for stages selects as many stages (up to four)
 * as keep two CTAs on an SM, else as many as one CTA holds (the default for
 * a new context). Results are bit-identical across every choice. WRS_ERR_ARG
 * if the stages do not fit in shared memory. */
int wrs_set_pipeline(wrs_ctx* ctx, int enable, int px_per_thread, int stages, int ctas_per_sm);
int wrs_get_pipeline(const wrs_ctx* ctx, int* enable, int* px_per_thread, int* stages,
                     int* ctas_per_sm);

/* Every device-side wait (the pipelined kernel's copy barriers) gives up after
 * timeout_ns (0: the 2 s default) and records WRS_ERR_TIMEOUT in the stream's
 * status word instead of hanging. test_extra_tx > 0 makes each wait expect
 * that many bytes more than are copied, so that it runs out: fault injection
 * for tests only (<= 4096). */
int wrs_set_wait_limit(wrs_ctx* ctx, uint64_t timeout_ns, uint32_t test_extra_tx);

/* Waits for `stream`, reads and clears the status word (and, in the checked
 * build, the check word). WRS_OK, WRS_ERR_TIMEOUT if a wait gave up since the
 * last check, or WRS_ERR_CHECK if the checked build skipped an access outside
 * its buffer. Either error leaves the reservoirs undefined (the push that
 * failed was partly applied, and the pipelined kernels leave the state alone
 * from then until this call): the context is marked failed, and every push,
 * batch containing it and resolve returns WRS_ERR_STATE until
 * wrs_import_state restores a saved state (or the context is destroyed and
 * created again). This is the one exception to "a call that fails leaves the
 * reservoir state as it was": such failures happen on the device, after the
 * call that launched the work has returned. */
int wrs_check_status(wrs_ctx* ctx, wrs_stream_t stream);

/* 1 in the checked build of the library (libwrs_checked.so, compiled with
 * WRS_CHECKED: every kernel tests the indices and copy ranges it uses against
 * their buffers, records a failed test in the stream's check word and skips
 * the access), 0 in the default build. Host only. */
int wrs_checked_build(void);

/* ------------------------------------------------------------------ batches */

/* A batch launcher: pushes one frame into each of up to max_streams streams
 * (any mix of sizes, K and colour precision, all on one device) with a single
 * persistent launch. The launch is a kernel node of a CUDA graph, built on
 * the first push and updated in place for every later push. The library owns
 * the launcher and its graphs (host objects and driver handles only: no
 * device memory). */
typedef struct wrs_batch wrs_batch;
int wrs_batch_create(int max_streams, wrs_batch** out);
int wrs_batch_destroy(wrs_batch* batch);

/* Tile and launch shape: tiles of 256 * px_per_thread pixels (1, 2 or 4),
 * `stages` shared-memory stages (0: two, or one if two do not fit),
 * ctas_per_sm persistent CTAs per SM (0: as many as fit), use_graph = 0 for a
 * plain launch instead of the graph. Chosen by the autotuner. */
int wrs_batch_set_launch(wrs_batch* batch, int px_per_thread, int stages, int ctas_per_sm,
                         int use_graph);
int wrs_batch_get_launch(const wrs_batch* batch, int* px_per_thread, int* stages,
                         int* ctas_per_sm, int* use_graph);

/* Pushes d_frames[i] with gaze (gaze_xy[2i], gaze_xy[2i+1]) into ctxs[i] for
 * i < n, the same per-pixel steps as wrs_push_frame (Sec. 4), with optional
 * flush maps (d_fov_maps NULL or per-stream NULL) and fused resolves into
 * d_outs[i] (d_outs NULL or per-stream NULL). Every frame must be unpadded
 * (pitch 3 * width), width % 4 == 0, frame and out 16-byte aligned; a stream
 * may appear once per batch. gaze_xy is host memory. Each stream's state and
 * output are bit-identical to pushing it alone. Every stream's frame counter
 * advances. Errors: WRS_ERR_ARG, WRS_ERR_STATE, WRS_ERR_CUDA (nothing is
 * launched on error). */
int wrs_push_batch(wrs_batch* batch, int n, wrs_ctx* const* ctxs, const float* const* d_frames,
                   const float* gaze_xy, const uint8_t* const* d_fov_maps, float* const* d_outs,
                   wrs_stream_t stream);

/* A rendered image and its mip levels: the source a stream's frame is
 * foveated from (Sec. 4.3), as wrs_foveate / wrs_push_foveated take it. */
typedef struct {
  const float* d_img;          /* device [height][img_pitch_elems] RGB floats, 4-byte aligned */
  int64_t img_pitch_elems;     /* >= 3 * width */
  const void* d_mip;           /* device mip buffer (wrs_mip_build) with >= nradii + 1 levels */
  size_t mip_bytes;
  int32_t nradii;              /* 1 .. WRS_MAX_MIP_LEVELS - 1 */
  float radii[WRS_MAX_MIP_LEVELS - 1]; /* ring radii in pixels, ascending; [0] the fovea */
} wrs_fov_source;

/* wrs_push_batch with every frame foveated on read (wrs_push_foveated's
 * update, batched): stream i's frame is foveated from sources[i] for its
 * gaze with `filter` (WRS_FILTER_*) by the update kernel itself, so no frame
 * is written to memory and no foveation launch precedes the batch. Results
 * are bit-identical to wrs_push_foveated of each stream alone (and so to
 * wrs_foveate + wrs_push_frame). Needs width % 4 == 0 and 16-byte aligned
 * outputs; always one pixel per thread (256-pixel tiles). Errors: as
 * wrs_push_batch and wrs_foveate (nothing is launched on error). */
int wrs_push_batch_foveated(wrs_batch* batch, int n, wrs_ctx* const* ctxs,
                            const wrs_fov_source* sources, int32_t filter, const float* gaze_xy,
                            const uint8_t* const* d_fov_maps, float* const* d_outs,
                            wrs_stream_t stream);

/* Slot replacements since create (over all pixels and frames; the stream's
 * reservoir churn: a pixel whose candidate entered a slot counts once per
 * frame). Waits for `stream`. */
int wrs_get_stats(wrs_ctx* ctx, uint64_t* replacements, wrs_stream_t stream);

/* ------------------------------------------------------------------------
 * Temporal reprojection (Sec. 4.3, "Implementation"): after camera or scene
 * motion each pixel continues the reservoir of the surface it now shows,
 * found through a motion vector, and a depth comparison between frames drops
 * that history where the surface was occluded or disoccluded.
 * ------------------------------------------------------------------------ */

/* Gives the stream a second state buffer (d_spare, wrs_state_bytes bytes,
 * 256-byte aligned, caller-owned, on the stream's device): a reprojected push
 * reads the previous reservoirs from one buffer and writes the new ones to
 * the other, and the two swap roles after every reprojected push. Plain
 * pushes, resolves, exports and imports always act on whichever buffer holds
 * the current reservoirs; the status word and counters stay in the header of
 * the buffer given to wrs_create. d_spare = NULL detaches the spare buffer,
 * first copying the current reservoirs back into the primary buffer if they
 * live in the spare (enqueued on `stream`). Errors: WRS_ERR_ARG, WRS_ERR_BUDGET
 * (buffer too small), WRS_ERR_CUDA. */
int wrs_set_reprojection_buffer(wrs_ctx* ctx, void* d_spare, size_t bytes, wrs_stream_t stream);

/* One frame with temporal reprojection. Pixel p = (x, y) continues the
 * previous frame's reservoir at the pixel q containing the point
 * (x + 0.5 - mx, y + 0.5 - my), (mx, my) = d_motion[p] the screen-space motion
 * in pixels of the surface seen at p since the previous frame (FP32 sub/add;
 * NULL = no motion). The history is flushed (reservoir emptied, as a 0xFF fov
 * map entry does) when that point lies outside [0, width) x [0, height), when
 * depth buffers are given and |d_prev_depth[q] - d_depth[p]| >
 * depth_tol * d_depth[p] (FP32; view depths of the surfaces at p now and at q
 * in the previous frame), or where d_fov_map is 0xFF. Then the frame's
 * candidate is combined exactly as wrs_push_frame does (same weight, uniform
 * and key race), every slot is written to the other state buffer and the
 * buffers swap. d_motion: [height][width] float pairs (8-byte aligned);
 * d_depth, d_prev_depth: [height][width] floats, both or neither; the rest as
 * for wrs_push_frame. Requires wrs_set_reprojection_buffer. Errors: as
 * wrs_push_frame, plus WRS_ERR_STATE without a spare buffer and WRS_ERR_ARG for
 * a bad depth_tol (negative or not finite) or a lone depth buffer. */
int wrs_push_frame_reproject(wrs_ctx* ctx, const float* d_frame, int64_t frame_pitch_elems,
                             float gaze_x, float gaze_y, const float* d_motion,
                             const float* d_depth, const float* d_prev_depth, float depth_tol,
                             const uint8_t* d_fov_map, float* d_out, wrs_stream_t stream);

/* ------------------------------------------------------------------------
 * Foveation post-process (Sec. 4.3, "Implementation"): the paper simulates
 * foveated rendering on the rendered frame by mip-mapping it and
 * reconstructing each ring around the gaze from a coarser level with
 * filtering. These calls produce, on the device, the foveated frames and
 * ring maps that wrs_push_frame consumes, from a full-resolution image.
 * ------------------------------------------------------------------------ */

/* Where each level of a mip buffer lives. Level L >= 1 holds one texel per
 * aligned 2^L x 2^L block of the image, [height[L]][width[L]] texels of
 * 16 bytes {r, g, b, 0} (float), row-major from offset[L]; offsets are
 * 256-byte aligned. Level 0 is the image itself (offset[0] = -1). */
typedef struct {
  int32_t levels;                        /* levels described, 1..WRS_MAX_MIP_LEVELS */
  int32_t width[WRS_MAX_MIP_LEVELS];     /* ceil(image width / 2^L) */
  int32_t height[WRS_MAX_MIP_LEVELS];    /* ceil(image height / 2^L) */
  int64_t offset[WRS_MAX_MIP_LEVELS];    /* byte offset of level L; -1 for level 0 */
  int64_t total_bytes;                   /* bytes the buffer must hold (0 when levels = 1) */
} wrs_mip_layout;

/* Layout of the mip buffer of a width x height image with `levels` levels
 * (levels 1..L-1 are stored). Levels 1..n of a buffer laid out for more levels
 * sit at the same offsets as in one laid out for n + 1 levels.
 * Returns WRS_ERR_ARG for sizes < 1, width * height >= 2^31 or levels outside
 * 1..WRS_MAX_MIP_LEVELS. */
int wrs_mip_layout_get(int32_t width, int32_t height, int32_t levels, wrs_mip_layout* out);

/* Builds levels 1..levels-1 of the mip buffer from an RGB float image
 * [height][img_pitch_elems] (RGB triples, pitch >= 3 * width, 4-byte aligned).
 * Texel = the block's mean: the FP32 sum over the block, formed as the quad
 * tree (s00 + s01) + (s10 + s11) of its four half-size quadrants (pixels
 * outside the image count as 0), divided by the number of image pixels in the
 * block. d_mip: caller-owned device buffer of at least the layout's
 * total_bytes, 256-byte aligned. Asynchronous on `stream`; the image must not
 * change until the call completes. Errors: WRS_ERR_ARG (NULL or unaligned
 * pointers, bad sizes), WRS_ERR_BUDGET (buffer too small), WRS_ERR_CUDA. */
int wrs_mip_build(const float* d_img, int64_t img_pitch_elems, int32_t width, int32_t height,
                  int32_t levels, void* d_mip, size_t mip_bytes, wrs_stream_t stream);

/* One foveated frame for the gaze (gaze_x, gaze_y) in pixels.
 * Ring level of pixel (x, y): the number of radii r_i with
 * dx*dx + dy*dy > r_i*r_i, dx = (x + 0.5) - gaze_x, dy likewise, all FP32
 * rounded once (a centre exactly on a radius stays inside it). radii: host
 * array of nradii (1..WRS_MAX_MIP_LEVELS-1) finite positive values in
 * ascending order; radii[0] is the foveal radius. Level 0 copies the image
 * pixel; level L reads the level-L texels of d_mip (built by wrs_mip_build
 * with at least nradii + 1 levels; mip_bytes its size): WRS_FILTER_BOX takes
 * the texel of the pixel's block; WRS_FILTER_BILINEAR samples at the level
 * coordinate u = (x + 0.5) * 2^-L - 0.5 (v likewise) clamped to
 * [0, width[L] - 1], with x0 = floor(u), fx = u - x0, x1 = min(x0 + 1,
 * width[L] - 1) and colour = top * (1 - fy) + bot * fy,
 * top = t00 * (1 - fx) + t01 * fx, bot = t10 * (1 - fx) + t11 * fx, each
 * product and sum one FP32 rounding. Writes d_frame [height][frame_pitch_elems]
 * (RGB triples) and, if d_ring_map is not NULL, the level of each pixel to
 * d_ring_map [height][width] (bytes 0..nradii: a valid fov map for
 * wrs_push_frame, no flushes). d_img and d_frame must not overlap.
 * Asynchronous on `stream`. Errors: WRS_ERR_ARG, WRS_ERR_BUDGET (mip_bytes
 * below the layout's size for nradii + 1 levels), WRS_ERR_CUDA. */
int wrs_foveate(const float* d_img, int64_t img_pitch_elems, const void* d_mip, size_t mip_bytes,
                int32_t width, int32_t height, int32_t nradii, const float* radii, float gaze_x,
                float gaze_y, int32_t filter, float* d_frame, int64_t frame_pitch_elems,
                uint8_t* d_ring_map, wrs_stream_t stream);

/* wrs_foveate followed by wrs_push_frame in one pass, without the frame in
 * memory: the update kernel foveates each pixel of the frame (same ring test,
 * texels and arithmetic as wrs_foveate, so the reservoirs and the output are
 * bit-identical to the two calls) as it reads the pixel's reservoir. d_img,
 * img_pitch_elems, d_mip, mip_bytes, nradii, radii and filter as for
 * wrs_foveate (the image is width x height of the stream); gaze, d_fov_map
 * (a flush map: only 0xFF matters) and d_out as for wrs_push_frame. Needs
 * width % 4 == 0 and d_out 16-byte aligned; always takes the pipelined kernel
 * with one pixel per thread. Errors: as wrs_foveate and wrs_push_frame. */
int wrs_push_foveated(wrs_ctx* ctx, const float* d_img, int64_t img_pitch_elems,
                      const void* d_mip, size_t mip_bytes, int32_t nradii, const float* radii,
                      int32_t filter, float gaze_x, float gaze_y, const uint8_t* d_fov_map,
                      float* d_out, wrs_stream_t stream);

/* Message of the last failed call on this thread ("" if none). */
const char* wrs_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* WRS_H */
