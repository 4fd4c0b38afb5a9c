/*
 * svgf.h -- C ABI of the GB300 (sm_103a) variance-guided denoiser of "Hybrid-Rendering
 * Techniques in GPU" (Granja & Pereira, 2021): Reinhard tone mapping (Sec. 3.4), temporal
 * accumulation with backward reprojection and moment/variance estimation (Sec. 2, Sec. 3 step 4),
 * history rectification by variance colour clamping (Sec. 3.1) with the adaptive blur start that
 * counters its artifacts (Sec. 3.2), the edge-avoiding a-trous wavelet passes (Sec. 2 Fig. 1,
 * Sec. 3 step 5) or their separable variant (Sec. 3.3), and the inverse tone map (Sec. 3.4).
 *
 * Conventions (all entry points):
 *  - Images are row-major, tightly packed, pixel (x, y) at index y*width + x; every buffer is
 *    FP32 with the channel count given per argument.  Device pointers must be 16-byte aligned.
 *  - All device memory is owned by the caller: frame inputs, outputs and the workspace bound
 *    with svgf_bind_workspace.  The library allocates no device memory; a handle is host state.
 *  - `stream` is a cudaStream_t passed as void* (NULL = the legacy default stream).  Calls on
 *    device buffers only enqueue work on `stream` and return; results are ready when the
 *    stream is.  Calls on one handle must be issued from one host thread, in order.
 *  - Argument errors are reported before anything is enqueued (SVGF_ERR_INVALID_ARG,
 *    SVGF_ERR_UNSUPPORTED, SVGF_ERR_NO_WORKSPACE) and leave the handle unchanged.  A failed
 *    launch returns SVGF_ERR_CUDA; svgf_last_error() then holds the CUDA error text.
 *  - No entry point throws, aborts or prints.
 *
 * Storage precision (svgf_config.precision).  The colour+variance images that pass between the
 * stages ("cv" buffers: svgf_reproject_accumulate's output, svgf_atrous' input and output,
 * svgf_inverse_tonemap's input) and the workspace's history and moments are stored as
 *  - SVGF_FP32: [H][W][4] float (R, G, B, variance), 16-byte aligned;
 *  - SVGF_FP16: [H][W] 8-byte records of four 16-bit fields: R, G, B as IEEE FP16 and the
 *    variance as BF16 (its 8-bit exponent keeps the small variances of the late passes), 8-byte
 *    aligned;
 *  - SVGF_BF16: the same record with all four fields BF16.
 * Every computation -- reprojection coordinates, the depth test, edge-stopping weights and their
 * sums, the variance step -- is FP32 in every mode; 16-bit values are widened on load and rounded
 * to nearest on store.  Frame inputs and rgb_out are FP32 in every mode.
 */
#ifndef SVGF_H
#define SVGF_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum svgf_status {
    SVGF_OK = 0,
    SVGF_ERR_INVALID_ARG = 1,   /* NULL/misaligned pointer, bad size or config value */
    SVGF_ERR_UNSUPPORTED = 2,   /* a valid but unimplemented option */
    SVGF_ERR_CUDA = 3,          /* a CUDA call failed (see svgf_last_error) */
    SVGF_ERR_TIMEOUT = 4,       /* a bounded device wait gave up */
    SVGF_ERR_DEVICE_CHECK = 5,  /* a device-side check raised the handle's error word */
    SVGF_ERR_NO_WORKSPACE = 6   /* no (or too small a) workspace is bound */
} svgf_status;

enum { SVGF_ATROUS_5X5 = 0, SVGF_SEPARABLE = 1 };          /* svgf_config.spatial_mode */
enum { SVGF_INVERSE_EXACT = 0, SVGF_INVERSE_PAPER = 1 };   /* svgf_config.inverse_mode */
enum { SVGF_FP32 = 0, SVGF_FP16 = 1, SVGF_BF16 = 2 };      /* svgf_config.precision */
enum { SVGF_RECTIFY_CLAMP = 0, SVGF_RECTIFY_CLIP = 1 };    /* svgf_config.rectify_mode */

/* Denoiser parameters.  svgf_default_config fills the values in brackets. */
typedef struct svgf_config {
    int width, height;          /* frame size in pixels, each in [1, 32768] */
    float alpha;                /* colour accumulation factor, a = max(alpha, 1/n) [0.2] (Sec. 2) */
    float alpha_moments;        /* moment accumulation factor [0.2] (Sec. 2) */
    float clamp_gamma;          /* clamp box m +- gamma*sigma over 3x3 [1.0] (Sec. 3.1) */
    int atrous_iters;           /* a-trous iterations, 0..8 [5] (Sec. 2, Sec. 3 step 5) */
    float sigma_z, sigma_n, sigma_l; /* depth, normal, luminance edge-stopping [1, 128, 4] */
    int spatial_mode;           /* SVGF_ATROUS_5X5 or SVGF_SEPARABLE (Sec. 3.3) [5X5] */
    int clamp_enable;           /* history rectification on/off [1] (Sec. 3.1) */
    int adaptive_start;         /* start one scale higher above the threshold [1] (Sec. 3.2) */
    float roughness_threshold;  /* [0.2] (Sec. 3.2) */
    int tonemap;                /* Reinhard before / inverse after denoising [1] (Sec. 3.4) */
    float luma_k;               /* lumaMultiplier of the forward map [1] (Sec. 3.4) */
    float inv_weight;           /* reinhardToneMappingWeight of the printed inverse [1] */
    int inverse_mode;           /* SVGF_INVERSE_EXACT or SVGF_INVERSE_PAPER [EXACT] */
    int history_from_pass;      /* a-trous pass whose output becomes the colour history; -1 =
                                   the accumulated colour [0] */
    float depth_rel_tol;        /* reprojection: |z_prev - z| <= tol * z [0.1] */
    float normal_cos_tol;       /* reprojection: cos(n, n_prev) >= tol [0.9] */
    float disocclusion_weight;  /* valid bilinear weight below which history is dropped [1e-4] */
    int max_history;            /* history length cap, 1..65535 [255] */
    int min_temporal_frames;    /* temporal variance once n >= this, else spatial [4] */
    int spatial_var_radius;     /* spatial variance window radius, 0..7 [3] */
    float eps;                  /* edge-stopping denominator guard [1e-10] */
    int precision;              /* storage of the colour+variance, history and moment images:
                                   SVGF_FP32, SVGF_FP16 or SVGF_BF16 [FP32]; see below */
    int rectify_mode;           /* history rectification when clamp_enable (Sec. 3.1, Fig. 3):
                                   SVGF_RECTIFY_CLAMP limits each channel to m +- gamma*sigma;
                                   SVGF_RECTIFY_CLIP moves the history toward m along the line
                                   from m until it lies in that box [CLAMP] */
    int iter_by_roughness;      /* roughness-adapted number of a-trous passes per pixel (Sec.
                                   3.5): roughness <= iter_rough_t0 -> iter_count0 passes,
                                   <= iter_rough_t1 -> iter_count1, otherwise atrous_iters; a
                                   pixel past its budget keeps its input colour and variance.
                                   Needs svgf_frame.roughness [0] */
    float iter_rough_t0, iter_rough_t1; /* [0, 0.05], t0 <= t1 */
    int iter_count0, iter_count1;       /* [0, 1], each in 0..8 (above atrous_iters: all) */
} svgf_config;

/* One frame's inputs (device pointers, caller-owned, read-only during the call's work).
 *  noisy_rgb     [H][W][3]  1-spp noisy radiance (linear HDR)
 *  gbuf_nz       [H][W][4]  world-space unit normal (x, y, z) and linear view-axis depth
 *  prev_gbuf_nz  [H][W][4]  the previous frame's gbuf_nz, or NULL: history is then dropped
 *  motion        [H][W][2]  screen motion mv = p_cur - p_prev in pixels
 *  roughness     [H][W]     per-pixel surface roughness (may be NULL if adaptive_start = 0
 *                           and iter_by_roughness = 0) */
typedef struct svgf_frame {
    const float* noisy_rgb;
    const float* gbuf_nz;
    const float* prev_gbuf_nz;
    const float* motion;
    const float* roughness;
} svgf_frame;

typedef struct svgf_handle svgf_handle;

/* Fill *out with the defaults above for a width x height frame. */
svgf_status svgf_default_config(int width, int height, svgf_config* out);

/* The hybrid renderer's denoised channels (Sec. 3 step 5: shadows and indirect specular are
 * filtered separately, each with the extra techniques of Sec. 3.1-3.4). */
enum { SVGF_CHANNEL_INDIRECT_SPECULAR = 0, SVGF_CHANNEL_SHADOW = 1 };

/* Fill *out with one channel's defaults for a width x height frame.
 *  INDIRECT_SPECULAR: svgf_default_config (Reinhard on; adaptive start above roughness 0.2).
 *  SHADOW: no tone mapping (Sec. 3.4 applies it to the specular channel only) and the adaptive
 *          start above a shadow angle of 6.0 (Sec. 3.2): the frame's `roughness` image then
 *          holds the light's angular size seen from each pixel, in degrees; the noisy input is
 *          the visibility replicated into RGB.
 * Returns SVGF_ERR_INVALID_ARG for an unknown channel or a size outside [1, 32768]. */
svgf_status svgf_channel_config(int channel, int width, int height, svgf_config* out);

/* Validate *cfg and create a host-side handle.  The handle needs a workspace
 * (svgf_workspace_size / svgf_bind_workspace) before any frame call. */
svgf_status svgf_create(const svgf_config* cfg, svgf_handle** out);

/* Destroy a handle (NULL is accepted).  The caller frees the workspace after the stream that
 * last used it has finished. */
svgf_status svgf_destroy(svgf_handle* h);

/* Bytes of device workspace the handle needs: colour history and moments (two slots each,
 * swapped per frame), two a-trous ping-pong buffers, the separable pass buffer, a per-tile
 * flag array and the device error word. */
svgf_status svgf_workspace_size(const svgf_handle* h, size_t* bytes);

/* Bind caller-owned device memory (256-byte aligned, >= svgf_workspace_size bytes).  Binding
 * resets the temporal history.  The memory must stay valid while the handle uses it. */
svgf_status svgf_bind_workspace(svgf_handle* h, void* dev, size_t bytes);

/* Drop the temporal history: the next frame starts with history length 1 (Sec. 2). */
svgf_status svgf_reset_history(svgf_handle* h);

/* Temporal stage of one frame (Sec. 2; Sec. 3 step 4; Sec. 3.1; Sec. 3.4 forward map):
 * tone-map the noisy colour, reproject the colour history and moments bilinearly with depth and
 * normal consistency tests, clamp the history colour to the 3x3 mean +- gamma*sigma box, blend
 * with a = max(alpha, 1/n), update the luminance moments and estimate the variance (temporal
 * for n >= min_temporal_frames, else 7x7 spatial).  Writes cv_out (storage precision) =
 * accumulated (tone-mapped) colour and variance; updates the moments and history length in the
 * workspace.
 * This call starts a new frame: the next svgf_atrous calls belong to it. */
svgf_status svgf_reproject_accumulate(svgf_handle* h, const svgf_frame* f, float* cv_out,
                                      void* stream);

/* Variance colour clamp alone (Sec. 3.1): hist_out = clamp(hist_in, m - gamma*s, m + gamma*s)
 * per RGB channel, m and s the mean and population standard deviation of f->noisy_rgb
 * (tone-mapped when cfg.tonemap) over the in-image 3x3 neighbourhood.  hist_in/hist_out are
 * [H][W][4]; channel 3 is copied.  Touches no handle state. */
svgf_status svgf_clamp(svgf_handle* h, const svgf_frame* f, const float* hist_in,
                       float* hist_out, void* stream);

/* One a-trous iteration `iter` (0-based) of the current frame (Sec. 2 Fig. 1; Sec. 3 step 5;
 * Sec. 3.2 adaptive start; Sec. 3.3 separable when spatial_mode = SVGF_SEPARABLE):
 * step 2^(iter + s_p), s_p = 1 where roughness > roughness_threshold (if adaptive_start);
 * weights h_j h_k w_z w_n w_l; colour = sum w c / sum w, variance = sum w^2 var / (sum w)^2.
 * cv_in/cv_out (colour, variance; storage precision) must not overlap.  When iter equals
 * history_from_pass the output colour also becomes the next frame's colour history. */
svgf_status svgf_atrous(svgf_handle* h, int iter, const svgf_frame* f, const float* cv_in,
                        float* cv_out, void* stream);

/* Inverse tone map (Sec. 3.4) of cv_in (storage precision) into rgb_out [H][W][4] float (colour,
 * channel 3 = variance): exact c'/(1 - k luma(c')) or the printed c'(1 + luma(c'))w per
 * inverse_mode; a plain copy when cfg.tonemap = 0.  In place (cv_in == rgb_out) is allowed in
 * FP32 storage only. */
svgf_status svgf_inverse_tonemap(svgf_handle* h, const float* cv_in, float* rgb_out,
                                 void* stream);

/* The whole frame: svgf_reproject_accumulate, atrous_iters x svgf_atrous, then the inverse tone
 * map fused into the last pass.  rgb_out [H][W][4] = denoised linear colour and the final
 * variance.  Bit-identical to the stage calls in that order. */
svgf_status svgf_denoise_frame(svgf_handle* h, const svgf_frame* f, float* rgb_out,
                               void* stream);

/* Copy the temporal state (colour history [H][W][4] float = RGB, 0; moments [H][W][4] float =
 * mu1, S = mu2 - mu1^2, history length n, 0; FP32 in every storage precision) of the last frame
 * to caller device buffers (export) or replace it (import; has_history = 0 drops it; imported
 * values are rounded to the storage precision).  The second moment is held in this central form
 * (S, the luminance variance of the history) so that FP32 storage does not lose the variance to
 * the cancellation of mu2 - mu1^2.  For checkpoint/resume and stage-level tests. */
svgf_status svgf_history_export(svgf_handle* h, float* hist_rgb, float* moments, void* stream);
svgf_status svgf_history_import(svgf_handle* h, const float* hist_rgb, const float* moments,
                                int has_history, void* stream);

/* ---- host-buffer entry points (end-to-end use without device-memory management) ---------
 * svgf_host_submit enqueues one frame given in host memory: it copies the frame's noisy colour,
 * G-buffer, motion and roughness (page-locked memory gives asynchronous copies) into a caller-
 * owned device staging area on a copy stream of the handle, denoises on `stream`
 * (svgf_denoise_frame), and copies rgb_out ([H][W][4] float) back to host_rgb_out on a second
 * copy stream; it returns without waiting.  Up to two frames are in flight: the uploads of frame
 * t + 1 and the download of frame t - 1 overlap the denoise of frame t (events order each
 * staging slot's reuse).  svgf_host_wait returns when every submitted frame's result is in host
 * memory; until then the host inputs must stay unchanged and host_rgb_out must not be read.
 * svgf_denoise_frame_host is submit + wait (the output is ready on return).  The previous
 * frame's G-buffer is kept in the staging area (host_frame->prev_gbuf_nz is ignored); the first
 * frame after creation, binding or svgf_reset_history has no history.  Staging needs
 * svgf_staging_size bytes, 256-byte aligned, bound with svgf_bind_staging (call svgf_host_wait
 * before rebinding or destroying while frames are in flight). */
svgf_status svgf_staging_size(const svgf_handle* h, size_t* bytes);
svgf_status svgf_bind_staging(svgf_handle* h, void* dev, size_t bytes);
svgf_status svgf_denoise_frame_host(svgf_handle* h, const svgf_frame* host_frame,
                                    float* host_rgb_out, void* stream);
svgf_status svgf_host_submit(svgf_handle* h, const svgf_frame* host_frame, float* host_rgb_out,
                             void* stream);
svgf_status svgf_host_wait(svgf_handle* h);

/* ---- per-kernel timing ------------------------------------------------------------------
 * With profiling on, every kernel this handle launches is bracketed by CUDA events on its
 * stream (up to 4096 launches between reads; later launches are not timed).  svgf_profile_read
 * must be called after the stream has finished: it returns, per kernel kind, the summed
 * device time in milliseconds and the launch count since the last read, then clears them.
 * Kinds: SVGF_K_TEMPORAL, SVGF_K_SPATIAL_VAR, SVGF_K_ATROUS_5X5, SVGF_K_ATROUS_H,
 * SVGF_K_ATROUS_V, SVGF_K_INVERSE, SVGF_K_CLAMP (SVGF_K_COUNT entries). */
enum { SVGF_K_TEMPORAL = 0, SVGF_K_SPATIAL_VAR = 1, SVGF_K_ATROUS_5X5 = 2, SVGF_K_ATROUS_H = 3,
       SVGF_K_ATROUS_V = 4, SVGF_K_INVERSE = 5, SVGF_K_CLAMP = 6, SVGF_K_COUNT = 7 };
svgf_status svgf_profile_enable(svgf_handle* h, int enable);
svgf_status svgf_profile_read(svgf_handle* h, double* total_ms, unsigned long long* counts,
                              int n_kinds);

/* ---- batched streams (one persistent launch per stage over many frames) --------------------
 * A batch groups n handles (1 <= n <= 1024), each with its own bound workspace (each handle is
 * one stream of frames).  They must share the storage precision, the spatial mode and
 * atrous_iters (these select the kernels and the launches); every other field, and the frame
 * size, may differ per handle -- e.g. the shadow and the indirect-specular channel of one frame
 * (Sec. 3 step 5), each with its own tone mapping and adaptive-start rule (svgf_channel_config),
 * denoised in the same launches.
 * svgf_batch_denoise denoises one frame of every stream -- frames[i] into outs[i] (device,
 * [H_i][W_i][4] float) for handle i -- with one persistent launch per stage (temporal, spatial
 * variance, each a-trous pass) over the tiles of up to 64 streams per launch; results are
 * bit-identical to svgf_denoise_frame on each handle.  Requires atrous_iters >= 1.
 *  - svgf_batch_use_graph(b, 1): every svgf_batch_denoise call captures its launches into a CUDA
 *    graph, updates the batch's executable graph with it (re-instantiating when the update is
 *    refused) and launches the graph: one host launch per frame step.  `stream` must then be a
 *    created stream (not the legacy default stream, which cannot be captured).
 *  - svgf_batch_autotune denoises one frame like svgf_batch_denoise and, on the way, times every
 *    compiled a-trous tile shape (32x8, 32x4, 16x16, 64x4) x grid (one block per tile, or a
 *    persistent grid of 1x, 2x, 4x the kernel's resident blocks per SM walking the tiles with a
 *    grid stride) on that
 *    frame's a-trous passes, keeps the fastest (blocks_per_sm = 0 is one block per tile), and
 *    writes a one-line
 *    report per candidate into `report` (may be NULL).  It waits for `stream`.  The choice is read
 *    and set with svgf_batch_get_tuning / svgf_batch_set_tuning (to reuse a tuning).
 * The handles must outlive the batch and must not be used on their own while it is in use. */
typedef struct svgf_batch svgf_batch;
svgf_status svgf_batch_create(svgf_handle* const* handles, int n, svgf_batch** out);
svgf_status svgf_batch_destroy(svgf_batch* b);
svgf_status svgf_batch_denoise(svgf_batch* b, const svgf_frame* frames, float* const* outs,
                               void* stream);
svgf_status svgf_batch_use_graph(svgf_batch* b, int enable);
svgf_status svgf_batch_autotune(svgf_batch* b, const svgf_frame* frames, float* const* outs,
                                void* stream, char* report, size_t report_len);
svgf_status svgf_batch_get_tuning(const svgf_batch* b, int* atrous_shape, int* blocks_per_sm);
svgf_status svgf_batch_set_tuning(svgf_batch* b, int atrous_shape, int blocks_per_sm);

/* ---- learned part: kernel-predicting network standing in for a-trous iterations 2.. --------
 * Not in the paper (an extension of the denoiser).  After the temporal stage and a-trous pass 0,
 * a small CNN predicts a 5x5 kernel per pixel from 10 features of the pass-0 output (tone-mapped
 * colour 3, sqrt of the variance 1, log2 depth 1, octahedral normal 2, albedo 3): four 3x3
 * convolutions 10 -> 32 -> 32 -> 32 -> 25 with ReLU between (BF16 operands, FP32 accumulation, on
 * the tensor cores), a softmax over the 25 logits, and the kernel applied to the pass-0 colour at
 * dilation 1 and then at dilation 4 (renormalised over in-image taps).  It is trained (MSE in
 * tone-mapped space against the plain pipeline's output, Adam) by the library's own backward
 * kernels.
 *
 * Parameters: SVGF_KPN_PARAM_COUNT FP32 values, caller-owned device memory, one flat array: for
 * layers l = 0..3, W_l [co][9][ci] (tap = (dy + 1) * 3 + (dx + 1)) then b_l [co].
 * Batches: features [B][H][W][16] BF16 (channels 10..15 zero; svgf_kpn_features makes them),
 * c0 and target [B][H][W][4] float (RGB in tone-mapped space, channel 3 ignored), c2 likewise.
 * Workspace: svgf_kpn_workspace_size(max_pixels) bytes (about 650 per pixel), 256-byte aligned,
 * for batches of up to max_pixels = B*H*W pixels or frames of up to max_pixels pixels.
 * grad, adam_m, adam_v (SVGF_KPN_PARAM_COUNT floats each) may be NULL for inference only. */
#define SVGF_KPN_PARAM_COUNT 28633
typedef struct svgf_kpn svgf_kpn;
svgf_status svgf_kpn_workspace_size(int max_pixels, size_t* bytes);
svgf_status svgf_kpn_create(float* params, float* grad, float* adam_m, float* adam_v,
                            void* workspace, size_t workspace_bytes, int max_pixels,
                            svgf_kpn** out);
svgf_status svgf_kpn_destroy(svgf_kpn* k);

/* Read and clear the learned part's device error word (zeroed on the stream before its first
 * convolution).  Value 2: a tensor-core convolution block gave up one of its bounded waits (for
 * a staged row, its MMAs or an accumulator slot; about a second each) and stopped, leaving the
 * rest of its rows unwritten.  Waits for `stream`; *word (may be
 * NULL) receives the value.  Returns SVGF_OK when it was 0, SVGF_ERR_TIMEOUT when it was 2,
 * SVGF_ERR_DEVICE_CHECK for any other value. */
svgf_status svgf_kpn_check_device(svgf_kpn* k, int* word, void* stream);

/* Failure-detection self-test of the bounded device wait above: enqueues on `stream` one block
 * that waits, with the convolutions' wait, on a barrier phase nothing completes; the wait gives
 * up after `tries` polls (1 .. 2^20; a poll is at most a few microseconds) and raises the error
 * word as a convolution block would, so that svgf_kpn_check_device then returns
 * SVGF_ERR_TIMEOUT with *word = 2 and clears it.  Touches nothing else; the context and the
 * handle stay usable.  SVGF_ERR_INVALID_ARG for a NULL handle or tries out of range. */
svgf_status svgf_kpn_wait_selftest(svgf_kpn* k, int tries, void* stream);
/* Checkpoint of the learned part in host memory: the parameters and, when the handle trains
 * (adam_m given), the Adam moments and step count, in a fixed little-endian layout: uint32
 * magic 0x504B5653, uint32 version 1, uint32 SVGF_KPN_PARAM_COUNT, uint32 flags (bit 0: Adam
 * state follows), uint64 Adam step count, float params[count], then float adam_m[count], float
 * adam_v[count] when flagged.
 * svgf_kpn_save: host_buf NULL -> *bytes = the size needed; otherwise *bytes is the buffer's
 * capacity on entry (too small: SVGF_ERR_INVALID_ARG with *bytes = the size needed) and the
 * size written on return; waits for `stream`.
 * svgf_kpn_load: checks magic, version, count and size (SVGF_ERR_INVALID_ARG otherwise), copies
 * the parameters (and the Adam state when both the checkpoint and the handle have it; else the
 * optimiser restarts from zero), refreshes the BF16 weights and waits for `stream`. */
svgf_status svgf_kpn_save(svgf_kpn* k, void* host_buf, size_t* bytes, void* stream);
svgf_status svgf_kpn_load(svgf_kpn* k, const void* host_buf, size_t bytes, void* stream);
/* Refresh the BF16 copies of the weights after `params` was written (initialised or loaded);
 * the training step refreshes them itself.  Zeroes the Adam step count when reset_adam != 0. */
svgf_status svgf_kpn_params_changed(svgf_kpn* k, int reset_adam, void* stream);
/* Network forward of a batch: c2_out [B][H][W][4] float. */
svgf_status svgf_kpn_forward(svgf_kpn* k, const void* feats, const float* c0, int B, int H, int W,
                             float* c2_out, void* stream);
/* Loss (mean squared error, device float *loss_out) and its gradient into `grad`. */
svgf_status svgf_kpn_grad(svgf_kpn* k, const void* feats, const float* c0, const float* target,
                          int B, int H, int W, float* loss_out, void* stream);
/* svgf_kpn_grad followed by one Adam update of `params` (beta 0.9 / 0.999, eps 1e-8). */
svgf_status svgf_kpn_train_step(svgf_kpn* k, const void* feats, const float* c0,
                                const float* target, int B, int H, int W, float lr,
                                float* loss_out, void* stream);
/* The network alone on a batch: the per-pixel 5x5 kernels (the softmax of the 25 logits) for
 * features [B][H][W][16] BF16, into kernels_out [B][H][W][32] FP16 (25 weights and 7 zeros, 64
 * bytes a pixel, 16-byte aligned), as svgf_kpn_denoise_frame hands them to its kernel
 * applications.  form 0: the four convolutions in one kernel, the activations kept in shared
 * memory (no activation buffers in device memory); form 1: layer by layer through device memory
 * (the convolutions of svgf_kpn_forward and svgf_kpn_denoise_frame); form 2: two kernels of two
 * layers each, only the layer-1 activation passing through device memory.  All forms give the
 * same bits.  SVGF_ERR_INVALID_ARG for a
 * NULL handle or pointer, a misaligned pointer, B*H*W above the workspace's max_pixels or
 * another form. */
svgf_status svgf_kpn_predict(svgf_kpn* k, const void* feats, int B, int H, int W, void* kernels_out,
                             int form, void* stream);
/* The two kernel applications of the learned frame on their own: the per-pixel kernels
 * `kernels` [H][W][32] FP16 (as svgf_kpn_predict writes them) applied to c0 [H][W][4] float (the
 * pass-0 colour in tone-mapped space and its variance, as svgf_kpn_features writes it) at
 * dilation 1 and then at dilation 4, each renormalised over its in-image taps, then the handle's
 * inverse tone map into rgb_out [H][W][4] float (channel 3 = c0's variance); H and W are the
 * handle's, and the dilation-1 result passes through the learned part's workspace.  The same
 * launches, and bits, as svgf_kpn_denoise_frame.  SVGF_ERR_INVALID_ARG for a NULL or misaligned
 * pointer; SVGF_ERR_NO_WORKSPACE when the learned part's workspace holds fewer than width*height
 * pixels. */
svgf_status svgf_kpn_apply(svgf_kpn* k, svgf_handle* h, const void* kernels, const float* c0, float* rgb_out,
                           void* stream);
/* Features of one frame from a pass-0 output `cv` (the handle's storage precision), the frame's
 * G-buffer and albedo [H][W][3] float: feats_out [H][W][16] BF16, c0_out [H][W][4] float (the
 * pass-0 colour and variance; may be NULL). */
svgf_status svgf_kpn_features(svgf_handle* h, const void* cv, const svgf_frame* f,
                              const float* albedo, void* feats_out, float* c0_out, void* stream);
/* A whole frame with the network standing in for a-trous iterations 2..: temporal stage, pass 0
 * (which still writes the colour history), features, network, the two kernel applications and
 * the inverse tone map into rgb_out [H][W][4] float (channel 3 = pass-0 variance).  The 25
 * per-pixel kernel weights pass between the network and the applications as FP16 (the forward
 * of svgf_kpn_forward / svgf_kpn_train_step keeps them FP32 for the gradients).  Fallback:
 * when detail_threshold is finite, every 32x32 tile in which the standard deviation of the
 * pass-0 luminance (tone-mapped, population form) exceeds it takes the plain a-trous passes
 * 1..atrous_iters-1 instead, bit-identical to svgf_denoise_frame there.  The call reads the
 * number of such tiles back (waiting for `stream` up to that point) into *fallback_tiles (host
 * int, may be NULL) and runs the plain passes only if it is non-zero, each pass only on the tiles
 * the flagged ones depend on (the whole frame when history_from_pass is one of passes
 * 1..atrous_iters-1, since that pass writes the colour history).  Requires atrous_iters >= 1 and
 * a KPN workspace of at least width*height pixels. */
svgf_status svgf_kpn_denoise_frame(svgf_kpn* k, svgf_handle* h, const svgf_frame* f,
                                   const float* albedo, float* rgb_out, float detail_threshold,
                                   int* fallback_tiles, void* stream);

/* ---- separable iteration without any allocation ---------------------------------------
 * The paper has no counterpart to this entry point; it exists for callers that cannot
 * allocate device memory -- code running where cudaMalloc is forbidden or unavailable, such as
 * inside a host callback, a real-time thread with a no-allocation rule, or an embedding that
 * only hands out its own fixed buffers -- and so cannot provide svgf_bind_workspace's memory.
 *
 * svgf_atrous_separable_noalloc runs one separable a-trous iteration `iter` (Sec. 3.3: the
 * horizontal then the vertical 5-tap pass, same weights and results as svgf_atrous with
 * spatial_mode = SVGF_SEPARABLE) of cv_in [H][W][4] into cv_out [H][W][4], whatever the
 * handle's spatial_mode.  The handle supplies the configuration only: no workspace needs to be
 * bound, and no temporal state is read or written (the colour history is not updated).  The
 * horizontal pass's output goes to a scratch array that is part of the library image: a
 * file-scope device array of SVGF_NOALLOC_MAX_PIXELS float4 (32 MiB), which every GPU that loads
 * the library holds until the process exits.  Frames larger than SVGF_NOALLOC_MAX_PIXELS
 * pixels are rejected with SVGF_ERR_INVALID_ARG (svgf_last_error(h) says why).  The call
 * allocates nothing: no cudaMalloc, no cudaFree, no allocating library routine.
 *  - The first call on a device looks up the array's device address on that device (the
 *    current device) and remembers it with the identity of the current CUDA context; make that
 *    first call before any stream capture.  A call in another context of the device (after
 *    cudaDeviceReset, for one) looks the address up again, so it too belongs outside a capture.
 *  - All calls in the process share the one array per device and it keeps the last call's
 *    contents; every pixel is rewritten before it is read, so nothing needs clearing.  Calls
 *    whose work overlaps on the GPU (other streams, other host threads) race on the array:
 *    order them on one stream or serialise them. */
#define SVGF_NOALLOC_MAX_PIXELS (1u << 21)
svgf_status svgf_atrous_separable_noalloc(svgf_handle* h, int iter, const svgf_frame* f,
                                          const float* cv_in, float* cv_out, void* stream);

/* Static text of a status code; the last CUDA error text of a handle ("" if none). */
const char* svgf_status_string(svgf_status s);
const char* svgf_last_error(const svgf_handle* h);

/* Number of kernel launches enqueued by this handle since creation (for launch accounting). */
unsigned long long svgf_launch_count(const svgf_handle* h);

#ifdef __cplusplus
}
#endif

#endif /* SVGF_H */
