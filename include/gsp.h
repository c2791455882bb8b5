/*
 * gsp.h - C ABI of the GB300 edge-guided densification library (libgsp.so).
 *
 * The library implements the data-parallel hot path of ImprovedGS+
 * (arXiv 2603.08661): the edge-importance map of Sec. 2.1, the tile-binned
 * Gaussian splatting pass that accumulates each Gaussian's edge score
 * (Sec. 1, "Edge-Score importance"), its adjoint, and the Long-Axis-Split of
 * Sec. 2.2 (Alg. 1 and Alg. 2); around it, the refinement set-up of Sec. 2.3
 * (gradient-threshold masking after a warm-up, importance sampling by edge
 * score, the learning-rate schedule and a Gaussian budget).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - Every pointer named as device memory must be a CUDA device (or managed)
 *   allocation on the current device.  The caller owns every buffer; the
 *   library never allocates device memory.  Scratch space comes from a
 *   caller-provided workspace whose size the matching *_workspace_size query
 *   returns (alignment: 256 bytes).
 * - Every call is asynchronous on the caller's stream and performs no host
 *   synchronisation.  Argument errors are detected on the host before any
 *   launch and returned synchronously; nothing is enqueued then.
 * - Errors that only the device can see (capacity exceeded, a bounded wait
 *   that ran out: grid barrier, sort look-back, bulk copy) are written as a
 *   gsp_status code to *dev_status (a
 *   device int32 the caller zeroes and reads after its own synchronisation);
 *   the first error wins.  dev_status may not be NULL.
 * - No C++ exception crosses this interface.  All floating point arithmetic
 *   on the device is FP32.
 */
#ifndef GSP_H
#define GSP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st *gsp_stream_t; /* a cudaStream_t; NULL = legacy default stream */

typedef enum gsp_status {
    GSP_OK = 0,
    GSP_ERR_INVALID_ARG = 1, /* a host-checked argument is invalid (nothing was launched) */
    GSP_ERR_CUDA = 2,        /* a CUDA runtime call failed (see gsp_last_cuda_error) */
    GSP_ERR_CAPACITY = 3,    /* device: pair list or Gaussian capacity exceeded; outputs untouched */
    GSP_ERR_TIMEOUT = 4,     /* device: a bounded grid-barrier wait ran out */
    GSP_ERR_WORKSPACE = 5,   /* workspace pointer NULL, misaligned or smaller than required */
    GSP_ERR_UNSUPPORTED = 6  /* valid request the build does not support (e.g. too many views) */
} gsp_status;

#define GSP_MAX_VIEWS 64
#define GSP_TILE 16 /* splatting tiles are GSP_TILE x GSP_TILE pixels */

/* Message for a status code (static string). */
const char *gsp_status_string(int32_t status);
/* Last CUDA error code seen by the library on this host thread (0 if none). */
int32_t gsp_last_cuda_error(void);
/* Library version, major * 10000 + minor * 100 + patch. */
int32_t gsp_version(void);

/* Instrumentation (host side, not thread-safe; no counterpart in the paper).
 * gsp_kernel_launch_count: kernels and memsets the library has enqueued in
 * this process since it was loaded (launches captured into a CUDA graph count
 * once, at capture).
 * gsp_stage_timer_arm: from now on, every occurrence of the named stage
 * ("edge_fused", "edge_plain", "project", "depth_sort", "bin", "composite_fwd",
 * "composite_bwd", "project_bwd", "topk", "las", "sgd"; NULL disarms) is bracketed by
 * a pair of CUDA events recorded on the caller's stream, up to max_records
 * occurrences; re-arming discards earlier records.
 * gsp_stage_timer_read: waits for the recorded events and returns the summed
 * milliseconds and the number of occurrences. */
int64_t gsp_kernel_launch_count(void);
gsp_status gsp_stage_timer_arm(const char *stage, int32_t max_records);
gsp_status gsp_stage_timer_read(float *total_ms, int32_t *occurrences);

/* ======================================================================
 * Edge-importance map (Sec. 2.1).
 *
 * Per view: grayscale (luma 0.299 / 0.587 / 0.114 of the uint8 channels,
 * divided by 255), 5x5 Gaussian blur, Sobel gradient, non-maximum
 * suppression along the gradient direction quantised to 8 directions
 * (kept iff M > 0, M >= M(uphill neighbour), M > M(downhill neighbour);
 * neighbours outside the image count as 0), then division by the lower
 * median of the kept magnitudes (Sec. 2.1, closing paragraph).  The image is
 * extended beyond its border by clamp-to-edge before blurring.  A view with
 * no kept pixel gets E = 0 and median 0.
 * ==================================================================== */

typedef struct gsp_image_desc {
    const uint8_t *rgb;    /* device, HWC uint8, `height` rows of `pitch_bytes` */
    int32_t width;         /* >= 1 */
    int32_t height;        /* >= 1 */
    int64_t pitch_bytes;   /* >= 3 * width */
    int64_t out_offset;    /* first element of this view in E_out / nms_mask_out */
} gsp_image_desc;

enum { GSP_EDGE_FUSED = 0, GSP_EDGE_PLAIN = 1 };

typedef struct gsp_edge_opts {
    int32_t mode;            /* GSP_EDGE_FUSED: all stages and views in one persistent
                                launch; GSP_EDGE_PLAIN: one launch per stage and view */
    int32_t use_custom_taps; /* 0: taps from sigma; 1: taps[] as given */
    float taps[5];           /* 1-D blur taps, symmetric (taps[k] == taps[4-k]) */
    float sigma;             /* blur sigma when use_custom_taps == 0 (> 0) */
    int64_t spin_limit;      /* grid-barrier polls before GSP_ERR_TIMEOUT; <= 0: default */
    int32_t test_expire;     /* failure-injection hook for tests (0 in normal use), fused mode:
                                bit 0: the first grid barrier is never opened, so every
                                block's bounded wait runs out; bit 1 (batches under 4 Mi
                                pixels, which stage their halo boxes by TMA): each wait for
                                a staged box gives up at once (the block still lets its
                                copies in flight land before it leaves).  Either way the
                                call reports GSP_ERR_TIMEOUT in dev_status and E_out /
                                median_out are unspecified; the next call works normally. */
    int32_t blocks_per_sm;   /* fused mode: at most this many blocks of the launch per SM
                                (<= 0: as many as fit).  A caller that runs the edge map
                                on a second stream beside other kernels leaves them room
                                with 1; the result does not depend on it. */
} gsp_edge_opts;

/* Default options: fused mode, sigma = 1. */
void gsp_edge_opts_default(gsp_edge_opts *opts);

/* Workspace bytes gsp_edge_map needs for these views (host array of num_views). */
size_t gsp_edge_map_workspace_size(const gsp_image_desc *imgs, int32_t num_views,
                                   const gsp_edge_opts *opts);

/*
 * imgs          host array of num_views descriptors (1 <= num_views <= GSP_MAX_VIEWS)
 * E_out         device float; view v occupies [out_offset, out_offset + width*height),
 *               row-major; receives E = M_thinned / median
 * median_out    device float[num_views]: the median, in units of the luma in [0, 1]
 * nms_mask_out  device uint8 laid out like E_out (1 = kept), or NULL
 * opts          NULL for the defaults
 * Views must not overlap in E_out.  Device errors: GSP_ERR_TIMEOUT (fused mode).
 */
gsp_status gsp_edge_map(const gsp_image_desc *imgs, int32_t num_views, float *E_out,
                        float *median_out, uint8_t *nms_mask_out, const gsp_edge_opts *opts,
                        void *workspace, size_t workspace_bytes, int32_t *dev_status,
                        gsp_stream_t stream);

/* ======================================================================
 * Tile-binned splatting with edge score (Sec. 1 "Edge-Score importance";
 * the 3DGS renderer the paper builds on is not described in the paper, so
 * its conventions are fixed here).
 *
 *   Sigma  = R S S^T R^T  (R of the normalised quaternion, S = diag(exp(log_scales)))
 *   t      = W mu + t_c; culled when t_z <= 0.2
 *   Sigma2 = J W Sigma W^T J^T + 0.3 I,  J the pinhole Jacobian at t
 *   colour = max(0, sum_k sh[k] Y_k(normalise(mu - camera centre)) + 0.5), real SH, k = l^2+l+m
 *   alpha  = min(0.99, sigmoid(o) exp(-1/2 d^T Sigma2^-1 d)), d = pixel centre - projected mean;
 *            skipped when alpha < 1/255; compositing stops before the Gaussian that
 *            would take T (1 - alpha) below 1e-4
 *   order  ascending camera depth t_z (compared as FP32), ties by ascending index
 *   C      = sum_i c_i alpha_i T_i (black background)
 *   score  s_i += sum over pixels of alpha_i T_i E(pixel)
 *   loss   L1: mean over all pixels of all views and 3 channels of |C - target/255|
 *          (over gsp_render_opts.loss_pixels pixels when the caller sets it)
 * ==================================================================== */

typedef struct gsp_gaussians {
    float *means;          /* device [capacity][3] */
    float *log_scales;     /* device [capacity][3] (storage space: log of the scale) */
    float *quats;          /* device [capacity][4] (w, x, y, z), any non-zero norm */
    float *opacity_logits; /* device [capacity]   (storage space: logit of the opacity) */
    float *sh;             /* device [capacity][K][3], K = (sh_degree + 1)^2 */
    int32_t *count;        /* device int32: number N of live Gaussians (0 <= N <= capacity) */
    int64_t capacity;      /* 1 <= capacity < 2^30 */
    int32_t sh_degree;     /* 0..3 */
} gsp_gaussians;

typedef struct gsp_camera {
    float viewmat[12];     /* world -> camera, 3x4 row-major [W | t_c]; image y points down */
    float fx, fy, cx, cy;  /* pinhole intrinsics; pixel (u, v) is sampled at (u+0.5, v+0.5) */
    int32_t width, height; /* >= 1 */
    int64_t pixel_offset;  /* first pixel of this view in the per-pixel buffers */
} gsp_camera;

typedef struct gsp_render_opts {
    int64_t pair_capacity; /* maximum tile-Gaussian pairs summed over views (>= 1, < 2^32); the
                              supertile entries of the binning (one per Gaussian, view and 8x8-tile
                              block its tile rectangle touches) share the same bound */
    int32_t fwd_variant;   /* forward compositing variant, 0 .. GSP_FWD_VARIANTS - 1 (0: default) */
    int32_t bwd_variant;   /* adjoint compositing variant, 0 .. GSP_BWD_VARIANTS - 1 (0: default) */
    /* Positional statistic of the gradient-threshold masking (Sec. 2.3, "Global Warm-up
     * Phase"), read by gsp_render_bwd only; both NULL or both device [capacity] arrays.
     * For every view in which Gaussian i's screen-space mean gradient g = dL/d(mean2D) is
     * nonzero: pos_grad_sum[i] += |g| (Euclidean norm, pixel units), pos_grad_count[i] += 1.
     * Accumulated over calls; the caller clears them (e.g. after each densification). */
    float *pos_grad_sum;
    int32_t *pos_grad_count;
    int64_t loss_pixels;   /* pixels the L1 loss averages over, for the loss of gsp_render_fwd and
                              the L1 upstream gradient of gsp_render_bwd; <= 0: the pixels of
                              this call's views.  A caller that shards the views of one loss
                              over several GPUs passes the pixel count of all of them, so that
                              the per-GPU results sum to the whole loss and its gradient. */
    int64_t spin_limit;    /* depth-sort look-back polls before GSP_ERR_TIMEOUT; <= 0: default */
    int32_t test_expire;   /* failure-injection hook for tests (0 in normal use), gsp_render_fwd:
                              bit 0: the first depth-sort tile never publishes its digit counts,
                              so every later tile's bounded look-back runs out (the forward
                              then skips its remaining stages and writes no output); bit 1:
                              the projection's wait for its bulk SH copy gives up at once (each
                              thread then reads its SH row from global memory, so the outputs
                              are complete and correct).  Either way dev_status receives
                              GSP_ERR_TIMEOUT. */
    void *score_event;     /* a cudaEvent_t, or NULL; read by gsp_render_bwd only, which records
                              it on its stream once the adjoint compositing has finished: the
                              edge score (and every screen-space gradient) is then complete,
                              while the chain to the parameters still runs.  A caller can start
                              the selection on another stream from it. */
    int64_t list_prefix;   /* read by gsp_render_fwd: entries of each tile's list (in depth order)
                              written before the compositing, <= 0: 2048.  A tile whose pixels
                              have not all stopped within them (T would drop below 1e-4) gets
                              the rest of its list afterwards and its compositing resumes from
                              where the prefix ended, so the results do not depend on this
                              value, only the speed does. */
} gsp_render_opts;

/* Compositing variants (pixels per thread, Gaussians staged per shared-memory batch,
 * warp-level culling of staged Gaussians by footprint box: c = on, n = off).
 * The results do not depend on the variant, only the speed does; an autotuner picks
 * one per workload.  Forward: (1, 256, c), (2, 256, c), (1, 128, c), (2, 128, c),
 * (1, 128, n), (2, 128, n).  Adjoint: (2, 256, c), (1, 256, c), (4, 256, c),
 * (2, 128, c), (2, 128, n), (4, 128, c). */
#define GSP_FWD_VARIANTS 6
#define GSP_BWD_VARIANTS 6

/* Workspace bytes for a fwd/bwd pair over these cameras (host array). */
size_t gsp_render_workspace_size(int64_t capacity, int32_t sh_degree, const gsp_camera *cams,
                                 int32_t num_views, const gsp_render_opts *opts);

/*
 * Forward pass over num_views views (host array cams, 1 <= num_views <= GSP_MAX_VIEWS).
 *
 * targets    host array of num_views image descriptors of the ground-truth views
 *            (out_offset ignored), or NULL: then no loss is computed
 * edge       device float per pixel (layout of rgb_out / 3), or NULL
 * rgb_out    device float [total_pixels][3], written
 * T_final    device float [total_pixels], written
 * last_idx   device int32 [total_pixels]: 1 + position in the tile's list of the last
 *            composited Gaussian (0 = none), written; consumed by gsp_render_bwd
 * score      device float [capacity], accumulated (+=) when edge != NULL, or NULL
 * loss_out   device float [1], written when targets != NULL, or NULL
 * workspace  holds the projected Gaussians and sorted tile lists; it must stay
 *            untouched until the matching gsp_render_bwd has been enqueued
 * Device errors: GSP_ERR_CAPACITY when the pairs exceed opts->pair_capacity
 * (then rgb_out / T_final / last_idx / score / loss are not written).
 */
gsp_status gsp_render_fwd(const gsp_gaussians *g, const gsp_camera *cams, int32_t num_views,
                          const gsp_image_desc *targets, const float *edge, float *rgb_out,
                          float *T_final, int32_t *last_idx, float *score, float *loss_out,
                          const gsp_render_opts *opts, void *workspace, size_t workspace_bytes,
                          int32_t *dev_status, gsp_stream_t stream);

/* Statistics of the last gsp_render_fwd on this workspace (device int64[3] inside
 * the workspace; valid after that call completes; no counterpart in the paper):
 * [0] tile-Gaussian pairs (exact, also when they exceeded pair_capacity),
 * [1] composited (pixel, Gaussian) pairs, i.e. the terms of the sums for C,
 * [2] tiles whose compositing went on past the written prefix of their list
 *     (gsp_render_opts.list_prefix) once the rest of the list was written. */
const int64_t *gsp_render_pair_count_ptr(const void *workspace, int64_t capacity,
                                         int32_t sh_degree, const gsp_camera *cams,
                                         int32_t num_views, const gsp_render_opts *opts);

/*
 * Adjoint of gsp_render_fwd, replayed back to front from T_final and last_idx.
 *
 * The upstream gradient is dL_drgb (device float [total_pixels][3]) when it is
 * not NULL; otherwise that of the L1 loss, sign(C - target/255) / (3 * P), P = opts->loss_pixels
 * when it is > 0, else the total pixels of these views,
 * with sign(0) = 0, from rgb and targets (both then required).
 * grad_*     device buffers shaped like the parameters; accumulate != 0 adds to
 *            them, accumulate == 0 overwrites rows [0, N)
 * score      device float [capacity] += edge score, or NULL (needs edge != NULL);
 *            lets a caller fuse the score into the backward pass instead of the forward
 * workspace  the workspace of the matching gsp_render_fwd (same sizes); the adjoint may be
 *            called any number of times after one forward pass (each call starts its
 *            screen-space sums from zero)
 */
gsp_status gsp_render_bwd(const gsp_gaussians *g, const gsp_camera *cams, int32_t num_views,
                          const gsp_image_desc *targets, const float *dL_drgb, const float *rgb,
                          const float *T_final, const int32_t *last_idx, const float *edge,
                          float *score, float *grad_means, float *grad_log_scales,
                          float *grad_quats, float *grad_opacity_logits, float *grad_sh,
                          int32_t accumulate, const gsp_render_opts *opts, void *workspace,
                          size_t workspace_bytes, int32_t *dev_status, gsp_stream_t stream);

/* ======================================================================
 * Selection and Long-Axis-Split (Sec. 2.2, Alg. 1 and Alg. 2).
 * ==================================================================== */

typedef struct gsp_las_params {
    float k_off;        /* offset = k_off * exp(log_scale[l]) along column l of R (Alg. 1: alpha) */
    float long_factor;  /* long axis physical scale factor (Alg. 1: alpha = 0.5) */
    float other_factor; /* other axes' factor (Alg. 1: gamma = 0.85) */
    float beta;         /* physical opacity factor (Alg. 1: beta = 0.6) */
} gsp_las_params;

/* The paper's preset (Sec. 2.2): k_off 0.5, long 0.5, other 0.85, beta 0.6. */
void gsp_las_params_paper(gsp_las_params *p);

size_t gsp_las_workspace_size(int64_t capacity);

/*
 * Top-k selection by score: mask_out[i] = 1 for the k largest scores[i],
 * i < N (device count), ties at the k-th value taken in ascending index order;
 * 0 for every other i < capacity.  k is clamped to [0, N].
 * selected_out (device int32, or NULL) receives the number selected.
 */
gsp_status gsp_topk_mask(const float *scores, const int32_t *count, int64_t capacity, int64_t k,
                         uint8_t *mask_out, int32_t *selected_out, void *workspace,
                         size_t workspace_bytes, int32_t *dev_status, gsp_stream_t stream);

/*
 * Top-k with gradient-threshold masking (Sec. 2.3, "Global Warm-up Phase": after the
 * warm-up events the split candidates must pass the gradient threshold; the paper
 * names neither the statistic nor the threshold).  Gaussian i < N is a candidate when
 * pos_grad_count[i] > 0 and pos_grad_sum[i] / pos_grad_count[i] >= threshold, the
 * quotient and comparison in FP32 (the statistic gsp_render_bwd accumulates through
 * gsp_render_opts).  mask_out selects the min(k, candidates) largest scores among the
 * candidates, ties in ascending index order; selected_out receives that number.
 * pos_grad_sum / pos_grad_count: device float / int32 [capacity].  threshold: not NaN
 * (+inf selects nothing).  Workspace: gsp_las_workspace_size(capacity) bytes, as for
 * gsp_topk_mask.  Errors: GSP_ERR_INVALID_ARG, GSP_ERR_WORKSPACE; device: GSP_ERR_TIMEOUT.
 */
gsp_status gsp_topk_mask_gated(const float *scores, const float *pos_grad_sum, const int32_t *pos_grad_count,
                               float threshold, const int32_t *count, int64_t capacity, int64_t k,
                               uint8_t *mask_out, int32_t *selected_out, void *workspace,
                               size_t workspace_bytes, int32_t *dev_status, gsp_stream_t stream);

/*
 * Importance sampling by edge score (Sec. 1, "Edge-Score importance sampling"): k
 * Gaussians drawn without replacement with probabilities proportional to scores[i],
 * by exponential clocks.  Gaussian i < N with scores[i] > 0 rings at
 * exp_variates[i] / scores[i] (one FP32 division); mask_out selects the min(k, number
 * of positive scores) earliest, ties in ascending index order.  exp_variates: device
 * float [capacity] of independent Exp(1) draws supplied by the caller (fresh ones for
 * each draw).  Workspace and errors as for gsp_topk_mask.
 */
gsp_status gsp_sample_mask(const float *scores, const float *exp_variates, const int32_t *count,
                           int64_t capacity, int64_t k, uint8_t *mask_out, int32_t *selected_out,
                           void *workspace, size_t workspace_bytes, int32_t *dev_status, gsp_stream_t stream);

/*
 * One selection entry for the densification schedule: top-k (exp_variates NULL) or
 * importance sampling (exp_variates given), optionally gated by the gradient threshold
 * (top-k only), and capped by a Gaussian budget (Conclusion: the 1M-budget variant, and
 * a 3M pre-allocated capacity):
 * with budget > 0 at most max(budget - N, 0) Gaussians are selected, so that the
 * split keeps N <= budget.  The selections are those of gsp_topk_mask,
 * gsp_topk_mask_gated and gsp_sample_mask with k reduced accordingly.
 */
typedef struct gsp_select_opts {
    const float *pos_grad_sum;     /* gating: device float [capacity], or NULL */
    const int32_t *pos_grad_count; /* gating: device int32 [capacity], or NULL (with pos_grad_sum) */
    float threshold;               /* gating threshold (not NaN) */
    const float *exp_variates;     /* sampling: device Exp(1) draws [capacity], or NULL for top-k */
    int64_t budget;                /* 0: none */
    int64_t spin_limit;            /* unused: the selection's launches wait on nothing (no grid
                                      barrier, no flag); kept so that the layout does not change */
    int32_t test_expire;           /* unused, as spin_limit */
} gsp_select_opts;

gsp_status gsp_select_mask(const float *scores, const int32_t *count, int64_t capacity, int64_t k,
                           const gsp_select_opts *opts, uint8_t *mask_out, int32_t *selected_out,
                           void *workspace, size_t workspace_bytes, int32_t *dev_status, gsp_stream_t stream);

/*
 * Allocation-free variant of gsp_topk_mask (the paper has no counterpart).
 *
 * For callers that cannot allocate device memory when they call: real-time
 * loops that forbid allocation once they run, and host applications whose
 * device memory is owned by their own allocator, where a plug-in may not take
 * memory behind the host's back.  Same arguments and result as
 * gsp_topk_mask, but no workspace: the scratch (about 89 KB) is a static
 * device array inside the library that every GPU which loads the library
 * holds until the process exits.  The caller still passes scores, count,
 * mask_out and selected_out.
 * - capacity must be <= GSP_TOPK_STATIC_MAX_CAPACITY, else GSP_ERR_INVALID_ARG
 *   is returned and nothing is enqueued.
 * - The first call on a device (that device current) looks up the array's
 *   device address on it with cudaGetSymbolAddress, a host-side runtime call;
 *   later calls on that device reuse the address.
 * - All calls share the one array and the kernels re-initialise what must
 *   start at zero; calls that overlap on the GPU (other streams, other host
 *   threads) race on it and must be serialised by the caller.
 * - No device memory is allocated or freed by this call.
 */
#define GSP_TOPK_STATIC_MAX_CAPACITY (1 << 24)
gsp_status gsp_topk_mask_static(const float *scores, const int32_t *count, int64_t capacity, int64_t k,
                                uint8_t *mask_out, int32_t *selected_out, int32_t *dev_status,
                                gsp_stream_t stream);

/*
 * Long-Axis-Split in place (Alg. 1, with Alg. 2's column read of R).
 *
 * mask       device uint8 [capacity]: split Gaussian i < N iff mask[i] != 0; or NULL,
 *            then the top-k by scores (gsp_topk_mask semantics) is split
 * scores     device float [capacity] (used only when mask == NULL)
 * For each selected Gaussian i with rank r among the selected (ascending index):
 * child 0 overwrites slot i at mu + d, child 1 is written to slot N + r at mu - d,
 * d = R[:, l] k_off exp(log_scale[l]), l = argmax log_scale (lowest index on ties);
 * both get log_scale[l] + log(long_factor), the others + log(other_factor),
 * opacity logit(beta * sigmoid(o)); quaternion and SH are copied.  *count
 * becomes N + (number selected).  When N + selected > capacity the device writes
 * GSP_ERR_CAPACITY and changes nothing.
 */
gsp_status gsp_las_split(const gsp_gaussians *g, const uint8_t *mask, const float *scores,
                         int64_t k, const gsp_las_params *p, void *workspace,
                         size_t workspace_bytes, int32_t *dev_status, gsp_stream_t stream);

/* ======================================================================
 * Optimiser step of the densification loop (the paper does not state its
 * optimiser; the workloads use plain SGD).
 * ==================================================================== */

/*
 * theta <- theta - lr * grad on rows [0, N) (device count) of every parameter
 * group, computed as one FMA per element (fma(-lr, grad, theta)); rows >= N
 * are not touched.  grad_* are device buffers shaped like the parameters.
 * One launch, asynchronous on the caller's stream.
 */
gsp_status gsp_sgd_step(const gsp_gaussians *g, float *grad_means, float *grad_log_scales,
                        float *grad_quats, float *grad_opacity_logits, float *grad_sh, float lr,
                        gsp_stream_t stream);

/*
 * Learning-rate schedule of the refinement (Sec. 2.3): per parameter group
 * (0 means, 1 log_scales, 2 quats, 3 opacity_logits, 4 sh) an exponential decay
 * lr(t) = lr_init * (lr_final / lr_init)^(min(t, steps) / steps); a group with
 * lr_init == lr_final keeps that rate.  The paper's values: log_scales 0.020 -> 0.002
 * ("Exponential Scale Scheduling", gamma = 0.1), means 1.28e-4 -> 1.28e-5
 * ("Positional Learning Rate Optimization"); the horizon `steps` is not stated.
 */
typedef struct gsp_lr_schedule {
    float lr_init[5];
    float lr_final[5];
    int32_t steps; /* >= 1 */
} gsp_lr_schedule;

/*
 * gsp_sgd_step with each group's rate taken from sched at t = *step (device int32),
 * computed on the device (FP32 expf / logf), then *step += 1: the same enqueued
 * step (e.g. a CUDA-graph replay) follows the schedule.  Both rates of a decaying
 * group must be > 0.  Two launches.
 */
gsp_status gsp_sgd_step_scheduled(const gsp_gaussians *g, float *grad_means, float *grad_log_scales,
                                  float *grad_quats, float *grad_opacity_logits, float *grad_sh,
                                  const gsp_lr_schedule *sched, int32_t *step, gsp_stream_t stream);

#ifdef __cplusplus
}
#endif

#endif /* GSP_H */
