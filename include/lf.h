/*
 * lf.h -- C ABI of the GB300-native semantic light-field EM.
 *
 * Method: Kaveti, Katt & Singh, "Removing Dynamic Objects for Static Scene
 * Reconstruction using Light Fields" (arXiv 2003.11076).  For every pixel of
 * the reference view of a rectified linear camera array the library
 *   1. rasterises the piecewise-planar disparity prior of the Delaunay
 *      triangulation of sparse support points (Sec. III-C "Disparity Prior"),
 *   2. runs the per-pixel hard EM (Sec. III-B schedule): an M-step that sweeps
 *      D disparity candidates and keeps the arg-max of the photometric-variance
 *      likelihood plus prior (Sec. III-C, M-step energy), and an E-step that
 *      enumerates all 2^K static/dynamic label vectors of the pixel's K rays
 *      (Sec. III-D "Segmentation update", Eq. e-step general),
 *   3. reports per-ray posteriors of the final labels and synthesises the
 *      refocused static image (Eq. 2, Sec. III-E "Refocused Image Synthesis").
 *
 * Conventions shared by every entry point:
 *   - No C++ exception crosses this ABI.  Every call returns an lf_status;
 *     lf_last_error() gives a one-line message for the calling thread.
 *   - Layouts are dense, row-major, C order.  "K" is the number of cameras,
 *     H x W the image size, C the number of image channels (1 or 3).
 *   - Geometry: camera k sits at signed position b_k on the line, relative to
 *     the reference camera (b_ref = 0).  A reference pixel (u, v) at disparity
 *     d sees camera k at column u - d * b_k of row v (Eq. 1 for a rectified
 *     linear array).  Out-of-image columns clamp to the border; fractional
 *     columns interpolate linearly (Sec. III-F: non-integral disparities).
 *   - Candidate disparities: d_j = d_min + j * (d_max - d_min) / (D - 1),
 *     j = 0..D-1 (D == 1: d_min).
 *   - Device pointers are read and written on the context's stream
 *     (lf_set_stream); the caller keeps them alive until that stream has
 *     passed the work.  Host pointers are copied within the call.
 *   - All compute runs in the library's sm_103a CUDA kernels; there is no CPU
 *     fallback.  Without a usable GPU every compute call returns LF_ECUDA.
 *   - Entry points that compute part of the method cite the paper passage
 *     they follow.  The others have no counterpart in the paper, which
 *     processes one frame at a time on one GPU: streams, synchronisation,
 *     page-locked buffers, tile and timing controls, statistics, errors, the
 *     uneven-batch API, the allocation-free entry and the failure hooks.
 */
#ifndef LF_H
#define LF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lf_ctx lf_ctx; /* opaque; created by lf_create, owned by the library */

typedef enum lf_status {
    LF_OK = 0,
    LF_EINVAL = 1,   /* an argument is out of range or inconsistent */
    LF_ENOMEM = 2,   /* a device or host allocation failed */
    LF_ECUDA = 3,    /* a CUDA call failed (message in lf_last_error) */
    LF_ESTATE = 4,   /* call order violated (e.g. run before inputs) */
    LF_ETIMEOUT = 5  /* a bounded device wait expired; results are invalid */
} lf_status;

typedef enum lf_dtype {
    LF_U8 = 0,       /* uint8, value / 255 is the intensity in [0, 1] */
    LF_F32 = 1,      /* float32 intensity in [0, 1] */
    LF_F16 = 2,      /* float16 intensity in [0, 1] */
    LF_BF16 = 3      /* bfloat16 intensity in [0, 1] */
} lf_dtype;

/* Storage precision of the staged descriptor maps the rays are sampled from
 * (luminance, Sobel responses, log segmentation priors) and of float32 input
 * images, which the reduced modes convert to 16 bits on the device.  Every
 * interpolation, likelihood, prior and posterior accumulation, the disparity
 * arg-max and the refocus normalisation stay in float32. */
typedef enum lf_precision {
    LF_PREC_F32 = 0, /* staged maps in float32 */
    LF_PREC_F16 = 1, /* staged maps and float32 images stored in float16 */
    LF_PREC_BF16 = 2 /* staged maps and float32 images stored in bfloat16 */
} lf_precision;

/*
 * How the hidden labels S are treated (Sec. III-B formulates EM over them;
 * Sec. III-C/III-D run it with hard assignments):
 *   LF_EM_HARD   the paper's EM: M-step at the labels of the last E-step,
 *                E-step = arg-max over the 2^K label vectors.
 *   LF_EM_SOFT   soft EM: the E-step keeps the posterior q(S) proportional to
 *                exp J(d_t, S) over all label vectors and every M-step after
 *                the first maximises sum_S q(S) J(d, S); the labels reported
 *                are the arg-max of J(d_T, S).  At most 8 cameras.
 *   LF_EM_JOINT  joint MAP: (d, S) = arg-max of J(d, S) over every candidate
 *                and label vector (lowest candidate, then smallest mask); the
 *                iteration count is not used.
 * The two variants stage float32 maps (precision must be LF_PREC_F32) and run
 * through lf_run_em only (not the batch API nor lf_run_em_static).
 */
typedef enum lf_em_mode {
    LF_EM_HARD = 0,
    LF_EM_SOFT = 1,
    LF_EM_JOINT = 2
} lf_em_mode;

/*
 * Model and run parameters.  The paper names beta, gamma, sigma and the
 * initial threshold (Sec. III-C energy, Sec. III-F) but prints a value only
 * for the threshold (0.7); the defaults of lf_default_params are
 * beta = 200, gamma = 0.1, sigma = 2, seg_threshold = 0.7, eps = 1e-4,
 * mstep_seg_term = 1, median = 0, precision = LF_PREC_F32, early_exit = 1,
 * dynamic_only = 0, em_mode = LF_EM_HARD, prune = 1.
 */
typedef struct lf_params {
    float beta;          /* weight of the static rays' descriptor variance */
    float gamma;         /* uniform floor of the disparity prior */
    float sigma;         /* width of the prior's sampled Gaussian (disparity units) */
    float seg_threshold; /* first M-step: a ray is dynamic iff P(dynamic) >= this */
    float eps;           /* floor inside log P and log(1 - P) */
    int mstep_seg_term;  /* 1: the M-step maximises the complete-data objective
                            (likelihood + disparity prior + segmentation prior);
                            0: likelihood + disparity prior only (Eq. mstep) */
    int median;          /* 1: 3x3 median on the refocused image (Sec. III-E) */
    int precision;       /* lf_precision */
    int early_exit;      /* 1: a pixel stops iterating once it reached an EM
                            fixed point (results are identical) */
    int dynamic_only;    /* 1: reconstruct only the reference pixels whose
                            P(dynamic) >= seg_threshold (Sec. III-F: the other
                            pixels already show the static background); see
                            lf_run_em for what the other pixels receive */
    int em_mode;         /* lf_em_mode: the paper's hard EM, or one of the two
                            variants of its formulation (see lf_em_mode) */
    int prune;           /* 1: each M-step of the hard EM (Sec. III-C arg-max
                            over the D candidates) evaluates only the
                            candidates whose upper bound -- disparity prior
                            plus the largest segmentation term, the variance
                            term being <= 0 -- reaches an objective already
                            computed; the arg-max, and so every output, is
                            identical to the full sweep's; from seven cameras
                            the E-step likewise skips blocks of label vectors
                            whose bound (the segmentation terms) is below the
                            all-static vector's objective.  0: full sweeps and
                            enumerations.  Hard EM on rectified arrays
                            (lf_create, the batch API, lf_run_em_static) and
                            on calibrated arrays; the soft-EM and joint-MAP
                            modes ignore it. */
} lf_params;

/* Statistics accumulated over the lf_run_em calls since the previous
 * lf_get_stats (which resets them). */
typedef struct lf_stats {
    uint64_t runs;                 /* lf_run_em calls covered */
    uint64_t nominal_ray_samples;  /* H * W * K * D * iters of the last run */
    uint64_t executed_ray_samples; /* sum over the runs: ray samples the M-steps
                                      evaluated, K per (pixel, candidate) objective
                                      (K x D per pixel-iteration without pruning) */
    int halo_left, halo_right;     /* staged column halo, pixels */
    int tile_rows, tile_cols;      /* sweep tile shape */
    int kernels_launched;          /* kernels one lf_run_em enqueues */
    float ms_prior, ms_sweep, ms_refocus, ms_median; /* mean device time per run
                                      of each kernel (lf_set_timing on), else 0 */
    int graph_captures;            /* batches: CUDA graphs captured so far */
    int tuned_signatures;          /* batches: tile shapes chosen by timing so far */
    float ms_support;              /* device time of the last support-point detection */
    float ms_set_inputs;           /* mean host time of lf_set_inputs (copies, detection,
                                      Delaunay, bins) over the calls covered */
    uint64_t executed_static_ray_samples; /* of executed_ray_samples, those whose ray was
                                      labelled static in its M-step (hard EM on a
                                      rectified array; 0 for the other modes) */
    uint64_t executed_pixel_iterations; /* sum over the runs: (pixel, EM iteration)
                                      pairs run, i.e. E-steps (after the exact
                                      early exit; hard EM on a rectified array,
                                      0 for the other modes) */
} lf_stats;

/* Fill *p with the documented defaults. */
void lf_default_params(lf_params *p);

/*
 * Create a context for one camera array and image size (Sec. III-A problem
 * setup).  baselines: [n_cams] host floats, exactly one of them 0 (the
 * reference camera; Sec. III-F takes the leftmost, any works).  p may be NULL
 * for the defaults; it is copied.  Allocates the context's device buffers on
 * the current CUDA device.
 * Errors: LF_EINVAL if n_cams < 1 or > 12, no baseline is 0, H or W < 3,
 * D < 1 or > 1024, d_max < d_min, a parameter is non-finite or out of its
 * range (sigma > 0 with 1 / (2 sigma^2) finite in float32, gamma >= 0,
 * eps > 0, beta >= 0, 0 < seg_threshold < 1, a known precision and em_mode,
 * float32 maps for the soft-EM and joint-MAP modes), or the disparity halo
 * does not fit the kernel's staging limit; LF_ENOMEM; LF_ECUDA.
 * On error *out is NULL.
 */
lf_status lf_create(lf_ctx **out, int n_cams, const float *baselines, int H, int W,
                    float d_min, float d_max, int D, const lf_params *p);

/*
 * Create a context for a calibrated, non-rectified camera array (Eq. 1:
 * x_k = pi_k [R_k | t_k] pi_ref^-1 (x_ref, d), written in generalized
 * disparity space so that the warping function of Sec. III-C is the
 * homography of the plane at disparity d).  cameras: [n_cams][3][4] host
 * floats, row-major; camera k sees reference pixel (u, v) at candidate
 * disparity d at (X / Z, Y / Z) with (X, Y, Z) = M_k (u, v, 1, d).  The
 * reference camera is the first whose matrix is exactly [I | 0]; the
 * rectified array is the special case M_k = [I | (-b_k, 0, 0)].  Rays are
 * sampled by bilinear interpolation with both coordinates clamped to the
 * image; everything else (inputs, outputs, lf_set_inputs, lf_run_em) is as
 * for lf_create.  The descriptor maps of all cameras are kept on the device
 * (20 bytes per camera pixel, allocated at the first lf_run_em).
 * Supports the hard EM on float32 maps only (em_mode = LF_EM_HARD,
 * precision = LF_PREC_F32), dynamic_only and median included.
 * Errors: as lf_create, and LF_EINVAL if cameras is NULL or non-finite, no
 * matrix is [I | 0], another em_mode or precision is asked for, some ray
 * of the frame at a candidate disparity projects behind its camera (Z <= 0
 * at a corner of [0, W-1] x [0, H-1] x [d_min, d_max]), or
 * n_cams * H * W + W + 1 exceeds 2^31 - 1 (the maps are indexed in 32 bits).
 */
lf_status lf_create_calibrated(lf_ctx **out, int n_cams, const float *cameras, int H, int W,
                               float d_min, float d_max, int D, const lf_params *p);

/* Use `stream` (a cudaStream_t; NULL = the legacy default stream) for every
 * later call on this context. */
lf_status lf_set_stream(lf_ctx *ctx, void *stream);

/*
 * Hand one frame to the context (Fig. 1 inputs: the K frames, the per-view
 * segmentation probabilities and the sparse support points).
 *   images       [K][H][W][C], dtype LF_U8, LF_F32, LF_F16 or LF_BF16, C = 1 (gray) or 3 (RGB;
 *                luminance Y = 0.299 R + 0.587 G + 0.114 B drives the
 *                likelihood, the refocus is per channel).
 *   seg_prior    [K][H][W] float32, P(pixel is dynamic) in [0, 1]
 *                (Sec. III-B; the Bodypix convention of Sec. III-F).
 *   sparse_points [M][3] float32 HOST memory, (u, v, d) in reference-view
 *                pixel units; triangulated on the host (Delaunay), repeated
 *                (u, v) keep their first occurrence; fewer than 3
 *                non-collinear points give a uniform prior everywhere.
 *                sparse_points = NULL with M = LF_DETECT_SUPPORT: the
 *                support points are detected on the device from these
 *                images and segmentation probabilities (Sec. III-C; see
 *                lf_support_params) and the call waits for them; they can
 *                be read back with lf_get_support_points.  Rectified arrays
 *                only.
 *   on_device    1: images and seg_prior are device pointers (borrowed until
 *                the stream passes the next lf_run_em); 0: host pointers
 *                (copied now, synchronously with respect to the caller);
 *                LF_HOST_ASYNC: host pointers copied to the device on the
 *                context's stream without waiting -- the caller keeps them
 *                unchanged until lf_synchronize (page-locked memory, e.g.
 *                from lf_host_alloc, makes the copy asynchronous; pageable
 *                memory works but the driver then stages it on the host).
 * Errors: LF_EINVAL (NULL pointer, C not 1 or 3, bad dtype, M < 0 other than
 * LF_DETECT_SUPPORT, non-finite point, detection on a calibrated array,
 * on_device not 0, 1 or LF_HOST_ASYNC), LF_ENOMEM, LF_ECUDA.
 */
lf_status lf_set_inputs(lf_ctx *ctx, const void *images, int C, int dtype,
                        const float *seg_prior, const float *sparse_points, int M,
                        int on_device);

#define LF_DETECT_SUPPORT (-1)

/* Transfer mode for lf_set_inputs (on_device) and lf_run_em
 * (outputs_on_device): host buffers moved by asynchronous copies on the
 * context's stream; completion through lf_synchronize. */
#define LF_HOST_ASYNC 2

/*
 * Support-point detection (Sec. III-C "Disparity Prior": points matched along
 * the epipolar lines over the full disparity range as in ELAS, points on
 * dynamic objects dropped, points of other views that re-project onto the
 * reference's occluded background added, duplicates and inconsistent points
 * removed).  The paper gives the steps, not their details; this library's
 * reading, all in integer or double arithmetic so that results are exact:
 *   - 8-bit luminance (uint8 RGB: (77 R + 150 G + 29 B + 128) >> 8; float
 *     inputs quantised per channel to rint(255 x) first), integer 3x3 Sobel
 *     responses, descriptor = both responses over the 3x3 window;
 *   - candidate pixels on a grid of step `grid` (offset grid / 2); a source
 *     camera is matched against target cameras at every candidate d_j, the
 *     target column being u + floor(-d_j (b_t - b_s) + 1/2); cost = summed
 *     L1 descriptor distance; candidates whose target leaves the image are
 *     skipped;
 *   - accepted iff the window texture (sum |Gx| + |Gy|) >= texture and
 *     100 * best < ratio_pct * (best cost at least one pixel of shift away
 *     on the widest pair);
 *   - reference points: the reference against all other cameras, the 3x3
 *     window static (P < seg_threshold); other views: each other camera
 *     against all cameras but itself and the reference, static in that view,
 *     kept where they re-project (u + d b_s, same row) onto a reference pixel
 *     with P >= seg_threshold;
 *   - one point per grid cell (the reference's own first, then other views
 *     in camera and raster order), then a point is kept iff at least
 *     min_support other points within `window` cells have |d - d'| <= delta;
 *   - each point is placed at its position plus a fixed offset of at most
 *     0.01 px that depends on its cell ((7 i + 13 j) mod 17 + 1) / 1800 in u,
 *     ((11 i + 5 j) mod 19 + 1) / 2000 in v), so that the grid's points are
 *     not cocircular and their Delaunay triangulation is unique.
 */
typedef struct lf_support_params {
    int grid;        /* grid step in pixels (default 5) */
    int ratio_pct;   /* uniqueness ratio, percent (85) */
    int texture;     /* minimum window texture (120) */
    int window;      /* consistency radius in cells (3) */
    float delta;     /* consistency tolerance, disparity units (3) */
    int min_support; /* agreeing neighbours needed (2) */
} lf_support_params;

/* Fill *p with the defaults listed above. */
void lf_default_support_params(lf_support_params *p);

/* Parameters of the next detections on this context (NULL = defaults).
 * Errors: LF_EINVAL on a NULL ctx or out-of-range values. */
lf_status lf_set_support_params(lf_ctx *ctx, const lf_support_params *p);

/* The points of the last detection: *n_points = their number; up to
 * max_points (u, v, d) triples are copied to the host array points (may be
 * NULL to query the count).  Points come in grid-cell raster order. */
lf_status lf_get_support_points(const lf_ctx *ctx, float *points, int max_points, int *n_points);

/*
 * Run the whole hot path on the last inputs: prior raster, `iters` EM
 * iterations (M-step first, Sec. III-B), posteriors, refocus (Eq. 2) and the
 * optional median.  Outputs (any may be NULL except disparity_idx):
 *   disparity_idx [H][W] int32   arg-max candidate index j of the last M-step
 *   disparity     [H][W] float32 d_j
 *   posteriors    [K][H][W] float32, marginal P(ray k static) under
 *                 q(S) proportional to exp J(d_T, S) over all 2^K label vectors
 *   labels        [H][W] uint16, bit k set = ray k static in the final E-step
 *   refocused     [H][W][C] float32 in [0, 1]; pixels with no static ray keep
 *                 the reference image
 * With dynamic_only, a reference pixel whose own P(dynamic) is below
 * seg_threshold is not reconstructed: disparity_idx = the candidate nearest
 * the prior centre mu (lower index on a tie; -1 outside the triangulation),
 * disparity = that d_j (NaN outside), labels = 0, posteriors = NaN, refocused
 * = the reference image; every other pixel gets exactly the full-mode result.
 * Tiles without such a pixel are filled by a classification kernel and never
 * staged.
 * The hard EM on a rectified array runs as one kernel: the sweep computes
 * the prior of its pixels while its staging copies are in flight and the
 * refocus from the raw rows it staged (lf_stats: ms_prior and ms_refocus ~ 0,
 * ms_sweep includes them); in dynamic_only mode the tile classifier
 * rasterises the prior and fills the static tiles before the sweep.  The
 * other modes run prior, sweep and refocus kernels in order.
 * outputs_on_device: 1 = device pointers (the call returns once the work is
 * enqueued; lf_synchronize waits and reports device errors); 0 = host pointers
 * (the call waits for the results); LF_HOST_ASYNC = host pointers written by
 * asynchronous copies on the context's stream (the call returns once the
 * work and the copies are enqueued; the results are there after
 * lf_synchronize).  With LF_HOST_ASYNC for inputs and outputs, two contexts
 * on two streams overlap one frame's copies with the other's kernels.
 * Errors: LF_ESTATE before lf_set_inputs, LF_EINVAL (iters < 1 or > 255, NULL
 * disparity_idx, outputs_on_device not 0, 1 or LF_HOST_ASYNC), LF_ETIMEOUT (a
 * bounded device wait expired), LF_ECUDA.
 */
lf_status lf_run_em(lf_ctx *ctx, int iters, int32_t *disparity_idx, float *disparity,
                    float *posteriors, uint16_t *labels, float *refocused,
                    int outputs_on_device);

/* Wait for the context's stream and report device-side errors of the last
 * run (LF_ETIMEOUT if a bounded wait expired). */
lf_status lf_synchronize(lf_ctx *ctx);

/* Fault injection for tests, on the host only: after `after` further
 * successful device allocations by the library (contexts and batches), the
 * next one reports LF_ENOMEM without being attempted, once; after < 0
 * switches the injection off.  Process-wide.  A call that fails this way
 * leaves its context usable: the next call allocates again. */
void lf_inject_alloc_failure(int after);

/* Page-locked host memory for the LF_HOST_ASYNC transfer mode, so that a C
 * caller needs no CUDA call of its own: *out receives `bytes` bytes (freed
 * with lf_host_free).  Errors: LF_EINVAL (NULL out, bytes == 0), LF_ENOMEM,
 * LF_ECUDA. */
lf_status lf_host_alloc(void **out, size_t bytes);
void lf_host_free(void *p);

/* Copy the rasterised prior of the last run (Sec. III-C "Disparity Prior"):
 * mu [H][W] float32, the interpolated disparity, NaN outside the
 * triangulation.  on_device as for lf_run_em outputs. */
lf_status lf_get_prior(lf_ctx *ctx, float *mu, int on_device);

/* Sweep tile shape: tile_rows x tile_cols reference pixels per CTA (one
 * thread each; tile_cols a multiple of 32, rows * cols <= 256 up to eight
 * cameras, <= 128 from nine, where the sweep kernel is compiled for three
 * 128-thread CTAs per SM).  0, 0 restores
 * the library's choice.  LF_EINVAL if the shape does not fit the staging
 * limits of the current inputs.  The batch autotuner uses this to time
 * candidate shapes. */
lf_status lf_set_tile(lf_ctx *ctx, int tile_rows, int tile_cols);

/* 1: record CUDA events on the context's stream around every kernel that
 * lf_run_em enqueues, so that lf_get_stats reports their mean device times
 * over the runs it covers; 0 (the default): no events. */
lf_status lf_set_timing(lf_ctx *ctx, int enable);

/* Statistics of the runs since the previous call (then reset); synchronises
 * the stream. */
lf_status lf_get_stats(lf_ctx *ctx, lf_stats *out);

/* One-line description of the calling thread's last error ("" if none).
 * ctx may be NULL.  The string stays valid until the thread's next call. */
const char *lf_last_error(const lf_ctx *ctx);

/* Free the context and its device buffers (waits for its stream). */
void lf_destroy(lf_ctx *ctx);

/*
 * Uneven batches (workload: many frames of different sizes, camera counts,
 * candidate and iteration counts in one go).  Same method (the per-pixel EM
 * of Sec. III-B to III-E) and results per frame as lf_run_em; the batch runs as one CUDA graph: a batched prior
 * raster, one persistent sweep launch per camera count present (its CTAs take
 * (frame, tile) items from a device-side queue, so small and large frames
 * share the GPU without tail effects) and a batched refocus / median.  The
 * graph reads its work lists from device memory and is captured again only
 * when the batch's shape changes (camera counts present, shared-memory size,
 * or a work list outgrowing its buffer); otherwise it is replayed.
 *
 * lf_batch_create: p as for lf_create (copied).  autotune = 1: before a
 *   frame whose signature (camera count, D, bytes per pixel, precision,
 *   halo width and width class) has not been seen in this process runs, its
 *   candidate 256-thread tile shapes are timed on that frame through the
 *   single-frame path and the fastest is kept for the signature (a one-off
 *   cost, synchronous); 0: the first shape that fits.
 * lf_batch_add: queue one frame.  images, seg_prior and every output are
 *   DEVICE pointers with the layouts of lf_set_inputs / lf_run_em, owned by
 *   the caller and kept alive until lf_batch_synchronize returns; outputs may
 *   be NULL except disparity_idx.  sparse_points is HOST memory (copied).
 *   iters is per frame.  *index (may be NULL) receives the frame's position.
 *   Rows need not be aligned: unaligned inputs are staged by the batch.
 * lf_batch_run: enqueue all queued frames on the batch's stream (async).
 * lf_batch_synchronize: wait; LF_ETIMEOUT if a bounded wait expired.
 * lf_batch_clear: forget the queued frames (device buffers are kept).
 * lf_batch_get_stats: runs since the last call, nominal and executed ray
 *   samples and kernel times (prior, all sweeps, refocus, median) of the last
 *   run, graph captures so far; synchronises.
 * Errors: LF_EINVAL (bad frame, halo too wide), LF_ESTATE (empty run),
 * LF_ENOMEM, LF_ECUDA, LF_ETIMEOUT.
 */
typedef struct lf_batch lf_batch;
lf_status lf_batch_create(lf_batch **out, const lf_params *p, int autotune);
lf_status lf_batch_set_stream(lf_batch *b, void *stream);
lf_status lf_batch_add(lf_batch *b, int n_cams, const float *baselines, int H, int W, float d_min,
                       float d_max, int D, int iters, const void *images, int C, int dtype,
                       const float *seg_prior, const float *sparse_points, int M,
                       int32_t *disparity_idx, float *disparity, float *posteriors, uint16_t *labels,
                       float *refocused, int *index);
lf_status lf_batch_run(lf_batch *b);
lf_status lf_batch_synchronize(lf_batch *b);
lf_status lf_batch_clear(lf_batch *b);
lf_status lf_batch_get_stats(lf_batch *b, lf_stats *out);
void lf_batch_destroy(lf_batch *b);

/*
 * Allocation-free EM sweep.  The paper has no counterpart of this entry
 * point; it exists for callers that cannot allocate device memory -- for
 * example a host framework whose own memory pool owns the GPU and forbids raw
 * cudaMalloc, or a latency-critical loop that must not trigger the
 * device-wide synchronisation a cudaMalloc or cudaFree can cause.
 *
 * It runs the same fused EM sweep kernel as lf_run_em (same results for the
 * same inputs), without the prior raster and the refocus.  Every input and
 * output is a caller-owned DEVICE pointer with the layouts of lf_set_inputs /
 * lf_run_em; mu is the caller's [H][W] float32 prior-centre map (NaN outside
 * the triangulation), e.g. the one lf_get_prior returns.  The kernel's other
 * scratch -- the per-(candidate, camera) sampling tables, the work counter and
 * the status word -- lives in one fixed 64 KiB device array inside the
 * library, which every GPU that loads the library keeps until the process
 * exits.  The call allocates nothing: no cudaMalloc, cudaFree or other
 * allocating routine.
 *   Limits: D <= 256 (the tables the array holds); images and seg_prior rows
 *   must start on 16-byte boundaries (W * bytes per pixel a multiple of 16),
 *   because they are read in place; hard EM on float32 maps, every pixel
 *   (em_mode = LF_EM_HARD, precision = LF_PREC_F32, dynamic_only = 0);
 *   p is checked as lf_create checks it.  Otherwise LF_EINVAL.
 *   Every call looks up the array's device address for the current device
 *   (nothing is cached between calls).
 *   The call is synchronous: it waits for `stream` (a cudaStream_t, NULL =
 *   legacy default stream) before returning, so it cannot be recorded into a
 *   CUDA graph (a call on a stream being captured fails with LF_ECUDA).
 *   All calls share the one array and leave their contents in it (each call
 *   clears the counter and status it needs); calls whose GPU work overlaps
 *   would race on it, so the call serialises its callers.
 * Errors as lf_run_em (message in lf_last_error).
 */
lf_status lf_run_em_static(int n_cams, const float *baselines, int H, int W, float d_min, float d_max,
                           int D, const lf_params *p, int iters, const void *images, int C, int dtype,
                           const float *seg_prior, const float *mu, int32_t *disparity_idx,
                           float *disparity, float *posteriors, uint16_t *labels, void *stream);

/*
 * Self-test of the bounded device waits (no fault is involved).  Every wait
 * of the sweep kernels on their TMA copies gives up after a time limit and
 * reports it through the context's status word, which lf_run_em turns into
 * LF_ETIMEOUT.  This call launches one CTA on the current device that arms
 * an mbarrier for bytes no copy will deliver and waits on it with the same
 * bounded wait for timeout_ns nanoseconds (0 < timeout_ns <= 1e10).
 * Returns LF_ETIMEOUT when the wait expired and was reported (the expected
 * outcome), LF_OK if it completed, LF_EINVAL / LF_ECUDA otherwise.  Nothing
 * stays in flight and the device stays usable.
 */
lf_status lf_selftest_bounded_wait(unsigned long long timeout_ns);

/*
 * Host utility (no GPU needed): Delaunay triangulation of the (u, v) of
 * `points` ([M][3] float32, (u, v, d)) as used for the prior (Sec. III-C,
 * triangulation of the support points, as in ELAS).  Writes up to max_tris
 * counter-clockwise index triples into tris ([max_tris][3] int32, indices into
 * `points`) and returns the number of triangles, or -1 on invalid arguments.
 */
int lf_triangulate(const float *points, int M, int32_t *tris, int max_tris);

#ifdef __cplusplus
}
#endif

#endif /* LF_H */
