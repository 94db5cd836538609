/*
 * liblp -- LP-SIFT hot path on one NVIDIA GB300 (sm_103a).
 *
 * Li, Wang, Zhao & Zhao, "Local-peak scale-invariant feature transform for
 * fast and random image stitching": multiscale local-peak detection (Sec. 2.1-
 * 2.2, Eq. 1-2), SIFT-style orientation and 128-d description (Sec. 2.3,
 * Eq. 3-5), nearest-neighbour matching with Eq. 6 distances (Sec. 2.4) and
 * RANSAC estimation of the homography of Eq. 7 or the rigid transform of
 * Eq. 8 (Sec. 2.5), plus the all-pairs homography matrix H_M and the mosaic of
 * Sec. 4.  Paper-literal variants (finite alpha in Eq. 1, border rejection,
 * Delta_s-only matching) are configuration options.  A learned RANSAC
 * proposal, not in the paper, is an addition.
 *
 * Conventions shared by every entry point
 *  - Pointers named d_* or documented as "device" are device pointers that the
 *    caller allocates and owns; the library never frees them.  Host pointers
 *    are documented as such.
 *  - Calls are asynchronous on `stream` (a cudaStream_t passed as void*;
 *    NULL = the legacy default stream) unless documented otherwise.
 *  - Every call returns an lp_status.  Argument errors that the host can see
 *    are returned synchronously and launch nothing.  Errors found on the device
 *    are recorded in a per-context status word; lp_sync_status() waits for the
 *    context's last stream and returns it.
 *  - Images are uint8, row-major, `pitch` bytes per row, pitch % 16 == 0 and a
 *    16-byte aligned base.  channels = 1 (intensity) or 3 (interleaved RGB).
 *    Coordinates are 0-based; x = column, y = row; a feature point is the
 *    raster index idx = y*W + x (H*W < 2^24 is required).
 *  - A context is not thread-safe; use one context per host thread / stream.
 */
#ifndef LP_H
#define LP_H
#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define LP_API __attribute__((visibility("default")))
#else
#define LP_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum lp_status {
    LP_OK = 0,
    LP_ERR_ARG = 1,          /* invalid argument (null, size, range) */
    LP_ERR_ALIGN = 2,        /* pointer or pitch not 16-byte aligned */
    LP_ERR_CUDA = 3,         /* a CUDA runtime call failed */
    LP_ERR_TIMEOUT = 4,      /* a bounded device-side wait gave up */
    LP_ERR_NOMEM = 5,        /* workspace allocation failed */
    LP_ERR_DEGENERATE = 6,   /* no model could be fitted (reported, not fatal) */
    LP_ERR_UNSUPPORTED = 7,  /* configuration outside what the library supports */
    LP_ERR_DEVICE = 8        /* a kernel recorded an internal inconsistency */
} lp_status;

typedef enum lp_precision {
    LP_PREC_FP32 = 0,        /* FP32 SIMT distances, exact top-2 */
    LP_PREC_BF16 = 1,        /* BF16 tcgen05 distances, top-k, FP32 re-rank */
    LP_PREC_FP8 = 2          /* E4M3 tcgen05 distances (descriptors x 2^8 rounded to E4M3 in the
                                matcher's workspace), the same certified candidate filter with the
                                E4M3 error bound, FP32 re-rank: results equal LP_PREC_FP32's */
} lp_precision;

/* Transform models of Sec. 2.5.  Eq. 7 maps points through a 3x3 homography
 * H; Eq. 8 prints H in rigid form (rotation theta and translation t_x, t_y).
 * LP_MODEL_HOMOGRAPHY estimates all eight degrees of freedom from samples of
 * four matches; LP_MODEL_RIGID estimates Eq. 8's three from samples of two
 * (the least-squares rotation and translation of the two) and refits them by
 * least squares.  Both report H as a row-major double[9] with h33 = 1. */
typedef enum lp_model {
    LP_MODEL_HOMOGRAPHY = 0,
    LP_MODEL_RIGID = 1
} lp_model;

#define LP_MAX_SCALES 8

/* Parameters of the method.  lp_config_default() fills the values used by the
 * 640x480 and 2688x1600 workloads. */
typedef struct lp_config {
    int32_t  nL;                  /* number of window sizes, 1..LP_MAX_SCALES */
    int32_t  Ls[LP_MAX_SCALES];   /* interrogation window sizes L (Eq. 2), >= 2 */
    double   beta0;               /* Eq. 3 beta0; <= 0 selects (1/d) sqrt(Lmin/Lmax) */
    float    ratio;               /* ratio test: accept Delta1 < ratio * Delta2; 0 = no ratio
                                     test (Sec. 2.4 literally: Delta1 < Delta_s alone) */
    float    delta_s;             /* Delta_s of Sec. 2.4; <= 0 or inf disables it */
    int32_t  ransac_iters;        /* RANSAC iterations T, 1..65536 */
    float    thresh_px;           /* inlier threshold on reprojection error (px) */
    uint64_t seed;                /* key of the Philox4x32-10 sampling stream */
    int32_t  min_inliers;         /* an H_M entry is non-zero iff n_in >= this */
    int32_t  precision;           /* lp_precision */
    int32_t  upright;             /* 1: every orientation is 0 (no rotation) */
    int32_t  model;               /* lp_model of lp_ransac and the stitch calls */
    /* Paper-literal variants (off by default). */
    double   alpha;               /* Eq. 1 ramp coefficient: 0 = the limit alpha -> 0+ (exact
                                     integer keys); > 0 = M + alpha * (raster index + 1) in
                                     FP64, ties to the earlier raster position */
    int32_t  border;              /* 1: a point whose describe neighbourhood (radius
                                     ceil(2 sqrt(2) w_s + 1.5) + 1) leaves the image is invalid */
    int32_t  hard_bins;           /* Sec. 2.3's 8-direction histogram: 0 = each magnitude split
                                     linearly between the two nearest bins; 1 = all of it in the
                                     45-degree sector [45k, 45(k+1)) holding atan2(b, a) */
} lp_config;

typedef struct lp_ctx lp_ctx;

/* Fill *cfg with L = {16, 32, 64, 128}, beta0 auto, ratio 0.8, Delta_s off,
 * T = 1000, 3 px, seed 0, min_inliers 8, LP_PREC_FP32 (select LP_PREC_BF16
 * for the tensor-core form), rotated descriptors, the homography model, and
 * the paper-literal variants off (alpha 0, border 0). */
LP_API int lp_config_default(lp_config* cfg);

/* Create a context on the current CUDA device.  The context owns a copy of the
 * configuration, a device status word and a grow-only device workspace, and
 * (created on first use) three streams of its own: lp_describe, lp_match and
 * lp_stitch_pair fork independent launches onto them and join them back to
 * the caller's stream with events before returning, so every call is ordered
 * on the caller's stream as if all its work ran there (also under graph
 * capture).  A context is not thread-safe: use one per host thread.
 * Errors: LP_ERR_ARG (bad config), LP_ERR_CUDA, LP_ERR_NOMEM. */
LP_API int lp_create(lp_ctx** ctx, const lp_config* cfg);

/* Synchronise the context's streams and free everything it owns. */
LP_API int lp_destroy(lp_ctx* ctx);

/* Number of feature points 2 * sum_L floor(H/L) * floor(W/L) (Eq. 2: one max
 * and one min per full L x L window; partial windows are dropped).  Returns -1
 * on bad arguments. */
LP_API int64_t lp_num_keypoints(int H, int W, const int* Ls, int nL);

/* Sec. 2.1-2.2, Eq. 1-2: multiscale local peaks.
 *  img      device, H x W x channels uint8, pitch bytes per row
 *  kp_idx   device, uint32[K], K = lp_num_keypoints(H, W, cfg.Ls): raster
 *           indices in canonical order -- L ascending, windows row-major,
 *           the window maximum then its minimum.  Eq. 1's ramp with
 *           alpha -> 0+ decides ties: the later raster index is the larger.
 *  gray     device, uint8[H*W] dense intensity output, required when
 *           channels == 3 (it feeds lp_describe), ignored when channels == 1.
 *           RGB -> intensity is (299 R + 587 G + 114 B + 500) / 1000.
 * Errors: LP_ERR_ARG, LP_ERR_ALIGN, LP_ERR_CUDA. */
LP_API int lp_detect(lp_ctx* ctx, const uint8_t* img, int H, int W, int pitch, int channels,
              uint32_t* kp_idx, uint8_t* gray, void* stream);

/* Sec. 2.3, Eq. 3-5: orientation and 128-d descriptor of every feature point.
 *  gray       device, H x W uint8 intensity, gray_pitch bytes per row
 *  kp_idx     device, uint32[K] from lp_detect (K must equal lp_num_keypoints;
 *             the scale of point k follows from its position)
 *  ori        device, uint8[K]: orientation bin k (theta = (k + 0.5) * 10 deg)
 *  desc       device, float[K*128], row-major, unit L2 norm (zeros if invalid)
 *  desc_bf16  device, uint16[K*128] bfloat16 copy of desc, or NULL
 *  valid      device, uint8[K]: 0 when the gradient histogram is all zero, or
 *             (cfg.border = 1) when the point's neighbourhood leaves the image
 * Errors: LP_ERR_ARG, LP_ERR_ALIGN, LP_ERR_CUDA. */
LP_API int lp_describe(lp_ctx* ctx, const uint8_t* gray, int H, int W, int gray_pitch, const uint32_t* kp_idx,
                int64_t K, uint8_t* ori, float* desc, uint16_t* desc_bf16, uint8_t* valid, void* stream);

/* Sec. 2.4, Eq. 6: each valid point i of image A takes its nearest valid point
 * j1 of image B (lowest j on exact ties) and keeps it when
 * Delta1 < ratio * Delta2 (and Delta1 < Delta_s when set).
 *  dA, dB           device float[N*128] descriptors
 *  dA_bf16, dB_bf16 device bf16 copies, required for LP_PREC_BF16, else unused
 *  vA, vB           device uint8 validity
 *  match            device int32[NA]: j1 or -1
 *  d1, d2           device float[NA]: Delta1, Delta2 (FP32, +inf if none)
 * With LP_PREC_BF16 or LP_PREC_FP8 the tensor cores rank candidates, every
 * candidate is re-scored exactly in FP32 and rows whose ranking cannot be
 * certified are re-scanned in FP32, so the result is that of the FP32 form.
 * LP_PREC_FP8 converts dA and dB to E4M3 itself (the bf16 copies are unused).
 * Errors: LP_ERR_ARG, LP_ERR_ALIGN, LP_ERR_NOMEM, LP_ERR_CUDA. */
LP_API int lp_match(lp_ctx* ctx, const float* dA, const uint16_t* dA_bf16, const uint8_t* vA, int64_t NA,
             const float* dB, const uint16_t* dB_bf16, const uint8_t* vB, int64_t NB,
             int32_t* match, float* d1, float* d2, void* stream);

/* Matched pairs p_v1, p_v2 of Sec. 2.4 as coordinates, in row order of A.
 *  kpA, kpB  device uint32 raster indices; WA, WB image widths
 *  match     device int32[NA] from lp_match
 *  pts       device float[NA*4] output rows (xA, yA, xB, yB); the first M used
 *  rows      device int32[NA] output: the A row of each compacted pair, or NULL
 *  d_M       device int32 output: M, the number of matched pairs
 * Errors: LP_ERR_ARG, LP_ERR_CUDA. */
LP_API int lp_compact(lp_ctx* ctx, const uint32_t* kpA, int WA, const uint32_t* kpB, int WB, const int32_t* match,
               int64_t NA, float* pts, int32_t* rows, int32_t* d_M, void* stream);

/* Sec. 2.5, Eq. 7: RANSAC with a full homography x_B ~ H x_A.
 *  pts       device float[M_cap*4] (xA, yA, xB, yB)
 *  M_cap     capacity of pts; the count used is *d_M when d_M != NULL, else M_cap
 *  H         device double[9], row-major, h33 = 1 (all zero if no model)
 *  inlier    device uint8[M_cap] final inlier mask (first M entries)
 *  n_inliers device int32: inliers of the refitted H
 *  best_t    device int32 or NULL: the winning iteration (-1 if none)
 * Iteration t draws 4 distinct matches from Philox4x32-10 keyed by
 * (lo32(seed), hi32(seed) ^ pair_id), counter (t, block, 0, 0), fits a
 * normalised 4-point DLT in FP64, and counts inliers (e < thresh_px).  The
 * most inliers win (earliest t on ties), decided in FP64 for every hypothesis
 * whose FP32 count could reach the maximum.  The winner's inliers are refitted
 * by least squares (FP64) and the final mask is taken from the refitted H.
 * With cfg.model = LP_MODEL_RIGID (Eq. 8) iteration t takes the first 2
 * distinct matches of the same stream, the hypothesis is their least-squares
 * rotation and translation, and the refit is the least-squares rotation and
 * translation of the winner's inliers.
 * Errors: LP_ERR_ARG, LP_ERR_NOMEM, LP_ERR_CUDA. */
LP_API int lp_ransac(lp_ctx* ctx, const float* pts, int64_t M_cap, const int32_t* d_M, uint32_t pair_id,
              double* H, uint8_t* inlier, int32_t* n_inliers, int32_t* best_t, void* stream);

/* lp_ransac for callers that cannot allocate device memory.  The paper has
 * no counterpart; this is a deployment variant of the same stage.
 *
 * Who needs it: code that may not call cudaMalloc -- a host application whose
 * own caching allocator already holds the device's memory, a real-time loop
 * that must not enter the driver's allocation path (it can synchronise the
 * device and take unbounded time), or a plug-in host that forbids device
 * allocations after start-up.  This call needs no lp_ctx (creating one
 * allocates) and allocates nothing: its scratch is a fixed 384 KiB array
 * compiled into the library, resident on every GPU that loads the library
 * until the process exits.
 *
 * Arguments are those of lp_ransac, with the configuration values passed
 * directly: iters = T (1..LP_RANSAC_STATIC_MAX_ITERS; more returns
 * LP_ERR_ARG), thresh_px, seed and pair_id.  The model is the full
 * 8-parameter homography.  The results equal lp_ransac's for the same inputs
 * and configuration.
 *
 * The first call on each device looks up the array's device address (once per
 * device, with that device current); make that first call before any stream
 * capture.  All calls share the one array, which keeps the last call's
 * contents: calls that overlap on the GPU (different streams, or host threads
 * without ordering) race on it and must be serialised by the caller.
 * Errors: LP_ERR_ARG, LP_ERR_ALIGN, LP_ERR_CUDA. */
#define LP_RANSAC_STATIC_MAX_ITERS 4096
LP_API int lp_ransac_static(const float* pts, int64_t M_cap, const int32_t* d_M, int iters, float thresh_px,
                            uint64_t seed, uint32_t pair_id, double* H, uint8_t* inlier, int32_t* n_inliers,
                            int32_t* best_t, void* stream);

/* The whole Sec. 2 path for one image pair held on the device: detect,
 * describe, match, compact and RANSAC, with every intermediate in the
 * context's workspace.  imgA/imgB as in lp_detect (same channels).
 *  H        device double[9]; n_in device int32; M_out device int32 or NULL
 * Errors: as the stages. */
LP_API int lp_stitch_pair(lp_ctx* ctx, const uint8_t* imgA, int HA, int WA, int pitchA, const uint8_t* imgB,
                   int HB, int WB, int pitchB, int channels, uint32_t pair_id, double* H, int32_t* n_in,
                   int32_t* M_out, void* stream);

/* lp_stitch_pair for images in HOST memory (pinned memory makes the copies
 * asynchronous): copies both images to the context's workspace, runs the
 * path, copies H, n_in and M back to the host buffers and synchronises
 * `stream` before returning.  H_host double[9], n_in_host / M_host int32. */
LP_API int lp_stitch_pair_host(lp_ctx* ctx, const uint8_t* imgA_host, int HA, int WA, int pitchA,
                        const uint8_t* imgB_host, int HB, int WB, int pitchB, int channels,
                        uint32_t pair_id, double* H_host, int32_t* n_in_host, int32_t* M_host, void* stream);

/* One independent pair in host memory, for lp_stitch_pairs_host. */
typedef struct lp_host_pair {
    const uint8_t* A;        /* host, HA x WA x channels, pitchA bytes per row (a multiple of 16) */
    const uint8_t* B;        /* host, HB x WB x channels, pitchB bytes per row */
    int32_t HA, WA, pitchA, HB, WB, pitchB;
} lp_host_pair;

/* lp_stitch_pair_host over a stream of P independent pairs (Fig. 2 for each):
 * the two images of pair q are copied to one of two upload slots on a copy
 * stream of the context while pair q - 1 is computed on `stream`, so with
 * pinned host images the copies hide behind the computation.  Pair q gets
 * pair id pair_id0 + q (its RANSAC sampling stream) and gives exactly what
 * lp_stitch_pair_host gives for it.  Results of all pairs are copied back at
 * the end and `stream` is synchronised before returning.
 *  pairs      host lp_host_pair[P] (the host images must stay valid until return)
 *  H_host     host double[9 P] (pair q's H at 9 q); n_in_host host int32[P];
 *  M_host     host int32[P] or NULL
 * Errors: LP_ERR_ARG (P < 0, null pointers), LP_ERR_ALIGN (pitch), as the stages. */
LP_API int lp_stitch_pairs_host(lp_ctx* ctx, const lp_host_pair* pairs, int P, int channels, uint32_t pair_id0,
                                double* H_host, int32_t* n_in_host, int32_t* M_host, void* stream);

/* One image of a batch: device data plus its geometry (lp_detect's rules). */
typedef struct lp_image {
    const uint8_t* data;     /* device, H x W x channels, pitch bytes per row */
    int32_t H, W, pitch, channels;
} lp_image;

/* lp_detect for N images at once (same configuration, same channel count):
 * on the fast path (nested window sizes, the largest <= 128, alpha = 0) the
 * images share launches of up to 12, so a batch fills the GPU that one image
 * cannot; otherwise the images are detected one by one.  Results are those of
 * lp_detect, bit for bit.
 *  imgs     host array of N images (device data pointers)
 *  kp_idx   host array of N device pointers, uint32[K_i] each
 *  gray     host array of N device pointers (uint8[H_i*W_i], required for RGB)
 * Errors: LP_ERR_ARG, LP_ERR_ALIGN, LP_ERR_CUDA. */
LP_API int lp_detect_batch(lp_ctx* ctx, const lp_image* imgs, int N, uint32_t* const* kp_idx, uint8_t* const* gray,
                           void* stream);

/* Sec. 4: the homography matrix H_M of a set of images, one entry per pair.
 *  imgs     host array of N image descriptors (device pixel pointers); every
 *           image uses the same channel count
 *  pairs    host int32[P*2] (i, j) with image i the reference of Eq. 7, or
 *           NULL for all N(N-1)/2 pairs i < j in row-major order (then P is
 *           ignored and the pair count is N(N-1)/2)
 *  HM       device double[P*9]: H of each pair (all zero without a model)
 *  n_in     device int32[P]: inliers of each pair
 *  valid    device uint8[P]: 1 iff n_in >= cfg.min_inliers (a non-zero H_M
 *           entry)
 *  M_out    device int32[P] matched pairs per image pair, or NULL
 * Every image is detected and described once; then each pair is matched,
 * compacted and fitted with RANSAC (Philox pair_id = pair index).  The whole
 * sequence is captured once as a CUDA graph and replayed while the images,
 * pairs and outputs stay the same.
 * Errors: as the stages; LP_ERR_ARG for N < 2 or a bad pair index. */
LP_API int lp_stitch_pairs(lp_ctx* ctx, const lp_image* imgs, int N, const int32_t* pairs, int P, double* HM,
                           int32_t* n_in, uint8_t* valid, int32_t* M_out, void* stream);

/* lp_stitch_pairs with explicit RANSAC pair ids (host uint32[P]; the Philox
 * key of pair q uses pair_ids[q] instead of q), so that a subset of a pair
 * list run on another GPU reproduces the full list's entries exactly.
 * `pairs` must not be NULL here. */
LP_API int lp_stitch_pairs_ids(lp_ctx* ctx, const lp_image* imgs, int N, const int32_t* pairs,
                               const uint32_t* pair_ids, int P, double* HM, int32_t* n_in, uint8_t* valid,
                               int32_t* M_out, void* stream);

/* Sec. 4 mosaic rounds (host only, synchronous).  The image of largest degree
 * (number of valid H_M entries; lowest index on ties) is the first reference;
 * it and every image matched with it are placed in its frame through their H_M
 * entries.  Each later round takes, among unmatched images with a valid entry
 * to a placed image, the one of largest degree, places it through that entry
 * (to the placed image of lowest index) and then its unmatched neighbours
 * through it.  Images that never connect stay unplaced.
 *  pairs, HM, valid  host: the P pairs (a, b), their H (x_b ~ H x_a, double[9]
 *                    each) and validity, as lp_stitch_pairs returns them
 *  Hs, Ws            host int32[N] image sizes
 *  G                 host double[N*9] out: image pixel -> canvas pixel (zero
 *                    for an unplaced image)
 *  round_of, ref_of  host int32[N] out: round of each image (-1 unplaced) and
 *                    the reference it was placed through
 *  canvas_w/h        out: the integer bounding box of the placed corner pixels
 * Errors: LP_ERR_ARG (N outside 1..64, bad pair index or size),
 * LP_ERR_UNSUPPORTED (canvas side above 32768). */
LP_API int lp_mosaic_plan(int N, const int32_t* pairs, int P, const double* HM, const uint8_t* valid,
                          const int32_t* Hs, const int32_t* Ws, double* G, int32_t* round_of, int32_t* ref_of,
                          int32_t* canvas_w, int32_t* canvas_h);

/* Warp every placed image onto the canvas: each canvas pixel is the mean of
 * the bilinear samples of the placed images whose inverse placement maps it
 * inside the image (rounded half up; 0 where none does).
 *  imgs      host array of N image descriptors (device pixels, same channels)
 *  G, round_of  lp_mosaic_plan's host outputs
 *  canvas    device uint8, canvas_h rows of canvas_pitch bytes (>= w * channels)
 *  cover     device uint8[canvas_w * canvas_h] images per pixel, or NULL
 * Errors: LP_ERR_ARG, LP_ERR_ALIGN, LP_ERR_CUDA. */
LP_API int lp_mosaic_render(lp_ctx* ctx, const lp_image* imgs, int N, const double* G, const int32_t* round_of,
                            uint8_t* canvas, int canvas_w, int canvas_h, int canvas_pitch, uint8_t* cover,
                            void* stream);

/* ---- learned RANSAC proposal (not in the paper) ----
 * A small network scores each matched pair's chance of being an inlier;
 * RANSAC can then draw its samples in proportion to the score.  Scoring of the
 * hypotheses is unchanged (every match votes), so the winner is judged exactly
 * as in uniform RANSAC, which remains the default. */

typedef struct lp_mlp lp_mlp;
#define LP_MLP_PARAMS 4801   /* W1[64][8], b1[64], W2[64][64], b2[64], w3[64], b3 */

/* Create a network on the current device: He-uniform weights from `seed`
 * (zero biases), FP32 master weights, a BF16-rounded copy used by every
 * forward pass, zero Adam state.  Errors: LP_ERR_ARG, LP_ERR_CUDA. */
LP_API int lp_mlp_create(lp_mlp** mlp, uint64_t seed);
LP_API int lp_mlp_destroy(lp_mlp* mlp);

/* Host copies of the FP32 master weights (float[LP_MLP_PARAMS]); set also
 * resets the Adam state and the step count.  Synchronous. */
LP_API int lp_mlp_set_params(lp_mlp* mlp, const float* host_params);
LP_API int lp_mlp_get_params(lp_mlp* mlp, float* host_params);

/* Host copy of the whole optimiser state, float[3 * LP_MLP_PARAMS]: master
 * weights, Adam first moments m, second moments v; *step = Adam steps taken
 * (may be NULL).  Synchronous. */
LP_API int lp_mlp_get_state(lp_mlp* mlp, float* host_state, int32_t* step);

/* Checkpoint: magic, step count, weights and Adam moments in one binary file. */
LP_API int lp_mlp_save(lp_mlp* mlp, const char* path);
LP_API int lp_mlp_load(lp_mlp* mlp, const char* path);

/* Features of the compacted matched pairs (see lp_compact; `rows` required):
 * d1/d2, d1, log2(L_A)/log2(Lmax), wrap(theta_B - theta_A)/pi in [-1, 1),
 * x_A/W_A, y_A/H_A, x_B/W_B, y_B/H_B.
 *  kpA, oriA / kpB, oriB   device outputs of lp_detect / lp_describe
 *  match, d1, d2           device outputs of lp_match (indexed by A row)
 *  rows, d_M               device outputs of lp_compact (A row per pair, M)
 *  feat                    device float[M_cap*8]
 * The scale L_A of a point follows from its index (the context's L set and
 * image A's size).  Errors: LP_ERR_ARG, LP_ERR_CUDA. */
LP_API int lp_mlp_features(lp_ctx* ctx, const uint32_t* kpA, const uint8_t* oriA, int HA, int WA,
                           const uint32_t* kpB, const uint8_t* oriB, int HB, int WB, const int32_t* match,
                           const float* d1, const float* d2, const int32_t* rows, const int32_t* d_M, int64_t M_cap,
                           float* feat, void* stream);

/* Inlier probability (sigmoid of the logit) of M = *d_M (or M_cap) matches;
 * prob / logit device float[M_cap], either may be NULL. */
LP_API int lp_mlp_forward(lp_mlp* mlp, const float* feat, int64_t M_cap, const int32_t* d_M, float* prob,
                          float* logit, void* stream);

/* One Adam step (lr, beta 0.9 / 0.999, eps 1e-8) on the mean binary
 * cross-entropy (with logits) of a minibatch of B samples.
 *  feat  device float[B*8]; label device uint8[B] (1 = inlier)
 *  loss  device float (the minibatch loss before the step) or NULL */
LP_API int lp_mlp_train_step(lp_mlp* mlp, const float* feat, const uint8_t* label, int64_t B, float lr, float* loss,
                             void* stream);

/* Failure injection for the batched distance passes of lp_stitch_pairs (BF16).
 * The paper has no counterpart.  Those passes run in one persistent launch in
 * which a pass-2 unit waits, for at most 2 s, until the pass-1 units of its
 * rows have published their values.  hold > 0 adds hold to the number of
 * completions every such wait expects, a number the launch never reaches: each
 * wait gives up, the device status word records LP_ERR_TIMEOUT (read it with
 * lp_sync_status), the launch drains and returns, and the context stays
 * usable.  hold = 0 restores normal operation.  For tests of the timeout path.
 * Errors: LP_ERR_ARG (hold < 0). */
LP_API int lp_diag_set_batch_hold(lp_ctx* ctx, int32_t hold);

/* Tile autotuning of the BF16 matcher, for batches of pairs of uneven sizes
 * (the paper has no counterpart).  on = 1: the first lp_match of a size class
 * -- (ceil(log2 NA), ceil(log2 NB)) -- that runs outside stream capture times
 * a few choices of the column-split count S and the pass-1 tile stride around
 * the built-in ones on the caller's own inputs (each once, after a warm-up
 * run; the call synchronises the stream for it), keeps the fastest for the
 * class in the context and uses it from then on (lp_stitch_pair tunes the
 * same way, inside its own lp_match).  lp_stitch_pairs runs the built-in
 * choice for a class it meets first, tunes the class on that call's
 * descriptors once its results are complete, and uses the tuned choice from
 * its next call on.  Every choice is certified against the FP32 form, so
 * outputs do not change.  Under capture, classes not yet tuned run the
 * built-in choice.  on = 0: the built-in choice everywhere (the table is
 * kept).
 * Errors: LP_ERR_ARG. */
LP_API int lp_set_autotune(lp_ctx* ctx, int32_t on);

/* The tuning table: *n = number of tuned classes; rows (host int32[cap * 6],
 * or NULL with cap = 0) receives up to cap rows (ceil(log2 NA), ceil(log2 NB),
 * S, pass-1 stride, tuned time in us, built-in choice's time in us).
 * Errors: LP_ERR_ARG. */
LP_API int lp_autotune_table(lp_ctx* ctx, int32_t* rows, int32_t cap, int32_t* n);

/* RANSAC guided by a prior, with uniform RANSAC as fallback and judge.
 * Guided phase: guided_iters hypotheses whose samples are drawn in proportion
 * to the prior -- match i gets the integer weight
 * q_i = floor(65536 * max(prior_i, 1e-3) + 1/2) (NaN counts as 1e-3), and
 * Philox word w of iteration t (the stream of lp_ransac) picks the match whose
 * interval of the inclusive prefix sums of q holds floor(w * sum(q) / 2^32);
 * repeated indices are redrawn.  Every hypothesis is scored by all matches, as
 * in lp_ransac.  Stop test: with w = (sum of q over the guided winner's
 * inliers) / sum(q), the chance that a guided draw is an inlier, the phase
 * stops when (1 - w^k)^guided_iters <= 0.01 -- the standard bound
 * T >= log(0.01) / log(1 - w^k), k = 4 matches per sample (2 for
 * LP_MODEL_RIGID) -- and the guided winner has at least the configuration's
 * min_inliers inliers (a prior concentrated on a few matches, any four of
 * which fit a homography, cannot end the search).  Then the guided winner is
 * refitted as in lp_ransac.  Otherwise the uniform phase runs: exactly lp_ransac with the
 * context's T (the test and the skipped work are decided on the device, so
 * the call never waits for the host).
 *  prior         device float[M_cap] (e.g. lp_mlp_forward's prob)
 *  guided_iters  1..65536
 *  best_t        winner: t < guided_iters (guided) or guided_iters + t
 *                (uniform iteration t); -1 if no model; device, or NULL
 *  iters_used    device int32: guided_iters, or guided_iters + T; or NULL
 * Other arguments and errors as lp_ransac. */
LP_API int lp_ransac_prior(lp_ctx* ctx, const float* pts, int64_t M_cap, const int32_t* d_M, const float* prior,
                           int32_t guided_iters, uint32_t pair_id, double* H, uint8_t* inlier, int32_t* n_inliers,
                           int32_t* best_t, int32_t* iters_used, void* stream);

/* Wait for the context's last stream, then return and clear the device
 * status word (LP_OK, LP_ERR_TIMEOUT or LP_ERR_DEVICE) or a CUDA error. */
LP_API int lp_sync_status(lp_ctx* ctx);

/* Text of the last host-side error of this context (static storage). */
LP_API const char* lp_last_error(lp_ctx* ctx);

/* ---- diagnostics used by the test-suite (no paper counterpart needed) ---- */

/* Rows that the last LP_PREC_BF16 or LP_PREC_FP8 lp_match of this context
 * re-scanned in FP32 because their tensor-core ranking could not be certified
 * (waits for the stream). */
LP_API int lp_diag_last_rescans(lp_ctx* ctx, int64_t* out);

/* Attach a network to the context (NULL detaches it): lp_stitch_pair and
 * lp_stitch_pairs then score every pair's matches with it (lp_mlp_features,
 * lp_mlp_forward) and run lp_ransac_prior with guided_iters instead of
 * lp_ransac.  The context does not own the network; keep it alive while it is
 * attached.  Errors: LP_ERR_ARG (guided_iters outside 1..65536). */
LP_API int lp_set_proposal(lp_ctx* ctx, lp_mlp* mlp, int32_t guided_iters);

/* Kernel timing for benchmarks.  With profiling on, every lp_match call that
 * is not being captured into a CUDA graph records two CUDA events on its
 * stream, immediately before and after its distance kernel (the tensor-core
 * passes of LP_PREC_BF16 and LP_PREC_FP8, the FP32 kernel of LP_PREC_FP32).
 * lp_diag_last_match_kernel_ms waits for the second event and returns the
 * elapsed milliseconds of the last such call.  Errors: LP_ERR_ARG (profiling
 * off, or no recorded call), LP_ERR_CUDA. */
LP_API int lp_set_profiling(lp_ctx* ctx, int on);
LP_API int lp_diag_last_match_kernel_ms(lp_ctx* ctx, float* ms);

/* FP32 inlier count (points certainly inside the threshold) of each hypothesis
 * of the context's last lp_ransac (n = T) or lp_ransac_prior
 * (n = guided_iters + T) call; -1 where no hypothesis was formed or the phase
 * was skipped.  host int32[n]; waits for the stream. */
LP_API int lp_diag_last_ransac_counts(lp_ctx* ctx, int32_t* host_counts, int n);

/* Orientation bin of every integer gradient (a, b) in [-255, 255]^2, written
 * to device int32[511*511] at (a + 255) * 511 + (b + 255). */
LP_API int lp_diag_orient_bins(int32_t* out, void* stream);
/* round(65536 * sqrt(s)) for s in [0, 130050], device uint32[130051]. */
LP_API int lp_diag_orient_weights(uint32_t* out, void* stream);
/* Philox4x32-10 blocks: n counters (device uint32[n*4]) under one key. */
LP_API int lp_diag_philox(const uint32_t* ctr, int64_t n, uint32_t key0, uint32_t key1, uint32_t* out, void* stream);
/* RGB -> intensity of n pixels (device uint8[n*3] -> uint8[n]). */
LP_API int lp_diag_gray(const uint8_t* rgb, int64_t n, uint8_t* gray, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* LP_H */
