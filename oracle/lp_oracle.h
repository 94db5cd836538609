/*
 * LP-SIFT oracle -- TEST INFRASTRUCTURE, NOT PRODUCT CODE.
 *
 * A plain, slow, single-threaded FP64 CPU statement of what the LP-SIFT hot
 * path computes (Li, Wang, Zhao & Zhao, "Local-peak scale-invariant feature
 * transform for fast and random image stitching", Sec. 2 and Sec. 4).  Only the
 * test-suite, the smoke check and the CPU-baseline leg of the benchmark may
 * load it.  It shares no code, header, table or constant generator with the
 * CUDA library.
 *
 * Conventions: images are uint8, row-major, `pitch` bytes per row; a keypoint
 * is its raster index idx = y*W + x (x = column, y = row, 0-based).  All
 * functions return 0 on success and a negative value on bad arguments.
 */
#ifndef LP_ORACLE_H
#define LP_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Colour -> intensity matrix M_k (Sec. 2.1): g = (299R + 587G + 114B + 500) / 1000. */
int or_gray_from_rgb(const uint8_t* rgb, int H, int W, int pitch, uint8_t* gray);

/* Number of feature points: 2 per full L x L interrogation window per scale (Eq. 2). */
int64_t or_num_keypoints(int H, int W, const int* Ls, int nL);

/* Multiscale local peaks (Eq. 1 ramp + Eq. 2).  alpha == 0 takes the limit
 * alpha -> 0+ (ties broken by the ramp only); alpha > 0 evaluates the FP64 ramp
 * literally.  Output order: L ascending, windows row-major, max then min. */
int or_detect(const uint8_t* gray, int H, int W, int pitch, const int* Ls, int nL,
              double alpha, uint32_t* idx);

/* Sub-region side w_s(L) (Eq. 3-4); beta0 <= 0 selects (1/d) sqrt(Lmin/Lmax). */
int or_region_ws(const int* Ls, int nL, double beta0, int d, int* ws);

/* Orientation helpers, exposed so they can be pinned on their own. */
int      or_orient_bin(int a, int b);          /* 10-degree bin of atan2(b, a) in [0, 360) */
uint32_t or_orient_weight(int s);             /* round(65536 * sqrt(s)) */

/* Orientation bin per keypoint (36-bin histogram over the upright window). */
int or_orient(const uint8_t* gray, int H, int W, int pitch, const uint32_t* idx, const int* ws,
              int64_t K, uint8_t* ori, uint64_t* hist36 /* K*36 or NULL */);

/* 128-d descriptor (Eq. 5 gradients on a rotated 4x4 grid, 8 soft bins).
 * ori == NULL: upright (theta = 0). */
int or_describe(const uint8_t* gray, int H, int W, int pitch, const uint32_t* idx, const int* ws,
                const uint8_t* ori, int64_t K, double* desc, uint8_t* valid);
int or_octant(double a, double b);               /* hard 8-direction sector of atan2(b, a) */
int or_turn_fx(int k, int* cq, int* sq);         /* round(2^11 cos), round(2^11 sin) of bin k's angle */
int or_describe_ex(const uint8_t* gray, int H, int W, int pitch, const uint32_t* idx, const int* ws,
                   const uint8_t* ori, int64_t K, int hard, double* desc, uint8_t* valid);

/* Nearest-neighbour matching with Eq. 6 distance, the ratio test and Delta_s.
 * rows == NULL: all NA rows; otherwise only rows[0..nrows) (outputs indexed by
 * position in rows). */
int or_match(const double* dA, const uint8_t* vA, int64_t NA, const double* dB, const uint8_t* vB,
             int64_t NB, double ratio, double delta_s, const int64_t* rows, int64_t nrows,
             int32_t* match, double* d1, double* d2, int32_t* j1, int32_t* j2);

/* Philox4x32-10 block function (Salmon, Moraes, Dror & Shaw, SC'11). */
void or_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);

/* The four sample indices of RANSAC iteration t; returns 0, or 1 if skipped. */
int or_ransac_sample(int64_t M, uint64_t seed, uint32_t pair_id, int t, int32_t* idx4);
/* The same stream's first k (2 or 4) distinct indices. */
int or_ransac_sample_k(int64_t M, uint64_t seed, uint32_t pair_id, int t, int k, int32_t* idx);

/* Models of Sec. 2.5: the homography of Eq. 7 (8 DOF, four matches per sample)
 * or the rigid transform of Eq. 8 (rotation + translation, two matches). */
#define OR_MODEL_HOMOGRAPHY 0
#define OR_MODEL_RIGID 1
int or_model_sample_size(int model);

/* Least-squares Eq. 8 (rotation + translation) over the masked correspondences;
 * returns 0, or 1 for fewer than two of them or a degenerate set. */
int or_rigid_fit(const double* pts /*M x 4*/, const uint8_t* mask, int64_t M, double* H /*9*/);

/* 4-point DLT (h33 = 1) with Hartley normalisation; returns 0, or 1 if singular. */
int or_dlt4(const double* src /*4x2 (x,y)*/, const double* dst /*4x2*/, double* H /*9*/);

/* Least-squares DLT over the masked correspondences; returns 0, or 1 on failure. */
int or_refit(const double* pts /*M x 4: xA yA xB yB*/, const uint8_t* mask, int64_t M, double* H);

/* Border rejection (paper-literal variant): clears valid[k] when the pixels
 * within ceil(2 sqrt(2) ws[k] + 1.5) + 1 of point k leave the image. */
int or_border_valid(const uint32_t* idx, const int* ws, int64_t K, int H, int W, uint8_t* valid);

/* Symmetric eigen-decomposition (cyclic Jacobi), ascending eigenvalues,
 * eigenvectors in the columns of evecs (row-major n x n). */
int or_eig_sym(int n, const double* A, double* evals, double* evecs);

/* Inlier count of H at threshold thresh (pixels); writes the mask if non-NULL. */
int64_t or_score(const double* H, const double* pts, int64_t M, double thresh, uint8_t* mask);

/* RANSAC with a homography model (Sec. 2.5, Eq. 7).  Returns 0, or 1 when no
 * model was found (H = 0, n_in = 0).  counts (T) and Hs (T*9) are optional. */
int or_ransac(const double* pts, int64_t M, int T, double thresh, uint64_t seed, uint32_t pair_id,
              double* H, uint8_t* inl, int32_t* n_in, int32_t* best_t, int32_t* counts, double* Hs);
/* The same with a model of Sec. 2.5 (OR_MODEL_*). */
int or_ransac_model(const double* pts, int64_t M, int model, int T, double thresh, uint64_t seed, uint32_t pair_id,
                    double* H, uint8_t* inl, int32_t* n_in, int32_t* best_t, int32_t* counts, double* Hs);


/* ---- learned RANSAC proposal (not in the paper) -- TEST INFRASTRUCTURE ---- */
#define OR_MLP_NPARAM 4801
/* Parameter layout: W1[64][8], b1[64], W2[64][64], b2[64], w3[64], b3. */

/* Eight features of one match (A point -> B point):
 * d1/d2, d1, log2(L_A)/log2(Lmax), wrap(theta_B - theta_A)/pi,
 * x_A/W_A, y_A/H_A, x_B/W_B, y_B/H_B. */
int or_mlp_features(int64_t M, const double* d1, const double* d2, const int32_t* LA, int Lmax,
                    const uint8_t* oriA, const uint8_t* oriB, const double* pts /*M x 4*/, int WA, int HA, int WB,
                    int HB, double* feat /*M x 8*/);

/* z = w3 . relu(W2 relu(W1 x + b1) + b2) + b3, p = sigmoid(z). */
int or_mlp_forward(const double* params, const double* x, int64_t M, double* logit, double* prob);

/* Mean binary cross-entropy with logits and its gradient. */
int or_mlp_loss_grad(const double* params, const double* x, const uint8_t* y, int64_t B, double* loss, double* grad);

/* One Adam step (t >= 1): m, v updated in place. */
int or_mlp_adam(double* params, double* m, double* v, const double* grad, int n, int t, double lr, double b1,
                double b2, double eps);

/* Guided draw of four distinct matches from integer weights (see lp_oracle.c). */
int or_ransac_sample_guided(int64_t M, const uint64_t* prefix /* inclusive prefix sums of q */, uint64_t seed,
                            uint32_t pair_id, int t, int32_t* idx4);
int or_ransac_sample_guided_k(int64_t M, const uint64_t* prefix, uint64_t seed, uint32_t pair_id, int t, int k,
                              int32_t* idx);
int or_guided_weights(const float* prob, int64_t M, uint64_t* prefix);

/* Stop test of the guided phase: (1 - w^4)^Tg <= 0.01 with w = s_in / total
 * (the standard bound T >= log(0.01) / log(1 - w^4)). */
int or_guided_stop(uint64_t s_in, uint64_t total, int Tg);
/* The same bound for samples of k matches: (1 - w^k)^Tg <= 0.01, k = 2 or 4. */
int or_guided_stop_k(uint64_t s_in, uint64_t total, int Tg, int k);

/* Tg guided hypotheses (samples drawn with probability proportional to the
 * prior), scored by all matches; the guided winner is refitted when
 * or_guided_stop holds for its prior-weighted inlier fraction and for its
 * plain inlier fraction (inliers / M), and it has at least min_support
 * inliers; otherwise the result is uniform or_ransac with T
 * iterations (best_t offset by Tg).  iters = Tg or Tg + T; counts (Tg + T,
 * optional) as or_ransac's. */
int or_ransac_prior(const double* pts, int64_t M, const float* prob, int Tg, int T, double thresh, uint64_t seed,
                    uint32_t pair_id, int min_support, double* H, uint8_t* inl, int32_t* n_in, int32_t* best_t,
                    int32_t* iters, int32_t* counts);
/* The same with a model of Sec. 2.5 (OR_MODEL_*). */
int or_ransac_prior_model(const double* pts, int64_t M, int model, const float* prob, int Tg, int T, double thresh,
                          uint64_t seed, uint32_t pair_id, int min_support, double* H, uint8_t* inl, int32_t* n_in,
                          int32_t* best_t, int32_t* iters, int32_t* counts);
/* Sec. 4 mosaic (readings in lp_oracle.c): rounds of reference selection over
 * H_M (pairs host int32[P*2], HM double[P*9], valid uint8[P]) and placements G
 * (double[N*9], image pixel -> canvas pixel) on a canvas_w x canvas_h canvas. */
int or_mosaic_plan(int N, const int32_t* pairs, int P, const double* HM, const uint8_t* valid, const int* Hs,
                   const int* Ws, double* G, int32_t* round_of, int32_t* ref_of, int* canvas_w, int* canvas_h);
/* Mean of the bilinear samples of every placed image covering each canvas
 * pixel (rounded half up, 0 where none); cover (or NULL) counts them. */
int or_mosaic_render(int N, const uint8_t* const* imgs, const int* Hs, const int* Ws, const int* pitches, int C,
                     const double* G, const int32_t* round_of, int cw, int ch, uint8_t* canvas, uint8_t* cover);

#ifdef __cplusplus
}
#endif
#endif
