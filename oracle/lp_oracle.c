/*
 * LP-SIFT oracle -- TEST INFRASTRUCTURE, NOT PRODUCT CODE.
 *
 * Plain FP64 CPU statement of the LP-SIFT hot path (Sec. 2.1-2.5, Sec. 4 of
 * the paper).  Each function cites the passage it follows and spells out the
 * readings taken where the paper is silent or garbled.  No blocking, no
 * vectorisation, no shortcuts: loops follow the definitions.  Only the tests,
 * the smoke check and the benchmark's CPU-baseline leg may load this file's
 * library; the CUDA path never does.
 *
 * Parity status of each function (pins live in tests/test_oracle_*.py):
 *   or_gray_from_rgb   pinned (closed form, exhaustive integer identity)
 *   or_detect          pinned (brute force, constant image, 2x replication)
 *   or_region_ws       pinned (closed form)
 *   or_orient_bin      pinned (exhaustive, high-precision angle)
 *   or_orient_weight   pinned (exhaustive, integer square-root bracket)
 *   or_orient          pinned (ramp images, 90-degree rotation)
 *   or_describe        pinned (ramp closed forms, unit norm, 90-degree rotation)
 *   or_octant / or_turn_fx / or_describe_ex (hard 8-direction bins)
 *                      pinned (edge and interior directions, atan2 sectors
 *                      away from edges, 40-digit turn table, ramp closed
 *                      forms, integer Eq. 5 with atan2 sectors, exact
 *                      90-degree rotation)
 *   or_match           pinned (brute force in numpy, permutation invariance)
 *   or_philox4x32_10   pinned (published known-answer vectors)
 *   or_dlt4 / or_refit pinned (known homographies, numpy SVD)
 *   or_ransac          pinned (synthetic inliers + outliers)
 *   or_border_valid    pinned (closed-form radius, padding invariance)
 *   or_rigid_fit / or_ransac_model (Eq. 8)
 *                      pinned (exact rotations, independent least squares,
 *                      special case of the homography model)
 *   or_mlp_*           pinned (finite differences, closed-form networks,
 *                      Adam first step, hand-computed features)
 *   or_guided_* / or_ransac_prior*
 *                      pinned (exact integer weights, chi-square of draws,
 *                      closed-form stop bound, uniform fallback)
 *   or_mosaic_plan / or_mosaic_render
 *                      pinned (star and chain graphs, identity and shifted
 *                      renders)
 */
#include "lp_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#define OR_PI 3.14159265358979323846

/* ------------------------------------------------------------------ */
/* Sec. 2.1: the image matrix M_k.  The paper works on intensity matrices and
 * is silent on colour; an RGB pixel becomes intensity with the integer form of
 * the 0.299/0.587/0.114 weights, rounded half up. */
int or_gray_from_rgb(const uint8_t* rgb, int H, int W, int pitch, uint8_t* gray)
{
    if (!rgb || !gray || H <= 0 || W <= 0 || pitch < 3 * W) return -1;
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x) {
            const uint8_t* p = rgb + (size_t)y * pitch + 3 * (size_t)x;
            unsigned v = 299u * p[0] + 587u * p[1] + 114u * p[2] + 500u;
            gray[(size_t)y * W + x] = (uint8_t)(v / 1000u);
        }
    return 0;
}

/* ------------------------------------------------------------------ */
/* Eq. 2: every full L x L interrogation window yields one maximum and one
 * minimum.  Reading: windows tile the image from (0, 0); a partial window at
 * the right or bottom edge is dropped; no de-duplication across scales. */
int64_t or_num_keypoints(int H, int W, const int* Ls, int nL)
{
    int64_t K = 0;
    for (int l = 0; l < nL; ++l) {
        if (Ls[l] < 2) return -1;
        K += 2 * (int64_t)(H / Ls[l]) * (int64_t)(W / Ls[l]);
    }
    return K;
}

static int cmp_int(const void* a, const void* b)
{
    int x = *(const int*)a, y = *(const int*)b;
    return (x > y) - (x < y);
}

/* Ramped intensity comparison of Eq. 1 in the limit alpha -> 0+:
 * M_n = M + alpha*(y*W + x + 1).  A larger intensity always wins; between
 * equal intensities the later raster position carries the larger ramp. */
static int ramp_greater(int g1, int64_t i1, int g2, int64_t i2)
{
    return g1 > g2 || (g1 == g2 && i1 > i2);
}

/* Eq. 1 + Eq. 2.  Reading of "i, j in [0, L]": the L x L pixels of window p. */
int or_detect(const uint8_t* gray, int H, int W, int pitch, const int* Ls_in, int nL,
              double alpha, uint32_t* idx)
{
    if (!gray || !idx || !Ls_in || nL <= 0 || nL > 64 || H <= 0 || W <= 0 || pitch < W) return -1;
    if ((int64_t)H * W > 0xFFFFFFFFll) return -1;
    int Ls[64];
    memcpy(Ls, Ls_in, sizeof(int) * nL);
    qsort(Ls, nL, sizeof(int), cmp_int);
    int64_t k = 0;
    for (int l = 0; l < nL; ++l) {
        int L = Ls[l];
        if (L < 2) return -1;
        int nwy = H / L, nwx = W / L;
        for (int wy = 0; wy < nwy; ++wy)
            for (int wx = 0; wx < nwx; ++wx) {
                int64_t imax = -1, imin = -1;
                int gmax = 0, gmin = 0;
                double vmax = 0, vmin = 0;
                for (int i = 0; i < L; ++i)
                    for (int j = 0; j < L; ++j) {
                        int y = wy * L + i, x = wx * L + j;
                        int64_t r = (int64_t)y * W + x;
                        int g = gray[(size_t)y * pitch + x];
                        if (alpha > 0) {
                            double v = (double)g + alpha * (double)(r + 1);
                            if (imax < 0 || v > vmax) { vmax = v; imax = r; }
                            if (imin < 0 || v < vmin) { vmin = v; imin = r; }
                        } else {
                            if (imax < 0 || ramp_greater(g, r, gmax, imax)) { gmax = g; imax = r; }
                            if (imin < 0 || ramp_greater(gmin, imin, g, r)) { gmin = g; imin = r; }
                        }
                    }
                idx[k++] = (uint32_t)imax;
                idx[k++] = (uint32_t)imin;
            }
    }
    return 0;
}

/* Eq. 3-4: w = beta*L*d, beta = beta0*(L/Lmax)^(-1/2), w_s = beta*L.
 * Readings: w_s is rounded to the nearest integer (at least 1); the exponent
 * printed in Eq. 4 contradicts Eq. 3, and w <= L for every L needs
 * beta0 <= (1/d) sqrt(L/Lmax), which binds at Lmin, so the default beta0 is
 * (1/d) sqrt(Lmin/Lmax). */
int or_region_ws(const int* Ls, int nL, double beta0, int d, int* ws)
{
    if (!Ls || !ws || nL <= 0 || d <= 0) return -1;
    int Lmin = Ls[0], Lmax = Ls[0];
    for (int l = 1; l < nL; ++l) {
        if (Ls[l] < Lmin) Lmin = Ls[l];
        if (Ls[l] > Lmax) Lmax = Ls[l];
    }
    if (beta0 <= 0) beta0 = sqrt((double)Lmin / (double)Lmax) / (double)d;
    for (int l = 0; l < nL; ++l) {
        double beta = beta0 * pow((double)Ls[l] / (double)Lmax, -0.5);
        int w = (int)floor(beta * (double)Ls[l] + 0.5);
        ws[l] = w < 1 ? 1 : w;
    }
    return 0;
}

/* ------------------------------------------------------------------ */
/* Clamp-to-edge pixel access (reading: border pixels are repeated). */
static int px(const uint8_t* g, int H, int W, int pitch, int y, int x)
{
    if (y < 0) y = 0;
    if (y >= H) y = H - 1;
    if (x < 0) x = 0;
    if (x >= W) x = W - 1;
    return g[(size_t)y * pitch + x];
}

/* Eq. 5: theta = "b/a" is read as the direction atan2(b, a), measured from
 * the +row axis towards the +column axis, in [0, 360) degrees.  The
 * orientation histogram has 36 bins of 10 degrees; bin k holds
 * k*10 <= phi < (k+1)*10.  On the axes the direction is exact. */
int or_orient_bin(int a, int b)
{
    if (a == 0 && b == 0) return 0;
    if (b == 0) return a > 0 ? 0 : 18;
    if (a == 0) return b > 0 ? 9 : 27;
    double phi = atan2((double)b, (double)a);
    if (phi < 0) phi += 2.0 * OR_PI;
    int k = (int)floor(phi * 36.0 / (2.0 * OR_PI));
    if (k > 35) k = 35;
    if (k < 0) k = 0;
    return k;
}

/* Magnitude f = sqrt(a^2 + b^2) of Eq. 5, in units of 2^-16, rounded. */
uint32_t or_orient_weight(int s)
{
    return (uint32_t)floor(65536.0 * sqrt((double)s) + 0.5);
}

/* Orientation assignment (not in the paper; SIFT's, needed for the rotation
 * invariance of Sec. 3.5).  Reading: one orientation per feature point, the
 * peak of a 36-bin magnitude-weighted histogram of Eq. 5 gradients over the
 * upright (4 w_s + 1)^2 window centred on the point; no Gaussian weight, no
 * smoothing, no secondary peaks; the lowest bin wins exact ties. */
int or_orient(const uint8_t* gray, int H, int W, int pitch, const uint32_t* idx, const int* ws,
              int64_t K, uint8_t* ori, uint64_t* hist36)
{
    if (!gray || !idx || !ws || !ori || K < 0) return -1;
    for (int64_t k = 0; k < K; ++k) {
        int y = (int)(idx[k] / (uint32_t)W), x = (int)(idx[k] % (uint32_t)W);
        int R = 2 * ws[k];
        uint64_t h[36];
        memset(h, 0, sizeof h);
        for (int u = -R; u <= R; ++u)
            for (int v = -R; v <= R; ++v) {
                int yy = y + u, xx = x + v;
                int a = px(gray, H, W, pitch, yy + 1, xx) - px(gray, H, W, pitch, yy - 1, xx);
                int b = px(gray, H, W, pitch, yy, xx + 1) - px(gray, H, W, pitch, yy, xx - 1);
                int s = a * a + b * b;
                if (s == 0) continue;
                h[or_orient_bin(a, b)] += or_orient_weight(s);
            }
        int best = 0;
        for (int j = 1; j < 36; ++j)
            if (h[j] > h[best]) best = j;
        ori[k] = (uint8_t)best;
        if (hist36) memcpy(hist36 + 36 * k, h, sizeof h);
    }
    return 0;
}

/* Bilinear intensity at real (row r, column c), clamp-to-edge taps.  Written
 * as nested linear interpolation v0 + f*(v1 - v0), which returns a flat
 * neighbourhood's value exactly (so its gradient is exactly zero). */
static double bil(const uint8_t* g, int H, int W, int pitch, double r, double c)
{
    double r0 = floor(r), c0 = floor(c);
    double fr = r - r0, fc = c - c0;
    int y = (int)r0, x = (int)c0;
    double v00 = px(g, H, W, pitch, y, x), v01 = px(g, H, W, pitch, y, x + 1);
    double v10 = px(g, H, W, pitch, y + 1, x), v11 = px(g, H, W, pitch, y + 1, x + 1);
    double top = v00 + fc * (v01 - v00);
    double bot = v10 + fc * (v11 - v10);
    return top + fr * (bot - top);
}

/* Sec. 2.3: a w x w region (w = d*w_s, d = 4) around the point, split into
 * d x d sub-regions of w_s x w_s samples; Eq. 5 gradients in each sub-region
 * feed an 8-direction histogram, giving 4*4*8 = 128 values.
 * Readings (the paper defers to SIFT): the grid is turned by the point's
 * orientation theta = (k + 0.5)*10 degrees; sample offsets are
 * u, v in {-2w_s, ..., 2w_s - 1} along the rotated axes e_u = (cos, sin),
 * e_v = (-sin, cos) in (row, column); intensities are bilinear; the gradient is
 * Eq. 5 taken along e_u and e_v; directions are relative to e_u; each
 * magnitude is split linearly between the two nearest of the 8 bins; the
 * vector is L2-normalised, clamped at 0.2 and normalised again.  A point whose
 * histogram is all zero is marked invalid (all-zero descriptor). */
int or_describe(const uint8_t* gray, int H, int W, int pitch, const uint32_t* idx, const int* ws,
                const uint8_t* ori, int64_t K, double* desc, uint8_t* valid)
{
    return or_describe_ex(gray, H, W, pitch, idx, ws, ori, K, 0, desc, valid);
}

/* Sec. 2.3 read literally (a paper-literal variant): the histogram has 8
 * directions, and a sample's whole magnitude goes to the direction whose
 * 45-degree sector [45k, 45(k + 1)) degrees holds atan2(b, a).  The sector is
 * decided by signs and magnitude comparisons, so a direction on a sector edge
 * belongs to the sector it starts.  (a, b) = 0 is never asked for. */
int or_octant(double a, double b)
{
    if (b >= 0 && a > 0) return b < a ? 0 : 1;
    if (a <= 0 && b > 0) return b > -a ? 2 : 3;
    if (b <= 0 && a < 0) return -b < -a ? 4 : 5;
    return a < -b ? 6 : 7;
}

/* The turned grid of the hard-bin variant in fixed point: cos and sin of
 * orientation bin k ((k + 0.5) * 10 degrees) rounded to multiples of 2^-11.
 * A hard bin is a discontinuous function of the gradient direction, so the
 * variant makes every sample position, intensity and gradient an exact
 * number: offsets (u cq - v sq, u sq + v cq) are multiples of 2^-11 px and
 * bilinear intensities multiples of 2^-22.  (The turn differs from the exact
 * angle by less than 2.5e-4 rad.) */
int or_turn_fx(int k, int* cq, int* sq)
{
    if (k < 0 || k > 35 || !cq || !sq) return -1;
    double th = ((double)k + 0.5) * (10.0 * OR_PI / 180.0);
    *cq = (int)floor(2048.0 * cos(th) + 0.5);
    *sq = (int)floor(2048.0 * sin(th) + 0.5);
    return 0;
}

static int64_t floor_div_2048(int64_t v)
{
    return v >= 0 ? v / 2048 : -((-v + 2047) / 2048);
}

/* 2^22 * bilinear intensity at (y + r / 2048, x + c / 2048), clamp-to-edge
 * taps, in exact integer arithmetic. */
static int64_t bil_fx(const uint8_t* g, int H, int W, int pitch, int y, int x, int64_t r, int64_t c)
{
    int64_t r0 = floor_div_2048(r), c0 = floor_div_2048(c);
    int64_t fr = r - 2048 * r0, fc = c - 2048 * c0;
    int yy = y + (int)r0, xx = x + (int)c0;
    int64_t v00 = px(g, H, W, pitch, yy, xx), v01 = px(g, H, W, pitch, yy, xx + 1);
    int64_t v10 = px(g, H, W, pitch, yy + 1, xx), v11 = px(g, H, W, pitch, yy + 1, xx + 1);
    int64_t top = v00 * (2048 - fc) + v01 * fc;
    int64_t bot = v10 * (2048 - fc) + v11 * fc;
    return top * (2048 - fr) + bot * fr;
}

/* or_describe with the bin rule chosen.  hard = 0: each magnitude is split
 * linearly between the two nearest bins (the default reading).  hard = 1: the
 * grid is the fixed-point one of or_turn_fx, each gradient an exact integer
 * (2^22 * Eq. 5), and its whole magnitude goes to its sector (or_octant). */
int or_describe_ex(const uint8_t* gray, int H, int W, int pitch, const uint32_t* idx, const int* ws,
                   const uint8_t* ori, int64_t K, int hard, double* desc, uint8_t* valid)
{
    if (!gray || !idx || !ws || !desc || !valid || K < 0) return -1;
    for (int64_t k = 0; k < K; ++k) {
        double y = (double)(idx[k] / (uint32_t)W), x = (double)(idx[k] % (uint32_t)W);
        int s_ = ws[k], R = 2 * ws[k];
        double th = ori ? ((double)ori[k] + 0.5) * (10.0 * OR_PI / 180.0) : 0.0;
        double c = ori ? cos(th) : 1.0, s = ori ? sin(th) : 0.0;
        double h[128];
        memset(h, 0, sizeof h);
        int cq = 2048, sq = 0;
        if (hard && ori) or_turn_fx(ori[k], &cq, &sq);
        for (int u = -R; u < R; ++u)
            for (int v = -R; v < R; ++v) {
                int cell = ((u + R) / s_) * 4 + (v + R) / s_;
                if (hard) {
                    int yi = (int)y, xi = (int)x;
                    int64_t pr = (int64_t)u * cq - (int64_t)v * sq, pc = (int64_t)u * sq + (int64_t)v * cq;
                    int64_t ai = bil_fx(gray, H, W, pitch, yi, xi, pr + cq, pc + sq) -
                                 bil_fx(gray, H, W, pitch, yi, xi, pr - cq, pc - sq);
                    int64_t bi = bil_fx(gray, H, W, pitch, yi, xi, pr - sq, pc + cq) -
                                 bil_fx(gray, H, W, pitch, yi, xi, pr + sq, pc - cq);
                    if (ai == 0 && bi == 0) continue;
                    double a = (double)ai, b = (double)bi;
                    h[cell * 8 + or_octant(a, b)] += sqrt(a * a + b * b) / 4194304.0;
                    continue;
                }
                double py = y + u * c - v * s;
                double pxx = x + u * s + v * c;
                double a = bil(gray, H, W, pitch, py + c, pxx + s) - bil(gray, H, W, pitch, py - c, pxx - s);
                double b = bil(gray, H, W, pitch, py - s, pxx + c) - bil(gray, H, W, pitch, py + s, pxx - c);
                double m = sqrt(a * a + b * b);
                if (m == 0) continue;
                double o = 8.0 * atan2(b, a) / (2.0 * OR_PI);
                if (o < 0) o += 8.0;
                if (o >= 8.0) o -= 8.0;
                double fo = floor(o);
                double t = o - fo;
                int b0 = (int)fo, b1 = (b0 + 1) % 8;
                h[cell * 8 + b0] += m * (1.0 - t);
                h[cell * 8 + b1] += m * t;
            }
        double n = 0;
        for (int j = 0; j < 128; ++j) n += h[j] * h[j];
        n = sqrt(n);
        double* out = desc + 128 * k;
        if (n == 0) {
            memset(out, 0, sizeof(double) * 128);
            valid[k] = 0;
            continue;
        }
        double n2 = 0;
        for (int j = 0; j < 128; ++j) {
            double q = h[j] / n;
            if (q > 0.2) q = 0.2;
            out[j] = q;
            n2 += q * q;
        }
        n2 = sqrt(n2);
        for (int j = 0; j < 128; ++j) out[j] /= n2;
        valid[k] = 1;
    }
    return 0;
}

/* Border rejection (a paper-literal variant of Sec. 2.3; the default reading
 * clamps to the edge): a point of region side w_s is invalid when the pixels
 * within P = ceil(2 sqrt(2) w_s + 1.5) + 1 of it do not all lie inside the
 * image.  P bounds every pixel that the orientation window (|u|, |v| <= 2 w_s,
 * plus one-pixel gradient taps) and the turned descriptor grid (radius
 * sqrt(2) (2 w_s + 1), plus bilinear taps) can read. */
int or_border_valid(const uint32_t* idx, const int* ws, int64_t K, int H, int W, uint8_t* valid)
{
    if ((K > 0 && (!idx || !ws || !valid)) || H <= 0 || W <= 0) return -1;
    for (int64_t k = 0; k < K; ++k) {
        const int P = (int)ceil(2.0 * sqrt(2.0) * ws[k] + 1.5) + 1;
        const int y = (int)(idx[k] / (uint32_t)W), x = (int)(idx[k] % (uint32_t)W);
        if (x - P < 0 || y - P < 0 || x + P > W - 1 || y + P > H - 1) valid[k] = 0;
    }
    return 0;
}

/* ------------------------------------------------------------------ */
/* Sec. 2.4, Eq. 6: Delta = |d_f1 - d_f2|.  Readings: every valid point of the
 * reference image queries all valid points of the registered image; the
 * nearest one (lowest index on ties) is kept when it passes the ratio test
 * Delta_1 < ratio * Delta_2 (Delta_2 = the next nearest) and, when set,
 * Delta_1 < Delta_s.  ratio = 0 drops the ratio test: the paper's own rule
 * keeps a nearest neighbour on Delta_1 < Delta_s alone (any valid candidate
 * when Delta_s is off). */
int or_match(const double* dA, const uint8_t* vA, int64_t NA, const double* dB, const uint8_t* vB,
             int64_t NB, double ratio, double delta_s, const int64_t* rows, int64_t nrows,
             int32_t* match, double* d1, double* d2, int32_t* j1o, int32_t* j2o)
{
    if (!dA || !vA || !dB || !vB || !match || !d1 || !d2 || NA < 0 || NB < 0) return -1;
    int64_t nq = rows ? nrows : NA;
    int64_t nbv = 0;
    for (int64_t j = 0; j < NB; ++j) nbv += vB[j] != 0;
    for (int64_t q = 0; q < nq; ++q) {
        int64_t i = rows ? rows[q] : q;
        if (i < 0 || i >= NA) return -1;
        match[q] = -1;
        d1[q] = INFINITY;
        d2[q] = INFINITY;
        if (j1o) j1o[q] = -1;
        if (j2o) j2o[q] = -1;
        if (!vA[i]) continue;
        double b1 = INFINITY, b2 = INFINITY;
        int64_t j1 = -1, j2 = -1;
        for (int64_t j = 0; j < NB; ++j) {
            if (!vB[j]) continue;
            double e = 0;
            for (int c = 0; c < 128; ++c) {
                double t = dA[128 * i + c] - dB[128 * j + c];
                e += t * t;
            }
            if (e < b1) {
                b2 = b1; j2 = j1;
                b1 = e; j1 = j;
            } else if (e < b2) {
                b2 = e; j2 = j;
            }
        }
        d1[q] = sqrt(b1);
        d2[q] = sqrt(b2);
        if (j1o) j1o[q] = (int32_t)j1;
        if (j2o) j2o[q] = (int32_t)j2;
        int ok = ratio > 0 ? (nbv >= 2 && b1 < ratio * ratio * b2) : nbv >= 1;
        if (delta_s > 0 && isfinite(delta_s)) ok = ok && sqrt(b1) < delta_s;
        if (ok) match[q] = (int32_t)j1;
    }
    return 0;
}

/* ------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon et al., SC'11): ten rounds of two 32x32->64
 * multiplications with a Weyl-sequence key schedule. */
void or_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int r = 0; r < 10; ++r) {
        if (r > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        uint64_t p0 = (uint64_t)0xD2511F53u * c0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
        c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* RANSAC's random draw (Fischler & Bolles; the paper cites RANSAC in
 * Sec. 2.5 without details).  Reading: iteration t draws four distinct match
 * indices from a Philox stream keyed by (lo32(seed), hi32(seed) ^ pair_id)
 * with counter (t, block, 0, 0); word j of the stream is word j%4 of block
 * j/4; index = floor(word * M / 2^32); repeated indices are redrawn, at most
 * 64 words per iteration, after which the iteration is skipped. */
int or_ransac_sample_k(int64_t M, uint64_t seed, uint32_t pair_id, int t, int k, int32_t* idx)
{
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32) ^ pair_id};
    uint32_t blk[4];
    int n = 0;
    for (int j = 0; j < 64 && n < k; ++j) {
        if (j % 4 == 0) {
            uint32_t ctr[4] = {(uint32_t)t, (uint32_t)(j / 4), 0u, 0u};
            or_philox4x32_10(ctr, key, blk);
        }
        int32_t i = (int32_t)(((uint64_t)blk[j % 4] * (uint64_t)M) >> 32);
        int dup = 0;
        for (int q = 0; q < n; ++q) dup |= idx[q] == i;
        if (!dup) idx[n++] = i;
    }
    return n == k ? 0 : 1;
}

int or_ransac_sample(int64_t M, uint64_t seed, uint32_t pair_id, int t, int32_t* idx4)
{
    return or_ransac_sample_k(M, seed, pair_id, t, 4, idx4);
}

/* Hartley normalisation: centroid to 0, mean distance to sqrt(2). */
static int hartley(const double* p, int stride, int n, double T[9])
{
    double cx = 0, cy = 0;
    for (int i = 0; i < n; ++i) { cx += p[i * stride]; cy += p[i * stride + 1]; }
    cx /= n; cy /= n;
    double md = 0;
    for (int i = 0; i < n; ++i) {
        double dx = p[i * stride] - cx, dy = p[i * stride + 1] - cy;
        md += sqrt(dx * dx + dy * dy);
    }
    md /= n;
    if (!(md > 0)) return 1;
    double s = sqrt(2.0) / md;
    T[0] = s; T[1] = 0; T[2] = -s * cx;
    T[3] = 0; T[4] = s; T[5] = -s * cy;
    T[6] = 0; T[7] = 0; T[8] = 1;
    return 0;
}

static void mat3_mul(const double* A, const double* B, double* C)
{
    double t[9];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double s = 0;
            for (int k = 0; k < 3; ++k) s += A[3 * i + k] * B[3 * k + j];
            t[3 * i + j] = s;
        }
    memcpy(C, t, sizeof t);
}

/* H = T_dst^-1 * Hn * T_src, scaled to h33 = 1. */
static int denormalise(const double* Ts, const double* Td, const double* Hn, double* H)
{
    double Tdi[9] = {1.0 / Td[0], 0, -Td[2] / Td[0], 0, 1.0 / Td[4], -Td[5] / Td[4], 0, 0, 1};
    double t[9];
    mat3_mul(Hn, Ts, t);
    mat3_mul(Tdi, t, H);
    double mx = 0;
    for (int i = 0; i < 9; ++i) mx = fmax(mx, fabs(H[i]));
    if (!(fabs(H[8]) > 1e-12 * mx)) return 1;
    double h = H[8];
    for (int i = 0; i < 9; ++i) H[i] /= h;
    return 0;
}

/* Eq. 7 from four correspondences: (x', y', 1)^T ~ H (x, y, 1)^T with h33 = 1,
 * an 8x8 linear system in normalised coordinates, solved by Gaussian
 * elimination with partial pivoting. */
int or_dlt4(const double* src, const double* dst, double* H)
{
    double Ts[9], Td[9];
    if (hartley(src, 2, 4, Ts) || hartley(dst, 2, 4, Td)) return 1;
    double A[8][9];
    for (int i = 0; i < 4; ++i) {
        double x = Ts[0] * src[2 * i] + Ts[2], y = Ts[4] * src[2 * i + 1] + Ts[5];
        double xp = Td[0] * dst[2 * i] + Td[2], yp = Td[4] * dst[2 * i + 1] + Td[5];
        double r0[9] = {x, y, 1, 0, 0, 0, -x * xp, -y * xp, xp};
        double r1[9] = {0, 0, 0, x, y, 1, -x * yp, -y * yp, yp};
        memcpy(A[2 * i], r0, sizeof r0);
        memcpy(A[2 * i + 1], r1, sizeof r1);
    }
    for (int c = 0; c < 8; ++c) {
        int p = c;
        for (int r = c + 1; r < 8; ++r)
            if (fabs(A[r][c]) > fabs(A[p][c])) p = r;
        if (!(fabs(A[p][c]) > 1e-10)) return 1;
        if (p != c)
            for (int j = 0; j < 9; ++j) { double t = A[c][j]; A[c][j] = A[p][j]; A[p][j] = t; }
        for (int r = c + 1; r < 8; ++r) {
            double f = A[r][c] / A[c][c];
            for (int j = c; j < 9; ++j) A[r][j] -= f * A[c][j];
        }
    }
    double h[9];
    for (int r = 7; r >= 0; --r) {
        double s = A[r][8];
        for (int j = r + 1; j < 8; ++j) s -= A[r][j] * h[j];
        h[r] = s / A[r][r];
    }
    h[8] = 1.0;
    return denormalise(Ts, Td, h, H);
}

/* Cyclic Jacobi rotations until the off-diagonal part vanishes. */
int or_eig_sym(int n, const double* Ain, double* evals, double* evecs)
{
    if (n <= 0 || n > 16) return -1;
    double a[16][16], v[16][16];
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) {
            a[i][j] = Ain[i * n + j];
            v[i][j] = i == j;
        }
    for (int sweep = 0; sweep < 100; ++sweep) {
        double off = 0, tot = 0;
        for (int i = 0; i < n; ++i)
            for (int j = 0; j < n; ++j) {
                tot += a[i][j] * a[i][j];
                if (i != j) off += a[i][j] * a[i][j];
            }
        if (off == 0 || off < 1e-30 * tot) break;
        for (int p = 0; p < n; ++p)
            for (int q = p + 1; q < n; ++q) {
                if (a[p][q] == 0) continue;
                double th = (a[q][q] - a[p][p]) / (2.0 * a[p][q]);
                double t = (th >= 0 ? 1.0 : -1.0) / (fabs(th) + sqrt(th * th + 1.0));
                double c = 1.0 / sqrt(t * t + 1.0), s = t * c;
                for (int k = 0; k < n; ++k) {
                    double akp = a[k][p], akq = a[k][q];
                    a[k][p] = c * akp - s * akq;
                    a[k][q] = s * akp + c * akq;
                }
                for (int k = 0; k < n; ++k) {
                    double apk = a[p][k], aqk = a[q][k];
                    a[p][k] = c * apk - s * aqk;
                    a[q][k] = s * apk + c * aqk;
                }
                for (int k = 0; k < n; ++k) {
                    double vkp = v[k][p], vkq = v[k][q];
                    v[k][p] = c * vkp - s * vkq;
                    v[k][q] = s * vkp + c * vkq;
                }
            }
    }
    /* selection sort, ascending */
    int ord[16];
    for (int i = 0; i < n; ++i) ord[i] = i;
    for (int i = 0; i < n; ++i)
        for (int j = i + 1; j < n; ++j)
            if (a[ord[j]][ord[j]] < a[ord[i]][ord[i]]) { int t = ord[i]; ord[i] = ord[j]; ord[j] = t; }
    for (int i = 0; i < n; ++i) {
        evals[i] = a[ord[i]][ord[i]];
        for (int k = 0; k < n; ++k) evecs[k * n + i] = v[k][ord[i]];
    }
    return 0;
}

/* Eq. 7 over all masked correspondences: minimise |A h| with |h| = 1 in
 * Hartley-normalised coordinates (the smallest eigenvector of A^T A), then
 * undo the normalisation and scale to h33 = 1. */
int or_refit(const double* pts, const uint8_t* mask, int64_t M, double* H)
{
    int64_t n = 0;
    for (int64_t i = 0; i < M; ++i) n += mask[i] != 0;
    if (n < 4) return 1;
    double* sa = (double*)malloc(sizeof(double) * 2 * n);
    double* sb = (double*)malloc(sizeof(double) * 2 * n);
    int64_t q = 0;
    for (int64_t i = 0; i < M; ++i)
        if (mask[i]) {
            sa[2 * q] = pts[4 * i]; sa[2 * q + 1] = pts[4 * i + 1];
            sb[2 * q] = pts[4 * i + 2]; sb[2 * q + 1] = pts[4 * i + 3];
            ++q;
        }
    double Ta[9], Tb[9];
    int bad = hartley(sa, 2, (int)n, Ta) || hartley(sb, 2, (int)n, Tb);
    double AtA[81];
    memset(AtA, 0, sizeof AtA);
    for (int64_t i = 0; i < n && !bad; ++i) {
        double x = Ta[0] * sa[2 * i] + Ta[2], y = Ta[4] * sa[2 * i + 1] + Ta[5];
        double xp = Tb[0] * sb[2 * i] + Tb[2], yp = Tb[4] * sb[2 * i + 1] + Tb[5];
        double r0[9] = {-x, -y, -1, 0, 0, 0, x * xp, y * xp, xp};
        double r1[9] = {0, 0, 0, -x, -y, -1, x * yp, y * yp, yp};
        for (int j = 0; j < 9; ++j)
            for (int k = 0; k < 9; ++k) AtA[9 * j + k] += r0[j] * r0[k] + r1[j] * r1[k];
    }
    free(sa);
    free(sb);
    if (bad) return 1;
    double ev[9], V[81], h[9];
    or_eig_sym(9, AtA, ev, V);
    for (int j = 0; j < 9; ++j) h[j] = V[9 * j + 0];
    return denormalise(Ta, Tb, h, H);
}

/* Reprojection error in the registered image, e^2 = |pi(H p_A) - p_B|^2;
 * a point is an inlier when e < thresh; a point projected to w <= 0 is not. */
int64_t or_score(const double* H, const double* pts, int64_t M, double thresh, uint8_t* mask)
{
    int64_t n = 0;
    double t2 = thresh * thresh;
    for (int64_t i = 0; i < M; ++i) {
        double x = pts[4 * i], y = pts[4 * i + 1];
        double w = H[6] * x + H[7] * y + H[8];
        int in = 0;
        if (w > 0) {
            double u = (H[0] * x + H[1] * y + H[2]) / w - pts[4 * i + 2];
            double v = (H[3] * x + H[4] * y + H[5]) / w - pts[4 * i + 3];
            in = u * u + v * v < t2;
        }
        if (mask) mask[i] = (uint8_t)in;
        n += in;
    }
    return n;
}

/* |cross(q - p, r - p)| relative to the spread: three points on one line. */
static int collinear(const double* p, const double* q, const double* r)
{
    double ux = q[0] - p[0], uy = q[1] - p[1], vx = r[0] - p[0], vy = r[1] - p[1];
    double cr = ux * vy - uy * vx;
    return fabs(cr) <= 1e-9 * (ux * ux + uy * uy + vx * vx + vy * vy);
}

/* Eq. 8 by least squares: the rotation theta and translation (t_x, t_y) that
 * minimise sum |R(theta) p_A + t - p_B|^2 over the masked correspondences.
 * With a and b the coordinates minus their centroids, the sum equals a
 * constant minus 2 (cos(theta) C + sin(theta) S), C = sum a.b and
 * S = sum (a_x b_y - a_y b_x), so (cos, sin) = (C, S) / sqrt(C^2 + S^2), and
 * t = centroid_B - R centroid_A.  Two correspondences give the minimal sample
 * of the rigid model.  Returns 0, or 1 for fewer than two correspondences or
 * C = S = 0 (all points of one image on one spot). */
int or_rigid_fit(const double* pts, const uint8_t* mask, int64_t M, double* H)
{
    int64_t n = 0;
    double sxa = 0, sya = 0, sxb = 0, syb = 0;
    for (int64_t i = 0; i < M; ++i)
        if (mask[i]) {
            ++n;
            sxa += pts[4 * i]; sya += pts[4 * i + 1]; sxb += pts[4 * i + 2]; syb += pts[4 * i + 3];
        }
    if (n < 2) return 1;
    const double cxa = sxa / n, cya = sya / n, cxb = sxb / n, cyb = syb / n;
    double Cs = 0, Ss = 0;
    for (int64_t i = 0; i < M; ++i)
        if (mask[i]) {
            const double ax = pts[4 * i] - cxa, ay = pts[4 * i + 1] - cya;
            const double bx = pts[4 * i + 2] - cxb, by = pts[4 * i + 3] - cyb;
            Cs += ax * bx + ay * by;
            Ss += ax * by - ay * bx;
        }
    const double r = sqrt(Cs * Cs + Ss * Ss);
    if (!(r > 0)) return 1;
    const double c = Cs / r, sn = Ss / r;
    H[0] = c;  H[1] = -sn; H[2] = cxb - (c * cxa - sn * cya);
    H[3] = sn; H[4] = c;   H[5] = cyb - (sn * cxa + c * cya);
    H[6] = 0;  H[7] = 0;   H[8] = 1;
    return 0;
}

int or_model_sample_size(int model) { return model == OR_MODEL_RIGID ? 2 : 4; }

/* The hypothesis of one minimal sample s[] (Sec. 2.5).  Eq. 7: four
 * correspondences by the DLT, skipped when three of them are collinear in
 * either image.  Eq. 8: two correspondences by or_rigid_fit.  Returns 0, or 1
 * when the sample is degenerate. */
static int hypothesis(int model, const double* pts, const int32_t* s, double* Ht)
{
    if (model == OR_MODEL_RIGID) {
        double sub[8];
        const uint8_t both[2] = {1, 1};
        for (int j = 0; j < 2; ++j) memcpy(sub + 4 * j, pts + 4 * (size_t)s[j], sizeof(double) * 4);
        return or_rigid_fit(sub, both, 2, Ht);
    }
    double src[8], dst[8];
    for (int j = 0; j < 4; ++j) {
        src[2 * j] = pts[4 * s[j]]; src[2 * j + 1] = pts[4 * s[j] + 1];
        dst[2 * j] = pts[4 * s[j] + 2]; dst[2 * j + 1] = pts[4 * s[j] + 3];
    }
    for (int a = 0; a < 4; ++a) {
        int i0 = (a + 1) % 4, i1 = (a + 2) % 4, i2 = (a + 3) % 4;
        if (collinear(src + 2 * i0, src + 2 * i1, src + 2 * i2) || collinear(dst + 2 * i0, dst + 2 * i1, dst + 2 * i2))
            return 1;
    }
    return or_dlt4(src, dst, Ht);
}

/* Least-squares fit of the model to the masked correspondences. */
static int refit_model(int model, const double* pts, const uint8_t* mask, int64_t M, double* H)
{
    return model == OR_MODEL_RIGID ? or_rigid_fit(pts, mask, M, H) : or_refit(pts, mask, M, H);
}

/* Sec. 2.5: RANSAC over the matched pairs with the homography of Eq. 7.
 * Readings: a full 8-DOF homography (Eq. 8's rigid form is a special case);
 * T iterations (no adaptive stop); a sample with three collinear points in
 * either image, or a singular system, is skipped; the hypothesis with the most
 * inliers wins, the earliest on ties; the winner's inliers are refitted once
 * by least squares, and the final inlier set is taken from the refitted H.
 * or_ransac_model runs the same loop with Eq. 8's rigid model, drawing two
 * matches per iteration (the first two distinct indices of the same stream). */
int or_ransac_model(const double* pts, int64_t M, int model, int T, double thresh, uint64_t seed, uint32_t pair_id,
                    double* H, uint8_t* inl, int32_t* n_in, int32_t* best_t, int32_t* counts, double* Hs)
{
    const int k = or_model_sample_size(model);
    memset(H, 0, sizeof(double) * 9);
    *n_in = 0;
    *best_t = -1;
    if (inl) memset(inl, 0, (size_t)M);
    if (counts)
        for (int t = 0; t < T; ++t) counts[t] = -1;
    if (Hs) memset(Hs, 0, sizeof(double) * 9 * (size_t)T);
    if (M < k) return 1;
    int64_t bestc = -1;
    double Hb[9];
    for (int t = 0; t < T; ++t) {
        int32_t s[4];
        if (or_ransac_sample_k(M, seed, pair_id, t, k, s)) continue;
        double Ht[9];
        if (hypothesis(model, pts, s, Ht)) continue;
        int64_t c = or_score(Ht, pts, M, thresh, NULL);
        if (counts) counts[t] = (int32_t)c;
        if (Hs) memcpy(Hs + 9 * t, Ht, sizeof Ht);
        if (c > bestc) {
            bestc = c;
            *best_t = t;
            memcpy(Hb, Ht, sizeof Hb);
        }
    }
    if (bestc < 0) return 1;
    uint8_t* m = (uint8_t*)malloc((size_t)M);
    or_score(Hb, pts, M, thresh, m);
    double Hf[9];
    if (refit_model(model, pts, m, M, Hf)) memcpy(Hf, Hb, sizeof Hf);
    *n_in = (int32_t)or_score(Hf, pts, M, thresh, m);
    if (inl) memcpy(inl, m, (size_t)M);
    free(m);
    memcpy(H, Hf, sizeof Hf);
    return 0;
}

int or_ransac(const double* pts, int64_t M, int T, double thresh, uint64_t seed, uint32_t pair_id,
              double* H, uint8_t* inl, int32_t* n_in, int32_t* best_t, int32_t* counts, double* Hs)
{
    return or_ransac_model(pts, M, OR_MODEL_HOMOGRAPHY, T, thresh, seed, pair_id, H, inl, n_in, best_t, counts, Hs);
}

/* ------------------------------------------------------------------ */
/* Learned RANSAC proposal (not in the paper).  A small network scores each
 * tentative match; RANSAC then draws its samples with probability
 * proportional to the score.  The scoring of hypotheses is unchanged, so the
 * winner is still judged by all matches. */

/* Features of one match: the ratio-test quantities, the scale of the
 * reference point, the orientation difference and both positions. */
int or_mlp_features(int64_t M, const double* d1, const double* d2, const int32_t* LA, int Lmax,
                    const uint8_t* oriA, const uint8_t* oriB, const double* pts, int WA, int HA, int WB, int HB,
                    double* feat)
{
    if (M < 0 || Lmax < 2) return -1;
    for (int64_t i = 0; i < M; ++i) {
        double* f = feat + 8 * i;
        f[0] = d2[i] > 0 ? d1[i] / d2[i] : 1.0;
        f[1] = d1[i];
        f[2] = log2((double)LA[i]) / log2((double)Lmax);
        int dk = ((int)oriB[i] - (int)oriA[i]) % 36;
        if (dk < 0) dk += 36;
        double dth = 10.0 * dk;                 /* degrees in [0, 360) */
        if (dth >= 180.0) dth -= 360.0;         /* [-180, 180) */
        f[3] = dth / 180.0;
        f[4] = pts[4 * i] / WA;
        f[5] = pts[4 * i + 1] / HA;
        f[6] = pts[4 * i + 2] / WB;
        f[7] = pts[4 * i + 3] / HB;
    }
    return 0;
}

static double sigmoid(double z)
{
    if (z >= 0) return 1.0 / (1.0 + exp(-z));
    double e = exp(z);
    return e / (1.0 + e);
}

/* One forward pass, keeping the hidden activations. */
static double mlp_fwd1(const double* P, const double* x, double* h1, double* h2)
{
    const double *W1 = P, *b1 = P + 512, *W2 = P + 576, *b2 = P + 4672, *w3 = P + 4736, *b3 = P + 4800;
    for (int i = 0; i < 64; ++i) {
        double s = b1[i];
        for (int j = 0; j < 8; ++j) s += W1[8 * i + j] * x[j];
        h1[i] = s > 0 ? s : 0;
    }
    for (int i = 0; i < 64; ++i) {
        double s = b2[i];
        for (int j = 0; j < 64; ++j) s += W2[64 * i + j] * h1[j];
        h2[i] = s > 0 ? s : 0;
    }
    double z = b3[0];
    for (int j = 0; j < 64; ++j) z += w3[j] * h2[j];
    return z;
}

int or_mlp_forward(const double* params, const double* x, int64_t M, double* logit, double* prob)
{
    double h1[64], h2[64];
    for (int64_t i = 0; i < M; ++i) {
        double z = mlp_fwd1(params, x + 8 * i, h1, h2);
        if (logit) logit[i] = z;
        if (prob) prob[i] = sigmoid(z);
    }
    return 0;
}

/* L = (1/B) sum_i max(z_i, 0) - z_i y_i + log(1 + exp(-|z_i|)); dL/dz_i =
 * (sigmoid(z_i) - y_i) / B, propagated back through the two ReLU layers. */
int or_mlp_loss_grad(const double* params, const double* x, const uint8_t* y, int64_t B, double* loss, double* grad)
{
    if (B <= 0) return -1;
    const double *W2 = params + 576, *w3 = params + 4736;
    double *gW1 = grad, *gb1 = grad + 512, *gW2 = grad + 576, *gb2 = grad + 4672, *gw3 = grad + 4736, *gb3 = grad + 4800;
    memset(grad, 0, sizeof(double) * OR_MLP_NPARAM);
    double L = 0;
    for (int64_t n = 0; n < B; ++n) {
        const double* xn = x + 8 * n;
        double h1[64], h2[64], d2[64], d1[64];
        double z = mlp_fwd1(params, xn, h1, h2);
        double yn = y[n] ? 1.0 : 0.0;
        L += (z > 0 ? z : 0) - z * yn + log1p(exp(-fabs(z)));
        double dz = (sigmoid(z) - yn) / (double)B;
        gb3[0] += dz;
        for (int j = 0; j < 64; ++j) {
            gw3[j] += dz * h2[j];
            d2[j] = h2[j] > 0 ? dz * w3[j] : 0;
        }
        for (int i = 0; i < 64; ++i) {
            gb2[i] += d2[i];
            for (int j = 0; j < 64; ++j) gW2[64 * i + j] += d2[i] * h1[j];
        }
        for (int j = 0; j < 64; ++j) {
            double s = 0;
            for (int i = 0; i < 64; ++i) s += W2[64 * i + j] * d2[i];
            d1[j] = h1[j] > 0 ? s : 0;
        }
        for (int i = 0; i < 64; ++i) {
            gb1[i] += d1[i];
            for (int j = 0; j < 8; ++j) gW1[8 * i + j] += d1[i] * xn[j];
        }
    }
    if (loss) *loss = L / (double)B;
    return 0;
}

/* Adam (Kingma & Ba): bias-corrected first and second moments. */
int or_mlp_adam(double* params, double* m, double* v, const double* grad, int n, int t, double lr, double b1,
                double b2, double eps)
{
    if (t < 1) return -1;
    double c1 = 1.0 - pow(b1, t), c2 = 1.0 - pow(b2, t);
    for (int i = 0; i < n; ++i) {
        m[i] = b1 * m[i] + (1 - b1) * grad[i];
        v[i] = b2 * v[i] + (1 - b2) * grad[i] * grad[i];
        params[i] -= lr * (m[i] / c1) / (sqrt(v[i] / c2) + eps);
    }
    return 0;
}

/* Guided sampling weights: q_i = round(65536 * max(p_i, 1e-3)) with p_i the
 * FP32 prior and 1e-3 the FP32 constant, as integers (no rounding can differ
 * between implementations); prefix holds the inclusive prefix sums. */
int or_guided_weights(const float* prob, int64_t M, uint64_t* prefix)
{
    uint64_t acc = 0;
    for (int64_t i = 0; i < M; ++i) {
        double p = (double)prob[i];
        double lo = (double)1e-3f;
        if (!(p > lo)) p = lo;      /* also maps NaN to the floor */
        acc += (uint64_t)floor(65536.0 * p + 0.5);
        prefix[i] = acc;
    }
    return 0;
}

/* Word j of iteration t's Philox stream (as or_ransac_sample) picks the
 * match whose prefix interval contains floor(word * total / 2^32): probability
 * proportional to q_i.  Repeated indices are redrawn (sampling without
 * replacement), at most 64 words. */
int or_ransac_sample_guided_k(int64_t M, const uint64_t* prefix, uint64_t seed, uint32_t pair_id, int t, int k,
                               int32_t* idx)
{
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32) ^ pair_id};
    uint32_t blk[4];
    const uint64_t total = prefix[M - 1];
    int n = 0;
    for (int j = 0; j < 64 && n < k; ++j) {
        if (j % 4 == 0) {
            uint32_t ctr[4] = {(uint32_t)t, (uint32_t)(j / 4), 0u, 0u};
            or_philox4x32_10(ctr, key, blk);
        }
        uint64_t target = (uint64_t)(((unsigned __int128)blk[j % 4] * total) >> 32);
        int64_t lo = 0, hi = M - 1;   /* first i with prefix[i] > target */
        while (lo < hi) {
            int64_t mid = (lo + hi) / 2;
            if (prefix[mid] > target) hi = mid; else lo = mid + 1;
        }
        int32_t i = (int32_t)lo;
        int dup = 0;
        for (int q = 0; q < n; ++q) dup |= idx[q] == i;
        if (!dup) idx[n++] = i;
    }
    return n == k ? 0 : 1;
}

int or_ransac_sample_guided(int64_t M, const uint64_t* prefix, uint64_t seed, uint32_t pair_id, int t, int32_t* idx4)
{
    return or_ransac_sample_guided_k(M, prefix, seed, pair_id, t, 4, idx4);
}

/* Stop test of the guided phase: the standard RANSAC bound T >= log(0.01) /
 * log(1 - w^k), rewritten as (1 - w^k)^T <= 0.01 (the chance that T samples
 * of k matches all contained an outlier), with w the prior-weighted inlier
 * fraction s_in / total of the guided winner: the probability that one guided
 * draw lands on an inlier.  k = 4 for Eq. 7, 2 for Eq. 8.  Powers by binary
 * exponentiation. */
int or_guided_stop_k(uint64_t s_in, uint64_t total, int Tg, int k)
{
    if (total == 0 || Tg <= 0 || (k != 2 && k != 4)) return 0;
    const double w = (double)s_in / (double)total;
    const double w2 = w * w;
    const double wk = k == 2 ? w2 : w2 * w2;
    double b = 1.0 - wk, r = 1.0;
    for (int e = Tg; e; e >>= 1) {
        if (e & 1) r = r * b;
        b = b * b;
    }
    return r <= 0.01;
}

int or_guided_stop(uint64_t s_in, uint64_t total, int Tg) { return or_guided_stop_k(s_in, total, Tg, 4); }

/* Learned-proposal RANSAC: Tg hypotheses from guided samples are scored by all
 * matches; when the stop test holds for the guided winner and the winner has at
 * least min_support inliers and an unweighted inlier fraction for which the
 * same bound holds, it is refitted as in or_ransac; otherwise the call
 * falls back to uniform RANSAC with T iterations (or_ransac itself, whose
 * best_t is reported offset by Tg).  The support floor keeps a prior that
 * concentrates on a handful of matches (any four of which fit a homography
 * exactly) from ending the search on them. */
int or_ransac_prior_model(const double* pts, int64_t M, int model, const float* prob, int Tg, int T, double thresh,
                          uint64_t seed, uint32_t pair_id, int min_support, double* H, uint8_t* inl, int32_t* n_in,
                          int32_t* best_t, int32_t* iters, int32_t* counts /* Tg + T or NULL */)
{
    const int k = or_model_sample_size(model);
    memset(H, 0, sizeof(double) * 9);
    *n_in = 0;
    *best_t = -1;
    *iters = Tg + T;
    if (inl) memset(inl, 0, (size_t)(M > 0 ? M : 0));
    if (counts)
        for (int t = 0; t < Tg + T; ++t) counts[t] = -1;
    int64_t bestc = -1;
    double Hb[9];
    int tg = -1;
    uint64_t* prefix = NULL;
    if (M >= k) {
        prefix = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)M);
        or_guided_weights(prob, M, prefix);
        for (int t = 0; t < Tg; ++t) {
            int32_t s[4];
            if (or_ransac_sample_guided_k(M, prefix, seed, pair_id, t, k, s)) continue;
            double Ht[9];
            if (hypothesis(model, pts, s, Ht)) continue;
            int64_t c = or_score(Ht, pts, M, thresh, NULL);
            if (counts) counts[t] = (int32_t)c;
            if (c > bestc) {
                bestc = c;
                tg = t;
                memcpy(Hb, Ht, sizeof Hb);
            }
        }
    }
    int stop = 0;
    uint8_t* m = (uint8_t*)malloc((size_t)(M > 0 ? M : 1));
    if (tg >= 0) {
        or_score(Hb, pts, M, thresh, m);
        uint64_t s_in = 0;
        for (int64_t i = 0; i < M; ++i)
            if (m[i]) s_in += prefix[i] - (i ? prefix[i - 1] : 0);
        stop = or_guided_stop_k(s_in, prefix[M - 1], Tg, k) && bestc >= (int64_t)min_support &&
               or_guided_stop_k((uint64_t)bestc, (uint64_t)M, Tg, k);
    }
    free(prefix);
    if (!stop) {
        free(m);
        int32_t bt;
        int r = or_ransac_model(pts, M, model, T, thresh, seed, pair_id, H, inl, n_in, &bt, counts ? counts + Tg : NULL,
                                NULL);
        *best_t = bt >= 0 ? Tg + bt : -1;
        return r;
    }
    *iters = Tg;
    *best_t = tg;
    double Hf[9];
    if (refit_model(model, pts, m, M, Hf)) memcpy(Hf, Hb, sizeof Hf);
    *n_in = (int32_t)or_score(Hf, pts, M, thresh, m);
    if (inl) memcpy(inl, m, (size_t)M);
    free(m);
    memcpy(H, Hf, sizeof Hf);
    return 0;
}

int or_ransac_prior(const double* pts, int64_t M, const float* prob, int Tg, int T, double thresh, uint64_t seed,
                    uint32_t pair_id, int min_support, double* H, uint8_t* inl, int32_t* n_in, int32_t* best_t,
                    int32_t* iters, int32_t* counts)
{
    return or_ransac_prior_model(pts, M, OR_MODEL_HOMOGRAPHY, prob, Tg, T, thresh, seed, pair_id, min_support, H, inl,
                                 n_in, best_t, iters, counts);
}

/* ------------------------------------------------------------------ */
/* Sec. 4 mosaic: rounds of reference selection over H_M, then every placed
 * image warped onto one canvas.
 * Readings:
 *  - the degree of an image is its number of valid H_M entries;
 *  - round 1: the reference is the image of largest degree (lowest index on
 *    ties); it is placed with the identity, every image matched with it is
 *    placed through their H_M entry;
 *  - round k > 1: among unmatched images with a valid entry to a placed image,
 *    the one of largest degree (lowest index on ties) is the reference; it is
 *    placed through its valid entry to the placed image of lowest index, then
 *    its unmatched neighbours through it;
 *  - images that never connect stay unplaced (round -1).
 * H_M entry q of pair (a, b) maps image a pixels to image b pixels
 * (x_b ~ H x_a, Eq. 7); the placement G_i maps image i pixels to the
 * reference frame of round 1.  The canvas is the integer bounding box of the
 * placed images' corner pixels; G is returned with the canvas shift applied. */

static int inv3(const double* M, double* R)
{
    const double c00 = M[4] * M[8] - M[5] * M[7], c01 = M[5] * M[6] - M[3] * M[8], c02 = M[3] * M[7] - M[4] * M[6];
    const double det = M[0] * c00 + M[1] * c01 + M[2] * c02;
    if (!(fabs(det) > 0)) return 1;
    R[0] = c00 / det; R[1] = (M[2] * M[7] - M[1] * M[8]) / det; R[2] = (M[1] * M[5] - M[2] * M[4]) / det;
    R[3] = c01 / det; R[4] = (M[0] * M[8] - M[2] * M[6]) / det; R[5] = (M[2] * M[3] - M[0] * M[5]) / det;
    R[6] = c02 / det; R[7] = (M[1] * M[6] - M[0] * M[7]) / det; R[8] = (M[0] * M[4] - M[1] * M[3]) / det;
    return 0;
}

/* map of image `from` into image `to` (x_to ~ M x_from) from entry q */
static int pair_map(const int32_t* pairs, const double* HM, int q, int from, double* M)
{
    if (pairs[2 * q] == from) { memcpy(M, HM + 9 * q, sizeof(double) * 9); return 0; }
    return inv3(HM + 9 * q, M);
}

int or_mosaic_plan(int N, const int32_t* pairs, int P, const double* HM, const uint8_t* valid, const int* Hs,
                   const int* Ws, double* G, int32_t* round_of, int32_t* ref_of, int* canvas_w, int* canvas_h)
{
    if (N < 1 || P < 0) return -1;
    int* deg = (int*)calloc((size_t)N, sizeof(int));
    for (int q = 0; q < P; ++q)
        if (valid[q]) { deg[pairs[2 * q]]++; deg[pairs[2 * q + 1]]++; }
    for (int i = 0; i < N; ++i) { round_of[i] = -1; ref_of[i] = -1; }
    double* Gr = (double*)calloc((size_t)N * 9, sizeof(double));
    int placed = 0;
    for (int rnd = 0; placed < N; ++rnd) {
        int ref = -1, via = -1;
        for (int i = 0; i < N; ++i) {
            if (round_of[i] >= 0) continue;
            int link = -1;
            if (rnd > 0)
                for (int q = 0; q < P; ++q) {
                    if (!valid[q]) continue;
                    int o = pairs[2 * q] == i ? pairs[2 * q + 1] : (pairs[2 * q + 1] == i ? pairs[2 * q] : -1);
                    if (o >= 0 && round_of[o] >= 0 && (link < 0 || o < pairs[2 * link] + pairs[2 * link + 1] - i))
                        link = q;
                }
            if (rnd > 0 && link < 0) continue;
            if (ref < 0 || deg[i] > deg[ref]) { ref = i; via = link; }
        }
        if (ref < 0) break;
        if (rnd == 0) {
            for (int k = 0; k < 9; ++k) Gr[9 * ref + k] = (k % 4 == 0) ? 1.0 : 0.0;
        } else {
            const int o = pairs[2 * via] == ref ? pairs[2 * via + 1] : pairs[2 * via];
            double M[9];
            if (pair_map(pairs, HM, via, ref, M)) break;          /* ref -> o */
            mat3_mul(Gr + 9 * o, M, Gr + 9 * ref);
        }
        round_of[ref] = rnd; ref_of[ref] = ref; ++placed;
        for (int q = 0; q < P; ++q) {
            if (!valid[q]) continue;
            int j = pairs[2 * q] == ref ? pairs[2 * q + 1] : (pairs[2 * q + 1] == ref ? pairs[2 * q] : -1);
            if (j < 0 || round_of[j] >= 0) continue;
            double M[9];
            if (pair_map(pairs, HM, q, j, M)) continue;            /* j -> ref */
            mat3_mul(Gr + 9 * ref, M, Gr + 9 * j);
            round_of[j] = rnd; ref_of[j] = ref; ++placed;
        }
    }
    double x0 = INFINITY, y0 = INFINITY, x1 = -INFINITY, y1 = -INFINITY;
    for (int i = 0; i < N; ++i) {
        if (round_of[i] < 0) continue;
        const double cx[4] = {0, Ws[i] - 1.0, 0, Ws[i] - 1.0}, cy[4] = {0, 0, Hs[i] - 1.0, Hs[i] - 1.0};
        for (int c = 0; c < 4; ++c) {
            const double* g = Gr + 9 * i;
            const double w = g[6] * cx[c] + g[7] * cy[c] + g[8];
            const double x = (g[0] * cx[c] + g[1] * cy[c] + g[2]) / w, y = (g[3] * cx[c] + g[4] * cy[c] + g[5]) / w;
            x0 = fmin(x0, x); x1 = fmax(x1, x); y0 = fmin(y0, y); y1 = fmax(y1, y);
        }
    }
    const double fx = floor(x0), fy = floor(y0);
    *canvas_w = placed ? (int)(ceil(x1) - fx) + 1 : 0;
    *canvas_h = placed ? (int)(ceil(y1) - fy) + 1 : 0;
    const double T[9] = {1, 0, -fx, 0, 1, -fy, 0, 0, 1};
    for (int i = 0; i < N; ++i) {
        if (round_of[i] < 0) { memset(G + 9 * i, 0, sizeof(double) * 9); continue; }
        mat3_mul(T, Gr + 9 * i, G + 9 * i);
    }
    free(deg);
    free(Gr);
    return 0;
}

/* Canvas pixel (x, y): every placed image i whose inverse placement maps the
 * pixel inside [0, W-1] x [0, H-1] (w > 0) contributes its bilinear sample;
 * the canvas value is the mean, rounded half up, and 0 where nothing covers;
 * cover[] counts the contributions. */
int or_mosaic_render(int N, const uint8_t* const* imgs, const int* Hs, const int* Ws, const int* pitches, int C,
                     const double* G, const int32_t* round_of, int cw, int ch, uint8_t* canvas, uint8_t* cover)
{
    double* Gi = (double*)malloc(sizeof(double) * 9 * (size_t)(N > 0 ? N : 1));
    for (int i = 0; i < N; ++i)
        if (round_of[i] >= 0 && inv3(G + 9 * i, Gi + 9 * i)) { free(Gi); return -1; }
    for (int y = 0; y < ch; ++y)
        for (int x = 0; x < cw; ++x) {
            double sum[4] = {0, 0, 0, 0};
            int n = 0;
            for (int i = 0; i < N; ++i) {
                if (round_of[i] < 0) continue;
                const double* m = Gi + 9 * i;
                const double w = m[6] * x + m[7] * y + m[8];
                if (!(w > 0)) continue;
                const double u = (m[0] * x + m[1] * y + m[2]) / w, v = (m[3] * x + m[4] * y + m[5]) / w;
                if (!(u >= 0 && v >= 0 && u <= Ws[i] - 1 && v <= Hs[i] - 1)) continue;
                const int u0 = (int)floor(u), v0 = (int)floor(v);
                const int u1 = u0 + 1 < Ws[i] ? u0 + 1 : u0, v1 = v0 + 1 < Hs[i] ? v0 + 1 : v0;
                const double fu = u - u0, fv = v - v0;
                for (int c = 0; c < C; ++c) {
                    const uint8_t* I = imgs[i];
                    const double p00 = I[(size_t)v0 * pitches[i] + (size_t)u0 * C + c];
                    const double p01 = I[(size_t)v0 * pitches[i] + (size_t)u1 * C + c];
                    const double p10 = I[(size_t)v1 * pitches[i] + (size_t)u0 * C + c];
                    const double p11 = I[(size_t)v1 * pitches[i] + (size_t)u1 * C + c];
                    const double top = p00 + fu * (p01 - p00), bot = p10 + fu * (p11 - p10);
                    sum[c] += top + fv * (bot - top);
                }
                ++n;
            }
            for (int c = 0; c < C; ++c) canvas[((size_t)y * cw + x) * C + c] = n ? (uint8_t)floor(sum[c] / n + 0.5) : 0;
            if (cover) cover[(size_t)y * cw + x] = (uint8_t)n;
        }
    free(Gi);
    return 0;
}
