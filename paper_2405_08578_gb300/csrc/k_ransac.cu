// Matched-pair compaction and RANSAC homography estimation (Sec. 2.4-2.5,
// Eq. 7) for sm_103a.
//
//  k_compact_count / k_compact_write  stable compaction of accepted rows into
//                 (xA, yA, xB, yB), tiles of 2048 rows: per-tile counts, then
//                 each tile adds the counts before it and writes in row order
//  k_ransac_hyp   eight lanes per iteration t: Philox4x32-10 draw of 4 distinct
//                 matches, collinearity test, Hartley normalisation, and the
//                 8x9 DLT system solved in FP64 with one row per lane (partial
//                 pivoting by warp shuffles, row-parallel back substitution)
//  k_ransac_score one CTA per hypothesis: FP32 reprojection errors; counts of
//                 points certainly inside (e^2 < t^2 - eps) and possibly inside
//                 (e^2 < t^2 + eps); the largest certain count c* by atomicMax
//  k_ransac_recount one CTA per hypothesis whose possible count reaches c*:
//                 the points in the band are re-tested in FP64, giving the
//                 exact FP64 inlier count
//  k_ransac_argmax most exact inliers, earliest t
//  k_refit_*      least-squares refit of the winner's FP64 inliers (Eq. 7):
//                 per-CTA partial sums reduced in a fixed order, the 9x9
//                 normal matrix's smallest eigenvector by Cholesky and shifted
//                 inverse iteration on one warp, denormalisation, final mask
#include <math.h>

#include <algorithm>

#include "lp_internal.cuh"

namespace lp {
namespace {

// ---------------------------------------------------------------- Philox
// Philox4x32-10 (Salmon, Moraes, Dror & Shaw, SC'11): ten rounds; each round
// multiplies words 0 and 2 by fixed odd constants (high/low halves), xors the
// high halves with words 1/3 and the round key; the key advances by the Weyl
// constants between rounds.
__device__ __forceinline__ uint4 philox(uint4 c, uint32_t k0, uint32_t k1)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
        const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
        c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return c;
}

__global__ void k_diag_philox(const uint4* ctr, long long n, uint32_t k0, uint32_t k1, uint4* out)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = philox(ctr[i], k0, k1);
}

// ---------------------------------------------------------------- compaction
constexpr int kCompactThreads = 256;
constexpr int kCompactPer = 8;                                  // consecutive rows per thread
constexpr int kCompactRows = kCompactThreads * kCompactPer;    // rows per tile

__device__ __forceinline__ int compact_rows(const int32_t* match, long long NA, long long r0, int (&m)[kCompactPer])
{
    int c = 0;
#pragma unroll
    for (int k = 0; k < kCompactPer; ++k) {
        const long long i = r0 + k;
        m[k] = i < NA ? match[i] : -1;
        c += m[k] >= 0;
    }
    return c;
}

// exclusive prefix of v over the CTA (thread order) and the CTA total
__device__ __forceinline__ int compact_scan(int v, int* wsum, int& total)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int u = __shfl_up_sync(0xFFFFFFFFu, incl, o);
        if (lane >= o) incl += u;
    }
    if (lane == 31) wsum[warp] = incl;
    __syncthreads();
    int before = 0;
    total = 0;
#pragma unroll
    for (int w = 0; w < kCompactThreads / 32; ++w) {
        const int x = wsum[w];
        before += w < warp ? x : 0;
        total += x;
    }
    return before + incl - v;
}

__global__ void __launch_bounds__(kCompactThreads)
k_compact_count(const int32_t* match, long long NA, int32_t* tile_cnt)
{
    __shared__ int wsum[kCompactThreads / 32];
    int m[kCompactPer];
    const long long r0 = (long long)blockIdx.x * kCompactRows + (long long)threadIdx.x * kCompactPer;
    int total;
    compact_scan(compact_rows(match, NA, r0, m), wsum, total);
    if (threadIdx.x == 0) tile_cnt[blockIdx.x] = total;
}

__global__ void __launch_bounds__(kCompactThreads)
k_compact_write(const uint32_t* kpA, int WA, const uint32_t* kpB, int WB, const int32_t* match, long long NA,
                const int32_t* tile_cnt, float4* pts, int32_t* rows, int32_t* dM)
{
    __shared__ int wsum[kCompactThreads / 32];
    __shared__ int before_s;
    int pre = 0;
    for (int b = threadIdx.x; b < (int)blockIdx.x; b += kCompactThreads) pre += tile_cnt[b];
    int tot_pre;
    compact_scan(pre, wsum, tot_pre);
    if (threadIdx.x == 0) before_s = tot_pre;
    __syncthreads();
    const int before = before_s;
    int m[kCompactPer];
    const long long r0 = (long long)blockIdx.x * kCompactRows + (long long)threadIdx.x * kCompactPer;
    const int c = compact_rows(match, NA, r0, m);
    int total;
    int pos = before + compact_scan(c, wsum, total);
#pragma unroll
    for (int k = 0; k < kCompactPer; ++k) {
        const int j = m[k];
        if (j < 0) continue;
        const uint32_t ia = kpA[r0 + k], ib = kpB[j];
        const uint32_t ya = ia / (uint32_t)WA, yb = ib / (uint32_t)WB;
        pts[pos] = make_float4((float)(ia - ya * WA), (float)ya, (float)(ib - yb * WB), (float)yb);
        if (rows) rows[pos] = (int32_t)(r0 + k);
        ++pos;
    }
    if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) *dM = before + total;
}

// ---------------------------------------------------------------- FP64 model
__device__ __forceinline__ long long m_count(const int32_t* dM, long long M_cap)
{
    if (!dM) return M_cap;
    const long long m = *dM;
    return m < 0 ? 0 : (m > M_cap ? M_cap : m);
}

// |cross(q - p, r - p)| small relative to the spread: the three are on a line.
__device__ __forceinline__ bool collinear(double px, double py, double qx, double qy, double rx, double ry)
{
    const double ux = qx - px, uy = qy - py, vx = rx - px, vy = ry - py;
    return fabs(ux * vy - uy * vx) <= 1e-9 * (ux * ux + uy * uy + vx * vx + vy * vy);
}

struct Norm2D { double s, cx, cy; };

// centroid to the origin, mean distance sqrt(2)
__device__ bool hartley4(const double* x, const double* y, Norm2D& n)
{
    double cx = 0, cy = 0;
    for (int i = 0; i < 4; ++i) { cx += x[i]; cy += y[i]; }
    cx /= 4; cy /= 4;
    double md = 0;
    for (int i = 0; i < 4; ++i) md += sqrt((x[i] - cx) * (x[i] - cx) + (y[i] - cy) * (y[i] - cy));
    md /= 4;
    if (!(md > 0)) return false;
    n.s = sqrt(2.0) / md; n.cx = cx; n.cy = cy;
    return true;
}

// H = Tb^-1 * Hn * Ta with T = [[s, 0, -s cx], [0, s, -s cy], [0, 0, 1]], h33 -> 1.
__device__ bool denorm(const Norm2D& na, const Norm2D& nb, const double* hn, double* H)
{
    // Hn * Ta
    double t[9];
    for (int r = 0; r < 3; ++r) {
        t[3 * r + 0] = hn[3 * r + 0] * na.s;
        t[3 * r + 1] = hn[3 * r + 1] * na.s;
        t[3 * r + 2] = hn[3 * r + 2] - hn[3 * r + 0] * na.s * na.cx - hn[3 * r + 1] * na.s * na.cy;
    }
    // Tb^-1 = [[1/s, 0, cx], [0, 1/s, cy], [0, 0, 1]]
    const double is = 1.0 / nb.s;
    for (int c = 0; c < 3; ++c) {
        H[0 + c] = is * t[0 + c] + nb.cx * t[6 + c];
        H[3 + c] = is * t[3 + c] + nb.cy * t[6 + c];
        H[6 + c] = t[6 + c];
    }
    double mx = 0;
    for (int i = 0; i < 9; ++i) mx = fmax(mx, fabs(H[i]));
    if (!(fabs(H[8]) > 1e-12 * mx)) return false;
    const double h = H[8];
    for (int i = 0; i < 9; ++i) H[i] /= h;
    return true;
}

// Slots of the per-call flags word array (int32).
constexpr int kFlagBest = 0, kFlagCount = 1, kFlagStop = 2, kFlagIters = 3, kFlagCmax = 4, kFlagWords = 8;

// The first K distinct match indices of iteration t's Philox stream: word j is
// word j % 4 of block j / 4 (counter (t, j / 4, 0, 0)); prefix == nullptr
// draws uniformly (index = floor(w * M / 2^32)), otherwise word w picks the
// match whose interval of the inclusive prefix sums of integer weights
// contains floor(w * total / 2^32).  Repeats are redrawn, at most 64 words.
// Returns how many indices were drawn (K, or fewer when the words ran out).
template <int K>
__device__ __forceinline__ int draw_sample(int t, uint32_t k0, uint32_t k1, long long M,
                                           const unsigned long long* prefix, int* idx)
{
    int n = 0;
    uint4 blk = make_uint4(0, 0, 0, 0);
    for (int j = 0; j < 64 && n < K; ++j) {
        if ((j & 3) == 0) blk = philox(make_uint4((uint32_t)t, (uint32_t)(j >> 2), 0u, 0u), k0, k1);
        const uint32_t w = (j & 3) == 0 ? blk.x : (j & 3) == 1 ? blk.y : (j & 3) == 2 ? blk.z : blk.w;
        int i;
        if (!prefix) {
            i = (int)(((unsigned long long)w * (unsigned long long)M) >> 32);
        } else {
            const unsigned long long total = prefix[M - 1];
            const unsigned long long target = __umul64hi((unsigned long long)w << 32, total);
            long long lo = 0, hi = M - 1;
            while (lo < hi) {
                const long long mid = (lo + hi) >> 1;
                if (prefix[mid] > target) hi = mid; else lo = mid + 1;
            }
            i = (int)lo;
        }
        bool dup = false;
#pragma unroll
        for (int q = 0; q < K - 1; ++q) dup |= q < n && idx[q] == i;
        if (!dup) {
#pragma unroll
            for (int q = 0; q < K; ++q)
                if (q == n) idx[q] = i;
            ++n;
        }
    }
    return n;
}

// Eight lanes per hypothesis, lane r owning row r of the normalised 8x9 DLT
// system (two rows per correspondence).
constexpr int kHypThreads = 64;

// prefix == nullptr: uniform draw; otherwise word w picks the match whose
// interval of the inclusive prefix sums of integer weights contains
// floor(w * total / 2^32) (probability proportional to the weight).
__global__ void __launch_bounds__(kHypThreads)
k_ransac_hyp(const float4* pts, long long M_cap, const int32_t* dM, int T, uint32_t k0, uint32_t k1,
             const unsigned long long* prefix, const int32_t* skip, double* Hs, int8_t* hok, int32_t* flags)
{
    const int g = (blockIdx.x * kHypThreads + threadIdx.x) >> 3;   // hypothesis t
    const int r = threadIdx.x & 7;
    const int base = threadIdx.x & 31 & ~7;                          // first lane of the group
    const unsigned gm = 0xFFu << base;
    if (skip && *skip) return;
    if (blockIdx.x == 0 && threadIdx.x == 0) flags[kFlagCmax] = -1;
    if (g >= T) return;                                              // whole groups
    const int t = g;
    if (r == 0) hok[t] = 0;
    const long long M = m_count(dM, M_cap);
    if (M < 4) return;
    // every lane of the group draws the same four indices
    int idx[4] = {0, 0, 0, 0};
    if (draw_sample<4>(t, k0, k1, M, prefix, idx) < 4) return;
    double xa[4], ya[4], xb[4], yb[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const float4 p = pts[idx[q]];
        xa[q] = p.x; ya[q] = p.y; xb[q] = p.z; yb[q] = p.w;
    }
#pragma unroll
    for (int a = 0; a < 4; ++a) {
        const int i0 = (a + 1) & 3, i1 = (a + 2) & 3, i2 = (a + 3) & 3;
        if (collinear(xa[i0], ya[i0], xa[i1], ya[i1], xa[i2], ya[i2])) return;
        if (collinear(xb[i0], yb[i0], xb[i1], yb[i1], xb[i2], yb[i2])) return;
    }
    Norm2D na, nb;
    if (!hartley4(xa, ya, na) || !hartley4(xb, yb, nb)) return;
    // this lane's row: correspondence q = r / 2, the u row (even) or v row (odd)
    const int q = r >> 1;
    const double pxa = q == 0 ? xa[0] : q == 1 ? xa[1] : q == 2 ? xa[2] : xa[3];
    const double pya = q == 0 ? ya[0] : q == 1 ? ya[1] : q == 2 ? ya[2] : ya[3];
    const double pxb = q == 0 ? xb[0] : q == 1 ? xb[1] : q == 2 ? xb[2] : xb[3];
    const double pyb = q == 0 ? yb[0] : q == 1 ? yb[1] : q == 2 ? yb[2] : yb[3];
    const double x = na.s * (pxa - na.cx), y = na.s * (pya - na.cy);
    const double u = nb.s * (pxb - nb.cx), v = nb.s * (pyb - nb.cy);
    double a[9];
    if ((r & 1) == 0) {
        a[0] = x; a[1] = y; a[2] = 1; a[3] = 0; a[4] = 0; a[5] = 0; a[6] = -x * u; a[7] = -y * u; a[8] = u;
    } else {
        a[0] = 0; a[1] = 0; a[2] = 0; a[3] = x; a[4] = y; a[5] = 1; a[6] = -x * v; a[7] = -y * v; a[8] = v;
    }
    // Gaussian elimination with partial pivoting (largest |a_rc| over rows
    // r >= c, the lowest row on ties); decisions are taken on group-uniform
    // values so the eight lanes never diverge around a shuffle
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        double pv = r >= c ? fabs(a[c]) : -1.0;
        int pr = r;
#pragma unroll
        for (int o = 1; o < 8; o <<= 1) {
            const double ov = __shfl_xor_sync(gm, pv, o);
            const int orr = __shfl_xor_sync(gm, pr, o);
            if (ov > pv || (ov == pv && orr < pr)) { pv = ov; pr = orr; }
        }
        pv = __shfl_sync(gm, pv, base);
        pr = __shfl_sync(gm, pr, base);
        if (!(pv > 1e-10)) return;
        const int src = base + (r == c ? pr : (r == pr ? c : r));
#pragma unroll
        for (int j = c; j < 9; ++j) a[j] = __shfl_sync(gm, a[j], src);
        double prow[9];
#pragma unroll
        for (int j = c; j < 9; ++j) prow[j] = __shfl_sync(gm, a[j], base + c);
        const double ip = 1.0 / prow[c];
        if (r > c) {
            const double f = a[c] * ip;
#pragma unroll
            for (int j = c; j < 9; ++j) a[j] -= f * prow[j];
        }
    }
    // back substitution, h_7 first; each h_k is broadcast as soon as known
    double acc = a[8];
    double h[9];
#pragma unroll
    for (int k = 7; k >= 0; --k) {
        double hk = r == k ? acc / a[k] : 0.0;
        hk = __shfl_sync(gm, hk, base + k);
        h[k] = hk;
        if (r < k) acc -= a[k] * hk;
    }
    h[8] = 1.0;
    if (r != 0) return;
    double H[9];
    if (!denorm(na, nb, h, H)) return;
    for (int i = 0; i < 9; ++i) Hs[9ll * t + i] = H[i];
    hok[t] = 1;
}

// Eq. 8 (rotation + translation): one thread per hypothesis.  The minimal
// sample is the first two distinct indices of the same stream; the model is
// their least-squares rigid fit: centroids, C = a.b and S = a x b of the
// centred coordinates, (cos, sin) = (C, S) / sqrt(C^2 + S^2), t = centroid_B -
// R centroid_A.  Every operation is one IEEE rounding in the order of the
// definition (no contraction), so the hypothesis is the same double on any
// conforming machine.  C = S = 0 (coincident points in one image) is skipped.
constexpr int kRigidThreads = 128;

__device__ bool rigid_fit2(const float4& p, const float4& q, double* H)
{
    const double cxa = __ddiv_rn(__dadd_rn(p.x, q.x), 2.0), cya = __ddiv_rn(__dadd_rn(p.y, q.y), 2.0);
    const double cxb = __ddiv_rn(__dadd_rn(p.z, q.z), 2.0), cyb = __ddiv_rn(__dadd_rn(p.w, q.w), 2.0);
    double Cs = 0.0, Ss = 0.0;
    const float4 r[2] = {p, q};
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        const double ax = __dsub_rn(r[i].x, cxa), ay = __dsub_rn(r[i].y, cya);
        const double bx = __dsub_rn(r[i].z, cxb), by = __dsub_rn(r[i].w, cyb);
        Cs = __dadd_rn(Cs, __dadd_rn(__dmul_rn(ax, bx), __dmul_rn(ay, by)));
        Ss = __dadd_rn(Ss, __dsub_rn(__dmul_rn(ax, by), __dmul_rn(ay, bx)));
    }
    const double rr = __dsqrt_rn(__dadd_rn(__dmul_rn(Cs, Cs), __dmul_rn(Ss, Ss)));
    if (!(rr > 0.0)) return false;
    const double c = __ddiv_rn(Cs, rr), s = __ddiv_rn(Ss, rr);
    H[0] = c; H[1] = -s; H[2] = __dsub_rn(cxb, __dsub_rn(__dmul_rn(c, cxa), __dmul_rn(s, cya)));
    H[3] = s; H[4] = c;  H[5] = __dsub_rn(cyb, __dadd_rn(__dmul_rn(s, cxa), __dmul_rn(c, cya)));
    H[6] = 0.0; H[7] = 0.0; H[8] = 1.0;
    return true;
}

__global__ void __launch_bounds__(kRigidThreads)
k_ransac_hyp_rigid(const float4* pts, long long M_cap, const int32_t* dM, int T, uint32_t k0, uint32_t k1,
                   const unsigned long long* prefix, const int32_t* skip, double* Hs, int8_t* hok, int32_t* flags)
{
    const int t = blockIdx.x * kRigidThreads + threadIdx.x;
    if (skip && *skip) return;
    if (blockIdx.x == 0 && threadIdx.x == 0) flags[kFlagCmax] = -1;
    if (t >= T) return;
    hok[t] = 0;
    const long long M = m_count(dM, M_cap);
    if (M < 2) return;
    int idx[2] = {0, 0};
    if (draw_sample<2>(t, k0, k1, M, prefix, idx) < 2) return;
    double H[9];
    if (!rigid_fit2(pts[idx[0]], pts[idx[1]], H)) return;
#pragma unroll
    for (int i = 0; i < 9; ++i) Hs[9ll * t + i] = H[i];
    hok[t] = 1;
}

// ---------------------------------------------------------------- scoring
constexpr int kScoreThreads = 256;

__device__ __forceinline__ int block_sum(int v, int* red)
{
#pragma unroll
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    __syncthreads();
    if (lane == 0) red[warp] = v;
    __syncthreads();
    int s = 0;
    for (int w = 0; w < nw; ++w) s += red[w];
    return s;
}

// FP32 inlier test against the band: 2 = certainly inside (e^2 < t^2 - eps),
// 1 = in the band, 0 = outside or w <= 0.  e^2 < t^2 <=> |(u, v) - w p_B|^2 <
// t^2 w^2 for w > 0 (no division).
__device__ __forceinline__ int band32(const float* h, const float4& p, float t2, float eps)
{
    const float w = fmaf(h[6], p.x, fmaf(h[7], p.y, h[8]));
    if (!(w > 0.f)) return 0;
    const float du = fmaf(-p.z, w, fmaf(h[0], p.x, fmaf(h[1], p.y, h[2])));
    const float dv = fmaf(-p.w, w, fmaf(h[3], p.x, fmaf(h[4], p.y, h[5])));
    const float d2 = du * du + dv * dv, w2 = w * w;
    return d2 < (t2 - eps) * w2 ? 2 : (d2 < (t2 + eps) * w2 ? 1 : 0);
}

__global__ void __launch_bounds__(kScoreThreads)
k_ransac_score(const float4* pts, long long M_cap, const int32_t* dM, const double* Hs, const int8_t* hok,
               float t2, float eps, const int32_t* skip, int32_t* lo, int32_t* hi, int32_t* flags)
{
    __shared__ int red[32];
    const int t = blockIdx.x;
    if ((skip && *skip) || !hok[t]) {
        if (threadIdx.x == 0) { lo[t] = -1; hi[t] = -1; }
        return;
    }
    const long long M = m_count(dM, M_cap);
    float h[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) h[i] = (float)Hs[9ll * t + i];
    int clo = 0, chi = 0;
    for (long long i = threadIdx.x; i < M; i += kScoreThreads) {
        const int b = band32(h, pts[i], t2, eps);
        clo += b == 2;
        chi += b != 0;
    }
    clo = block_sum(clo, red);
    chi = block_sum(chi, red);
    if (threadIdx.x == 0) {
        lo[t] = clo;
        hi[t] = chi;
        atomicMax(flags + kFlagCmax, clo);
    }
}

// FP64 inlier test of one correspondence (Eq. 7, one-sided error in B):
// |pi(H p_A) - p_B|^2 < t^2, written for w > 0 as |(u, v) - w p_B|^2 < t^2 w^2,
// which needs no division.
__device__ __forceinline__ bool inlier64(const double* H, const float4& p, double t2)
{
    const double x = p.x, y = p.y;
    const double w = H[6] * x + H[7] * y + H[8];
    if (!(w > 0)) return false;
    const double du = H[0] * x + H[1] * y + H[2] - (double)p.z * w;
    const double dv = H[3] * x + H[4] * y + H[5] - (double)p.w * w;
    return du * du + dv * dv < t2 * (w * w);
}

// Exact count of every hypothesis that can still win: its possible count
// reaches c* (the largest certain count).  Points certainly inside count as
// inliers, points in the band are decided in FP64.  hi[t] <- the exact count,
// or -1 for a hypothesis that cannot win.
constexpr int kRecountThreads = 256;

__global__ void __launch_bounds__(kRecountThreads)
k_ransac_recount(const float4* pts, long long M_cap, const int32_t* dM, const double* Hs, const int32_t* lo,
                 int32_t* hi, const int32_t* flags, float t2f, float eps, double t2, const int32_t* skip)
{
    __shared__ int red[32];
    __shared__ int mode;
    const int t = blockIdx.x;
    if (skip && *skip) return;
    if (threadIdx.x == 0) {
        const int l = lo[t], h = hi[t], cmax = flags[kFlagCmax];
        mode = (l < 0 || h < cmax) ? 0 : (h == l ? 1 : 2);
        if (mode == 0) hi[t] = -1;
    }
    __syncthreads();
    if (mode != 2) return;   // mode 1: no point in the band, hi[t] is already exact
    const long long M = m_count(dM, M_cap);
    double H[9];
    float h[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) { H[i] = Hs[9ll * t + i]; h[i] = (float)H[i]; }
    int n = 0;
    for (long long i = threadIdx.x; i < M; i += kRecountThreads) {
        const float4 p = pts[i];
        const int b = band32(h, p, t2f, eps);
        n += b == 2 ? 1 : (b == 1 ? (int)inlier64(H, p, t2) : 0);
    }
    n = block_sum(n, red);
    if (threadIdx.x == 0) hi[t] = n;
}

constexpr int kSelThreads = 1024;

// key = (count + 1) << 32 | (0xFFFFFFFF - t): the largest key is the most
// inliers at the earliest iteration.
__global__ void __launch_bounds__(kSelThreads)
k_ransac_argmax(const int32_t* exact, int T, const int32_t* skip, int t_off, int32_t* flags)
{
    __shared__ unsigned long long part[kSelThreads / 32];
    if (skip && *skip) return;
    unsigned long long key = 0;
    for (int t = threadIdx.x; t < T; t += kSelThreads) {
        const int c = exact[t];
        if (c >= 0) key = max(key, ((unsigned long long)(c + 1) << 32) | (0xFFFFFFFFull - (unsigned)t));
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) key = max(key, __shfl_xor_sync(0xFFFFFFFFu, key, o));
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = key;
    __syncthreads();
    if (threadIdx.x != 0) return;
    for (int w = 0; w < kSelThreads / 32; ++w) key = max(key, part[w]);
    if (key == 0) {
        flags[kFlagBest] = -1;
        flags[kFlagCount] = -1;
    } else {
        flags[kFlagBest] = t_off + (int)(0xFFFFFFFFull - (key & 0xFFFFFFFFull));
        flags[kFlagCount] = (int)(key >> 32) - 1;
    }
}

// Stop test of the guided phase.  w = (prior weight of the guided winner's
// FP64 inliers) / (total weight) is the chance that one guided draw is an
// inlier; the phase stops when (1 - w^4)^Tg <= 0.01, the standard bound
// T >= log(0.01) / log(1 - w^4) without logarithms.  Every operation is a
// single IEEE-rounded one (no contraction), powers by binary exponentiation.
// flags[kFlagStop] = stop, flags[kFlagIters] = iterations used.
// (1 - w^k)^Tg <= 0.01 for w = num / den: the standard stop bound
// T >= log(0.01) / log(1 - w^k), each operation one IEEE rounding in the
// order the CPU reference takes them, powers by binary exponentiation.
__device__ __forceinline__ bool guided_bound(double num, double den, int Tg, int k)
{
    const double w = __ddiv_rn(num, den);
    const double w2 = __dmul_rn(w, w);
    const double wk = k == 2 ? w2 : __dmul_rn(w2, w2);
    double b = __dsub_rn(1.0, wk), r = 1.0;
    for (int e = Tg; e; e >>= 1) {
        if (e & 1) r = __dmul_rn(r, b);
        b = __dmul_rn(b, b);
    }
    return r <= 0.01;
}

__global__ void __launch_bounds__(kSelThreads)
k_guided_decide(const float4* pts, long long M_cap, const int32_t* dM, const double* Hs,
                const unsigned long long* prefix, int Tg, int T, int k, double t2, int min_support, int32_t* flags)
{
    __shared__ unsigned long long part[kSelThreads / 32];
    __shared__ long long cpart[kSelThreads / 32];
    const int tb = flags[kFlagBest];
    const long long M = m_count(dM, M_cap);
    if (tb < 0 || M < k) {
        if (threadIdx.x == 0) { flags[kFlagStop] = 0; flags[kFlagIters] = Tg + T; }
        return;
    }
    double H[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) H[i] = Hs[9ll * tb + i];
    // prior mass and number of the guided winner's inliers
    unsigned long long sw = 0;
    long long cnt = 0;
    for (long long i = threadIdx.x; i < M; i += kSelThreads)
        if (inlier64(H, pts[i], t2)) {
            sw += prefix[i] - (i ? prefix[i - 1] : 0ull);
            ++cnt;
        }
#pragma unroll
    for (int o = 16; o; o >>= 1) {
        sw += __shfl_xor_sync(0xFFFFFFFFu, sw, o);
        cnt += __shfl_xor_sync(0xFFFFFFFFu, cnt, o);
    }
    if ((threadIdx.x & 31) == 0) {
        part[threadIdx.x >> 5] = sw;
        cpart[threadIdx.x >> 5] = cnt;
    }
    __syncthreads();
    if (threadIdx.x != 0) return;
    unsigned long long s_in = 0;
    long long n_win = 0;
    for (int w = 0; w < kSelThreads / 32; ++w) {
        s_in += part[w];
        n_win += cpart[w];
    }
    // the search ends on the guided winner only when the bound holds for its
    // prior-weighted and its plain inlier fraction, with enough support
    const int stop = guided_bound((double)s_in, (double)prefix[M - 1], Tg, k) && n_win >= (long long)min_support &&
                     guided_bound((double)n_win, (double)M, Tg, k);
    flags[kFlagStop] = stop;
    flags[kFlagIters] = stop ? Tg : Tg + T;
}

// ---------------------------------------------------------------- refit
// Least-squares refit of the winner's inliers (Eq. 7), spread over kRefitCTAs
// CTAs.  Each pass writes per-CTA partial sums; the next pass reduces them in
// a fixed order, so results do not depend on scheduling.
constexpr int kRefitThreads = 256;
constexpr int kRefitWarps = kRefitThreads / 32;
// The summing passes are FP64 reductions, and FP64 issue is scarce: a CTA has
// ~M / 32 points, so two warps per CTA keep the per-point work and halve
// nothing but the reduction.
constexpr int kSumThreads = 64;
constexpr int kSumWarps = kSumThreads / 32;
constexpr int kRefitCTAs = 32;
constexpr int kPartStride = 64;   // doubles per CTA partial row

struct RefitWS {
    double* part;     // [kRefitCTAs][kPartStride]
    double* Hf;       // [9] refitted homography
};

template <int N>
__device__ void block_sum_n(double* v, double (*part)[N], double* tot)
{
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
    for (int q = 0; q < N; ++q) {
        double x = v[q];
#pragma unroll
        for (int o = 16; o; o >>= 1) x += __shfl_xor_sync(0xFFFFFFFFu, x, o);
        v[q] = x;
    }
    if (lane == 0)
#pragma unroll
        for (int q = 0; q < N; ++q) part[warp][q] = v[q];
    __syncthreads();
    for (int q = threadIdx.x; q < N; q += kSumThreads) {
        double s = 0;
        for (int w = 0; w < kSumWarps; ++w) s += part[w][q];
        tot[q] = s;
    }
    __syncthreads();
}

__device__ __forceinline__ void cta_range(long long M, long long& b, long long& e)
{
    const long long chunk = (M + kRefitCTAs - 1) / kRefitCTAs;
    b = min(M, (long long)blockIdx.x * chunk);
    e = min(M, b + chunk);
}

// fixed-order sum of column q of the CTAs' partial rows
__device__ __forceinline__ double sum_col(const double* part, int q)
{
    double s = 0;
#pragma unroll 8
    for (int c = 0; c < kRefitCTAs; ++c) s += part[c * kPartStride + q];
    return s;
}

// pass 1: inlier mask of the winning hypothesis, count and coordinate sums
__global__ void __launch_bounds__(kSumThreads)
k_refit_p1(const float4* pts, long long M_cap, const int32_t* dM, const double* Hs, const int32_t* best_in,
           double t2, uint8_t* inl, RefitWS ws)
{
    __shared__ double part[kSumWarps][5];
    __shared__ double tot[5];
    const int best = *best_in;
    if (best < 0) return;
    const long long M = m_count(dM, M_cap);
    long long b, e;
    cta_range(M, b, e);
    double Hb[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) Hb[i] = Hs[9ll * best + i];
    double v5[5] = {0, 0, 0, 0, 0};
    for (long long i = b + threadIdx.x; i < e; i += kSumThreads) {
        const float4 p = pts[i];
        const bool in = inlier64(Hb, p, t2);
        inl[i] = in;
        if (in) { v5[0] += 1; v5[1] += p.x; v5[2] += p.y; v5[3] += p.z; v5[4] += p.w; }
    }
    block_sum_n<5>(v5, part, tot);
    if (threadIdx.x < 5) ws.part[blockIdx.x * kPartStride + threadIdx.x] = tot[threadIdx.x];
}

// pass 2: mean distances to the centroids (Hartley normalisation)
__global__ void __launch_bounds__(kSumThreads)
k_refit_p2(const float4* pts, long long M_cap, const int32_t* dM, const int32_t* best_in, const uint8_t* inl,
           RefitWS ws)
{
    __shared__ double part[kSumWarps][2];
    __shared__ double tot[2];
    __shared__ double c5[5];
    if (*best_in < 0) return;
    const long long M = m_count(dM, M_cap);
    if (threadIdx.x < 5) c5[threadIdx.x] = sum_col(ws.part, threadIdx.x);
    __syncthreads();
    const double n = c5[0];
    const double cxa = c5[1] / n, cya = c5[2] / n, cxb = c5[3] / n, cyb = c5[4] / n;
    long long b, e;
    cta_range(M, b, e);
    double v2[2] = {0, 0};
    for (long long i = b + threadIdx.x; i < e; i += kSumThreads) {
        if (!inl[i]) continue;
        const float4 p = pts[i];
        v2[0] += sqrt((p.x - cxa) * (p.x - cxa) + (p.y - cya) * (p.y - cya));
        v2[1] += sqrt((p.z - cxb) * (p.z - cxb) + (p.w - cyb) * (p.w - cyb));
    }
    block_sum_n<2>(v2, part, tot);
    if (threadIdx.x < 2) ws.part[blockIdx.x * kPartStride + 5 + threadIdx.x] = tot[threadIdx.x];
}

// Hartley normalisations of the inliers from the summed columns 0..6
// (count, coordinate sums, distance sums)
__device__ void norms_from_sums(const double* c7, Norm2D& na, Norm2D& nb, double& n, bool& good)
{
    n = c7[0];
    const double cxa = c7[1] / n, cya = c7[2] / n, cxb = c7[3] / n, cyb = c7[4] / n;
    const double da = c7[5] / n, db = c7[6] / n;
    na = Norm2D{sqrt(2.0) / da, cxa, cya};
    nb = Norm2D{sqrt(2.0) / db, cxb, cyb};
    good = n >= 4 && da > 0 && db > 0;
}

// pass 3: A^T A in normalised coordinates.  With a = (x, y, 1) of the A point
// and (u, v) of the B point, the two rows of a correspondence are (-a, 0, u a)
// and (0, -a, v a), so A^T A has the blocks sum a a^T (twice), -sum u a a^T,
// -sum v a a^T and sum (u^2 + v^2) a a^T: 4 x 6 distinct sums (columns 8..31:
// for each of 1, u, v, u^2 + v^2 the products xx, xy, x, yy, y, 1).
__global__ void __launch_bounds__(kSumThreads)
k_refit_p3(const float4* pts, long long M_cap, const int32_t* dM, const int32_t* best_in, const uint8_t* inl,
           RefitWS ws)
{
    __shared__ double part[kSumWarps][24];
    __shared__ double tot[24];
    __shared__ double nrm[6];
    __shared__ double c7[7];
    __shared__ int good_s;
    if (*best_in < 0) return;
    const long long M = m_count(dM, M_cap);
    if (threadIdx.x < 7) c7[threadIdx.x] = sum_col(ws.part, threadIdx.x);
    __syncthreads();
    if (threadIdx.x == 0) {
        Norm2D na, nb;
        double n;
        bool good;
        norms_from_sums(c7, na, nb, n, good);
        nrm[0] = na.s; nrm[1] = na.cx; nrm[2] = na.cy; nrm[3] = nb.s; nrm[4] = nb.cx; nrm[5] = nb.cy;
        good_s = good;
    }
    __syncthreads();
    const Norm2D na{nrm[0], nrm[1], nrm[2]}, nb{nrm[3], nrm[4], nrm[5]};
    long long b, e;
    cta_range(M, b, e);
    double acc[24];
#pragma unroll
    for (int q = 0; q < 24; ++q) acc[q] = 0;
    if (good_s) {
        for (long long i = b + threadIdx.x; i < e; i += kSumThreads) {
            if (!inl[i]) continue;
            const float4 p = pts[i];
            const double x = na.s * (p.x - na.cx), y = na.s * (p.y - na.cy);
            const double u = nb.s * (p.z - nb.cx), v = nb.s * (p.w - nb.cy);
            const double m[6] = {x * x, x * y, x, y * y, y, 1.0};
            const double f[4] = {1.0, u, v, u * u + v * v};
#pragma unroll
            for (int g = 0; g < 4; ++g)
#pragma unroll
                for (int q = 0; q < 6; ++q) acc[6 * g + q] += f[g] * m[q];
        }
    }
    block_sum_n<24>(acc, part, tot);
    if (threadIdx.x < 24) ws.part[blockIdx.x * kPartStride + 8 + threadIdx.x] = tot[threadIdx.x];
}

// Smallest eigenvector of the symmetric positive semi-definite 9x9 normal
// matrix S (assembled from the summed columns 8..31), as the dominant
// eigenvector of (S + mu I)^-1 (mu = 1e-12 trace S keeps the matrix positive
// definite for exact data and leaves the eigenvectors unchanged):
//   Gauss-Jordan inversion of [S + mu I | I] (9 pivot steps over the whole
//   block in parallel; positive pivots, as S + mu I is positive definite);
//   eight squarings of the inverse, each rescaled by a power of two (exact) so
//   its largest diagonal entry is in [1, 2): the result is (S + mu I)^-256 up
//   to scale, numerically rank one;
//   its column of largest diagonal entry, then two products with the inverse.
// FP64 issue is scarce, so the work is spread over few, wide steps instead of
// long serial chains.
constexpr int kSolveThreads = 192;

__global__ void __launch_bounds__(kSolveThreads)
k_refit_solve(const double* Hs, const int32_t* best_in, RefitWS ws, double* Hout, int32_t* n_in, int32_t* best_t)
{
    __shared__ double col[32];
    __shared__ double Sm[9][9];
    __shared__ double Ab[9][18];
    __shared__ double X[9][9];
    __shared__ double Y[9][9];
    __shared__ double vv[9];
    __shared__ double ipiv;
    __shared__ int ok_s;
    const int tid = threadIdx.x;
    const int best = *best_in;
    if (best < 0) {
        if (tid == 0) {
            if (best_t) *best_t = best;
            *n_in = 0;
        }
        if (tid < 9) { Hout[tid] = 0.0; ws.Hf[tid] = 0.0; }
        return;
    }
    if (tid < 7 || (tid >= 8 && tid < 32)) col[tid] = sum_col(ws.part, tid);
    __syncthreads();
    // S from the blocks: [[M1, 0, -Mu], [0, M1, -Mv], [-Mu, -Mv, Mw]], each M
    // the symmetric 3x3 of its six sums (xx, xy, x, yy, y, 1)
    for (int e = tid; e < 81; e += kSolveThreads) {
        const int r = e / 9, c = e % 9, br = r / 3, bc = c / 3, i = r % 3, j = c % 3;
        const int lo = i < j ? i : j, hi = i < j ? j : i;
        const int q = lo == 0 ? hi : (lo == 1 ? 2 + hi : 5);   // (0,0..2) -> 0..2, (1,1..2) -> 3..4, (2,2) -> 5
        double v = 0.0;
        if (br == bc && br < 2) v = col[8 + q];
        else if ((br == 0 && bc == 2) || (br == 2 && bc == 0)) v = -col[8 + 6 + q];
        else if ((br == 1 && bc == 2) || (br == 2 && bc == 1)) v = -col[8 + 12 + q];
        else if (br == 2 && bc == 2) v = col[8 + 18 + q];
        Sm[r][c] = v;
    }
    __syncthreads();
    Norm2D na, nb;
    double n;
    bool good;
    norms_from_sums(col, na, nb, n, good);
    double tr = 0;
    for (int i = 0; i < 9; ++i) tr += Sm[i][i];
    const double mu = 1e-12 * tr;
    const int r = tid / 18, c = tid - (tid / 18) * 18;   // this thread's entry of the 9 x 18 block
    const bool mine = tid < 162;
    if (mine) Ab[r][c] = c < 9 ? Sm[r][c] + (r == c ? mu : 0.0) : (c - 9 == r ? 1.0 : 0.0);
    if (tid == 0) ok_s = good ? 1 : 0;
    __syncthreads();
    for (int k = 0; k < 9; ++k) {
        if (tid == 0) {
            const double pv = Ab[k][k];
            if (!(pv > 0.0)) ok_s = 0;
            ipiv = pv > 0.0 ? 1.0 / pv : 0.0;
        }
        __syncthreads();
        double nv = 0.0;
        if (mine) {
            const double akc = Ab[k][c] * ipiv;
            nv = r == k ? akc : Ab[r][c] - Ab[r][k] * akc;
        }
        __syncthreads();
        if (mine) Ab[r][c] = nv;
        __syncthreads();
    }
    const bool ok = ok_s != 0;
    const int e = tid, er = e / 9, ec = e - (e / 9) * 9;   // this thread's entry of a 9 x 9 matrix
    if (ok) {
        // X = (S + mu I)^-1, then X <- X^2 eight times, each scaled by a power of two
        if (e < 81) X[er][ec] = Ab[er][9 + ec];
        __syncthreads();
        for (int it = 0; it < 8; ++it) {
            double acc = 0.0;
            if (e < 81)
                for (int k = 0; k < 9; ++k) acc += X[er][k] * X[k][ec];
            if (e < 81) Y[er][ec] = acc;
            __syncthreads();
            double dmax = 0.0;
            for (int i = 0; i < 9; ++i) dmax = fmax(dmax, Y[i][i]);
            if (e < 81) X[er][ec] = dmax > 0.0 ? scalbn(Y[er][ec], -ilogb(dmax)) : Y[er][ec];
            __syncthreads();
        }
        // the column of largest diagonal entry, normalised
        if (tid == 0) {
            int cb = 0;
            for (int i = 1; i < 9; ++i)
                if (X[i][i] > X[cb][cb]) cb = i;
            double nrm = 0.0;
            for (int i = 0; i < 9; ++i) nrm += X[i][cb] * X[i][cb];
            const double sc = nrm > 0.0 ? 1.0 / sqrt(nrm) : 0.0;
            for (int i = 0; i < 9; ++i) vv[i] = X[i][cb] * sc;
        }
        __syncthreads();
        // two inverse-iteration products: v <- (S + mu I)^-1 v, normalised
        for (int it = 0; it < 2; ++it) {
            double z = 0.0;
            if (tid < 9)
                for (int k = 0; k < 9; ++k) z += Ab[tid][9 + k] * vv[k];
            __syncthreads();
            if (tid < 9) Y[0][tid] = z;
            __syncthreads();
            if (tid == 0) {
                double nrm = 0.0;
                for (int i = 0; i < 9; ++i) nrm += Y[0][i] * Y[0][i];
                const double sc = nrm > 0.0 ? 1.0 / sqrt(nrm) : 0.0;
                for (int i = 0; i < 9; ++i) vv[i] = Y[0][i] * sc;
            }
            __syncthreads();
        }
    }
    if (tid != 0) return;
    if (best_t) *best_t = best;
    *n_in = 0;
    double h[9], H[9];
    for (int i = 0; i < 9; ++i) h[i] = vv[i];
    const bool fit = ok && denorm(na, nb, h, H);
    for (int i = 0; i < 9; ++i) {
        const double v = fit ? H[i] : Hs[9ll * best + i];
        ws.Hf[i] = v;
        Hout[i] = v;
    }
}

// Eq. 8 refit, pass 2 (after k_refit_p1's mask, count and coordinate sums):
// C = sum a.b and S = sum a x b of the inliers' coordinates minus their
// centroids, into columns 5 and 6.
__global__ void __launch_bounds__(kSumThreads)
k_rigid_p2(const float4* pts, long long M_cap, const int32_t* dM, const int32_t* best_in, const uint8_t* inl,
           RefitWS ws)
{
    __shared__ double part[kSumWarps][2];
    __shared__ double tot[2];
    __shared__ double c5[5];
    if (*best_in < 0) return;
    const long long M = m_count(dM, M_cap);
    if (threadIdx.x < 5) c5[threadIdx.x] = sum_col(ws.part, threadIdx.x);
    __syncthreads();
    const double n = c5[0];
    const double cxa = c5[1] / n, cya = c5[2] / n, cxb = c5[3] / n, cyb = c5[4] / n;
    long long b, e;
    cta_range(M, b, e);
    double v2[2] = {0, 0};
    for (long long i = b + threadIdx.x; i < e; i += kSumThreads) {
        if (!inl[i]) continue;
        const float4 p = pts[i];
        const double ax = p.x - cxa, ay = p.y - cya, bx = p.z - cxb, by = p.w - cyb;
        v2[0] += ax * bx + ay * by;
        v2[1] += ax * by - ay * bx;
    }
    block_sum_n<2>(v2, part, tot);
    if (threadIdx.x < 2) ws.part[blockIdx.x * kPartStride + 5 + threadIdx.x] = tot[threadIdx.x];
}

// Eq. 8 refit, solve: (cos, sin) = (C, S) / sqrt(C^2 + S^2), t = centroid_B -
// R centroid_A; fewer than two inliers or C = S = 0 keeps the hypothesis.
__global__ void __launch_bounds__(32)
k_rigid_solve(const double* Hs, const int32_t* best_in, RefitWS ws, double* Hout, int32_t* n_in, int32_t* best_t)
{
    if (threadIdx.x != 0) return;
    const int best = *best_in;
    if (best_t) *best_t = best;
    *n_in = 0;
    if (best < 0) {
        for (int i = 0; i < 9; ++i) { Hout[i] = 0.0; ws.Hf[i] = 0.0; }
        return;
    }
    double c7[7];
    for (int q = 0; q < 7; ++q) c7[q] = sum_col(ws.part, q);
    const double n = c7[0];
    const double cxa = c7[1] / n, cya = c7[2] / n, cxb = c7[3] / n, cyb = c7[4] / n;
    const double r = sqrt(c7[5] * c7[5] + c7[6] * c7[6]);
    const bool ok = n >= 2 && r > 0;
    double H[9];
    if (ok) {
        const double c = c7[5] / r, s = c7[6] / r;
        H[0] = c; H[1] = -s; H[2] = cxb - (c * cxa - s * cya);
        H[3] = s; H[4] = c;  H[5] = cyb - (s * cxa + c * cya);
        H[6] = 0.0; H[7] = 0.0; H[8] = 1.0;
    }
    for (int i = 0; i < 9; ++i) {
        const double v = ok ? H[i] : Hs[9ll * best + i];
        ws.Hf[i] = v;
        Hout[i] = v;
    }
}

// final inlier set of the refitted H
__global__ void __launch_bounds__(kRefitThreads)
k_refit_final(const float4* pts, long long M_cap, const int32_t* dM, RefitWS ws, double t2, uint8_t* inl,
              int32_t* n_in)
{
    __shared__ int red[kRefitWarps];
    const long long M = m_count(dM, M_cap);
    double H[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) H[i] = ws.Hf[i];
    const bool have = H[8] != 0.0;
    const long long chunk = (M_cap + gridDim.x - 1) / gridDim.x;
    const long long b = min(M_cap, (long long)blockIdx.x * chunk), e = min(M_cap, b + chunk);
    int n = 0;
    for (long long i = b + threadIdx.x; i < e; i += kRefitThreads) {
        const bool in = have && i < M && inlier64(H, pts[i], t2);
        inl[i] = in;
        n += in;
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) n += __shfl_xor_sync(0xFFFFFFFFu, n, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = n;
    __syncthreads();
    if (threadIdx.x == 0) {
        int s = 0;
        for (int w = 0; w < kRefitWarps; ++w) s += red[w];
        if (s) atomicAdd(n_in, s);
    }
}

}  // namespace

size_t compact_workspace(int64_t NA) { return sizeof(int32_t) * (size_t)((NA + kCompactRows - 1) / kCompactRows + 1); }

cudaError_t launch_compact(const uint32_t* kpA, int WA, const uint32_t* kpB, int WB, const int32_t* match,
                           int64_t NA, float* pts, int32_t* rows, int32_t* d_M, int32_t* tile_cnt, cudaStream_t s)
{
    const unsigned tiles = (unsigned)std::max<long long>(1, (NA + kCompactRows - 1) / kCompactRows);
    k_compact_count<<<tiles, kCompactThreads, 0, s>>>(match, NA, tile_cnt);
    k_compact_write<<<tiles, kCompactThreads, 0, s>>>(kpA, WA, kpB, WB, match, NA, tile_cnt,
                                                      reinterpret_cast<float4*>(pts), rows, d_M);
    return cudaGetLastError();
}

namespace {

struct RansacWS {
    double* Hs;       // [Ttot][9]
    int32_t* lo;      // [Ttot] certain FP32 counts (-1: no hypothesis)
    int32_t* hi;      // [Ttot] possible FP32 counts
    int32_t* flags;   // [4]: winner t, winner count, guided stop, iterations used
    int8_t* hok;      // [Ttot]
    RefitWS rw;
};

RansacWS carve(void* ws, int Ttot)
{
    RansacWS r;
    uint8_t* w = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(ws) + 255) & ~uintptr_t(255));
    r.Hs = reinterpret_cast<double*>(w);
    r.lo = reinterpret_cast<int32_t*>(r.Hs + 9ll * Ttot);
    r.hi = r.lo + Ttot;
    r.flags = r.hi + Ttot;
    r.hok = reinterpret_cast<int8_t*>(r.flags + kFlagWords);
    r.rw.part = reinterpret_cast<double*>((reinterpret_cast<uintptr_t>(r.hok + Ttot) + 255) & ~uintptr_t(255));
    r.rw.Hf = r.rw.part + kRefitCTAs * kPartStride + 1;
    return r;
}

void refit_launch(int model, const float4* p4, int64_t M_cap, const int32_t* d_M, double t2, const RansacWS& w,
                  double* H, uint8_t* inlier, int32_t* n_in, int32_t* best_t, cudaStream_t s)
{
    k_refit_p1<<<kRefitCTAs, kSumThreads, 0, s>>>(p4, M_cap, d_M, w.Hs, w.flags, t2, inlier, w.rw);
    if (model == LP_MODEL_RIGID) {
        k_rigid_p2<<<kRefitCTAs, kSumThreads, 0, s>>>(p4, M_cap, d_M, w.flags, inlier, w.rw);
        k_rigid_solve<<<1, 32, 0, s>>>(w.Hs, w.flags, w.rw, H, n_in, best_t);
    } else {
        k_refit_p2<<<kRefitCTAs, kSumThreads, 0, s>>>(p4, M_cap, d_M, w.flags, inlier, w.rw);
        k_refit_p3<<<kRefitCTAs, kSumThreads, 0, s>>>(p4, M_cap, d_M, w.flags, inlier, w.rw);
        k_refit_solve<<<1, kSolveThreads, 0, s>>>(w.Hs, w.flags, w.rw, H, n_in, best_t);
    }
    const unsigned gfin = (unsigned)std::max<long long>(1, std::min<long long>(kRefitCTAs, (M_cap + 1023) / 1024));
    k_refit_final<<<gfin, kRefitThreads, 0, s>>>(p4, M_cap, d_M, w.rw, t2, inlier, n_in);
}

// One batch of T hypotheses at rows [t_off, t_off + T) of the workspace,
// Philox counters 0..T-1; skipped entirely while *skip is non-zero.
void hyp_batch(int model, const float4* p4, int64_t M_cap, const int32_t* d_M, const unsigned long long* prefix,
               int T, int t_off, uint32_t k0, uint32_t k1, float t2f, float eps, double t2, const int32_t* skip,
               const RansacWS& w, cudaStream_t s)
{
    if (model == LP_MODEL_RIGID) {
        const unsigned gh = (unsigned)((T + kRigidThreads - 1) / kRigidThreads);
        k_ransac_hyp_rigid<<<gh, kRigidThreads, 0, s>>>(p4, M_cap, d_M, T, k0, k1, prefix, skip, w.Hs + 9ll * t_off,
                                                        w.hok + t_off, w.flags);
    } else {
        const unsigned gh = (unsigned)((8ll * T + kHypThreads - 1) / kHypThreads);
        k_ransac_hyp<<<gh, kHypThreads, 0, s>>>(p4, M_cap, d_M, T, k0, k1, prefix, skip, w.Hs + 9ll * t_off,
                                                w.hok + t_off, w.flags);
    }
    k_ransac_score<<<T, kScoreThreads, 0, s>>>(p4, M_cap, d_M, w.Hs + 9ll * t_off, w.hok + t_off, t2f, eps, skip,
                                               w.lo + t_off, w.hi + t_off, w.flags);
    k_ransac_recount<<<T, kRecountThreads, 0, s>>>(p4, M_cap, d_M, w.Hs + 9ll * t_off, w.lo + t_off, w.hi + t_off,
                                                   w.flags, t2f, eps, t2, skip);
    k_ransac_argmax<<<1, kSelThreads, 0, s>>>(w.hi + t_off, T, skip, t_off, w.flags);
}

}  // namespace

// Ttot = the number of hypotheses of one call (T, or Tg + T with a prior)
size_t ransac_workspace(int64_t M_cap, int Ttot)
{
    (void)M_cap;
    return 256 + (size_t)Ttot * (9 * sizeof(double) + 2 * sizeof(int32_t) + 1) + 256 +
           sizeof(double) * (kRefitCTAs * kPartStride + 16) + 256;
}

cudaError_t launch_ransac(const float* pts, int64_t M_cap, const int32_t* d_M, int T, int model, float thresh,
                          uint64_t seed, uint32_t pair_id, double* H, uint8_t* inlier, int32_t* n_in,
                          int32_t* best_t, void* ws, size_t ws_bytes, cudaStream_t s)
{
    if (ws_bytes < ransac_workspace(M_cap, T)) return cudaErrorInvalidValue;
    const RansacWS w = carve(ws, T);
    const float4* p4 = reinterpret_cast<const float4*>(pts);
    const uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32) ^ pair_id;
    const double t2 = (double)thresh * (double)thresh;
    const float t2f = (float)t2;
    const float eps = fmaxf(0.05f, 0.01f * t2f);
    hyp_batch(model, p4, M_cap, d_M, nullptr, T, 0, k0, k1, t2f, eps, t2, nullptr, w, s);
    refit_launch(model, p4, M_cap, d_M, t2, w, H, inlier, n_in, best_t, s);
    return cudaGetLastError();
}

// Guided phase (Tg hypotheses drawn by the prior's prefix sums), the stop test,
// then the uniform fallback (T hypotheses, the plain RANSAC stream), skipped on
// the device when the guided phase stopped.  Hypothesis rows: guided [0, Tg),
// uniform [Tg, Tg + T).
cudaError_t launch_ransac_prior(const float* pts, int64_t M_cap, const int32_t* d_M, const unsigned long long* prefix,
                                int Tg, int T, int model, float thresh, uint64_t seed, uint32_t pair_id,
                                int min_support, double* H,
                                uint8_t* inlier, int32_t* n_in, int32_t* best_t, int32_t* iters, void* ws,
                                size_t ws_bytes, cudaStream_t s)
{
    if (ws_bytes < ransac_workspace(M_cap, Tg + T)) return cudaErrorInvalidValue;
    const RansacWS w = carve(ws, Tg + T);
    const float4* p4 = reinterpret_cast<const float4*>(pts);
    const uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32) ^ pair_id;
    const double t2 = (double)thresh * (double)thresh;
    const float t2f = (float)t2;
    const float eps = fmaxf(0.05f, 0.01f * t2f);
    const int k = model == LP_MODEL_RIGID ? 2 : 4;
    hyp_batch(model, p4, M_cap, d_M, prefix, Tg, 0, k0, k1, t2f, eps, t2, nullptr, w, s);
    k_guided_decide<<<1, kSelThreads, 0, s>>>(p4, M_cap, d_M, w.Hs, prefix, Tg, T, k, t2, min_support, w.flags);
    hyp_batch(model, p4, M_cap, d_M, nullptr, T, Tg, k0, k1, t2f, eps, t2, w.flags + kFlagStop, w, s);
    refit_launch(model, p4, M_cap, d_M, t2, w, H, inlier, n_in, best_t, s);
    if (iters) {
        cudaError_t e = cudaMemcpyAsync(iters, w.flags + kFlagIters, sizeof(int32_t), cudaMemcpyDeviceToDevice, s);
        if (e != cudaSuccess) return e;
    }
    return cudaGetLastError();
}

// Certain inlier counts of the last RANSAC's hypotheses (-1: none or skipped).
cudaError_t ransac_counts(void* ws, int Ttot, int32_t* host_counts, cudaStream_t s)
{
    const RansacWS w = carve(ws, Ttot);
    cudaError_t e = cudaMemcpyAsync(host_counts, w.lo, sizeof(int32_t) * (size_t)Ttot, cudaMemcpyDeviceToHost, s);
    if (e != cudaSuccess) return e;
    return cudaStreamSynchronize(s);
}

cudaError_t launch_diag_philox(const uint32_t* ctr, int64_t n, uint32_t k0, uint32_t k1, uint32_t* out, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    k_diag_philox<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(reinterpret_cast<const uint4*>(ctr), n, k0, k1,
                                                              reinterpret_cast<uint4*>(out));
    return cudaGetLastError();
}

}  // namespace lp
